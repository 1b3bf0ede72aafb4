// Per-tile memory, features and error-map refresh for the learned tile-error
// predictor (an extension; the paper refreshes stale error maps by rendering,
// Sec. 3.3).  A view keeps, per tile, what it last observed there: the length
// of the tile's splat list, the mean final transmittance and the mean error
// of the sampled pixels, and the iteration of the observation.  Features for
// the network are formed from that memory; its predictions can rescale a stale
// error map tile by tile before selection.
#include "tgs_common.cuh"

namespace tgs {

// One warp per active rank: means over the rank's sampled pixels.
__global__ void __launch_bounds__(128) k_tile_observe(const int32_t* __restrict__ active_tiles,
                                                      const int32_t* __restrict__ n_active, int n_active_max,
                                                      const int32_t* __restrict__ pix_off,
                                                      const int2* __restrict__ ranges,
                                                      const float* __restrict__ T_final,
                                                      const float* __restrict__ err_pix,
                                                      const uint64_t* __restrict__ iter_dev, uint64_t iter,
                                                      float4* __restrict__ mem, int64_t* __restrict__ mem_iter,
                                                      float* __restrict__ target, int residual) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n_active_max) return;
  if (j >= *n_active) {
    if (target && lane == 0) target[j] = 0.f;
    return;
  }
  const int p0 = pix_off[j], p1 = pix_off[j + 1];
  float st = 0.f, se = 0.f;
  for (int p = p0 + lane; p < p1; p += 32) {
    st += T_final[p];
    se += err_pix[p];
  }
  st = warp_sum(st);
  se = warp_sum(se);
  if (lane == 0) {
    const int n = max(1, p1 - p0);
    const int t = active_tiles[j];
    const int2 r = ranges[j];
    const float me = se / (float)n;
    const float4 old = mem[t];
    mem[t] = make_float4((float)(r.y - r.x), st / (float)n, me, 1.f);
    mem_iter[t] = (int64_t)(iter_dev ? *iter_dev : iter);
    // residual: the change since the tile's previous observation
    if (target) target[j] = log1pf(me) - (residual && old.w > 0.f ? log1pf(old.z) : 0.f);
  }
}

constexpr int kFeat = 16;

// Features of tile rows[r] (or tile r when rows is NULL): log(1 + list
// length), mean final transmittance, log(1 + error), cosine between the view
// and the reference direction, log(1 + iterations since the observation), the
// cosine of the tile centre's ray to the optical axis, and whether the tile
// was ever observed; the remaining slots are zero.  Rows past the device count
// are zero.
__global__ void __launch_bounds__(256) k_tile_features(const float4* __restrict__ mem,
                                                       const int64_t* __restrict__ mem_iter,
                                                       const int32_t* __restrict__ rows,
                                                       const int32_t* __restrict__ n_rows, int n_rows_max,
                                                       int tiles_x, float fx, float fy, float cx, float cy,
                                                       float view_cos, const uint64_t* __restrict__ iter_dev,
                                                       uint64_t iter, float* __restrict__ x) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows_max) return;
  float f[kFeat];
#pragma unroll
  for (int k = 0; k < kFeat; ++k) f[k] = 0.f;
  const int t = rows ? (r < *n_rows ? rows[r] : -1) : r;
  if (t >= 0) {
    const float4 m = mem[t];
    const int64_t now = (int64_t)(iter_dev ? *iter_dev : iter);
    const bool seen = m.w > 0.f;
    const int64_t d = now - mem_iter[t];
    const float age = seen ? (float)(d > 0 ? d : 0) : 1e6f;
    const float u = ((t % tiles_x) * TGS_TILE + 0.5f * TGS_TILE - cx) / fx;
    const float v = ((t / tiles_x) * TGS_TILE + 0.5f * TGS_TILE - cy) / fy;
    f[0] = log1pf(m.x);
    f[1] = seen ? m.y : 1.f;
    f[2] = log1pf(m.z);
    f[3] = view_cos;
    f[4] = log1pf(age);
    f[5] = rsqrtf(1.f + u * u + v * v);
    f[6] = seen ? 1.f : 0.f;
  }
  float4* o = reinterpret_cast<float4*>(x + (size_t)r * kFeat);
#pragma unroll
  for (int k = 0; k < kFeat / 4; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// One block per tile: scale the tile's error values so their mean is the
// predicted exp(pred + base) - 1, base = the tile's feature 2 (its last
// observed log error) when predictions are residuals (all set to it when the
// tile's current mean is 0).
__global__ void __launch_bounds__(256) k_tile_refresh(const float* __restrict__ pred,
                                                      const float* __restrict__ base, uint16_t* __restrict__ err,
                                                      int W, int H, int tiles_x) {
  __shared__ float part[8];
  const int t = blockIdx.x, l = threadIdx.x;
  const int x = (t % tiles_x) * TGS_TILE + (l & 15), y = (t / tiles_x) * TGS_TILE + (l >> 4);
  const bool valid = x < W && y < H;
  const size_t k = (size_t)y * W + x;
  const float e = valid ? __half2float(__ushort_as_half(err[k])) : 0.f;
  float s = warp_sum(e);
  const int nv = __syncthreads_count(valid);
  if ((l & 31) == 0) part[l >> 5] = s;
  __syncthreads();
  float tot = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) tot += part[w];
  const float mean = tot / (float)max(1, nv);
  const float want = expm1f(fmaxf(pred[t] + (base ? base[16 * (size_t)t + 2] : 0.f), 0.f));
  if (!valid) return;
  const float v = mean > 0.f ? e * (want / mean) : want;
  err[k] = __half_as_ushort(__float2half_rn(v));
}

}  // namespace tgs

using namespace tgs;

extern "C" tgs_status tgs_tile_observe(const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                                       const int32_t* pix_off, const int32_t* tile_ranges, const float* T_final,
                                       const float* err_pix, uint64_t iter, const uint64_t* iter_dev, float* mem,
                                       int64_t* mem_iter, float* target, int32_t residual, tgs_stream stream) {
  if (n_active_max < 0 || !active_tiles || !n_active || !pix_off || !tile_ranges || !T_final || !err_pix || !mem ||
      !mem_iter || !aligned16(mem) || !aligned8(tile_ranges))
    return TGS_ERR_INVALID_ARG;
  if (n_active_max == 0) return TGS_OK;
  const int blocks = (int)((32ll * n_active_max + 127) / 128);
  k_tile_observe<<<blocks, 128, 0, (cudaStream_t)stream>>>(active_tiles, n_active, n_active_max, pix_off,
                                                          reinterpret_cast<const int2*>(tile_ranges), T_final,
                                                          err_pix, iter_dev, iter, reinterpret_cast<float4*>(mem),
                                                          mem_iter, target, residual);
  return check_launch();
}

extern "C" tgs_status tgs_tile_features(const float* mem, const int64_t* mem_iter, const int32_t* rows,
                                        const int32_t* n_rows, int32_t n_rows_max, const tgs_camera* cam,
                                        float view_cos, uint64_t iter, const uint64_t* iter_dev, float* x,
                                        tgs_stream stream) {
  if (!mem || !mem_iter || !cam || !x || n_rows_max < 0 || !aligned16(mem) || !aligned16(x) || cam->width <= 0 ||
      cam->height <= 0 || !(cam->fx > 0.f) || !(cam->fy > 0.f) || (rows && !n_rows))
    return TGS_ERR_INVALID_ARG;
  if (!rows && n_rows_max > tiles_x(cam->width) * tiles_y(cam->height)) return TGS_ERR_INVALID_ARG;
  if (n_rows_max == 0) return TGS_OK;
  k_tile_features<<<(n_rows_max + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4*>(mem), mem_iter, rows, n_rows, n_rows_max, tiles_x(cam->width), cam->fx,
      cam->fy, cam->cx, cam->cy, view_cos, iter_dev, iter, x);
  return check_launch();
}

extern "C" tgs_status tgs_tile_refresh(const float* pred, const float* base, uint16_t* err_map, int32_t width,
                                       int32_t height, tgs_stream stream) {
  if (!pred || !err_map || width <= 0 || height <= 0) return TGS_ERR_INVALID_ARG;
  const int T = tiles_x(width) * tiles_y(height);
  k_tile_refresh<<<T, 256, 0, (cudaStream_t)stream>>>(pred, base, err_map, width, height, tiles_x(width));
  return check_launch();
}
