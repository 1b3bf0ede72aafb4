// Fused sparse supervision (Sec. 3.7, Eqs. 9-11; App. A): Charbonnier L1,
// tile-level sparse NCC (or, for Table 4's S-SSIM variant, SSIM) with the
// gradient-balanced weight, the per-pixel error
// of Eq. 2 and the error/age map updates of Eqs. 3-4.  One thread block per
// active tile, one thread per sampled pixel; tile moments are two-pass block
// reductions.
#include "tgs_common.cuh"

namespace tgs {

// Block-wide sum of K floats per thread; every thread receives the totals.
template <int K>
__device__ __forceinline__ void block_sum(float (&v)[K], float (*sm)[K]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sm[w][k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float s = 0.f;
    for (int q = 0; q < nw; ++q) s += sm[q][k];
    v[k] = s;
  }
  __syncthreads();
}

struct LossArgs {
  const float* rgb;
  const float* target;
  int W, H, tiles_x;
  const int32_t* active_tiles;
  const int32_t* n_active;
  const int32_t* pix_off;
  const uint8_t* pix_idx;
  float eps_c2, eps_n, beta, weight;
  uint16_t* err_map;
  uint16_t* age_map;
  float* dL;
  float* lambda;
  float* err_pix;
  double* loss;
};

// SSIM constants (Wang et al. 2004, dynamic range 1) of the S-SSIM variant.
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;

// STRUCT 0: the sparse NCC term (Sec. 3.7); 1: the SSIM term of Table 4's
// S-SSIM variant, per channel from the same tile moments:
// SSIM = (2 mx my + C1)(2 cov + C2) / ((mx^2 + my^2 + C1)(var_x + var_y + C2)).
template <int STRUCT>
__global__ void k_loss(LossArgs a) {
  __shared__ float sm[8][9];
  const int j = blockIdx.x;
  const int A = *a.n_active;
  if (j >= A) return;
  const int P = a.pix_off[A];
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  const int n = p1 - p0;
  const int s = p0 + threadIdx.x;
  const bool on = (int)threadIdx.x < n;
  float x[3] = {0.f, 0.f, 0.f}, y[3] = {0.f, 0.f, 0.f};
  size_t pix = 0;
  if (on) {
    const int l = a.pix_idx[s];
    const int px = (t % a.tiles_x) * TGS_TILE + (l & 15), py = (t / a.tiles_x) * TGS_TILE + (l >> 4);
    pix = (size_t)py * a.W + px;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c] = a.rgb[3 * (size_t)s + c];
      y[c] = a.target[3 * pix + c];
    }
  }
  // the pixel's error-map entry, read now so that the load overlaps the
  // block reductions (the barriers between would otherwise hold it back)
  uint16_t old_err = 0;
  if (on && a.err_map) old_err = a.err_map[pix];
  if (n <= 0) return;  // uniform per block
  const float inv_n = 1.f / (float)n;
  // pass 1: means
  float m[6] = {x[0], x[1], x[2], y[0], y[1], y[2]};
  block_sum<6>(m, reinterpret_cast<float(*)[6]>(&sm[0][0]));
  float mx[3], my[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mx[c] = m[c] * inv_n;
    my[c] = m[3 + c] * inv_n;
  }
  // pass 2: variances and covariances
  float dx[3], dy[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dx[c] = on ? x[c] - mx[c] : 0.f;
    dy[c] = on ? y[c] - my[c] : 0.f;
  }
  float mom[9] = {dx[0] * dx[0], dx[1] * dx[1], dx[2] * dx[2], dy[0] * dy[0], dy[1] * dy[1],
                  dy[2] * dy[2], dx[0] * dy[0], dx[1] * dy[1], dx[2] * dy[2]};
  block_sum<9>(mom, sm);
  // NCC: D = sqrt(var_x var_y + eps), ncc = cov / D.  SSIM: ncc holds SSIM,
  // q1 = 1 / (b1 b2), q2 = mx / b1, D = b2 (a1, a2, b1, b2 as in the SSIM formula)
  float vy[3], D[3], ncc[3], a1[3], a2[3], q1[3], q2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float vx = mom[c] * inv_n;
    vy[c] = mom[3 + c] * inv_n;
    const float cv = mom[6 + c] * inv_n;
    if (STRUCT == 0) {
      D[c] = sqrtf(vx * vy[c] + a.eps_n);
      ncc[c] = cv / D[c];
    } else {
      a1[c] = 2.f * mx[c] * my[c] + kC1;
      a2[c] = 2.f * cv + kC2;
      const float b1 = mx[c] * mx[c] + my[c] * my[c] + kC1;
      D[c] = vx + vy[c] + kC2;
      q1[c] = 1.f / (b1 * D[c]);
      q2[c] = mx[c] / b1;
      ncc[c] = a1[c] * a2[c] * q1[c];
    }
  }
  // per-pixel gradients of both terms and the balancing weight
  float d1[3], dn[3], l1 = 0.f, e = 0.f;
  float gs[2] = {0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float d = x[c] - y[c];
    const float r = sqrtf(d * d + a.eps_c2);
    d1[c] = d / r;                                             // dl1/dx
    if (STRUCT == 0)
      dn[c] = (dy[c] - ncc[c] * vy[c] * dx[c] / D[c]) / D[c];  // n dNCC_c/dx
    else                                                        // n dSSIM_c/dx
      dn[c] = 2.f * ((my[c] * a2[c] + a1[c] * dy[c]) * q1[c] - ncc[c] * (q2[c] + dx[c] / D[c]));
    if (on) {
      l1 += r;
      e += fabsf(d);
      gs[0] += fabsf(d1[c]);
      gs[1] += fabsf(dn[c]);
    }
  }
  float g2[2] = {gs[0], gs[1]};
  {
    float v9[9] = {g2[0], g2[1], on ? l1 : 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    block_sum<9>(v9, sm);
    g2[0] = v9[0];
    g2[1] = v9[1];
    l1 = v9[2];
  }
  const float lam = fminf(1.f, fmaxf(0.f, (g2[0] * inv_n) / (g2[1] * inv_n + 1e-8f)));
  if (on) {
    const float invP = 1.f / (float)P;
    const float cn = lam / (3.f * (float)A) * inv_n;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.dL[3 * (size_t)s + c] = (d1[c] * invP - cn * dn[c]) * a.weight;
    a.err_pix[s] = e;
    if (a.err_map) {
      const float old = __half2float(__ushort_as_half(old_err));
      a.err_map[pix] = __half_as_ushort(__float2half_rn((1.f - a.beta) * old + a.beta * e));
    }
    if (a.age_map) a.age_map[pix] = 0;
  }
  if (threadIdx.x == 0) {
    a.lambda[j] = lam;
    const double tile_loss = (double)l1 / (double)P +
                             (double)lam * (1.0 - ((double)ncc[0] + (double)ncc[1] + (double)ncc[2]) / 3.0) / (double)A;
    atomicAdd(a.loss, tile_loss * (double)a.weight);
  }
}

// A <- min(A + 1, 65535) on every pixel, eight at a time; the first thread
// also clears the loss accumulator the loss kernel adds to next.
__global__ void k_age_inc(uint16_t* __restrict__ age, int64_t n, double* __restrict__ loss) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *loss = 0.0;
  const int64_t n8 = n / 8;
  if (i < n8) {
    uint4 v = reinterpret_cast<uint4*>(age)[i];
    v.x = __vaddus2(v.x, 0x00010001u);
    v.y = __vaddus2(v.y, 0x00010001u);
    v.z = __vaddus2(v.z, 0x00010001u);
    v.w = __vaddus2(v.w, 0x00010001u);
    reinterpret_cast<uint4*>(age)[i] = v;
  } else {
    const int64_t k = n8 * 8 + (i - n8);
    if (i >= n8 && k < n) age[k] = (uint16_t)min(65535, (int)age[k] + 1);
  }
}

}  // namespace tgs

using namespace tgs;

static tgs_status loss_impl(int structure, const float* rgb, const float* target, int32_t width, int32_t height,
                            const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                            const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                            const tgs_loss_params* params, uint16_t* err_map, uint16_t* age_map, float* dL_drgb,
                            float* lambda_tile, float* err_pix, double* loss, tgs_stream stream) {
  if (!rgb || !target || width <= 0 || height <= 0 || !n_active || n_active_max < 0 || !pix_off || !pix_idx ||
      n_pix_max < 1 || n_pix_max > 256 || !params || !dL_drgb || !lambda_tile || !err_pix || !loss)
    return TGS_ERR_INVALID_ARG;
  if (age_map && !aligned16(age_map)) return TGS_ERR_INVALID_ARG;
  if (!(params->eps_charbonnier >= 0.f) || !(params->eps_ncc >= 0.f) || !(params->beta >= 0.f) ||
      !(params->view_weight >= 0.f) ||
      !(params->beta <= 1.f))
    return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (age_map) {
    const int64_t n = (int64_t)width * height;
    const int64_t threads = n / 8 + (n % 8);
    k_age_inc<<<(int)((threads + 255) / 256), 256, 0, s>>>(age_map, n, loss);
  } else {
    cudaMemsetAsync(loss, 0, sizeof(double), s);
  }
  if (n_active_max > 0) {
    LossArgs a;
    a.rgb = rgb; a.target = target; a.W = width; a.H = height; a.tiles_x = tiles_x(width);
    a.active_tiles = active_tiles; a.n_active = n_active; a.pix_off = pix_off; a.pix_idx = pix_idx;
    a.eps_c2 = params->eps_charbonnier * params->eps_charbonnier;
    a.eps_n = params->eps_ncc;
    a.beta = params->beta;
    a.weight = params->view_weight;
    a.err_map = err_map; a.age_map = age_map; a.dL = dL_drgb; a.lambda = lambda_tile; a.err_pix = err_pix;
    a.loss = loss;
    const int B = std::min(256, std::max(32, (n_pix_max + 31) / 32 * 32));
    if (structure == 0) k_loss<0><<<n_active_max, B, 0, s>>>(a);
    else k_loss<1><<<n_active_max, B, 0, s>>>(a);
  }
  return check_launch();
}

extern "C" tgs_status tgs_loss_sparse_ncc(const float* rgb, const float* target, int32_t width, int32_t height,
                                          const int32_t* active_tiles, const int32_t* n_active,
                                          int32_t n_active_max, const int32_t* pix_off, const uint8_t* pix_idx,
                                          int32_t n_pix_max, const tgs_loss_params* params, uint16_t* err_map,
                                          uint16_t* age_map, float* dL_drgb, float* lambda_tile, float* err_pix,
                                          double* loss, tgs_stream stream) {
  return loss_impl(0, rgb, target, width, height, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                   n_pix_max, params, err_map, age_map, dL_drgb, lambda_tile, err_pix, loss, stream);
}

extern "C" tgs_status tgs_loss_sparse_ssim(const float* rgb, const float* target, int32_t width, int32_t height,
                                           const int32_t* active_tiles, const int32_t* n_active,
                                           int32_t n_active_max, const int32_t* pix_off, const uint8_t* pix_idx,
                                           int32_t n_pix_max, const tgs_loss_params* params, uint16_t* err_map,
                                           uint16_t* age_map, float* dL_drgb, float* lambda_tile, float* err_pix,
                                           double* loss, tgs_stream stream) {
  return loss_impl(1, rgb, target, width, height, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                   n_pix_max, params, err_map, age_map, dL_drgb, lambda_tile, err_pix, loss, stream);
}
