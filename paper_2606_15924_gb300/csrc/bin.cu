// Tile binning: the per-tile Gaussian lists ordered by depth (Sec. 3.1),
// built as a device LSD radix sort of (tile | depth) keys.  The low (depth)
// digits are sorted once per visible Gaussian before the splats are
// duplicated per tile; duplication keeps that order, so the remaining
// (tile) digits finish the same stable sort on the much longer pair list.
#include "radix.cuh"
#include "scan.cuh"

namespace tgs {

struct BinWs {
  int32_t* counts;     // [N] active tiles covered per Gaussian
  int32_t* vis_pos;    // [N] compacted position of visible Gaussians
  uint32_t* dk[2];     // [N] depth keys
  uint32_t* dv[2];     // [N] Gaussian ids
  int64_t* offs;       // [N] emission offsets in depth order
  int64_t* n_vis;      // [1]
  int32_t* n_vis32;    // [1]
  int32_t* n_sort;     // [1] min(n_isect, capacity)
  int32_t* inv_rank;   // [n_active_max] tile id of each rank
  uint32_t* tk[2];     // [C] tile-rank keys
  uint32_t* tv[2];     // [C] Gaussian ids
  int64_t* scan_sums;  // [scan blocks of N]
  uint32_t* hist;      // radix histograms
  uint32_t* bin_total; // [256]
};

static BinWs carve_bin(void* base, int64_t n, int64_t cap, int32_t n_active_max, size_t* total) {
  Carver c(base);
  BinWs w;
  size_t nn = (size_t)std::max<int64_t>(n, 1), cc = (size_t)std::max<int64_t>(cap, 1);
  w.counts = c.take<int32_t>(nn);
  w.vis_pos = c.take<int32_t>(nn);
  w.dk[0] = c.take<uint32_t>(nn);
  w.dk[1] = c.take<uint32_t>(nn);
  w.dv[0] = c.take<uint32_t>(nn);
  w.dv[1] = c.take<uint32_t>(nn);
  w.offs = c.take<int64_t>(nn);
  w.n_vis = c.take<int64_t>(1);
  w.n_vis32 = c.take<int32_t>(1);
  w.n_sort = c.take<int32_t>(1);
  w.inv_rank = c.take<int32_t>((size_t)std::max(n_active_max, 1));
  w.tk[0] = c.take<uint32_t>(cc);
  w.tk[1] = c.take<uint32_t>(cc);
  w.tv[0] = c.take<uint32_t>(cc);
  w.tv[1] = c.take<uint32_t>(cc);
  w.scan_sums = c.take<int64_t>((size_t)std::max(1, scan_blocks(n)));
  w.hist = c.take<uint32_t>(std::max(radix_hist_elems(n), radix_hist_elems(cap)));
  w.bin_total = c.take<uint32_t>(RS_BINS);
  *total = c.size();
  return w;
}

struct BinGeom {
  int tx, ty;
  int n_ranks;  // ranks >= n_ranks count as inactive
};

__device__ __forceinline__ bool rank_active(int r, const BinGeom& g) { return r >= 0 && r < g.n_ranks; }

// Number of active tiles in the rectangle of each Gaussian.
__global__ void __launch_bounds__(256) k_count_tiles(const float2* __restrict__ xy, const int32_t* __restrict__ radius,
                                                     int64_t n, BinGeom geo, const int32_t* __restrict__ tile_rank,
                                                     int32_t* __restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = radius[i];
  int c = 0;
  if (r > 0) {
    const float2 p = xy[i];
    int x0, x1, y0, y1;
    tile_span(p.x, r, geo.tx, x0, x1);
    tile_span(p.y, r, geo.ty, y0, y1);
    if (!tile_rank) {
      c = (x1 - x0) * (y1 - y0);
    } else {
      for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) c += rank_active(__ldg(tile_rank + ty * geo.tx + tx), geo);
    }
  }
  counts[i] = c;
}

__global__ void k_inv_rank(const int32_t* __restrict__ tile_rank, int T, int32_t* __restrict__ inv, int n_max) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int r = tile_rank ? tile_rank[t] : t;
  if (r >= 0 && r < n_max) inv[r] = t;
}

// Emit (tile rank, Gaussian) pairs for each visible Gaussian in depth order.
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ dv, const int64_t* __restrict__ offs,
                                              const int32_t* __restrict__ n_vis, const float2* __restrict__ xy,
                                              const int32_t* __restrict__ radius, BinGeom geo,
                                              const int32_t* __restrict__ tile_rank, int64_t cap,
                                              uint32_t* __restrict__ tk, uint32_t* __restrict__ tv, int64_t n_max) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= min((int64_t)*n_vis, n_max)) return;
  const uint32_t id = dv[j];
  int64_t o = offs[j];
  if (o >= cap) return;
  const float2 p = xy[id];
  const int r = radius[id];
  int x0, x1, y0, y1;
  tile_span(p.x, r, geo.tx, x0, x1);
  tile_span(p.y, r, geo.ty, y0, y1);
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx) {
      const int t = ty * geo.tx + tx;
      const int rank = tile_rank ? __ldg(tile_rank + t) : t;
      if (!rank_active(rank, geo)) continue;
      if (o >= cap) return;
      tk[o] = (uint32_t)rank;
      tv[o] = id;
      ++o;
    }
}

__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ tk, const int32_t* __restrict__ n_sort,
                                                int64_t n_max, int2* __restrict__ ranges) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = min((int64_t)*n_sort, n_max);
  if (i >= n) return;
  const uint32_t k = tk[i];
  if (i == 0 || tk[i - 1] != k) ranges[k].x = (int)i;
  if (i == n - 1 || tk[i + 1] != k) ranges[k].y = (int)(i + 1);
}

__global__ void __launch_bounds__(256) k_full_keys(const uint32_t* __restrict__ tk, const int32_t* __restrict__ vals,
                                                   const int32_t* __restrict__ n_sort, int64_t n_max,
                                                   const int32_t* __restrict__ inv_rank,
                                                   const float* __restrict__ depth, uint64_t* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= min((int64_t)*n_sort, n_max)) return;
  const uint32_t t = (uint32_t)inv_rank[tk[i]];
  keys[i] = ((uint64_t)t << 32) | (uint64_t)__float_as_uint(depth[vals[i]]);
}

__global__ void k_finish_counts(const int64_t* n_vis, int32_t* n_vis32, const int64_t* n_isect, int64_t cap,
                                int32_t* n_sort) {
  if (n_vis32) *n_vis32 = (int32_t)*n_vis;
  if (n_sort) *n_sort = (int32_t)min(*n_isect, cap);
}

}  // namespace tgs

using namespace tgs;

extern "C" size_t tgs_bin_tiles_workspace_size(int64_t n, int64_t capacity, int32_t n_active_max) {
  size_t total = 0;
  carve_bin(nullptr, n, capacity, n_active_max, &total);
  return total;
}

extern "C" tgs_status tgs_bin_tiles(const tgs_projected* proj, int64_t n, const tgs_camera* cam,
                                    const int32_t* tile_rank, int32_t n_active_max, void* workspace,
                                    size_t workspace_bytes, int64_t capacity, int32_t* vals, uint64_t* keys,
                                    int32_t* tile_ranges, int64_t* n_isect, tgs_stream stream) {
  if (!proj || !cam || n < 0 || capacity < 0 || capacity >= (int64_t)INT32_MAX || n >= (int64_t)INT32_MAX ||
      cam->width <= 0 || cam->height <= 0 || !n_isect || !tile_ranges || n_active_max < 0)
    return TGS_ERR_INVALID_ARG;
  const int T = tiles_x(cam->width) * tiles_y(cam->height);
  if (!tile_rank && n_active_max < T) return TGS_ERR_INVALID_ARG;
  if (n > 0 && (!proj->xy || !proj->radius || !proj->depth || !aligned8(proj->xy))) return TGS_ERR_INVALID_ARG;
  if (capacity > 0 && !vals) return TGS_ERR_INVALID_ARG;
  size_t need = tgs_bin_tiles_workspace_size(n, capacity, n_active_max);
  if (!workspace || workspace_bytes < need) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  size_t tot;
  BinWs w = carve_bin(workspace, n, capacity, n_active_max, &tot);
  BinGeom geo{tiles_x(cam->width), tiles_y(cam->height), n_active_max};
  if (n_active_max > 0) cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)n_active_max, s);
  cudaMemsetAsync(n_isect, 0, sizeof(int64_t), s);
  cudaMemsetAsync(w.n_sort, 0, sizeof(int32_t), s);
  if (n == 0) return check_launch();
  const float2* xy = reinterpret_cast<const float2*>(proj->xy);
  const int gb = (int)((n + 255) / 256);
  // 1. active tiles covered per Gaussian
  k_count_tiles<<<gb, 256, 0, s>>>(xy, proj->radius, n, geo, tile_rank, w.counts);
  // 2. compact the visible Gaussians with their depth keys
  {
    const int32_t* counts = w.counts;
    const float* depth = proj->depth;
    uint32_t* dk = w.dk[0];
    uint32_t* dv = w.dv[0];
    auto load = [=] __device__(int64_t i) -> int64_t { return counts[i] > 0 ? 1 : 0; };
    auto store = [=] __device__(int64_t i, int64_t pre, int64_t v) {
      if (v) {
        dk[pre] = __float_as_uint(depth[i]);
        dv[pre] = (uint32_t)i;
      }
    };
    exclusive_scan<int64_t>(load, store, nullptr, n, w.scan_sums, w.n_vis, s);
  }
  k_finish_counts<<<1, 1, 0, s>>>(w.n_vis, w.n_vis32, w.n_vis, 0, nullptr);
  // 3. stable sort of the visible Gaussians by depth (positive floats order as uint32)
  RadixScratch rsc{w.hist, w.bin_total};
  int cur = radix_sort_pairs(w.dk[0], w.dv[0], w.dk[1], w.dv[1], w.n_vis32, (int32_t)n, 0, 32, rsc, nullptr, s);
  const uint32_t* dv_sorted = w.dv[cur];
  // 4. emission offsets in depth order; n_isect = total
  {
    const int32_t* counts = w.counts;
    int64_t* offs = w.offs;
    auto load = [=] __device__(int64_t j) -> int64_t { return counts[dv_sorted[j]]; };
    auto store = [=] __device__(int64_t j, int64_t pre, int64_t) { offs[j] = pre; };
    exclusive_scan<int64_t>(load, store, w.n_vis, n, w.scan_sums, n_isect, s);
  }
  k_finish_counts<<<1, 1, 0, s>>>(w.n_vis, nullptr, n_isect, capacity, w.n_sort);
  if (capacity == 0) return check_launch();
  // 5. duplicate per active tile
  k_emit<<<gb, 256, 0, s>>>(dv_sorted, w.offs, w.n_vis32, xy, proj->radius, geo, tile_rank, capacity, w.tk[0],
                            w.tv[0], n);
  // 6. stable sort by tile rank (the high digits of the (tile | depth) key)
  int bits = 0;
  while ((1ll << bits) < (int64_t)std::max(n_active_max, 1)) ++bits;
  bits = std::max(8, (bits + 7) / 8 * 8);
  int tcur = radix_sort_pairs(w.tk[0], w.tv[0], w.tk[1], w.tv[1], w.n_sort, (int32_t)capacity, 0, bits, rsc,
                              reinterpret_cast<uint32_t*>(vals), s);
  const uint32_t* tk_sorted = w.tk[tcur];
  // 7. per-rank ranges, optional full keys
  const int cb = (int)((capacity + 255) / 256);
  k_ranges<<<cb, 256, 0, s>>>(tk_sorted, w.n_sort, capacity, reinterpret_cast<int2*>(tile_ranges));
  if (keys) {
    k_inv_rank<<<(T + 255) / 256, 256, 0, s>>>(tile_rank, T, w.inv_rank, std::max(n_active_max, 1));
    k_full_keys<<<cb, 256, 0, s>>>(tk_sorted, vals, w.n_sort, capacity, w.inv_rank, proj->depth, keys);
  }
  return check_launch();
}
