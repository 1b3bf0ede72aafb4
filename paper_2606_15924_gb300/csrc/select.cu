// Tile selection and tile-wise error-guided pixel sampling (Sec. 3.5).
//
// Both levels choose n items as: round(r_hard n) by the error-proportional
// draw without replacement, round(r_stable n) of the rest with the largest age,
// the remainder uniformly.  The weighted draw is realised as the
// Efraimidis-Spirakis order (ascending E_i / w_i with E_i = -log2 U_i an
// exponential clock in 32-bit fixed point), so every item's fate is decided
// by counting the items that precede it in a total order - no sequential
// loop, and integer-only arithmetic, hence bit-identical on every run.
#include "block_select.cuh"
#include "scan.cuh"

namespace tgs {

struct SelWs {
  uint64_t* tile_w;   // [T] sum of pixel weights
  uint64_t* tile_key; // [T] hard key: bits of the double L / w (exponential clock over weight)
  uint64_t* tile_u;   // [T] uniform key
  uint32_t* tile_age; // [T] smallest pixel age
  int32_t* rank_h;    // [T]
  int32_t* rank_s;    // [T]
  int32_t* rank_u;    // [T]
  int64_t* scan_sums;
  int64_t* total;     // [1]
};

static SelWs carve_sel(void* base, int T, size_t* total) {
  Carver c(base);
  SelWs w;
  w.tile_w = c.take<uint64_t>(T);
  w.tile_key = c.take<uint64_t>(T);
  w.tile_u = c.take<uint64_t>(T);
  w.tile_age = c.take<uint32_t>(T);
  w.rank_h = c.take<int32_t>(3 * (size_t)T);
  w.rank_s = w.rank_h + T;
  w.rank_u = w.rank_h + 2 * T;
  w.scan_sums = c.take<int64_t>((size_t)std::max(1, scan_blocks(T)));
  w.total = c.take<int64_t>(1);
  *total = c.size();
  return w;
}

struct SelGeom {
  int W, H, tx, T;
};

__device__ __forceinline__ int tile_valid(const SelGeom& g, int t) {
  int tx = t % g.tx, ty = t / g.tx;
  return min(TGS_TILE, g.W - tx * TGS_TILE) * min(TGS_TILE, g.H - ty * TGS_TILE);
}

// Hard order: ascending L / w in IEEE double (exact operands, correctly
// rounded division, so every machine computes the same key); weight 0 maps to
// L * 2^900, after every positive weight.  Positive doubles order like their
// bit patterns, so the key is used as an unsigned 64-bit integer; equal keys
// go to the lower index.
__device__ __forceinline__ uint64_t hard_key(uint64_t w, uint64_t L) {
  const double k = w ? __ddiv_rn(__ull2double_rn(L), __ull2double_rn(w)) : __ull2double_rn(L) * 0x1p900;
  return (uint64_t)__double_as_longlong(k);
}

// Per-tile weight (sum), age (min) and the tile's random keys.
// Hash prefixes of the call: the iteration comes from the host or, for graph
// replays, from device memory.
struct HashKeys {
  uint64_t seed, iter;
  const uint64_t* iter_dev;
  uint32_t view;
  __device__ __forceinline__ uint64_t prefix(uint32_t stream) const {
    return hash_prefix(seed, iter_dev ? *iter_dev : iter, view, stream);
  }
};

// 32 tiles per block of 8 warps, 4 tiles per warp: lane l sums the error
// weights and takes the minimum age of eight pixels of each (row l / 2,
// columns 8 (l % 2) .. + 7; one 16-byte load per map where the row allows
// it), all four tiles' loads in flight together, then the warp reduces.  The
// draws (-log2 of a hash, 32 dependent squarings) then run one tile per lane
// of the first warp.
constexpr int kStatsTiles = 32;
constexpr int kStatsPerWarp = kStatsTiles / 8;

__device__ __forceinline__ void pixel_row8(const uint16_t* __restrict__ err, const uint16_t* __restrict__ age,
                                           const SelGeom& g, int t, int lane, bool vec, uint64_t& wv,
                                           uint32_t& av) {
  wv = 0;
  av = 0xFFFFFFFFu;
  if (t >= g.T) return;
  const int y = (t / g.tx) * TGS_TILE + (lane >> 1), x0 = (t % g.tx) * TGS_TILE + 8 * (lane & 1);
  if (y >= g.H) return;
  const size_t p = (size_t)y * g.W + x0;
  uint16_t e[8], a[8];
  if (vec && x0 + 8 <= g.W) {  // 16-byte aligned: both maps are, and x0 and W are multiples of 8
    const uint4 ev = *reinterpret_cast<const uint4*>(err + p), avv = *reinterpret_cast<const uint4*>(age + p);
    const uint32_t ew[4] = {ev.x, ev.y, ev.z, ev.w}, aw[4] = {avv.x, avv.y, avv.z, avv.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      e[2 * u] = (uint16_t)(ew[u] & 0xFFFFu);
      e[2 * u + 1] = (uint16_t)(ew[u] >> 16);
      a[2 * u] = (uint16_t)(aw[u] & 0xFFFFu);
      a[2 * u + 1] = (uint16_t)(aw[u] >> 16);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      wv += err_weight(e[u]);
      av = min(av, (uint32_t)a[u]);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (x0 + u < g.W) {
        wv += err_weight(err[p + u]);
        av = min(av, (uint32_t)age[p + u]);
      }
  }
}

__global__ void __launch_bounds__(256) k_tile_stats(const uint16_t* __restrict__ err,
                                                    const uint16_t* __restrict__ age, SelGeom g, HashKeys hk,
                                                    SelWs w, bool vec) {
  __shared__ uint64_t s_w[kStatsTiles];
  __shared__ uint32_t s_a[kStatsTiles];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t0 = blockIdx.x * kStatsTiles;
  uint64_t wv[kStatsPerWarp];
  uint32_t av[kStatsPerWarp];
#pragma unroll
  for (int q = 0; q < kStatsPerWarp; ++q)
    pixel_row8(err, age, g, t0 + kStatsPerWarp * warp + q, lane, vec, wv[q], av[q]);
#pragma unroll
  for (int q = 0; q < kStatsPerWarp; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      wv[q] += __shfl_xor_sync(0xffffffffu, wv[q], o);
      av[q] = min(av[q], __shfl_xor_sync(0xffffffffu, av[q], o));
    }
  }
  if (lane < kStatsPerWarp) {
    // lane q keeps tile q of the warp (register arrays indexed by constants)
    uint64_t ww = wv[0];
    uint32_t aa = av[0];
#pragma unroll
    for (int q = 1; q < kStatsPerWarp; ++q)
      if (lane == q) {
        ww = wv[q];
        aa = av[q];
      }
    s_w[kStatsPerWarp * warp + lane] = ww;
    s_a[kStatsPerWarp * warp + lane] = aa;
  }
  __syncthreads();
  const int t = t0 + lane;
  if (warp == 0 && t < g.T) {
    w.tile_w[t] = s_w[lane];
    w.tile_age[t] = s_a[lane];
    // the FP64 division runs here, spread over the grid, and not in the
    // single-block selection (FP64 throughput is low on this part)
    w.tile_key[t] = hard_key(s_w[lane], neglog2_q32(hash_item(hk.prefix(STREAM_TILE_HARD), (uint32_t)t, 0)));
    w.tile_u[t] = hash_item(hk.prefix(STREAM_TILE_UNIF), (uint32_t)t, 0);
  }
}

// rank[i] += #{j in this block's chunk, eligible, preceding i} for the phase.
// phase 0: hard order among all; 1: age order among those not taken by phase
// 0; 2: uniform order among those not taken by phases 0 and 1.
constexpr int RANK_CHUNK = 64;

__global__ void __launch_bounds__(256) k_rank_tiles(SelWs w, int T, int phase, int kh, int ks) {
  __shared__ uint64_t s_k[RANK_CHUNK];
  __shared__ uint8_t s_e[RANK_CHUNK];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * RANK_CHUNK;
  // phase key, ascending, ties to the lower index:
  //  0: hard key; 1: (2^32 - 1 - age) (older first); 2: top 32 hash bits
  auto key = [&](int t) -> uint64_t {
    if (phase == 0) return w.tile_key[t];
    if (phase == 1) return 0xFFFFFFFFull - w.tile_age[t];
    return w.tile_u[t] >> 32;
  };
  if (threadIdx.x < RANK_CHUNK) {
    const int j = j0 + threadIdx.x;
    bool e = j < T;
    if (e && phase >= 1) e = w.rank_h[j] >= kh;
    if (e && phase >= 2) e = w.rank_s[j] >= ks;
    s_e[threadIdx.x] = e;
    s_k[threadIdx.x] = j < T ? key(j) : 0;
  }
  __syncthreads();
  if (i >= T) return;
  if (phase >= 1 && w.rank_h[i] < kh) return;
  if (phase >= 2 && w.rank_s[i] < ks) return;
  const uint64_t ki = key(i);
  int cnt = 0;
  const int jn = min(RANK_CHUNK, T - j0);
  for (int k = 0; k < jn; ++k) {
    const uint64_t kj = s_k[k];
    cnt += s_e[k] && (kj < ki || (kj == ki && j0 + k < i));
  }
  if (cnt) atomicAdd(phase == 0 ? &w.rank_h[i] : phase == 1 ? &w.rank_s[i] : &w.rank_u[i], cnt);
}

// Tile level in one block of 1024 threads (up to 1024 * ITEMS tiles): the
// three phases, then the ascending compaction into active_tiles, tile_rank,
// pix_off and n_active.
constexpr int kSelThreads = 1024;
constexpr int kSelBlockMaxTiles = kSelThreads * 16;

template <int ITEMS>
__global__ void __launch_bounds__(kSelThreads) k_select_block(SelWs w, SelGeom g, int n_sel, int kh, int ks,
                                                              int n_pix, int32_t* __restrict__ active_tiles,
                                                              int32_t* __restrict__ n_active,
                                                              int32_t* __restrict__ tile_rank,
                                                              int32_t* __restrict__ pix_off) {
  __shared__ RadixSelSmem sm;
  __shared__ int64_t s64[32];
  const int T = g.T;
  const bool all = n_sel >= T;
  uint64_t key[ITEMS];
  bool valid[ITEMS], elig[ITEMS], th[ITEMS], ts[ITEMS], tu[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int i = threadIdx.x * ITEMS + j;
    valid[j] = i < T;
    elig[j] = valid[j];
    key[j] = (valid[j] && !all && n_sel > 0) ? w.tile_key[i] : 0;
  }
  if (all || n_sel <= 0) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      th[j] = all && valid[j];
      ts[j] = tu[j] = false;
    }
  } else {
    block_radix_select<ITEMS>(key, elig, kh, 64, th, sm, s64, 0);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int i = threadIdx.x * ITEMS + j;
      elig[j] = valid[j] && !th[j];
      key[j] = valid[j] ? 0xFFFFull - min(w.tile_age[i], 0xFFFFu) : 0;
    }
    block_radix_select<ITEMS>(key, elig, ks, 16, ts, sm, s64, 1);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int i = threadIdx.x * ITEMS + j;
      elig[j] = valid[j] && !th[j] && !ts[j];
      key[j] = valid[j] ? (w.tile_u[i] >> 32) : 0;
    }
    block_radix_select<ITEMS>(key, elig, n_sel - kh - ks, 32, tu, sm, s64, 2);
  }
  // compaction: (taken count << 32 | pixel count) prefix in tile order
  int64_t mine = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int i = threadIdx.x * ITEMS + j;
    if (th[j] || ts[j] || tu[j]) mine += (1ll << 32) | (int64_t)min(n_pix, tile_valid(g, i));
  }
  int64_t total;
  int64_t pre = block_excl_sum(mine, s64, total);
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int i = threadIdx.x * ITEMS + j;
    if (!valid[j]) continue;
    if (th[j] || ts[j] || tu[j]) {
      const int r = (int)(pre >> 32);
      tile_rank[i] = r;
      active_tiles[r] = i;
      pix_off[r] = (int)(pre & 0xFFFFFFFFll);
      pre += (1ll << 32) | (int64_t)min(n_pix, tile_valid(g, i));
    } else {
      tile_rank[i] = -1;
    }
  }
  if (threadIdx.x == 0) {
    *n_active = (int32_t)(total >> 32);
    pix_off[total >> 32] = (int32_t)(total & 0xFFFFFFFFll);
  }
}

// Pixel sampling inside one chosen tile: one block of 256 threads (one per
// local pixel); each phase is one exact block-wide k-selection.
__global__ void __launch_bounds__(256) k_sample_pixels(const uint16_t* __restrict__ err,
                                                       const uint16_t* __restrict__ age, SelGeom g, int n_pix,
                                                       int hard_pm, int stable_pm, HashKeys hk,
                                                       const int32_t* __restrict__ active_tiles,
                                                       const int32_t* __restrict__ n_active,
                                                       const int32_t* __restrict__ pix_off,
                                                       uint8_t* __restrict__ pix_idx) {
  __shared__ uint32_t s_cnt[8];
  __shared__ RadixSelSmem sm;
  __shared__ int64_t s64[32];
  const int j = blockIdx.x;
  if (j >= *n_active) return;
  const int t = active_tiles[j];
  const int l = threadIdx.x;
  const int lane = l & 31;
  const int x = (t % g.tx) * TGS_TILE + (l & 15), y = (t / g.tx) * TGS_TILE + (l >> 4);
  const bool valid = x < g.W && y < g.H;
  const int nv = tile_valid(g, t);
  const int n = min(n_pix, nv);
  int kh, ks;
  split_counts(n, hard_pm, stable_pm, kh, ks);
  bool taken;
  if (n >= nv) {
    taken = valid;  // every valid pixel
  } else {
    uint64_t kh_key = 0, ku_key = 0;
    uint32_t av = 0;
    if (valid) {
      const size_t k = (size_t)y * g.W + x;
      av = age[k];
      kh_key = hard_key(err_weight(err[k]),
                        neglog2_q32(hash_item(hk.prefix(STREAM_PIX_HARD), (uint32_t)t, (uint32_t)l)));
      ku_key = hash_item(hk.prefix(STREAM_PIX_UNIF), (uint32_t)t, (uint32_t)l) >> 32;
    }
    // phase 0: error-proportional draw; 1: oldest of the rest; 2: uniform of the rest
    uint64_t key[1] = {kh_key};
    bool el[1] = {valid}, th[1], ts[1], tu[1];
    block_radix_select<1>(key, el, kh, 64, th, sm, s64, 0);
    key[0] = 0xFFFFull - av;
    el[0] = valid && !th[0];
    block_radix_select<1>(key, el, ks, 16, ts, sm, s64, 1);
    key[0] = ku_key;
    el[0] = valid && !th[0] && !ts[0];
    block_radix_select<1>(key, el, n - kh - ks, 32, tu, sm, s64, 2);
    taken = th[0] || ts[0] || tu[0];
  }
  // ascending compaction of the taken local indices
  const unsigned b = __ballot_sync(0xffffffffu, taken);
  if (lane == 0) s_cnt[l >> 5] = __popc(b);
  __syncthreads();
  int off = 0;
  for (int k = 0; k < (l >> 5); ++k) off += s_cnt[k];
  off += __popc(b & ((1u << lane) - 1u));
  if (taken) pix_idx[pix_off[j] + off] = (uint8_t)l;
}

__global__ void k_sel_finish(const int64_t* __restrict__ total, int32_t* __restrict__ n_active,
                             int32_t* __restrict__ pix_off) {
  const int64_t v = *total;
  *n_active = (int32_t)(v >> 32);
  pix_off[v >> 32] = (int32_t)(v & 0xFFFFFFFFll);
}

}  // namespace tgs

using namespace tgs;

// The launch sequence shared by both entry points (arguments checked).
static tgs_status launch_select(const uint16_t* err_map, const uint16_t* age_map, int32_t width, int32_t height,
                                int n_sel, int32_t n_pix, const tgs_sampling* cfg, uint64_t seed, uint64_t iter,
                                const uint64_t* iter_dev, uint32_t view, void* scratch, int32_t* active_tiles,
                                int32_t* n_active, int32_t* tile_rank, int32_t* pix_off, uint8_t* pix_idx,
                                cudaStream_t s) {
  const int T = tiles_x(width) * tiles_y(height);
  size_t tot;
  SelWs w = carve_sel(scratch, T, &tot);
  SelGeom g{width, height, tiles_x(width), T};
  const HashKeys hk{seed, iter, iter_dev, view};
  int kh, ks;
  split_counts(n_sel, cfg->tile_hard_pm, cfg->tile_stable_pm, kh, ks);
  if (n_sel < T && n_sel > 0)
    k_tile_stats<<<(T + kStatsTiles - 1) / kStatsTiles, 256, 0, s>>>(
        err_map, age_map, g, hk, w, aligned16(err_map) && aligned16(age_map) && width % 8 == 0);
  if (T <= kSelBlockMaxTiles) {
    // one block: the three phases and the compaction
    if (T <= kSelThreads * 4)
      k_select_block<4><<<1, kSelThreads, 0, s>>>(w, g, n_sel, kh, ks, n_pix, active_tiles, n_active, tile_rank,
                                                   pix_off);
    else if (T <= kSelThreads * 8)
      k_select_block<8><<<1, kSelThreads, 0, s>>>(w, g, n_sel, kh, ks, n_pix, active_tiles, n_active, tile_rank,
                                                   pix_off);
    else
      k_select_block<16><<<1, kSelThreads, 0, s>>>(w, g, n_sel, kh, ks, n_pix, active_tiles, n_active, tile_rank,
                                                    pix_off);
  } else {
    // many tiles: ranks by pairwise counting, then a device-wide scan.  A
    // tile is taken when rank_h < kh, or (not hard) rank_s < ks, or
    // (neither) rank_u < n_sel - kh - ks.
    cudaMemsetAsync(w.rank_h, 0, sizeof(int32_t) * 3 * (size_t)T, s);
    if (n_sel < T && n_sel > 0) {
      dim3 grid((T + 255) / 256, (T + RANK_CHUNK - 1) / RANK_CHUNK);
      if (kh > 0) k_rank_tiles<<<grid, 256, 0, s>>>(w, T, 0, kh, ks);
      if (ks > 0) k_rank_tiles<<<grid, 256, 0, s>>>(w, T, 1, kh, ks);
      if (n_sel - kh - ks > 0) k_rank_tiles<<<grid, 256, 0, s>>>(w, T, 2, kh, ks);
    }
    const int32_t* rh = w.rank_h;
    const int32_t* rs = w.rank_s;
    const int32_t* ru = w.rank_u;
    const int all = n_sel >= T ? 1 : 0, none = n_sel == 0 ? 1 : 0;
    const int ku = n_sel - kh - ks;
    const int npx = n_pix;
    int32_t* at = active_tiles;
    int32_t* tr = tile_rank;
    int32_t* po = pix_off;
    auto load = [=] __device__(int64_t t) -> int64_t {
      const bool taken = !none && (all || rh[t] < kh || rs[t] < ks || (rs[t] >= ks && ru[t] < ku));
      if (!taken) return 0;
      return (1ll << 32) | (int64_t)min(npx, tile_valid(g, (int)t));
    };
    auto store = [=] __device__(int64_t t, int64_t pre, int64_t v) {
      if (v) {
        const int r = (int)(pre >> 32);
        tr[t] = r;
        at[r] = (int)t;
        po[r] = (int)(pre & 0xFFFFFFFFll);
      } else {
        tr[t] = -1;
      }
    };
    exclusive_scan<int64_t>(load, store, nullptr, T, w.scan_sums, w.total, s);
    k_sel_finish<<<1, 1, 0, s>>>(w.total, n_active, pix_off);
  }
  if (n_sel > 0)
    k_sample_pixels<<<n_sel, 256, 0, s>>>(err_map, age_map, g, n_pix, cfg->pix_hard_pm, cfg->pix_stable_pm, hk,
                                          active_tiles, n_active, pix_off, pix_idx);
  return check_launch();
}

extern "C" size_t tgs_select_tiles_workspace_size(int32_t width, int32_t height) {
  size_t total = 0;
  if (width <= 0 || height <= 0) return 0;
  carve_sel(nullptr, tiles_x(width) * tiles_y(height), &total);
  return total;
}

extern "C" tgs_status tgs_select_tiles(const uint16_t* err_map, const uint16_t* age_map, int32_t width,
                                       int32_t height, int32_t n_select, int32_t n_pix, const tgs_sampling* cfg,
                                       uint64_t seed, uint64_t iter, const uint64_t* iter_dev, uint32_t view,
                                       void* workspace, size_t workspace_bytes, int32_t* active_tiles, int32_t* n_active,
                                       int32_t* tile_rank, int32_t* pix_off, uint8_t* pix_idx,
                                       tgs_stream stream) {
  if (width <= 0 || height <= 0 || width > (1 << 16) || height > (1 << 16) || n_select < 0 || n_pix < 1 ||
      n_pix > 256 || !cfg || !err_map || !age_map || !n_active || !tile_rank || !pix_off)
    return TGS_ERR_INVALID_ARG;
  const int pms[4] = {cfg->tile_hard_pm, cfg->tile_stable_pm, cfg->pix_hard_pm, cfg->pix_stable_pm};
  for (int k = 0; k < 4; ++k)
    if (pms[k] < 0 || pms[k] > 1000) return TGS_ERR_INVALID_ARG;
  const int T = tiles_x(width) * tiles_y(height);
  const int n_sel = std::min(n_select, T);
  if (n_sel > 0 && (!active_tiles || !pix_idx)) return TGS_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < tgs_select_tiles_workspace_size(width, height)) return TGS_ERR_INVALID_ARG;
  return launch_select(err_map, age_map, width, height, n_sel, n_pix, cfg, seed, iter, iter_dev, view, workspace,
                       active_tiles, n_active, tile_rank, pix_off, pix_idx, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// select_tiles without a caller workspace.
//
// For callers that cannot allocate device memory - for example code running
// inside a host framework that hands out all device memory from its own fixed
// pool and forbids any other allocation, or a latency-critical path where an
// allocation could block or synchronise the device.  The scratch that
// tgs_select_tiles carves out of `workspace` lives here in one file-scope
// device array of fixed size instead; every GPU that loads this library holds
// it until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

__device__ __align__(256) unsigned char g_select_scratch[TGS_SELECT_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void* g_scratch_ptr[TGS_SELECT_NOALLOC_MAX_DEVICES] = {};

// Device address of g_select_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
tgs_status select_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    tgs::set_cuda_error(e);
    return TGS_ERR_CUDA;
  }
  if (dev < 0 || dev >= TGS_SELECT_NOALLOC_MAX_DEVICES) return TGS_ERR_CAPACITY;  // the cache's size
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_select_scratch);
    if (e != cudaSuccess || !p) {
      tgs::set_cuda_error(e);
      return TGS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TGS_OK;
}

}  // namespace

extern "C" tgs_status tgs_select_tiles_noalloc(const uint16_t* err_map, const uint16_t* age_map, int32_t width,
                                               int32_t height, int32_t n_select, int32_t n_pix,
                                               const tgs_sampling* cfg, uint64_t seed, uint64_t iter,
                                               const uint64_t* iter_dev, uint32_t view, int32_t* active_tiles,
                                               int32_t* n_active, int32_t* tile_rank, int32_t* pix_off,
                                               uint8_t* pix_idx, tgs_stream stream) {
  if (width <= 0 || height <= 0 || width > (1 << 16) || height > (1 << 16) || n_select < 0 || n_pix < 1 ||
      n_pix > 256 || !cfg || !err_map || !age_map || !n_active || !tile_rank || !pix_off)
    return TGS_ERR_INVALID_ARG;
  const int pms[4] = {cfg->tile_hard_pm, cfg->tile_stable_pm, cfg->pix_hard_pm, cfg->pix_stable_pm};
  for (int k = 0; k < 4; ++k)
    if (pms[k] < 0 || pms[k] > 1000) return TGS_ERR_INVALID_ARG;
  const int T = tiles_x(width) * tiles_y(height);
  if (T > TGS_SELECT_NOALLOC_MAX_TILES) return TGS_ERR_CAPACITY;
  size_t need = 0;
  carve_sel(nullptr, T, &need);
  if (need > sizeof(g_select_scratch)) return TGS_ERR_CAPACITY;
  const int n_sel = std::min(n_select, T);
  if (n_sel > 0 && (!active_tiles || !pix_idx)) return TGS_ERR_INVALID_ARG;
  void* scratch = nullptr;
  tgs_status st = select_scratch_address(&scratch);
  if (st != TGS_OK) return st;
  return launch_select(err_map, age_map, width, height, n_sel, n_pix, cfg, seed, iter, iter_dev, view, scratch,
                       active_tiles, n_active, tile_rank, pix_off, pix_idx, (cudaStream_t)stream);
}
