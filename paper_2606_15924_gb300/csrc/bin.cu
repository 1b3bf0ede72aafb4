// Tile binning: the per-tile Gaussian lists ordered by depth (Sec. 3.1, the
// depth-ordered sets K(p)) as a sort of (tile | depth | id) keys:
//   0. when the lists are long (the caller's capacity averages more than 2048
//      pairs per tile), the visible Gaussians are first sorted by depth
//      (stable LSD radix sort of the depth bits, ids ascending within equal
//      depths); otherwise the chunks below are runs of ids and step 4 sorts
//      every tile's whole list (in shared memory up to kSortSmem keys);
//   1. blocks take consecutive chunks of that order and count their pairs per
//      active tile in shared memory (a tile x block table of counts),
//   2. one scan of that table in tile-major order gives every (tile, block)
//      its output offset, hence each tile's range,
//   3. each block scatters (depth bits << 32 | id) into its offsets with
//      shared-memory cursors (no contended global atomics),
//   4. because block b's chunk lies wholly before block b + 1's in (depth,
//      id) order, a tile's range is a run of G segments that are already in
//      order with respect to each other; only each (tile, block) segment needs
//      sorting, which one warp does in registers (or shared memory for longer
//      segments; a whole-block bitonic network for the rare long ones).
// Positive float depths order like their bit patterns, so the result is the
// order (tile, depth, Gaussian id).  With more active tiles than the shared
// table holds, a global-atomic count/scatter and a per-tile sort of the whole
// range take over.
#include "radix.cuh"
#include "scan.cuh"

namespace tgs {

constexpr int kSortThreads = 256;
constexpr int kSortSmem = 4096;  // keys sorted in shared memory (32 KB)

constexpr int kHistBlocks = 1216;         // at most 8 chunks per SM in the count/scatter passes
constexpr int kHistChunk = 1536;          // Gaussians per chunk below that (before the rounding to SM waves)
constexpr int kHistMaxRanks = 49152;      // shared-memory table limit (192 KB)

// Chunks of about kHistChunk Gaussians, rounded up to whole waves of the SMs
// (every SM then holds the same number of chunks).
static int hist_blocks(int64_t n) {
  const int64_t c = (n + kHistChunk - 1) / kHistChunk;
  const int64_t sms = std::max(1, device_sm_count());
  return (int)std::max<int64_t>(1, std::min<int64_t>(kHistBlocks, (c + sms - 1) / sms * sms));
}

struct BinWs {
  int32_t* tile_cnt;   // [R] pairs per rank (global-atomic path)
  int32_t* tile_fill;  // [R] scatter cursors (global-atomic path)
  int64_t* tile_start; // [R] (global-atomic path)
  int64_t* table;      // [R * G] counts, then offsets (shared-memory path)
  uint64_t* keys;      // [C] (depth bits << 32 | id), grouped by tile
  int32_t* inv_rank;   // [R] tile id of each rank
  int64_t* scan_sums;
  uint32_t* dk[2];     // [N] depth keys (radix sort buffers)
  uint32_t* dv[2];     // [N] Gaussian ids
  int32_t* n_vis;      // [1] visible Gaussians
  RadixScratch rs;
};

static BinWs carve_bin(void* base, int64_t n, int64_t cap, int32_t n_ranks, size_t* total) {
  Carver c(base);
  BinWs w;
  const size_t R = (size_t)std::max(n_ranks, 1), C = (size_t)std::max<int64_t>(cap, 1);
  const size_t RG = R * (size_t)hist_blocks(n);
  const size_t N = (size_t)std::max<int64_t>(n, 1);
  w.tile_cnt = c.take<int32_t>(R);
  w.tile_fill = c.take<int32_t>(R);
  w.tile_start = c.take<int64_t>(R);
  w.table = c.take<int64_t>(RG);
  w.keys = c.take<uint64_t>(C);
  w.inv_rank = c.take<int32_t>(R);
  w.scan_sums = c.take<int64_t>((size_t)std::max(1, scan_blocks((int64_t)std::max(RG, R))));
  for (int b = 0; b < 2; ++b) {
    w.dk[b] = c.take<uint32_t>(N);
    w.dv[b] = c.take<uint32_t>(N);
  }
  w.n_vis = c.take<int32_t>(1);
  w.rs.hist = c.take<uint32_t>(radix_hist_elems(n));
  w.rs.bin_total = c.take<uint32_t>(RS_BINS);
  *total = c.size();
  return w;
}

// 0. depth keys of the visible Gaussians (invisible ones sort last) and the
// visible count
__global__ void __launch_bounds__(256) k_depth_keys(const int32_t* __restrict__ radius,
                                                    const float* __restrict__ depth, int64_t n,
                                                    uint32_t* __restrict__ keys, uint32_t* __restrict__ ids,
                                                    int32_t* __restrict__ n_vis) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool vis = false;
  if (i < n) {
    vis = radius[i] > 0;
    keys[i] = vis ? __float_as_uint(depth[i]) : 0xFFFFFFFFu;
    ids[i] = (uint32_t)i;
  }
  const int c = __syncthreads_count(vis);
  if (threadIdx.x == 0 && c) atomicAdd(n_vis, c);
}

struct BinGeom {
  int tx, ty;
  int n_ranks;  // ranks >= n_ranks count as inactive
};

__device__ __forceinline__ int rank_of(const int32_t* __restrict__ tile_rank, int t, const BinGeom& g) {
  const int r = tile_rank ? __ldg(tile_rank + t) : t;
  return (r >= 0 && r < g.n_ranks) ? r : -1;
}

// Calls f(gaussian id, rank) for every (Gaussian, active tile) pair of the
// block's Gaussians at positions [i0, i1) (of `order`, or the ids themselves).
// The pairs of a warp's 32 Gaussians are dealt out evenly: an inclusive warp
// prefix of the rectangle areas numbers them, and in each round lane l takes
// pair q = round * 32 + l, finding its Gaussian by binary search over the
// prefix (so a few large splats do not leave the other lanes idle).
template <typename F>
__device__ __forceinline__ void for_each_pair(const float2* __restrict__ xy, const int32_t* __restrict__ radius,
                                              int64_t i0, int64_t i1, const BinGeom& geo,
                                              const int32_t* __restrict__ tile_rank, F f,
                                              const uint32_t* __restrict__ order = nullptr) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t wave = blockDim.x;
  for (int64_t base = i0 + (threadIdx.x & ~31); base < i1; base += wave) {
    const int64_t pos = base + lane;
    int id = 0;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    if (pos < i1) {
      id = order ? (int)order[pos] : (int)pos;
      const int r = radius[id];
      if (r > 0) {
        const float2 p = xy[id];
        tile_span(p.x, r, geo.tx, x0, x1);
        tile_span(p.y, r, geo.ty, y0, y1);
      }
    }
    const int w = x1 - x0;
    const int area = w * (y1 - y0);
    int incl = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(full, incl, 31);
    for (int q0 = 0; q0 < total; q0 += 32) {
      const int q = q0 + lane;
      int lo = 0;  // first lane whose inclusive prefix exceeds q
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(full, incl, lo + step - 1);
        if (v <= q) lo += step;
      }
      const int o_incl = __shfl_sync(full, incl, lo), o_area = __shfl_sync(full, area, lo);
      const int o_w = __shfl_sync(full, w, lo), o_x0 = __shfl_sync(full, x0, lo);
      const int o_y0 = __shfl_sync(full, y0, lo), o_id = __shfl_sync(full, id, lo);
      if (q < total) {
        const int rem = q - (o_incl - o_area);
        const int ty = o_y0 + rem / o_w, tx = o_x0 + rem % o_w;
        const int k = rank_of(tile_rank, ty * geo.tx + tx, geo);
        if (k >= 0) f((int64_t)o_id, k);
      }
    }
  }
}

// 1''. pairs per active tile with global atomics, 256 Gaussians per block,
// their pairs dealt out evenly over the lanes.
__global__ void __launch_bounds__(256) k_count_pairs(const float2* __restrict__ xy,
                                                     const int32_t* __restrict__ radius, int64_t n, BinGeom geo,
                                                     const int32_t* __restrict__ tile_rank,
                                                     int32_t* __restrict__ tile_cnt) {
  const int64_t i0 = (int64_t)blockIdx.x * 256, i1 = min(n, i0 + 256);
  for_each_pair(xy, radius, i0, i1, geo, tile_rank, [&](int64_t, int k) { atomicAdd(tile_cnt + k, 1); });
}

// 3''. scatter with global cursors (order inside a tile arbitrary: the
// per-tile sort that follows orders it).
__global__ void __launch_bounds__(256) k_scatter_pairs(const float2* __restrict__ xy,
                                                       const int32_t* __restrict__ radius,
                                                       const float* __restrict__ depth, int64_t n, BinGeom geo,
                                                       const int32_t* __restrict__ tile_rank,
                                                       const int64_t* __restrict__ tile_start,
                                                       int32_t* __restrict__ tile_fill, uint64_t* __restrict__ keys,
                                                       int64_t cap) {
  const int64_t i0 = (int64_t)blockIdx.x * 256, i1 = min(n, i0 + 256);
  for_each_pair(xy, radius, i0, i1, geo, tile_rank, [&](int64_t i, int k) {
    const int64_t pos = tile_start[k] + atomicAdd(tile_fill + k, 1);
    if (pos < cap) keys[pos] = ((uint64_t)__float_as_uint(depth[i]) << 32) | (uint64_t)(uint32_t)i;
  });
}

// 1'. shared-memory path: block b counts the pairs of Gaussians
// [b * chunk, (b + 1) * chunk) per rank; table[r * G + b] = count.
constexpr int kHistThreads = 512;

// Block b's chunk of the depth order: [b * chunk, min(n_vis, (b + 1) * chunk)).
__device__ __forceinline__ void vis_chunk(const int32_t* n_vis, int64_t n_host, int64_t& i0, int64_t& i1) {
  const int64_t nv = n_vis ? *n_vis : n_host, G = gridDim.x;
  const int64_t chunk = (nv + G - 1) / G;
  i0 = (int64_t)blockIdx.x * chunk;
  i1 = min(nv, i0 + chunk);
}

// With reserve (per-rank counters, zeroed): instead of its counts, the block
// stores in table[r * G + b] the offset of its pairs inside rank r's list,
// reserved with one atomic per rank it touches (blocks land in any order
// within a list: only for lists that are sorted whole afterwards).
__global__ void __launch_bounds__(kHistThreads) k_hist_count(const float2* __restrict__ xy,
                                                             const int32_t* __restrict__ radius,
                                                             const uint32_t* __restrict__ order,
                                                             const int32_t* __restrict__ n_vis, int64_t n,
                                                             BinGeom geo, const int32_t* __restrict__ tile_rank,
                                                             int64_t* __restrict__ table,
                                                             int32_t* __restrict__ reserve) {
  extern __shared__ uint32_t sh[];
  const int R = geo.n_ranks, G = gridDim.x, b = blockIdx.x;
  for (int r = threadIdx.x; r < R; r += blockDim.x) sh[r] = 0;
  __syncthreads();
  int64_t i0, i1;
  vis_chunk(n_vis, n, i0, i1);
  for_each_pair(xy, radius, i0, i1, geo, tile_rank, [&](int64_t, int k) { atomicAdd(sh + k, 1u); }, order);
  __syncthreads();
  if (reserve) {
    for (int r = threadIdx.x; r < R; r += blockDim.x)
      if (sh[r]) table[(size_t)r * G + b] = atomicAdd(reserve + r, (int32_t)sh[r]);
  } else {
    for (int r = threadIdx.x; r < R; r += blockDim.x) table[(size_t)r * G + b] = sh[r];
  }
}

// 3'. shared-memory path: scatter with shared cursors that start at the
// block's offsets table[r * G + b] (clamped to the capacity; positions at or
// past the capacity are dropped).
// With rank_cnt (the ranks' totals, reserve mode): every block first takes
// the exclusive prefix of the totals itself (R values, from L2), the ranks'
// starts; block 0 also writes them to rank_start and their sum to n_total for
// the sort that follows.  This replaces a separate scan launch.
__global__ void __launch_bounds__(kHistThreads) k_hist_scatter(const float2* __restrict__ xy,
                                                               const int32_t* __restrict__ radius,
                                                               const float* __restrict__ depth,
                                                               const uint32_t* __restrict__ order,
                                                               const int32_t* __restrict__ n_vis, int64_t n,
                                                               BinGeom geo, const int32_t* __restrict__ tile_rank,
                                                               const int64_t* __restrict__ table,
                                                               int64_t* __restrict__ rank_start,
                                                               const int32_t* __restrict__ rank_cnt,
                                                               int64_t* __restrict__ n_total,
                                                               uint64_t* __restrict__ keys, int64_t cap) {
  extern __shared__ uint32_t sh[];
  __shared__ int64_t s_wt[32];
  const int R = geo.n_ranks, G = gridDim.x, b = blockIdx.x;
  if (rank_cnt) {
    // thread t scans the contiguous run [t * per, (t + 1) * per) of the totals
    const int per = (R + (int)blockDim.x - 1) / (int)blockDim.x;
    const int r0 = (int)threadIdx.x * per, r1 = min(R, r0 + per);
    int64_t run = 0;
    for (int r = r0; r < r1; ++r) run += rank_cnt[r];
    int64_t total;
    int64_t pre = block_exclusive_scan<int64_t>(run, s_wt, total);
    for (int r = r0; r < r1; ++r) {
      const int64_t c = rank_cnt[r];
      if (b == 0) rank_start[r] = pre;
      sh[r] = (uint32_t)min(table[(size_t)r * G + b] + pre, cap);
      pre += c;
    }
    if (b == 0 && threadIdx.x == 0) *n_total = total;
  } else {
    // the table holds absolute offsets, or (rank_start given) offsets within
    // each rank's list; entries of ranks the block has no pair in are not read
    // back as positions
    for (int r = threadIdx.x; r < R; r += blockDim.x)
      sh[r] = (uint32_t)min(table[(size_t)r * G + b] + (rank_start ? rank_start[r] : 0), cap);
  }
  __syncthreads();
  int64_t i0, i1;
  vis_chunk(n_vis, n, i0, i1);
  for_each_pair(xy, radius, i0, i1, geo, tile_rank, [&](int64_t i, int k) {
    const uint32_t pos = atomicAdd(sh + k, 1u);
    if ((int64_t)pos < cap) keys[pos] = ((uint64_t)__float_as_uint(depth[i]) << 32) | (uint64_t)(uint32_t)i;
  }, order);
}

// Ascending-only bitonic network over n keys padded (virtually) with +inf to
// a power of two: every compare-exchange puts the smaller key at the lower
// index, so padding never moves.  K is shared or global memory.
__device__ __forceinline__ void cmp_swap(uint64_t* K, int i, int j, int n) {
  if (j < n) {
    const uint64_t a = K[i], b = K[j];
    if (b < a) {
      K[i] = b;
      K[j] = a;
    }
  }
}

__device__ void bitonic_sort(uint64_t* K, int n) {
  int lg2 = 0;
  while ((1 << lg2) < n) ++lg2;
  const int n2 = 1 << lg2;
  for (int lk = 1; lk <= lg2; ++lk) {
    const int k = 1 << lk, lh = lk - 1, half = k >> 1;
    for (int t = threadIdx.x; t < n2 / 2; t += blockDim.x) {
      const int blk = t >> lh, off = t & (half - 1);
      cmp_swap(K, blk * k + off, blk * k + k - 1 - off, n);
    }
    __syncthreads();
    for (int ld = lk - 2; ld >= 0; --ld) {
      const int d = 1 << ld;
      for (int t = threadIdx.x; t < n2 / 2; t += blockDim.x) {
        const int i = ((t >> ld) << (ld + 1)) + (t & (d - 1));
        cmp_swap(K, i, i + d, n);
      }
      __syncthreads();
    }
  }
}

// 4. one block per active rank: sort its keys, write ids (and full keys)
// Range of rank r: from the offset table (stride G, shared-memory path) or
// from per-tile starts and counts (global-atomic path).
struct RangeSrc {
  const int64_t* table;
  int G, R;
  const int64_t* total;
  const int64_t* start;
  const int32_t* cnt;
  __device__ __forceinline__ void get(int r, int64_t& s0, int64_t& e0) const {
    if (table) {
      s0 = table[(size_t)r * G];
      e0 = r + 1 < R ? table[(size_t)(r + 1) * G] : *total;
    } else {
      s0 = start[r];
      e0 = s0 + cnt[r];
    }
  }
};

// Register-tiled bitonic sort of N = kSortThreads * E keys (E a power of two
// up to 16) for the tile lists that fit in shared memory.  Thread t holds the
// keys at positions t E .. t E + E - 1 in registers.  A compare-exchange
// stage at distance j runs in registers for j < E, through warp shuffles for
// E <= j < 32 E, and through shared memory only for j >= 32 E: of the
// log2(N) (log2(N) + 1) / 2 stages, at most 6 touch shared memory (the
// whole-list network in shared memory reads and writes every key at every
// stage, which is what bounded it).  The shared-memory layout pads one word
// after every E, so that both the blocked (t E + r) and the exchange accesses
// hit distinct banks.
__device__ __forceinline__ int pad_idx(int i, int E) { return E > 1 ? i + i / E : i; }

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
  return ((uint64_t)hi << 32) | lo;
}

// Sorts sm[pad_idx(0 .. N - 1, E)] ascending in place (N = kSortThreads E).
// Both stage loops have compile-time trip counts and are unrolled, so every
// distance j, and with it the kind of stage, is a constant.
template <int E>
__device__ __forceinline__ void bitonic_tile(uint64_t* sm) {
  constexpr int N = kSortThreads * E;
  constexpr int L = (N >= 4096) ? 12 : (N >= 2048) ? 11 : (N >= 1024) ? 10 : (N >= 512) ? 9 : 8;
  static_assert((1 << L) == N, "N is a power of two from 256 to 4096");
  const int t = threadIdx.x, base = t * E;
  uint64_t k[E];
#pragma unroll
  for (int r = 0; r < E; ++r) k[r] = sm[pad_idx(base + r, E)];
#pragma unroll
  for (int lk = 1; lk <= L; ++lk) {
    const int kk = 1 << lk;
    const bool up = (base & kk) == 0;  // for kk > E the direction is the thread's
#pragma unroll
    for (int lj = lk - 1; lj >= 0; --lj) {
      const int j = 1 << lj;
      if (j < E) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if (r & j) continue;
          const bool u = ((base + r) & kk) == 0;
          const uint64_t a = k[r], b = k[r | j];
          const bool sw = (b < a) == u;  // a == b: no change either way
          k[r] = sw ? b : a;
          k[r | j] = sw ? a : b;
        }
        continue;
      }
      const int m = j / E;  // partner thread t ^ m
      const bool keep_min = ((t & m) == 0) == up;
      if (m < 32) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const uint64_t y = shfl_xor_u64(k[r], m);
          k[r] = ((y < k[r]) == keep_min) ? y : k[r];
        }
      } else {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < E; ++r) sm[pad_idx(base + r, E)] = k[r];
        __syncthreads();
        const int pb = (t ^ m) * E;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const uint64_t y = sm[pad_idx(pb + r, E)];
          k[r] = ((y < k[r]) == keep_min) ? y : k[r];
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < E; ++r) sm[pad_idx(base + r, E)] = k[r];
  __syncthreads();
}

__global__ void __launch_bounds__(kSortThreads) k_tile_sort(uint64_t* __restrict__ keys, RangeSrc src,
                                                            const int32_t* __restrict__ inv_rank, int64_t cap,
                                                            int32_t* __restrict__ vals, uint64_t* __restrict__ full_keys,
                                                            int2* __restrict__ ranges) {
  __shared__ uint64_t sk[kSortSmem + kSortSmem / 16];
  const int r = blockIdx.x;
  int64_t s0, e0;
  src.get(r, s0, e0);
  const int64_t s = min(s0, cap), e = min(e0, cap);  // pairs past the capacity are dropped
  if (threadIdx.x == 0) ranges[r] = make_int2((int)s, (int)e);
  const int n = (int)(e - s);
  if (n <= 0) return;
  const uint64_t tile_hi = full_keys ? ((uint64_t)(uint32_t)inv_rank[r] << 32) : 0;
  if (n > kSortSmem) {  // long list: the whole-list network in global memory
    bitonic_sort(keys + s, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const uint64_t k = keys[s + i];
      vals[s + i] = (int32_t)(uint32_t)k;
      if (full_keys) full_keys[s + i] = tile_hi | (k >> 32);
    }
    return;
  }
  const int E = n <= kSortThreads ? 1 : n <= 2 * kSortThreads ? 2 : n <= 4 * kSortThreads ? 4
              : n <= 8 * kSortThreads ? 8 : 16;
  const int N = kSortThreads * E;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sk[pad_idx(i, E)] = i < n ? keys[s + i] : ~0ull;
  __syncthreads();
  switch (E) {
    case 1: bitonic_tile<1>(sk); break;
    case 2: bitonic_tile<2>(sk); break;
    case 4: bitonic_tile<4>(sk); break;
    case 8: bitonic_tile<8>(sk); break;
    default: bitonic_tile<16>(sk); break;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t k = sk[pad_idx(i, E)];
    vals[s + i] = (int32_t)(uint32_t)k;
    if (full_keys) full_keys[s + i] = tile_hi | (k >> 32);
  }
}

// 4'. one block per active rank: sort each (rank, block) segment.  Segments
// of up to kLaneKeys keys are sorted by one lane each (a bitonic network in
// registers), up to 32 by a warp in registers (a network across the lanes),
// up to kSegWarpKeys by a warp in its slice of shared memory, longer ones by
// the whole block afterwards.
constexpr int kSegThreads = 256;
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegWarpKeys = kSortSmem / kSegWarps;  // 512
constexpr int kSegMaxBig = 64;
constexpr int kLaneKeys = 8;

__device__ __forceinline__ void emit_sorted(uint64_t k, int64_t pos, uint64_t tile_hi, int32_t* __restrict__ vals,
                                            uint64_t* __restrict__ full_keys) {
  vals[pos] = (int32_t)(uint32_t)k;
  if (full_keys) full_keys[pos] = tile_hi | (k >> 32);
}

__device__ __forceinline__ void cx(uint64_t& a, uint64_t& b) {
  const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}

// One lane sorts len <= kLaneKeys keys at keys[ss...] (padding with +inf).
__device__ __forceinline__ void lane_sort(const uint64_t* __restrict__ keys, int64_t ss, int len, uint64_t tile_hi,
                                          int32_t* __restrict__ vals, uint64_t* __restrict__ full_keys) {
  if (len == 1) {
    emit_sorted(keys[ss], ss, tile_hi, vals, full_keys);
    return;
  }
  uint64_t k[kLaneKeys];
#pragma unroll
  for (int i = 0; i < kLaneKeys; ++i) k[i] = i < len ? keys[ss + i] : ~0ull;
  if (len <= 2) {
    cx(k[0], k[1]);
  } else if (len <= 4) {
    cx(k[0], k[1]); cx(k[2], k[3]); cx(k[0], k[2]); cx(k[1], k[3]); cx(k[1], k[2]);
  } else {
    // bitonic network for 8
#pragma unroll
    for (int kk = 2; kk <= 8; kk <<= 1)
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int l = i ^ j;
          if (l > i) {
            if ((i & kk) == 0) cx(k[i], k[l]);
            else cx(k[l], k[i]);
          }
        }
  }
#pragma unroll
  for (int i = 0; i < kLaneKeys; ++i)
    if (i < len) emit_sorted(k[i], ss + i, tile_hi, vals, full_keys);
}

__device__ __forceinline__ uint64_t warp_sort32(uint64_t key, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t other = __shfl_xor_sync(0xffffffffu, key, j);
      const bool up = (lane & k) == 0 || k == 32;
      const bool lower = (lane & j) == 0;
      const uint64_t lo = other < key ? other : key, hi = other < key ? key : other;
      key = (lower == up) ? lo : hi;
    }
  }
  return key;
}

// Ascending-only bitonic network run by one warp over n keys in K (shared).
__device__ void warp_bitonic(uint64_t* K, int n, int lane) {
  int lg2 = 0;
  while ((1 << lg2) < n) ++lg2;
  const int n2 = 1 << lg2;
  for (int lk = 1; lk <= lg2; ++lk) {
    const int k = 1 << lk, lh = lk - 1, half = k >> 1;
    for (int t = lane; t < n2 / 2; t += 32) {
      const int blk = t >> lh, off = t & (half - 1);
      cmp_swap(K, blk * k + off, blk * k + k - 1 - off, n);
    }
    __syncwarp();
    for (int ld = lk - 2; ld >= 0; --ld) {
      const int d = 1 << ld;
      for (int t = lane; t < n2 / 2; t += 32) {
        const int i = ((t >> ld) << (ld + 1)) + (t & (d - 1));
        cmp_swap(K, i, i + d, n);
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ void seg_bounds(const int64_t* row, int b, int G, int64_t e0, int64_t cap, int64_t& ss,
                                           int& len) {
  ss = min(row[b], cap);
  const int64_t ee = min(b + 1 < G ? row[b + 1] : e0, cap);
  len = ee > ss ? (int)(ee - ss) : 0;
}

__global__ void __launch_bounds__(kSegThreads) k_seg_sort(uint64_t* __restrict__ keys, RangeSrc src,
                                                          const int32_t* __restrict__ inv_rank, int64_t cap,
                                                          int32_t* __restrict__ vals,
                                                          uint64_t* __restrict__ full_keys,
                                                          int2* __restrict__ ranges) {
  __shared__ uint64_t sk[kSortSmem];
  __shared__ int big[kSegMaxBig];
  __shared__ int n_big;
  const int r = blockIdx.x, G = src.G;
  int64_t s0, e0;
  src.get(r, s0, e0);
  const int64_t s = min(s0, cap), e = min(e0, cap);
  if (threadIdx.x == 0) {
    ranges[r] = make_int2((int)s, (int)e);
    n_big = 0;
  }
  __syncthreads();
  if (e <= s) return;  // uniform across the block
  const uint64_t tile_hi = full_keys ? ((uint64_t)(uint32_t)inv_rank[r] << 32) : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t* row = src.table + (size_t)r * G;
  uint64_t* wk = sk + w * kSegWarpKeys;
  for (int b0 = w * 32; b0 < G; b0 += kSegWarps * 32) {
    const int b = b0 + lane;
    int64_t ss = 0;
    int len = 0;
    if (b < G) seg_bounds(row, b, G, e0, cap, ss, len);
    if (len > 0 && len <= kLaneKeys) lane_sort(keys, ss, len, tile_hi, vals, full_keys);
    unsigned longer = __ballot_sync(0xffffffffu, len > kLaneKeys);
    while (longer) {
      const int src_lane = __ffs(longer) - 1;
      longer &= longer - 1;
      const int64_t ls = __shfl_sync(0xffffffffu, ss, src_lane);
      const int ll = __shfl_sync(0xffffffffu, len, src_lane);
      if (ll <= 32) {
        uint64_t k = lane < ll ? keys[ls + lane] : ~0ull;
        k = warp_sort32(k, lane);
        if (lane < ll) emit_sorted(k, ls + lane, tile_hi, vals, full_keys);
      } else if (ll <= kSegWarpKeys) {
        for (int i = lane; i < ll; i += 32) wk[i] = keys[ls + i];
        __syncwarp();
        warp_bitonic(wk, ll, lane);
        for (int i = lane; i < ll; i += 32) emit_sorted(wk[i], ls + i, tile_hi, vals, full_keys);
        __syncwarp();
      } else if (lane == 0) {
        const int q = atomicAdd(&n_big, 1);
        if (q < kSegMaxBig) big[q] = b0 + src_lane;
      }
    }
  }
  __syncthreads();
  const int nb = n_big;
  if (nb > kSegMaxBig) {
    // many long segments: sort the whole range at once (it holds them all)
    const int n = (int)(e - s);
    uint64_t* K = n <= kSortSmem ? sk : keys + s;
    if (n <= kSortSmem) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = keys[s + i];
      __syncthreads();
    }
    bitonic_sort(K, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) emit_sorted(K[i], s + i, tile_hi, vals, full_keys);
    return;
  }
  for (int q = 0; q < nb; ++q) {
    int64_t ss;
    int len;
    seg_bounds(row, big[q], G, e0, cap, ss, len);
    uint64_t* K = len <= kSortSmem ? sk : keys + ss;
    if (len <= kSortSmem) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) sk[i] = keys[ss + i];
      __syncthreads();
    }
    bitonic_sort(K, len);
    for (int i = threadIdx.x; i < len; i += blockDim.x) emit_sorted(K[i], ss + i, tile_hi, vals, full_keys);
    __syncthreads();
  }
}

__global__ void k_inv_rank(const int32_t* __restrict__ tile_rank, int T, int32_t* __restrict__ inv, int n_max) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int r = tile_rank ? tile_rank[t] : t;
  if (r >= 0 && r < n_max) inv[r] = t;
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
  if (!aligned8(tile_ranges) || (keys && !aligned8(keys))) return TGS_ERR_INVALID_ARG;
  size_t need = tgs_bin_tiles_workspace_size(n, capacity, n_active_max);
  if (!workspace || workspace_bytes < need) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  size_t tot;
  BinWs w = carve_bin(workspace, n, capacity, n_active_max, &tot);
  BinGeom geo{tiles_x(cam->width), tiles_y(cam->height), n_active_max};
  const int R = n_active_max;
  // the scan writes n_isect and the per-rank sort writes every range; they
  // are cleared here only where those kernels do not run
  if (n == 0 || R == 0) {
    if (R > 0) cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)R, s);
    cudaMemsetAsync(n_isect, 0, sizeof(int64_t), s);
    return check_launch();
  }
  const float2* xy = reinterpret_cast<const float2*>(proj->xy);
  RangeSrc src{};
  // Per-chunk histograms in shared memory and an offset table, while the
  // ranks fit in shared memory: global per-tile counters and cursors take
  // every pair's atomic on a few hundred addresses, several times slower.
  const bool shared_path = R <= kHistMaxRanks;
  const int G = hist_blocks(n);
  const size_t smem = sizeof(int32_t) * (size_t)R;
  const uint32_t* order = nullptr;
  // The depth presort pays off only when tile lists outgrow the shared-memory
  // sort: it is used when the capacity (sized by the caller from the pairs of
  // all tiles) averages more than half of kSortSmem per tile.  Without it the
  // chunks are runs of ids and every tile's whole list is sorted.
  const bool presort = shared_path && capacity > 0 && capacity > (int64_t)(kSortSmem / 2) * T;
  const int32_t* n_vis = presort ? w.n_vis : nullptr;
  if (shared_path) {
    if (smem > 48 * 1024) {  // opt in to more than 48 KB of dynamic shared memory (per device)
      static bool attr_set[64] = {};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
      if (!attr_set[dev]) {
        cudaFuncSetAttribute(k_hist_count, cudaFuncAttributeMaxDynamicSharedMemorySize, kHistMaxRanks * 4);
        cudaFuncSetAttribute(k_hist_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kHistMaxRanks * 4);
        attr_set[dev] = true;
      }
    }
    if (presort) {
      cudaMemsetAsync(w.n_vis, 0, sizeof(int32_t), s);
      k_depth_keys<<<(int)((n + 255) / 256), 256, 0, s>>>(proj->radius, proj->depth, n, w.dk[0], w.dv[0],
                                                          w.n_vis);
      const int cur = radix_sort_pairs(w.dk[0], w.dv[0], w.dk[1], w.dv[1], nullptr, (int32_t)n, 0, 32, w.rs,
                                       nullptr, s);
      order = w.dv[cur];
    }
    if (presort) {
      // segments must follow the chunk order: a scan of the whole table
      k_hist_count<<<G, kHistThreads, smem, s>>>(xy, proj->radius, order, n_vis, n, geo, tile_rank, w.table,
                                                 nullptr);
      int64_t* tab = w.table;
      auto load = [=] __device__(int64_t i) -> int64_t { return tab[i]; };
      auto store = [=] __device__(int64_t i, int64_t pre, int64_t) { tab[i] = pre; };
      exclusive_scan<int64_t>(load, store, nullptr, (int64_t)R * G, w.scan_sums, n_isect, s);
      src.table = w.table;
      src.G = G;
      src.R = R;
      src.total = n_isect;
    } else {
      // lists are sorted whole afterwards: blocks reserve their runs with
      // per-rank atomics; the scatter scans the R rank totals itself
      cudaMemsetAsync(w.tile_cnt, 0, sizeof(int32_t) * (size_t)R, s);
      k_hist_count<<<G, kHistThreads, smem, s>>>(xy, proj->radius, order, n_vis, n, geo, tile_rank, w.table,
                                                 w.tile_cnt);
      src.start = w.tile_start;
      src.cnt = w.tile_cnt;
    }
  } else {
    const int gb = (int)((n + 255) / 256);
    cudaMemsetAsync(w.tile_cnt, 0, sizeof(int32_t) * (size_t)R, s);
    cudaMemsetAsync(w.tile_fill, 0, sizeof(int32_t) * (size_t)R, s);
    k_count_pairs<<<gb, 256, 0, s>>>(xy, proj->radius, n, geo, tile_rank, w.tile_cnt);
    const int32_t* cnt = w.tile_cnt;
    int64_t* start = w.tile_start;
    auto load = [=] __device__(int64_t r) -> int64_t { return cnt[r]; };
    auto store = [=] __device__(int64_t r, int64_t pre, int64_t) { start[r] = pre; };
    exclusive_scan<int64_t>(load, store, nullptr, R, w.scan_sums, n_isect, s);
    src.start = w.tile_start;
    src.cnt = w.tile_cnt;
  }
  const bool scan_in_scatter = shared_path && !presort;
  if (capacity == 0) {
    if (scan_in_scatter) {  // the pair count still comes from the totals
      const int32_t* cnt = w.tile_cnt;
      int64_t* start = w.tile_start;
      auto load = [=] __device__(int64_t r) -> int64_t { return cnt[r]; };
      auto store = [=] __device__(int64_t r, int64_t pre, int64_t) { start[r] = pre; };
      exclusive_scan<int64_t>(load, store, nullptr, R, w.scan_sums, n_isect, s);
    }
    cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)R, s);
    return check_launch();
  }
  if (shared_path) {
    k_hist_scatter<<<G, kHistThreads, smem, s>>>(xy, proj->radius, proj->depth, order, n_vis, n, geo, tile_rank,
                                                 w.table, presort ? nullptr : w.tile_start,
                                                 scan_in_scatter ? w.tile_cnt : nullptr, n_isect, w.keys, capacity);
  } else {
    k_scatter_pairs<<<(int)((n + 255) / 256), 256, 0, s>>>(xy, proj->radius, proj->depth, n, geo, tile_rank,
                                                           w.tile_start, w.tile_fill, w.keys, capacity);
  }
  if (keys) k_inv_rank<<<(T + 255) / 256, 256, 0, s>>>(tile_rank, T, w.inv_rank, R);
  if (presort)
    k_seg_sort<<<R, kSegThreads, 0, s>>>(w.keys, src, w.inv_rank, capacity, vals, keys,
                                         reinterpret_cast<int2*>(tile_ranges));
  else
    k_tile_sort<<<R, kSortThreads, 0, s>>>(w.keys, src, w.inv_rank, capacity, vals, keys,
                                           reinterpret_cast<int2*>(tile_ranges));
  return check_launch();
}
