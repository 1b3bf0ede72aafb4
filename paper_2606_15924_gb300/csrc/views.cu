// Geometry-aware view sampling (Sec. 3.4, Eqs. 5-6; Alg. 1 step 2).
//
// Two calls: the per-view error totals (an HBM-bound pass over every view's
// fp16 error map, summed exactly in integers), and the draw itself (one
// block: anchor by largest total, then K - 1 views by the Efraimidis-Spirakis
// order of the geometric weights, with the same counter-based hash and
// integer logarithm recurrence as the tile draw).
#include "block_select.cuh"

namespace tgs {

constexpr uint32_t kStreamView = 5;  // hash stream of the view draw
constexpr int kSumThreads = 256;
constexpr int kSumVec = 4;           // 16-byte loads in flight per thread
constexpr int kViewThreads = 1024;

// E * 2^24 of an fp16 value h with sign-and-exponent field s = h >> 10 is
// ((h & 1023) | imp[s]) * mul[s]: a normal value (1024 + m) 2^(e - 25) counts
// (1024 + m) << (e - 1), a subnormal m, and negative, infinite or NaN
// values nothing (mul = 0).  tab[s] = (mul, imp).
__device__ __forceinline__ uint2 half_units_entry(uint32_t s) {
  if (s == 0u) return make_uint2(1u, 0u);
  if (s < 31u) return make_uint2(1u << (s - 1u), 1024u);
  return make_uint2(0u, 0u);
}

// Adds E * 2^24 of the two fp16 values packed in x (one table lookup and
// one widening multiply-add each).
__device__ __forceinline__ uint64_t pair_units(uint32_t x, const uint2* tab, uint64_t acc) {
  const uint2 lo = tab[(x >> 10) & 63u];
  const uint2 hi = tab[x >> 26];
  acc += (uint64_t)((x & 0x3FFu) | lo.y) * lo.x;
  acc += (uint64_t)(((x >> 16) & 0x3FFu) | hi.y) * hi.x;
  return acc;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block-wide total added to sums[v] (one atomic per block).
__device__ __forceinline__ void block_add_u64(uint64_t acc, unsigned long long* dst) {
  __shared__ uint64_t s[kSumThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  acc = warp_sum_u64(acc);
  if (lane == 0) s[w] = acc;
  __syncthreads();
  if (w == 0) {
    acc = lane < kSumThreads / 32 ? s[lane] : 0;
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(dst, (unsigned long long)acc);
  }
}

// blockIdx.y = view; the view's n16 16-byte words are strided over the
// blocks of its row of the grid, kSumVec loads in flight per thread.
__global__ void __launch_bounds__(kSumThreads) k_view_error_sums_v16(const uint4* __restrict__ maps,
                                                                   int64_t stride16, int64_t n16,
                                                                   unsigned long long* __restrict__ sums) {
  __shared__ uint2 tab[64];
  if (threadIdx.x < 64) tab[threadIdx.x] = half_units_entry(threadIdx.x);
  __syncthreads();
  const uint4* m = maps + (int64_t)blockIdx.y * stride16;
  const int64_t step = (int64_t)gridDim.x * kSumThreads;
  int64_t i = (int64_t)blockIdx.x * kSumThreads + threadIdx.x;
  uint64_t acc = 0;
  for (; i + (kSumVec - 1) * step < n16; i += kSumVec * step) {
    uint4 q[kSumVec];
#pragma unroll
    for (int u = 0; u < kSumVec; ++u) q[u] = __ldcs(m + i + u * step);
#pragma unroll
    for (int u = 0; u < kSumVec; ++u) {
      acc = pair_units(q[u].x, tab, acc);
      acc = pair_units(q[u].y, tab, acc);
      acc = pair_units(q[u].z, tab, acc);
      acc = pair_units(q[u].w, tab, acc);
    }
  }
  for (; i < n16; i += step) {
    const uint4 q = __ldcs(m + i);
    acc = pair_units(q.x, tab, acc);
    acc = pair_units(q.y, tab, acc);
    acc = pair_units(q.z, tab, acc);
    acc = pair_units(q.w, tab, acc);
  }
  block_add_u64(acc, sums + blockIdx.y);
}

// Any alignment: one fp16 value per thread and step.
__global__ void __launch_bounds__(kSumThreads) k_view_error_sums_h(const uint16_t* __restrict__ maps, int64_t stride,
                                                                 int64_t n, unsigned long long* __restrict__ sums) {
  const uint16_t* m = maps + (int64_t)blockIdx.y * stride;
  const int64_t step = (int64_t)gridDim.x * kSumThreads;
  uint64_t acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * kSumThreads + threadIdx.x; i < n; i += step) acc += err_weight(m[i]);
  block_add_u64(acc, sums + blockIdx.y);
}

// log2(x) * 2^32 for x >= 1 (integer part: the leading bit; fraction: one
// bit per squaring of the normalised mantissa, the recurrence of neglog2_q32).
__device__ __forceinline__ uint64_t log2_q32(uint64_t x) {
  const int lz = __clzll(x);
  uint64_t m = x << lz;
  uint64_t frac = 0;
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    const uint64_t hi = __umul64hi(m, m);
    const uint64_t bit = hi >> 63;
    frac = (frac << 1) | bit;
    m = bit ? hi : (hi << 1);
  }
  return ((uint64_t)(63 - lz) << 32) | frac;
}

// Camera centre -R^T t and unit forward axis (third row of R) of a
// row-major world-to-camera matrix, in double with every rounding explicit.
__device__ __forceinline__ void view_pose(const tgs_camera& cam, double c[3], double d[3]) {
  const float* M = cam.viewmat;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double s = __dadd_rn(__dadd_rn(__dmul_rn((double)M[j], (double)M[3]), __dmul_rn((double)M[4 + j], (double)M[7])),
                               __dmul_rn((double)M[8 + j], (double)M[11]));
    c[j] = -s;
  }
  const double f0 = M[8], f1 = M[9], f2 = M[10];
  const double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(f0, f0), __dmul_rn(f1, f1)), __dmul_rn(f2, f2)));
  d[0] = __ddiv_rn(f0, n);
  d[1] = __ddiv_rn(f1, n);
  d[2] = __ddiv_rn(f2, n);
}

// Total order of doubles as unsigned integers (finite keys).
__device__ __forceinline__ uint64_t ordered_bits(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// (eligible, sum, index) ordering of the anchor: eligible first, then the
// larger sum, then the lower index.
__device__ __forceinline__ bool anchor_better(bool ea, uint64_t sa, int ia, bool eb, uint64_t sb, int ib) {
  if (ea != eb) return ea;
  if (sa != sb) return sa > sb;
  return ia < ib;
}

template <int ITEMS>
__global__ void __launch_bounds__(kViewThreads) k_sample_views(const uint64_t* __restrict__ err_sums,
                                                              const tgs_camera* __restrict__ cams, int V, int K,
                                                              double lambda_d, double lambda_theta, uint64_t prefix,
                                                              uint8_t* __restrict__ stack,
                                                              int32_t* __restrict__ views) {
  __shared__ RadixSelSmem sm;
  __shared__ int64_t s64[32];
  __shared__ int s_cnt[32];
  __shared__ uint64_t s_bs[32];
  __shared__ int s_bi[32], s_be[32];
  __shared__ int s_anchor;
  __shared__ double s_pose[6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  bool on[ITEMS];
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int v = threadIdx.x * ITEMS + j;
    on[j] = v < V && stack[v] != 0;
    cnt += on[j];
  }
  // 1. refill when fewer than K views remain on the stack
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) s_cnt[w] = cnt;
  __syncthreads();
  const int on_stack = __reduce_add_sync(0xffffffffu, lane < nw ? s_cnt[lane] : 0);
  if (on_stack < K) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) on[j] = threadIdx.x * ITEMS + j < V;
  }
  // 2. anchor: the stack view with the largest error total (Eq. 5)
  bool be = false;
  uint64_t bs = 0;
  int bi = 0x7fffffff;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int v = threadIdx.x * ITEMS + j;
    const uint64_t s = on[j] ? err_sums[v] : 0;
    if (anchor_better(on[j], s, v, be, bs, bi)) {
      be = on[j];
      bs = s;
      bi = v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const bool oe = __shfl_xor_sync(0xffffffffu, (int)be, o);
    const uint64_t os = __shfl_xor_sync(0xffffffffu, bs, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (anchor_better(oe, os, oi, be, bs, bi)) {
      be = oe;
      bs = os;
      bi = oi;
    }
  }
  if (lane == 0) {
    s_be[w] = be;
    s_bs[w] = bs;
    s_bi[w] = bi;
  }
  __syncthreads();
  if (w == 0) {
    be = lane < nw ? s_be[lane] : 0;
    bs = lane < nw ? s_bs[lane] : 0;
    bi = lane < nw ? s_bi[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const bool oe = __shfl_xor_sync(0xffffffffu, (int)be, o);
      const uint64_t os = __shfl_xor_sync(0xffffffffu, bs, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (anchor_better(oe, os, oi, be, bs, bi)) {
        be = oe;
        bs = os;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_anchor = bi;
      double c[3], d[3];
      view_pose(cams[bi], c, d);
      for (int q = 0; q < 3; ++q) {
        s_pose[q] = c[q];
        s_pose[3 + q] = d[q];
      }
    }
  }
  __syncthreads();
  const int anchor = s_anchor;
  // 3. Efraimidis-Spirakis keys of the geometric weights (Eq. 6)
  uint64_t key[ITEMS];
  bool elig[ITEMS], taken[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int v = threadIdx.x * ITEMS + j;
    elig[j] = on[j] && v != anchor;
    key[j] = 0;
    if (elig[j]) {
      double c[3], d[3];
      view_pose(cams[v], c, d);
      const double dx = __dsub_rn(c[0], s_pose[0]), dy = __dsub_rn(c[1], s_pose[1]), dz = __dsub_rn(c[2], s_pose[2]);
      const double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
      const double cosv = __dadd_rn(__dadd_rn(__dmul_rn(d[0], s_pose[3]), __dmul_rn(d[1], s_pose[4])),
                                    __dmul_rn(d[2], s_pose[5]));
      const double s = __dadd_rn(__dmul_rn(lambda_d, dist), __dmul_rn(lambda_theta, __dsub_rn(1.0, cosv)));
      // log2 of the exponential clock -log2 U (a Q32 value, >= 2^-32)
      const uint64_t L = neglog2_q32(hash_item(prefix, (uint32_t)v, 0));
      const double lg = __dmul_rn((double)(int64_t)(log2_q32(L) - (32ull << 32)), 2.3283064365386963e-10);
      // + 0.0 turns a -0 into +0, so that the bit order is the numeric order
      key[j] = ordered_bits(__dadd_rn(__dadd_rn(lg, __dmul_rn(s, 1.4426950408889634)), 0.0));
    }
  }
  block_radix_select<ITEMS>(key, elig, K - 1, 64, taken, sm, s64, 0);
  // 4. outputs: anchor first, then the draws ascending; the K views leave the stack
  int mine = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) mine += taken[j];
  int64_t total;
  int off = 1 + (int)block_excl_sum(mine, s64, total);
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int v = threadIdx.x * ITEMS + j;
    if (taken[j]) views[off++] = v;
    if (v < V) stack[v] = (uint8_t)(on[j] && !taken[j] && v != anchor);
  }
  if (threadIdx.x == 0) views[0] = anchor;
}

}  // namespace tgs

using namespace tgs;

extern "C" tgs_status tgs_view_error_sums(const uint16_t* err_maps, int32_t n_views, int64_t view_stride,
                                          int32_t width, int32_t height, uint64_t* sums, tgs_stream stream) {
  if (!err_maps || !sums || n_views < 1 || n_views > 65535 || width < 1 || height < 1) return TGS_ERR_INVALID_ARG;
  const int64_t n = (int64_t)width * height;
  if (n > TGS_VIEW_MAX_PIXELS || view_stride < n || !aligned8(sums)) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(sums, 0, sizeof(uint64_t) * (size_t)n_views, s) != cudaSuccess) return check_launch();
  const bool vec = aligned16(err_maps) && (view_stride % 8) == 0 && (n % 8) == 0;
  const int64_t units = vec ? n / 8 : n;
  // about kSumVec * 8 loads per thread (a few waves of blocks over the SMs
  // for the full-size maps), at least one block per view
  const int64_t per_block = (int64_t)kSumThreads * (vec ? kSumVec * 8 : 16);
  const int nbx = (int)std::min<int64_t>(std::max<int64_t>((units + per_block - 1) / per_block, 1), 65535);
  const dim3 grid(nbx, n_views);
  if (vec)
    k_view_error_sums_v16<<<grid, kSumThreads, 0, s>>>(reinterpret_cast<const uint4*>(err_maps), view_stride / 8,
                                                       units, reinterpret_cast<unsigned long long*>(sums));
  else
    k_view_error_sums_h<<<grid, kSumThreads, 0, s>>>(err_maps, view_stride, n,
                                                     reinterpret_cast<unsigned long long*>(sums));
  return check_launch();
}

extern "C" tgs_status tgs_sample_views(const uint64_t* err_sums, const tgs_camera* cams, int32_t n_views, int32_t k,
                                       double lambda_d, double lambda_theta, uint64_t seed, uint64_t iter,
                                       uint8_t* stack, int32_t* views, tgs_stream stream) {
  if (!err_sums || !cams || !stack || !views || n_views < 1 || n_views > TGS_VIEW_SAMPLE_MAX_VIEWS || k < 1 ||
      k > n_views)
    return TGS_ERR_INVALID_ARG;
  // finite and non-negative (NaN fails both comparisons)
  if (!(lambda_d >= 0.0 && lambda_d <= 1e300) || !(lambda_theta >= 0.0 && lambda_theta <= 1e300))
    return TGS_ERR_INVALID_ARG;
  const uint64_t prefix = hash_prefix(seed, iter, 0, kStreamView);
  cudaStream_t s = (cudaStream_t)stream;
  if (n_views <= kViewThreads)
    k_sample_views<1><<<1, kViewThreads, 0, s>>>(err_sums, cams, n_views, k, lambda_d, lambda_theta, prefix, stack,
                                                 views);
  else if (n_views <= 2 * kViewThreads)
    k_sample_views<2><<<1, kViewThreads, 0, s>>>(err_sums, cams, n_views, k, lambda_d, lambda_theta, prefix, stack,
                                                 views);
  else if (n_views <= 4 * kViewThreads)
    k_sample_views<4><<<1, kViewThreads, 0, s>>>(err_sums, cams, n_views, k, lambda_d, lambda_theta, prefix, stack,
                                                 views);
  else
    k_sample_views<8><<<1, kViewThreads, 0, s>>>(err_sums, cams, n_views, k, lambda_d, lambda_theta, prefix, stack,
                                                 views);
  return check_launch();
}
