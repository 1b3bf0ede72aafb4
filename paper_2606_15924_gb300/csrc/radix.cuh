// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits,
// three launches per digit: per-block digit histograms, a scan of each digit's
// row of block counts, and a stable scatter.  The pair count may live on the
// device (grids are sized from the host bound).
#pragma once
#include "tgs_common.cuh"

namespace tgs {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 4;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // pairs per block
constexpr int RS_BINS = 256;

inline int rs_blocks(int64_t n_host) { return (int)((n_host + RS_TILE - 1) / RS_TILE); }

__device__ __forceinline__ int rs_count(const int32_t* n_dev, int32_t n_host) {
  return n_dev ? min(*n_dev, n_host) : n_host;
}

// hist[digit * nb + block] = count of that digit in the block's pairs
static __global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const uint32_t* __restrict__ keys, const int32_t* n_dev,
                                                           int32_t n_host, int shift, uint32_t* __restrict__ hist,
                                                           int nb) {
  __shared__ uint32_t h[RS_WARPS][RS_BINS];
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&h[0][0])[i] = 0;
  __syncthreads();
  const int n = rs_count(n_dev, n_host);
  const int base = blockIdx.x * RS_TILE;
  if (base < n) {
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
      int idx = base + r * RS_THREADS + threadIdx.x;
      if (idx < n) atomicAdd(&h[w][(keys[idx] >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < RS_WARPS; ++k) s += h[k][threadIdx.x];
  hist[threadIdx.x * nb + blockIdx.x] = s;
}

// One block per digit: exclusive scan of the digit's nb block counts in place;
// bin_total[digit] = total.
static __global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ hist, int nb,
                                                  uint32_t* __restrict__ bin_total) {
  __shared__ uint32_t wt[32];
  uint32_t* row = hist + (size_t)blockIdx.x * nb;
  uint32_t carry = 0;
  for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
    int b = b0 + threadIdx.x;
    uint32_t v = b < nb ? row[b] : 0u;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t s = lane < nw ? wt[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < nw) wt[lane] = s;
    }
    __syncthreads();
    uint32_t off = (w > 0 ? wt[w - 1] : 0u) + x - v;
    if (b < nb) row[b] = carry + off;
    carry += wt[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) bin_total[blockIdx.x] = carry;
}

// Stable scatter.  Pairs are taken in rounds of 256 (thread t of round r
// holds pair base + 256 r + t); equal digits keep their input order through
// the running per-digit counts, the per-warp prefix and the lane rank.
static __global__ void __launch_bounds__(RS_THREADS) k_rs_downsweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const int32_t* n_dev, int32_t n_host, int shift,
    const uint32_t* __restrict__ hist, int nb, const uint32_t* __restrict__ bin_total) {
  __shared__ uint32_t wt[32];
  __shared__ uint32_t blk_off[RS_BINS];
  __shared__ uint32_t warp_cnt[RS_WARPS][RS_BINS];
  const int n = rs_count(n_dev, n_host);
  const int base = blockIdx.x * RS_TILE;
  if (base >= n) return;  // uniform across the block
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  {
    // digit bases: exclusive scan of the digit totals, plus this block's offset
    uint32_t v = bin_total[t];
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t s = lane < RS_WARPS ? wt[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < RS_WARPS) wt[lane] = s;
    }
    __syncthreads();
    blk_off[t] = (w > 0 ? wt[w - 1] : 0u) + x - v + hist[t * nb + blockIdx.x];
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
#pragma unroll
    for (int k = 0; k < RS_WARPS; ++k) warp_cnt[k][t] = 0;
    __syncthreads();
    const int idx = base + r * RS_THREADS + t;
    const bool valid = idx < n;
    const uint32_t key = valid ? keys_in[idx] : 0u;
    const uint32_t d = (key >> shift) & 255u;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
    const uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) warp_cnt[w][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = blk_off[t];
#pragma unroll
      for (int k = 0; k < RS_WARPS; ++k) {
        uint32_t c = warp_cnt[k][t];
        warp_cnt[k][t] = run;
        run += c;
      }
      blk_off[t] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = warp_cnt[w][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = vals_in[idx];
    }
    __syncthreads();
  }
}

struct RadixScratch {
  uint32_t* hist;       // [256 * nb]
  uint32_t* bin_total;  // [256]
};

inline size_t radix_hist_elems(int64_t n_host) { return (size_t)RS_BINS * (size_t)std::max(1, rs_blocks(n_host)); }

// Sorts pairs by key bits [begin_bit, end_bit).  Pass p reads (k[p%2], v[p%2])
// and writes (k[(p+1)%2], v[(p+1)%2]); last_vals (nullable) replaces the value
// destination of the final pass.  Returns the index of the buffer holding the
// sorted keys.
inline int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const int32_t* n_dev,
                            int32_t n_host, int begin_bit, int end_bit, RadixScratch sc, uint32_t* last_vals,
                            cudaStream_t s) {
  int nb = std::max(1, rs_blocks(n_host));
  uint32_t* K[2] = {k0, k1};
  uint32_t* V[2] = {v0, v1};
  int cur = 0;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    bool last = shift + 8 >= end_bit;
    uint32_t* vout = (last && last_vals) ? last_vals : V[cur ^ 1];
    k_rs_upsweep<<<nb, RS_THREADS, 0, s>>>(K[cur], n_dev, n_host, shift, sc.hist, nb);
    k_rs_scan<<<RS_BINS, 1024, 0, s>>>(sc.hist, nb, sc.bin_total);
    k_rs_downsweep<<<nb, RS_THREADS, 0, s>>>(K[cur], V[cur], K[cur ^ 1], vout, n_dev, n_host, shift, sc.hist, nb,
                                             sc.bin_total);
    cur ^= 1;
  }
  return cur;
}

}  // namespace tgs
