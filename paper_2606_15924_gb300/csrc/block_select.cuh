// Block-wide exact k-selection shared by the tile selection (Sec. 3.5) and
// the view sampling (Sec. 3.4).
#pragma once
#include "tgs_common.cuh"

namespace tgs {

// Exact block-wide k-selection by radix select: the k smallest (key, index)
// pairs among the eligible items of the block, keys < 2^nbits, items held
// ITEMS per thread in index order (thread t holds t * ITEMS + j).  The k-th
// smallest key K is found one 8-bit digit at a time from the top: a pass
// first takes the block-wide minimum and maximum of the digit over the keys
// that match the digits found so far (one digit: nothing to count), else
// counts them in a shared histogram, and every warp then locates the digit
// where the running count reaches k by itself (no second barrier).  Once the
// chosen bin holds exactly the keys still wanted, those are taken and the
// lower digits are never looked at; otherwise every key below K is taken, and
// the ties at K in index order until k are reached.  Every thread of the
// block must call it (it synchronises); k is the same on all threads.
// Buffers that a pass writes before a barrier and reads after it alternate
// between two copies, so that the next pass never overwrites what a slower
// warp still reads.
struct RadixSelSmem {
  uint32_t hist[2][256];
  uint32_t wmin[2][32], wmax[2][32];
  int32_t wcnt[2][32];
};

// Exclusive prefix over threads of v (thread order); total receives the sum.
__device__ __forceinline__ int64_t block_excl_sum(int64_t v, int64_t* s64, int64_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s64[w] = x;
  __syncthreads();
  int64_t t = lane < nw ? s64[lane] : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
    if (lane >= o) t += y;
  }
  const int64_t upto = __shfl_sync(0xffffffffu, t, w > 0 ? w - 1 : 0);  // warps 0 .. w - 1
  total = __shfl_sync(0xffffffffu, t, nw - 1);
  __syncthreads();
  return (w > 0 ? upto : 0) + x - v;
}

// call: 0, 1, 2 ... for consecutive selections of one kernel (buffer parity).
template <int ITEMS>
__device__ void block_radix_select(const uint64_t (&key)[ITEMS], const bool (&elig)[ITEMS], int k, int nbits,
                                   bool (&taken)[ITEMS], RadixSelSmem& sm, int64_t* s64, int call) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) taken[j] = false;
  if (k <= 0) return;
  int mine = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) mine += elig[j];
  mine = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) sm.wcnt[call & 1][w] = mine;
  __syncthreads();
  const int n_elig = __reduce_add_sync(0xffffffffu, lane < nw ? sm.wcnt[call & 1][lane] : 0);
  if (k >= n_elig) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) taken[j] = elig[j];
    return;
  }
  uint64_t prefix = 0, mask = 0;
  int kk = k;  // rank (from 1) of the sought key among the keys matching the prefix
  int hp = 0;  // histogram passes so far (buffer parity)
  for (int shift = ((nbits + 7) / 8) * 8 - 8; shift >= 0; shift -= 8) {
    const int par = (shift >> 3) & 1;
    uint32_t dmin = 255u, dmax = 0u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j)
      if (elig[j] && (key[j] & mask) == prefix) {
        const uint32_t d = (uint32_t)((key[j] >> shift) & 255u);
        dmin = min(dmin, d);
        dmax = max(dmax, d);
      }
    dmin = __reduce_min_sync(0xffffffffu, dmin);
    dmax = __reduce_max_sync(0xffffffffu, dmax);
    if (lane == 0) {
      sm.wmin[par][w] = dmin;
      sm.wmax[par][w] = dmax;
    }
    uint32_t* h = sm.hist[hp & 1];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const uint32_t lo = __reduce_min_sync(0xffffffffu, lane < nw ? sm.wmin[par][lane] : 255u);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, lane < nw ? sm.wmax[par][lane] : 0u);
    if (lo == hi) {  // one digit: every key in play has it
      prefix |= (uint64_t)lo << shift;
      mask |= 255ull << shift;
      continue;
    }
    const uint32_t span = hi - lo + 1u;
    if (span <= 32u) {
      // few distinct digits (exponent bits, small ages): counted per warp by
      // ballots, lane q holding digit lo + q, then one atomic per warp and
      // digit (shared atomics on a few hot bins would serialise)
      uint32_t cnt = 0;
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const uint32_t d = elig[j] && (key[j] & mask) == prefix ? (uint32_t)((key[j] >> shift) & 255u) - lo : 32u;
        for (uint32_t q = 0; q < span; ++q) {
          const uint32_t b = __ballot_sync(0xffffffffu, d == q);
          if ((uint32_t)lane == q) cnt += __popc(b);
        }
      }
      if (cnt) atomicAdd(&h[lo + lane], cnt);
    } else {
#pragma unroll
      for (int j = 0; j < ITEMS; ++j)
        if (elig[j] && (key[j] & mask) == prefix) atomicAdd(&h[(key[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    ++hp;
    // every warp: the digit where the running count reaches kk
    uint32_t c[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      c[q] = h[lane * 8 + q];
      sum += c[q];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - sum;
    const unsigned at = __ballot_sync(0xffffffffu, excl < (uint32_t)kk && (uint32_t)kk <= incl);
    const int src = __ffs(at) - 1;  // exactly one lane: 1 <= kk <= keys in play
    int digit = 0, below = 0, count = 0;
    if (lane == src) {
      uint32_t run = excl;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (run + c[q] >= (uint32_t)kk) {
          digit = lane * 8 + q;
          below = (int)run;
          count = (int)c[q];
          break;
        }
        run += c[q];
      }
    }
    digit = __shfl_sync(0xffffffffu, digit, src);
    below = __shfl_sync(0xffffffffu, below, src);
    count = __shfl_sync(0xffffffffu, count, src);
    prefix |= (uint64_t)digit << shift;
    mask |= 255ull << shift;
    kk -= below;
    if (kk == count) {
      // every key matching the prefix is taken, so the digits below decide
      // nothing: the k smallest are the keys whose leading digits are at most
      // the prefix
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) taken[j] = elig[j] && (key[j] & mask) <= prefix;
      return;
    }
  }
  // every key below K = prefix is taken; of the keys equal to K, the first kk
  int ties = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) ties += elig[j] && key[j] == prefix;
  int64_t all_ties;
  int before = (int)block_excl_sum(ties, s64, all_ties);
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const bool tie = elig[j] && key[j] == prefix;
    taken[j] = elig[j] && (key[j] < prefix || (tie && before < kk));
    before += tie;
  }
}

}  // namespace tgs
