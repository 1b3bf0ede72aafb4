// Device-wide exclusive prefix sum in three launches (reduce, scan of block
// sums, downsweep), or one for up to SCAN_CHUNK elements.  The element count may live on the device; grids are
// sized from a host-side upper bound so the sequence can be graph-captured.
#pragma once
#include "tgs_common.cuh"

namespace tgs {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_tot[lane] = s;
  }
  __syncthreads();
  T off = w > 0 ? warp_tot[w - 1] : T(0);
  total = warp_tot[nw - 1];
  __syncthreads();
  return off + x - v;
}

// Count source: n_dev (device, nullable) else n_host.
__device__ __forceinline__ int64_t load_count(const int64_t* n_dev, int64_t n_host) {
  return n_dev ? min(*n_dev, n_host) : n_host;
}

template <typename T, typename Load>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(Load load, const int64_t* n_dev, int64_t n_host,
                                                              T* block_sums) {
  __shared__ T wt[32];
  const int64_t n = load_count(n_dev, n_host);
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  T s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) s += load(base + k);
  T total;
  block_exclusive_scan<T>(s, wt, total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of nb block sums in place; *total_out = sum.
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_block_sums(T* block_sums, int nb, T* total_out) {
  __shared__ T wt[32];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  T s = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) s += block_sums[b0 + k];
  T total;
  T run = block_exclusive_scan<T>(s, wt, total);
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) {
      T v = block_sums[b0 + k];
      block_sums[b0 + k] = run;
      run += v;
    }
  if (threadIdx.x == 0 && total_out) *total_out = total;
}

template <typename T, typename Load, typename Store>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(Load load, Store store, const int64_t* n_dev,
                                                            int64_t n_host, const T* block_sums) {
  __shared__ T wt[32];
  const int64_t n = load_count(n_dev, n_host);
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? load(base + k) : T(0);
    s += v[k];
  }
  T total;
  T run = block_exclusive_scan<T>(s, wt, total) + block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) {
      store(base + k, run, v[k]);
      run += v[k];
    }
}

// Up to SCAN_CHUNK elements: the whole scan in one block and one launch.
template <typename T, typename Load, typename Store>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_single(Load load, Store store, const int64_t* n_dev,
                                                              int64_t n_host, T* total_out) {
  __shared__ T wt[32];
  const int64_t n = load_count(n_dev, n_host);
  const int64_t base = (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? load(base + k) : T(0);
    s += v[k];
  }
  T total;
  T run = block_exclusive_scan<T>(s, wt, total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) {
      store(base + k, run, v[k]);
      run += v[k];
    }
  if (threadIdx.x == 0 && total_out) *total_out = total;
}

inline int scan_blocks(int64_t n_host) { return (int)((n_host + SCAN_CHUNK - 1) / SCAN_CHUNK); }

// Exclusive scan: store(i, prefix_i, value_i) for i < n; *total_out = sum.
// block_sums needs scan_blocks(n_host) elements.
template <typename T, typename Load, typename Store>
void exclusive_scan(Load load, Store store, const int64_t* n_dev, int64_t n_host, T* block_sums, T* total_out,
                    cudaStream_t s) {
  int nb = scan_blocks(n_host);
  if (nb <= 1) {
    k_scan_single<T, Load, Store><<<1, SCAN_THREADS, 0, s>>>(load, store, n_dev, n_host, total_out);
    return;
  }
  k_scan_reduce<T, Load><<<nb, SCAN_THREADS, 0, s>>>(load, n_dev, n_host, block_sums);
  k_scan_block_sums<T><<<1, 1024, 0, s>>>(block_sums, nb, total_out);
  k_scan_down<T, Load, Store><<<nb, SCAN_THREADS, 0, s>>>(load, store, n_dev, n_host, block_sums);
}

}  // namespace tgs
