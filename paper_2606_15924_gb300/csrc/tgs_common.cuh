// Shared device helpers of the TurboGS GB300 library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>

#include "turbogs.h"

#define TGS_TILE 16
#define TGS_TILE_PIX 256

namespace tgs {

// Records the CUDA error of the calling thread's last failed call.
void set_cuda_error(cudaError_t e);
// Streaming multiprocessors of the current device (cached per device; 1 on error).
int device_sm_count();

// Returns TGS_ERR_CUDA (and records the error) when the last launch failed.
inline tgs_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TGS_ERR_CUDA;
  }
  return TGS_OK;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
inline bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

// ---------------------------------------------------------------------------
// Geometric fields of Gaussian i (means, log-scales, quats, opacity logits)
// in either layout of tgs_gaussians::geo_stride: four packed arrays (stride
// 0: 3, 3, 4 and 1 floats per Gaussian) or views into one array of rows of
// geo_stride floats.
// ---------------------------------------------------------------------------
inline bool geo_stride_ok(int32_t s) { return s == 0 || (s >= 12 && s % 4 == 0); }

struct GeoC {  // read-only view
  const float* m;
  const float* l;
  const float4* q;
  const float* o;
  int s3, s4, s1;  // strides: means / log-scales (floats), quats (float4s), opacity (floats)
  __device__ __forceinline__ float3 mean(int64_t i) const {
    const float* p = m + i * s3;
    return make_float3(p[0], p[1], p[2]);
  }
  __device__ __forceinline__ float3 lsc(int64_t i) const {
    const float* p = l + i * s3;
    return make_float3(p[0], p[1], p[2]);
  }
  __device__ __forceinline__ float4 quat(int64_t i) const { return q[i * s4]; }
  __device__ __forceinline__ float opac(int64_t i) const { return o[i * s1]; }
};

struct GeoW {  // writable view
  float* m;
  float* l;
  float4* q;
  float* o;
  int s3, s4, s1;
  __device__ __forceinline__ float* mean(int64_t i) const { return m + i * s3; }
  __device__ __forceinline__ float* lsc(int64_t i) const { return l + i * s3; }
  __device__ __forceinline__ float4* quat(int64_t i) const { return q + i * s4; }
  __device__ __forceinline__ float* opac(int64_t i) const { return o + i * s1; }
};

__host__ __device__ inline GeoC geo_of(const tgs_gaussians& g) {
  const int s = g.geo_stride;
  return GeoC{g.means, g.log_scales, reinterpret_cast<const float4*>(g.quats), g.opacity_logits, s ? s : 3,
              s ? s / 4 : 1, s ? s : 1};
}

__host__ __device__ inline GeoW geo_of(const tgs_param_ptrs& p) {
  const int s = p.geo_stride;
  return GeoW{p.means, p.log_scales, reinterpret_cast<float4*>(p.quats), p.opacity_logits, s ? s : 3,
              s ? s / 4 : 1, s ? s : 1};
}

__host__ __device__ inline GeoC geo_const(const GeoW& w) { return GeoC{w.m, w.l, w.q, w.o, w.s3, w.s4, w.s1}; }

// Pointers, alignment and stride of a parameter set (quats and sh 16-byte
// aligned, the rest 4-byte aligned).
inline bool param_ptrs_ok(const tgs_param_ptrs* p) {
  return p && p->means && p->log_scales && p->quats && p->opacity_logits && p->sh && aligned4(p->means) &&
         aligned4(p->log_scales) && aligned16(p->quats) && aligned4(p->opacity_logits) && aligned16(p->sh) &&
         geo_stride_ok(p->geo_stride);
}

inline int tiles_x(int w) { return (w + TGS_TILE - 1) / TGS_TILE; }
inline int tiles_y(int h) { return (h + TGS_TILE - 1) / TGS_TILE; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves aligned sub-buffers out of a caller-provided workspace.
struct Carver {
  char* base;
  size_t off;
  explicit Carver(void* b) : base(static_cast<char*>(b)), off(0) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return align_up(off, 256); }
};

// ---------------------------------------------------------------------------
// tile rectangle: tiles [lo, hi) along one axis covered by [c - r, c + r]
// (tile k covers [16k, 16k + 16)), decided in single precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_span(float c, int r, int ntiles, int& lo, int& hi) {
  float rf = (float)r;
  float a = floorf(__fmul_rn(__fsub_rn(c, rf), 0.0625f));
  float b = __fadd_rn(floorf(__fmul_rn(__fadd_rn(c, rf), 0.0625f)), 1.0f);
  a = fminf(fmaxf(a, 0.0f), (float)ntiles);
  b = fminf(fmaxf(b, 0.0f), (float)ntiles);
  lo = (int)a;
  hi = (int)b;
}

// ---------------------------------------------------------------------------
// counter-based random stream (SplitMix64 output function)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum : uint32_t { STREAM_TILE_HARD = 1, STREAM_TILE_UNIF = 2, STREAM_PIX_HARD = 3, STREAM_PIX_UNIF = 4 };

// Hash of (seed, iteration, view, stream, tile, item); the first three
// rounds depend only on the call, so kernels pass them in precomputed.
__host__ __device__ inline uint64_t hash_prefix(uint64_t seed, uint64_t iter, uint32_t view, uint32_t stream) {
  auto mix = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  uint64_t h = mix(seed + 0x9E3779B97F4A7C15ull);
  h = mix(h ^ iter);
  h = mix(h ^ (((uint64_t)view << 8) | stream));
  return h;
}
__device__ __forceinline__ uint64_t hash_item(uint64_t prefix, uint32_t tile, uint32_t item) {
  return splitmix_mix(prefix ^ (((uint64_t)tile << 16) | item));
}

// -log2(U) of U = (h | 1) / 2^64 with 32 fractional bits: normalise the
// mantissa to [1, 2) and read one bit per squaring (integer only).
__device__ __forceinline__ uint64_t neglog2_q32(uint64_t h) {
  uint64_t u = h | 1ull;
  int lz = __clzll(u);
  uint64_t m = u << lz;
  uint64_t frac = 0;
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    uint64_t hi = __umul64hi(m, m);
    uint64_t bit = hi >> 63;
    frac = (frac << 1) | bit;
    m = bit ? hi : (hi << 1);
  }
  return ((uint64_t)(lz + 1) << 32) - frac;   // (64 - (63 - lz)) << 32
}

// fp16 error value -> exact integer E * 2^24 (0 for negative, NaN, inf).
__device__ __forceinline__ uint64_t err_weight(uint16_t h) {
  if (h & 0x8000u) return 0;
  uint32_t e = (h >> 10) & 31u, m = h & 1023u;
  if (e == 31u) return 0;
  if (e == 0u) return m;
  return (uint64_t)(1024u + m) << (e - 1u);
}

// a < b for 128-bit products a1*a2 vs b1*b2 (unsigned)
__device__ __forceinline__ bool mul128_less(uint64_t a1, uint64_t a2, uint64_t b1, uint64_t b2) {
  uint64_t ah = __umul64hi(a1, a2), al = a1 * a2;
  uint64_t bh = __umul64hi(b1, b2), bl = b1 * b2;
  return ah < bh || (ah == bh && al < bl);
}

// split of n draws into hard / stable / rest (ratios in 1/1000)
__host__ __device__ inline void split_counts(int n, int hard_pm, int stable_pm, int& kh, int& ks) {
  int h = (hard_pm * n + 500) / 1000;
  if (h > n) h = n;
  int s = (stable_pm * n + 500) / 1000;
  if (s > n - h) s = n - h;
  kh = h;
  ks = s;
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 16-byte load through the read-only path as a volatile asm statement, so
// that a run of them is issued in program order, ahead of the arithmetic that
// uses them (the compiler otherwise sinks each load to its first use).
__device__ __forceinline__ float4 ldg_f4_now(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// vector atomic add of 4 floats (sm_90+ red.global.add.v4.f32)
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Position of this thread's entry in a list appended to by every block, with
// one atomic on the length counter per block (a counter hit once per warp by
// thousands of warps serialises in L2).  Entries of a block keep thread
// order.  Every thread of the block calls it, once per kernel; blockDim.x is
// a multiple of 32.  The result is meaningful only where on is true.
__device__ __forceinline__ int64_t block_append(bool on, int32_t* count) {
  __shared__ int s_off[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, on);
  if (lane == 0) s_off[w] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int k = 0; k < nw; ++k) {
      const int c = s_off[k];
      s_off[k] = tot;
      tot += c;
    }
    s_off[32] = tot ? atomicAdd(count, tot) : 0;
  }
  __syncthreads();
  return (int64_t)s_off[32] + s_off[w] + __popc(b & ((1u << lane) - 1u));
}

}  // namespace tgs
