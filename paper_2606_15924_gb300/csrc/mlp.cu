// Tile-error predictor: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with
// x in R^16 (per-tile features, zero padded), 128 hidden units, bf16 weights
// and activations, fp32 accumulation.  The dense layers run on the tensor
// cores (mma m16n8k16, bf16 in, fp32 accumulate): one warp takes 16 rows, and
// the fp32 accumulator fragments of one layer, rounded to bf16, are exactly
// the A-operand fragments of the next (two n8 tiles = one k16 chunk), so
// activations never leave registers.  The backward computes the input
// adjoint of layer 2 on the tensor cores too; the weight gradients (a
// reduction over rows, small) on the CUDA cores.
#include <cuda_bf16.h>

#include "tgs_common.cuh"

namespace tgs {

constexpr int MI = 16, MH = 128;
// packed fp32 parameter vector: W1 [128,16] | b1 | W2 [128,128] | b2 | W3 [128] | b3
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MH * MI, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH,
              OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MH, N_PARAMS = OFF_B3 + 1;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// D = A (16x16, row) * B (16x8, col) + C, bf16 inputs, fp32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct MlpK {
  const uint16_t *w1, *w2, *w3;
  const float *b1, *b2, *b3;
};

// Weights staged in shared memory (bf16 bits): W1 [128][16], W2 [128][128]
// (plus W2^T for the backward), W3 [128]; biases fp32.
// Rows are padded (W1: 24, W2: 136 halves) so that the B-fragment loads of a
// warp hit 32 different banks.
constexpr int S1 = 24, S2 = 136;

struct MlpSmem {
  uint16_t w1[MH * S1];
  uint16_t w2[MH * S2];
  uint16_t w3[MH];
  float b1[MH], b2[MH], b3;
};

__device__ void load_weights(const MlpK& w, MlpSmem& s) {
  for (int i = threadIdx.x; i < MH * MI; i += blockDim.x) s.w1[(i / MI) * S1 + i % MI] = w.w1[i];
  for (int i = threadIdx.x; i < MH * MH; i += blockDim.x) s.w2[(i / MH) * S2 + i % MH] = w.w2[i];
  for (int i = threadIdx.x; i < MH; i += blockDim.x) {
    s.w3[i] = w.w3[i];
    s.b1[i] = w.b1[i];
    s.b2[i] = w.b2[i];
  }
  if (threadIdx.x == 0) s.b3 = w.b3[0];
  __syncthreads();
}

// B fragment of W[n][k] (row-major, row stride S halves) for n-tile nt,
// k-chunk kc.
__device__ __forceinline__ void bfrag(const uint16_t* W, int S, int nt, int kc, int lane, uint32_t& b0,
                                      uint32_t& b1) {
  const int g = lane >> 2, t = lane & 3;
  const uint16_t* p = W + (nt * 8 + g) * S + kc * 16 + 2 * t;
  b0 = *reinterpret_cast<const uint32_t*>(p);
  b1 = *reinterpret_cast<const uint32_t*>(p + 8);
}

// Forward of one 16-row tile by one warp.  Returns the hidden activations as
// bf16 A fragments (h1a, h2a: 8 k-chunks x 4 registers) and y for rows g and
// g + 8 (valid in lanes with t == 0).
__device__ __forceinline__ void mlp_tile_forward(const MlpSmem& s, const float* __restrict__ x, int64_t row0,
                                                 int64_t R, int lane, uint32_t (&h1a)[8][4], uint32_t (&h2a)[8][4],
                                                 float& y_lo, float& y_hi) {
  const int g = lane >> 2, t = lane & 3;
  const int64_t r_lo = row0 + g, r_hi = row0 + g + 8;
  auto xv = [&](int64_t r, int c) -> float { return r < R ? x[r * MI + c] : 0.f; };
  uint32_t a[4];
  a[0] = pack_bf16(xv(r_lo, 2 * t), xv(r_lo, 2 * t + 1));
  a[1] = pack_bf16(xv(r_hi, 2 * t), xv(r_hi, 2 * t + 1));
  a[2] = pack_bf16(xv(r_lo, 2 * t + 8), xv(r_lo, 2 * t + 9));
  a[3] = pack_bf16(xv(r_hi, 2 * t + 8), xv(r_hi, 2 * t + 9));
  // layer 1
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t b0, b1;
    bfrag(s.w1, S1, nt, 0, lane, b0, b1);
    mma16816(d, a, b0, b1);
    const int c = nt * 8 + 2 * t;
    const float v0 = fmaxf(d[0] + s.b1[c], 0.f), v1 = fmaxf(d[1] + s.b1[c + 1], 0.f);
    const float v2 = fmaxf(d[2] + s.b1[c], 0.f), v3 = fmaxf(d[3] + s.b1[c + 1], 0.f);
    h1a[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(v0, v1);
    h1a[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(v2, v3);
  }
  // layer 2 (+ layer 3 partial dot products)
  float p_lo = 0.f, p_hi = 0.f;
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      uint32_t b0, b1;
      bfrag(s.w2, S2, nt, kc, lane, b0, b1);
      const uint32_t ak[4] = {h1a[kc][0], h1a[kc][1], h1a[kc][2], h1a[kc][3]};
      mma16816(d, ak, b0, b1);
    }
    const int c = nt * 8 + 2 * t;
    const uint32_t lo = pack_bf16(fmaxf(d[0] + s.b2[c], 0.f), fmaxf(d[1] + s.b2[c + 1], 0.f));
    const uint32_t hi = pack_bf16(fmaxf(d[2] + s.b2[c], 0.f), fmaxf(d[3] + s.b2[c + 1], 0.f));
    h2a[nt >> 1][(nt & 1) * 2 + 0] = lo;
    h2a[nt >> 1][(nt & 1) * 2 + 1] = hi;
    const uint32_t w3p = *reinterpret_cast<const uint32_t*>(s.w3 + c);
    const float w3a = bf16_lo(w3p), w3b = bf16_hi(w3p);
    p_lo += bf16_lo(lo) * w3a + bf16_hi(lo) * w3b;
    p_hi += bf16_lo(hi) * w3a + bf16_hi(hi) * w3b;
  }
  p_lo += __shfl_xor_sync(0xffffffffu, p_lo, 1);
  p_lo += __shfl_xor_sync(0xffffffffu, p_lo, 2);
  p_hi += __shfl_xor_sync(0xffffffffu, p_hi, 1);
  p_hi += __shfl_xor_sync(0xffffffffu, p_hi, 2);
  y_lo = p_lo + s.b3;
  y_hi = p_hi + s.b3;
}

// Stores the A fragments of a 16 x 128 activation tile as bf16 rows.
__device__ __forceinline__ void store_act(uint16_t* __restrict__ h, const uint32_t (&ha)[8][4], int64_t row0,
                                          int64_t R, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int kc = 0; kc < 8; ++kc) {
    const int c = kc * 16 + 2 * t;
    if (row0 + g < R) {
      *reinterpret_cast<uint32_t*>(h + (row0 + g) * MH + c) = ha[kc][0];
      *reinterpret_cast<uint32_t*>(h + (row0 + g) * MH + c + 8) = ha[kc][2];
    }
    if (row0 + g + 8 < R) {
      *reinterpret_cast<uint32_t*>(h + (row0 + g + 8) * MH + c) = ha[kc][1];
      *reinterpret_cast<uint32_t*>(h + (row0 + g + 8) * MH + c + 8) = ha[kc][3];
    }
  }
}

__global__ void __launch_bounds__(128) k_mlp_forward(MlpK w, const float* __restrict__ x, int64_t R,
                                                     float* __restrict__ y, uint16_t* __restrict__ h1,
                                                     uint16_t* __restrict__ h2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
  load_weights(w, s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles = (R + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t row0 = tile * 16;
    uint32_t h1a[8][4], h2a[8][4];
    float ylo, yhi;
    mlp_tile_forward(s, x, row0, R, lane, h1a, h2a, ylo, yhi);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
      if (row0 + g < R) y[row0 + g] = ylo;
      if (row0 + g + 8 < R) y[row0 + g + 8] = yhi;
    }
    if (h1) store_act(h1, h1a, row0, R, lane);
    if (h2) store_act(h2, h2a, row0, R, lane);
  }
}

// Backward, part 1 (per 16-row tile, one warp): dy = (y - t) / R;
// dh2 = [h2 > 0] dy W3 (bf16); dh1 = [h1 > 0] dh2 W2 (tensor cores, bf16);
// stores dh2 and dh1 rows (bf16) and the per-row dy for the weight gradients,
// and accumulates the loss.
__global__ void __launch_bounds__(128) k_mlp_backward_act(MlpK w, const uint16_t* __restrict__ h1,
                                                          const uint16_t* __restrict__ h2,
                                                          const float* __restrict__ y, const float* __restrict__ t,
                                                          int64_t R, const int32_t* __restrict__ R_dev,
                                                          float* __restrict__ dy_out,
                                                          uint16_t* __restrict__ dh2_out,
                                                          uint16_t* __restrict__ dh1_out, double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
  uint16_t* w2t = reinterpret_cast<uint16_t*>(smem_raw + sizeof(MlpSmem));  // W2^T [in][out], stride S2
  load_weights(w, s);
  for (int i = threadIdx.x; i < MH * MH; i += blockDim.x) {
    const int o = i / MH, k = i % MH;
    w2t[k * S2 + o] = s.w2[o * S2 + k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t tiles = (R + 15) / 16;
  // rows past Re are padding: no error, no gradient
  const int64_t Re = R_dev ? (*R_dev > 0 ? (*R_dev < R ? (int64_t)*R_dev : R) : 0) : R;
  const float inv = Re > 0 ? 1.f / (float)Re : 0.f;
  double lsum = 0.0;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t row0 = tile * 16, r_lo = row0 + g, r_hi = row0 + g + 8;
    const float e_lo = r_lo < Re ? y[r_lo] - t[r_lo] : 0.f, e_hi = r_hi < Re ? y[r_hi] - t[r_hi] : 0.f;
    if (tq == 0) lsum += 0.5 * ((double)e_lo * e_lo + (double)e_hi * e_hi) * (double)inv;
    const float dy_lo = e_lo * inv, dy_hi = e_hi * inv;
    if (tq == 0) {
      if (r_lo < R) dy_out[r_lo] = dy_lo;
      if (r_hi < R) dy_out[r_hi] = dy_hi;
    }
    // dh2 in A-fragment layout (rows g, g+8; cols kc*16 + 2t (+1), +8 (+9))
    uint32_t da[8][4];
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int c = kc * 16 + half * 8 + 2 * tq;
        const uint32_t w3p = *reinterpret_cast<const uint32_t*>(s.w3 + c);
        uint32_t hl = 0, hh = 0;
        if (r_lo < R) hl = *reinterpret_cast<const uint32_t*>(h2 + r_lo * MH + c);
        if (r_hi < R) hh = *reinterpret_cast<const uint32_t*>(h2 + r_hi * MH + c);
        const float a0 = bf16_lo(hl) > 0.f ? dy_lo * bf16_lo(w3p) : 0.f;
        const float a1 = bf16_hi(hl) > 0.f ? dy_lo * bf16_hi(w3p) : 0.f;
        const float a2 = bf16_lo(hh) > 0.f ? dy_hi * bf16_lo(w3p) : 0.f;
        const float a3 = bf16_hi(hh) > 0.f ? dy_hi * bf16_hi(w3p) : 0.f;
        da[kc][half * 2 + 0] = pack_bf16(a0, a1);
        da[kc][half * 2 + 1] = pack_bf16(a2, a3);
      }
    }
    // dh1 = dh2 W2 (B[k = out][n = in] = W2[out][in] = W2^T[in][out])
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) {
        uint32_t b0, b1;
        bfrag(w2t, S2, nt, kc, lane, b0, b1);
        const uint32_t ak[4] = {da[kc][0], da[kc][1], da[kc][2], da[kc][3]};
        mma16816(d, ak, b0, b1);
      }
      const int c = nt * 8 + 2 * tq;
      uint32_t hl = 0, hh = 0;
      if (r_lo < R) hl = *reinterpret_cast<const uint32_t*>(h1 + r_lo * MH + c);
      if (r_hi < R) hh = *reinterpret_cast<const uint32_t*>(h1 + r_hi * MH + c);
      const uint32_t lo = pack_bf16(bf16_lo(hl) > 0.f ? d[0] : 0.f, bf16_hi(hl) > 0.f ? d[1] : 0.f);
      const uint32_t hi = pack_bf16(bf16_lo(hh) > 0.f ? d[2] : 0.f, bf16_hi(hh) > 0.f ? d[3] : 0.f);
      if (r_lo < R) *reinterpret_cast<uint32_t*>(dh1_out + r_lo * MH + c) = lo;
      if (r_hi < R) *reinterpret_cast<uint32_t*>(dh1_out + r_hi * MH + c) = hi;
    }
    // dh2 rows for the weight gradients
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      const int c = kc * 16 + 2 * tq;
      if (r_lo < R) {
        *reinterpret_cast<uint32_t*>(dh2_out + r_lo * MH + c) = da[kc][0];
        *reinterpret_cast<uint32_t*>(dh2_out + r_lo * MH + c + 8) = da[kc][2];
      }
      if (r_hi < R) {
        *reinterpret_cast<uint32_t*>(dh2_out + r_hi * MH + c) = da[kc][1];
        *reinterpret_cast<uint32_t*>(dh2_out + r_hi * MH + c + 8) = da[kc][3];
      }
    }
  }
  lsum = warp_sum_d(lsum);
  if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum);
}

// Backward, part 2: weight gradients, sums over rows of outer products.  A
// block takes a chunk of rows, stages kWgRows of them at a time in shared
// memory (each row read once), and every thread accumulates a fixed set of
// weights in registers: thread t owns dW2[t / 2][64 (t % 2) ... + 63],
// dW1[t / 2][8 (t % 2) ... + 7], the biases of unit t / 2 (even t) and dW3[t]
// (t < 128).  One atomic flush per block and weight.
constexpr int kWgThreads = 256;
constexpr int kWgRows = 32;

__global__ void __launch_bounds__(kWgThreads) k_mlp_wgrad(const float* __restrict__ x,
                                                          const uint16_t* __restrict__ h1,
                                                          const uint16_t* __restrict__ h2,
                                                          const float* __restrict__ dy,
                                                          const uint16_t* __restrict__ dh2,
                                                          const uint16_t* __restrict__ dh1, int64_t R,
                                                          int64_t chunk, float* __restrict__ grads) {
  __shared__ __align__(16) uint16_t s_h1[kWgRows][MH];
  __shared__ __align__(16) uint16_t s_h2[kWgRows][MH];
  __shared__ __align__(16) uint16_t s_d2[kWgRows][MH];
  __shared__ __align__(16) uint16_t s_d1[kWgRows][MH];
  __shared__ float s_x[kWgRows][MI];
  __shared__ float s_dy[kWgRows];
  const int t = threadIdx.x, j = t >> 1, half = t & 1;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(R, r0 + chunk);
  float a2[64], a1[8];
#pragma unroll
  for (int k = 0; k < 64; ++k) a2[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) a1[k] = 0.f;
  float b1 = 0.f, b2 = 0.f, w3 = 0.f, b3 = 0.f;
  auto bf = [](uint32_t bits16) { return __uint_as_float(bits16 << 16); };
  for (int64_t rb = r0; rb < r1; rb += kWgRows) {
    const int n = r1 - rb < kWgRows ? (int)(r1 - rb) : kWgRows;
    __syncthreads();
    // stage the rows: 16-byte loads of the bf16 rows, scalar for x and dy
    for (int i = t; i < kWgRows * (MH / 8); i += kWgThreads) {
      const int r = i / (MH / 8), c = (i % (MH / 8)) * 8;
      uint4 z = make_uint4(0u, 0u, 0u, 0u);
      const bool in = r < n;
      const size_t g = (size_t)(rb + r) * MH + c;
      *reinterpret_cast<uint4*>(&s_h1[r][c]) = in ? *reinterpret_cast<const uint4*>(h1 + g) : z;
      *reinterpret_cast<uint4*>(&s_h2[r][c]) = in ? *reinterpret_cast<const uint4*>(h2 + g) : z;
      *reinterpret_cast<uint4*>(&s_d2[r][c]) = in ? *reinterpret_cast<const uint4*>(dh2 + g) : z;
      *reinterpret_cast<uint4*>(&s_d1[r][c]) = in ? *reinterpret_cast<const uint4*>(dh1 + g) : z;
    }
    for (int i = t; i < kWgRows * MI; i += kWgThreads) {
      const int r = i / MI, c = i % MI;
      s_x[r][c] = r < n ? round_bf16(x[(size_t)(rb + r) * MI + c]) : 0.f;
    }
    if (t < kWgRows) s_dy[t] = t < n ? dy[rb + t] : 0.f;
    __syncthreads();
    for (int r = 0; r < n; ++r) {
      const float d2 = bf(s_d2[r][j]), d1 = bf(s_d1[r][j]);
      const uint4* hp = reinterpret_cast<const uint4*>(&s_h1[r][64 * half]);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint4 v = hp[q];
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a2[8 * q + 2 * e] += d2 * bf(u[e] & 0xFFFFu);
          a2[8 * q + 2 * e + 1] += d2 * bf(u[e] >> 16);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) a1[k] += d1 * s_x[r][8 * half + k];
      if (!half) {
        b2 += d2;
        b1 += d1;
      }
      if (t < MH) w3 += s_dy[r] * bf(s_h2[r][t]);
      if (t == 0) b3 += s_dy[r];
    }
  }
#pragma unroll
  for (int k = 0; k < 64; ++k) atomicAdd(grads + OFF_W2 + j * MH + 64 * half + k, a2[k]);
#pragma unroll
  for (int k = 0; k < 8; ++k) atomicAdd(grads + OFF_W1 + j * MI + 8 * half + k, a1[k]);
  if (!half) {
    atomicAdd(grads + OFF_B2 + j, b2);
    atomicAdd(grads + OFF_B1 + j, b1);
  }
  if (t < MH) atomicAdd(grads + OFF_W3 + t, w3);
  if (t == 0) atomicAdd(grads + OFF_B3, b3);
}

// Adam on the fp32 master parameters; refreshes the bf16 weight copies.
__global__ void k_mlp_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                           float* __restrict__ V, int n, float lr, float b1, float b2, float eps, float bc1,
                           float bc2, uint16_t* __restrict__ w1, uint16_t* __restrict__ w2,
                           uint16_t* __restrict__ w3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  const float p = P[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  P[i] = p;
  const uint16_t hb = __bfloat16_as_ushort(__float2bfloat16_rn(p));
  if (i >= OFF_W1 && i < OFF_B1) w1[i - OFF_W1] = hb;
  else if (i >= OFF_W2 && i < OFF_B2) w2[i - OFF_W2] = hb;
  else if (i >= OFF_W3 && i < OFF_B3) w3[i - OFF_W3] = hb;
}

static bool mlp_ok(const tgs_mlp* w) {
  return w && w->w1 && w->w2 && w->w3 && w->b1 && w->b2 && w->b3 && aligned4(w->w1) && aligned4(w->w2) &&
         aligned4(w->w3);
}

static MlpK mlp_k(const tgs_mlp* w) { return MlpK{w->w1, w->w2, w->w3, w->b1, w->b2, w->b3}; }

static int mlp_grid(int64_t R) {
  const int64_t tiles = (R + 15) / 16;
  return (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 3) / 4, (int64_t)device_sm_count() * 8));
}

tgs_status launch_mlp_backward_tc(const tgs_mlp* w, const float* x, const uint16_t* h1, const uint16_t* h2,
                                  const float* y, const float* target, int64_t R, const int32_t* R_dev,
                                  float* grads, double* loss, int32_t* status, cudaStream_t s);
tgs_status launch_mlp_train_tc(const tgs_mlp* w, const float* x, const float* target, int64_t R,
                               const int32_t* R_dev, float* y, float* grads, double* loss, int32_t* status,
                               cudaStream_t s);

}  // namespace tgs

using namespace tgs;

extern "C" int32_t tgs_mlp_param_count(void) { return N_PARAMS; }

extern "C" tgs_status tgs_mlp_forward(const tgs_mlp* w, int64_t rows, const float* x, float* y, uint16_t* h1,
                                      uint16_t* h2, tgs_stream stream) {
  if (!mlp_ok(w) || rows < 0 || (rows > 0 && (!x || !y))) return TGS_ERR_INVALID_ARG;
  if ((h1 && !aligned4(h1)) || (h2 && !aligned4(h2))) return TGS_ERR_INVALID_ARG;
  if (rows == 0) return TGS_OK;
  const size_t smem = sizeof(MlpSmem);
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr[dev] = true;
  }
  k_mlp_forward<<<mlp_grid(rows), 128, smem, (cudaStream_t)stream>>>(mlp_k(w), x, rows, y, h1, h2);
  return check_launch();
}

extern "C" size_t tgs_mlp_backward_workspace_size(int64_t rows) {
  const size_t R = (size_t)std::max<int64_t>(rows, 1);
  return align_up(R * 4, 256) + 2 * align_up(R * MH * 2, 256);
}

static tgs_status mlp_backward_impl(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                                    const uint16_t* h1, const uint16_t* h2, const float* y, const float* target,
                                    float* grads, double* loss, void* workspace, size_t workspace_bytes,
                                    bool tc, int32_t* status, tgs_stream stream) {
  if (!mlp_ok(w) || rows < 0 || !grads || !loss) return TGS_ERR_INVALID_ARG;
  if (rows > 0 && (!x || !h1 || !h2 || !y || !target || !aligned4(h1) || !aligned4(h2))) return TGS_ERR_INVALID_ARG;
  if (tc && rows > 0 && (!aligned16(x) || !aligned16(h1) || !aligned16(h2) || !aligned16(workspace)))
    return TGS_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < tgs_mlp_backward_workspace_size(rows)) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(grads, 0, sizeof(float) * N_PARAMS, s);
  cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (rows == 0) return check_launch();
  Carver c(workspace);
  float* dy = c.take<float>((size_t)rows);
  uint16_t* dh2 = c.take<uint16_t>((size_t)rows * MH);
  uint16_t* dh1 = c.take<uint16_t>((size_t)rows * MH);
  if (tc) return launch_mlp_backward_tc(w, x, h1, h2, y, target, rows, rows_dev, grads, loss, status, s);
  const size_t smem = sizeof(MlpSmem) + MH * S2 * sizeof(uint16_t);
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaFuncSetAttribute(k_mlp_backward_act, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr[dev] = true;
  }
  k_mlp_backward_act<<<mlp_grid(rows), 128, smem, s>>>(mlp_k(w), h1, h2, y, target, rows, rows_dev, dy, dh2, dh1,
                                                        loss);
  // chunks: whole kWgRows groups, at most 4 blocks per SM's worth

  const int64_t groups = (rows + kWgRows - 1) / kWgRows;
  const int64_t waves = (int64_t)device_sm_count() * 4;
  const int64_t per = std::max<int64_t>(1, (groups + waves - 1) / waves);
  const int64_t chunk = per * kWgRows;
  k_mlp_wgrad<<<(unsigned)((rows + chunk - 1) / chunk), kWgThreads, 0, s>>>(x, h1, h2, dy, dh2, dh1, rows, chunk,
                                                                          grads);
  return check_launch();
}

extern "C" tgs_status tgs_mlp_backward(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                                       const uint16_t* h1, const uint16_t* h2, const float* y, const float* target,
                                       float* grads, double* loss, void* workspace, size_t workspace_bytes,
                                       tgs_stream stream) {
  return mlp_backward_impl(w, rows, rows_dev, x, h1, h2, y, target, grads, loss, workspace, workspace_bytes, false,
                           nullptr, stream);
}

extern "C" tgs_status tgs_mlp_backward_tc(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                                          const uint16_t* h1, const uint16_t* h2, const float* y,
                                          const float* target, float* grads, double* loss, int32_t* status,
                                          void* workspace, size_t workspace_bytes, tgs_stream stream) {
  return mlp_backward_impl(w, rows, rows_dev, x, h1, h2, y, target, grads, loss, workspace, workspace_bytes, true,
                           status, stream);
}

extern "C" tgs_status tgs_mlp_train_tc(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                                       const float* target, float* y, float* grads, double* loss, int32_t* status,
                                       tgs_stream stream) {
  if (!mlp_ok(w) || rows < 0 || !grads || !loss) return TGS_ERR_INVALID_ARG;
  if (rows > 0 && (!x || !target || !aligned16(x) || !aligned16(w->w1) || !aligned16(w->w2)))
    return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(grads, 0, sizeof(float) * N_PARAMS, s);
  cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (rows == 0) return check_launch();
  return launch_mlp_train_tc(w, x, target, rows, rows_dev, y, grads, loss, status, s);
}

extern "C" tgs_status tgs_mlp_adam(float* params, const float* grads, float* m, float* v, int32_t step, float lr,
                                   float beta1, float beta2, float eps, uint16_t* w1, uint16_t* w2, uint16_t* w3,
                                   tgs_stream stream) {
  if (!params || !grads || !m || !v || step < 1 || !w1 || !w2 || !w3 || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f))
    return TGS_ERR_INVALID_ARG;
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)step));
  k_mlp_adam<<<(N_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, N_PARAMS, lr, beta1,
                                                                       beta2, eps, bc1, bc2, w1, w2, w3);
  return check_launch();
}
