// Forward of the tile-error MLP on the 5th-generation tensor cores
// (tcgen05): 128-row tiles, bf16 operands in shared memory, fp32
// accumulators in tensor memory (TMEM).
//
// One CTA of 128 threads (4 warps) loops over 128-row tiles:
//   1. every thread converts its row of x to bf16 into the A tile of layer 1;
//   2. one thread issues D1 = X W1^T (M 128, N 128, K 16) into TMEM columns
//      0-127 and commits to an mbarrier;
//   3. every thread reads its row of D1 (tcgen05.ld, 32 columns at a time),
//      adds b1, applies ReLU, rounds to bf16 and writes the row into the A
//      tile of layer 2 (and to h1);
//   4. one thread issues D2 = H1 W2^T as eight K-16 steps into columns
//      128-255;
//   5. every thread reads its row of D2, adds b2, applies ReLU, rounds to
//      bf16 (h2) and takes the dot product with W3 (bf16) in fp32: y.
// The arithmetic is that of the mma.sync forward: bf16 products, fp32 sums.
//
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices stored as 128 contiguous bytes; consecutive core matrices
// along K are LBO = 128 bytes apart, consecutive 8-row groups SBO bytes apart.
// Waits on the mbarrier are bounded: on a timeout the CTA records it in the
// status word, waits (bounded) for its MMAs, frees its TMEM and stops.
#include <cuda_bf16.h>

#include "tgs_common.cuh"

namespace tgs {
namespace {

constexpr int TI = 16, TH = 128, TM = 128;  // input width, hidden width, rows per tile
// packed parameter / gradient vector: W1 [128,16] | b1 | W2 [128,128] | b2 | W3 [128] | b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + TH * TI, kOffW2 = kOffB1 + TH, kOffB2 = kOffW2 + TH * TH,
              kOffW3 = kOffB2 + TH, kOffB3 = kOffW3 + TH;
constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 256;         // D1 (0-127) and D2 (128-255)
constexpr long long kWaitLimit = 1ll << 22; // try_wait rounds before giving up
constexpr long long kDrillLimit = 1024;     // the same for the timeout drill

// byte offsets of the shared-memory operand tiles
constexpr uint32_t SBO_K16 = (TI / 8) * 128;    // 8-row group stride of a K = 16 tile
constexpr uint32_t SBO_K128 = (TH / 8) * 128;   // of a K = 128 tile
constexpr uint32_t OFF_W1S = 0;                             // W1 [128 n][16 k]
constexpr uint32_t OFF_W2S = OFF_W1S + TH * TI * 2;         // W2 [128 n][128 k]
constexpr uint32_t OFF_XS = OFF_W2S + TH * TH * 2;          // X  [128 m][16 k]
constexpr uint32_t OFF_HS = OFF_XS + TM * TI * 2;           // H1 [128 m][128 k]
constexpr uint32_t OFF_PAR = OFF_HS + TM * TH * 2;          // b1, b2, w3 (fp32), b3
constexpr uint32_t SMEM_USED = OFF_PAR + (3 * TH + 4) * 4;
// requested dynamic shared memory: more than a third of the SM's, so that at
// most two CTAs (2 x 256 TMEM columns = all 512) share an SM and an
// allocation never waits for another CTA
constexpr uint32_t SMEM_REQ = 100 * 1024;
static_assert(SMEM_USED <= SMEM_REQ, "shared memory layout");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) in a K-major no-swizzle tile
__device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// shared-memory matrix descriptor: start, LBO, SBO (all >> 4), version 1,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: fp32 accumulate, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TH >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Bounded wait for the mbarrier's phase `parity` to complete.
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity, long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

struct TcArgs {
  const uint16_t *w1, *w2, *w3;
  const float *b1, *b2, *b3;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_forward_tc(TcArgs w, const float* __restrict__ x, int64_t R,
                                                                  float* __restrict__ y, uint16_t* __restrict__ h1,
                                                                  uint16_t* __restrict__ h2,
                                                                  int32_t* __restrict__ status, int drill) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar;
  const int t = threadIdx.x, warp = t >> 5;
  float* par = reinterpret_cast<float*>(sm + OFF_PAR);  // b1 [128], b2 [128], w3 [128], b3
  // weights into the canonical layouts (each 16-byte chunk = 8 k-values of one row)
  for (int i = t; !drill && i < TH * (TI / 8); i += kTcThreads) {
    const int n = i / (TI / 8), k8 = (i % (TI / 8)) * 8;
    *reinterpret_cast<uint4*>(sm + OFF_W1S + core_off(n, k8, SBO_K16)) =
        *reinterpret_cast<const uint4*>(w.w1 + n * TI + k8);
  }
  for (int i = t; !drill && i < TH * (TH / 8); i += kTcThreads) {
    const int n = i / (TH / 8), k8 = (i % (TH / 8)) * 8;
    *reinterpret_cast<uint4*>(sm + OFF_W2S + core_off(n, k8, SBO_K128)) =
        *reinterpret_cast<const uint4*>(w.w2 + n * TH + k8);
  }
  for (int i = t; !drill && i < TH; i += kTcThreads) {
    par[i] = w.b1[i];
    par[TH + i] = w.b2[i];
    par[2 * TH + i] = __uint_as_float((uint32_t)w.w3[i] << 16);
  }
  if (t == 0) {
    if (!drill) par[3 * TH] = w.b3[0];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t mbar = smem_u32(&s_mbar);
  const uint32_t base = smem_u32(sm);
  const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
  uint32_t phase = 0;
  bool failed = false;   // uniform across the CTA (decided by __syncthreads_or)
  bool pending = false;  // MMAs committed whose completion was not observed
  // drill: the timeout path on a phase that nothing completes (no MMA issued)
  if (drill && __syncthreads_or(!wait_parity(mbar, phase, kDrillLimit))) failed = true;
  const int64_t tiles = drill ? 0 : (R + TM - 1) / TM;
  // the x row of the CTA's next tile is loaded while the current one runs
  float4 xn[TI / 4];
  auto load_x = [&](int64_t tl) {
    const int64_t rw = tl * TM + t;
#pragma unroll
    for (int k4 = 0; k4 < TI / 4; ++k4)
      xn[k4] = tl < tiles && rw < R ? *reinterpret_cast<const float4*>(x + rw * TI + 4 * k4)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  load_x(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * TM + t;
    const bool valid = row < R;
    // 1. x row -> bf16 A tile of layer 1
    {
      float xv[TI];
#pragma unroll
      for (int k = 0; k < TI; k += 4) {
        const float4 v = xn[k / 4];
        xv[k] = v.x; xv[k + 1] = v.y; xv[k + 2] = v.z; xv[k + 3] = v.w;
      }
#pragma unroll
      for (int k8 = 0; k8 < TI; k8 += 8)
        *reinterpret_cast<uint4*>(sm + OFF_XS + core_off(t, k8, SBO_K16)) =
            make_uint4(pack2(xv[k8], xv[k8 + 1]), pack2(xv[k8 + 2], xv[k8 + 3]), pack2(xv[k8 + 4], xv[k8 + 5]),
                       pack2(xv[k8 + 6], xv[k8 + 7]));
    }
    load_x(tile + gridDim.x);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // 2. layer 1 (one K-16 step)
    if (t == 0) {
      mma_bf16(tmem, sdesc(base + OFF_XS, 128, SBO_K16), sdesc(base + OFF_W1S, 128, SBO_K16), 0u);
      commit(mbar);
    }
    if (__syncthreads_or(!wait_parity(mbar, phase))) {
      failed = pending = true;
      break;
    }
    phase ^= 1u;
    fence_after();
    // 3. epilogue 1: h1 = bf16(relu(D1 + b1)) -> A tile of layer 2 (and h1)
#pragma unroll 1
    for (int c0 = 0; c0 < TH; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_addr + (uint32_t)c0, v);
      uint32_t pk[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2)
        pk[k / 2] = pack2(fmaxf(v[k] + par[c0 + k], 0.f), fmaxf(v[k + 1] + par[c0 + k + 1], 0.f));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 u = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        *reinterpret_cast<uint4*>(sm + OFF_HS + core_off(t, c0 + 8 * q, SBO_K128)) = u;
        if (h1 && valid) *reinterpret_cast<uint4*>(h1 + row * TH + c0 + 8 * q) = u;
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // 4. layer 2 (eight K-16 steps)
    if (t == 0) {
#pragma unroll
      for (int kk = 0; kk < TH / 16; ++kk)
        mma_bf16(tmem + TH, sdesc(base + OFF_HS + kk * 256, 128, SBO_K128),
                 sdesc(base + OFF_W2S + kk * 256, 128, SBO_K128), kk > 0 ? 1u : 0u);
      commit(mbar);
    }
    if (__syncthreads_or(!wait_parity(mbar, phase))) {
      failed = pending = true;
      break;
    }
    phase ^= 1u;
    fence_after();
    // 5. epilogue 2: h2 = bf16(relu(D2 + b2)), y = W3 . h2 + b3
    float acc = 0.f;
#pragma unroll 1
    for (int c0 = 0; c0 < TH; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_addr + (uint32_t)(TH + c0), v);
      uint32_t pk[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        pk[k / 2] = pack2(fmaxf(v[k] + par[TH + c0 + k], 0.f), fmaxf(v[k + 1] + par[TH + c0 + k + 1], 0.f));
        acc += __uint_as_float(pk[k / 2] << 16) * par[2 * TH + c0 + k] +
               __uint_as_float(pk[k / 2] & 0xffff0000u) * par[2 * TH + c0 + k + 1];
      }
      if (h2 && valid) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(h2 + row * TH + c0 + 8 * q) =
              make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
      }
    }
    if (valid) y[row] = acc + par[3 * TH];
    // every thread is done reading TMEM and the A tiles before the next MMAs
    fence_before();
    __syncthreads();
    fence_after();
  }
  if (failed) {
    if (t == 0 && status) atomicExch(status, 1);
    if (pending) wait_parity(mbar, phase);  // the MMAs still in flight (phase not yet observed; bounded)
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// Weight gradients as tensor-core contractions over the row index.  For a
// 128-row tile
//   dW2 [128 k][128 j] += dH2^T H1,   db2 [k] += sum_r dH2 [r][k],
//   dW1 [128 j][16 i]  += dH1^T X,    db1 [j] += sum_r dH1 [r][j],
// with M = 128 hidden units, K = 128 rows and N = 144 (128 units, a column
// of ones for the bias, 15 zero columns) or N = 32 (16 features, ones, 15
// zeros).  The operands are the row tiles themselves, read MN-major: a core
// matrix of a row tile (8 rows x 8 consecutive units or features) is, for a
// contraction over the rows, 8 K-rows x 8 contiguous M (or N) values.
constexpr uint32_t N2 = TH + 16, N1 = 32;       // B widths: units + ones + zeros, features + ones + zeros
// instruction descriptors of the two contractions (as kIdesc, N = N2 and N1)
constexpr uint32_t kIdescN2 = (1u << 4) | (1u << 7) | (1u << 10) | ((N2 >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t kIdescN1 = (1u << 4) | (1u << 7) | (1u << 10) | ((N1 >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// Row tiles, rows r of the 128-row tile in 8-row core-matrix groups (core_off):
// read K-major (rows = M) by the forward's contractions and MN-major (rows =
// K) by the weight gradients, so nothing is copied transposed.
constexpr uint32_t XW = 32, HW = TH + 16;                 // widths: 16 features | 1 | 15 zeros; 128 units | 1 | 15 zeros
constexpr uint32_t SBO_X = (XW / 8) * 128, SBO_H = (HW / 8) * 128;
// the weight-gradient contractions read both operands MN-major (transpose bits 15, 16)
constexpr uint32_t kIdescN2T = kIdescN2 | (1u << 15) | (1u << 16);
constexpr uint32_t kIdescN1T = kIdescN1 | (1u << 15) | (1u << 16);

__device__ __forceinline__ void mma_bf16_n(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// ---------------------------------------------------------------------------
// The whole backward in one pass over the rows: per 128-row tile the
// activation adjoint (dH1 = [H1 > 0] (dH2 W2), the forward's second layer run
// backwards) and the weight gradients above, with dH2 and dH1 kept in shared
// memory, so the rows are read once and no adjoint goes to memory; dW3 and
// db3 (fp32 dy, not a bf16 operand) on the CUDA cores.  256 threads: thread t takes row t % 128
// and hidden units 64 (t / 128) .. + 63.  dH2, H1, dH1 and X are written once
// each, as row tiles: dH2 is the A operand of dH1 = dH2 W2 (K-major) and of
// dW2 (MN-major); H1, dH1 and X are read MN-major by the weight gradients.
// TMEM: dH1 in columns 0-127, dW2 | db2 in 128-271, dW1 |
// db1 in 288-319.  The roundings and products are those of the mma.sync and
// CUDA-core backward: dH2 and dH1 rounded to bf16, bf16 x bf16 products with
// fp32 sums, x rounded to bf16.
constexpr int kBwThreads = 256;
constexpr uint32_t FB_W2T = 0;                            // W2^T [128 j][128 k] (B of dH1)
constexpr uint32_t FB_DA = FB_W2T + TH * TH * 2;          // dH2 [128 r][128 k]: A of dH1 (K-major) and of dW2 (MN-major)
constexpr uint32_t FB_H1 = FB_DA + TM * TH * 2;           // [H1 | 1 | 0] [128 r][144]: B of dW2 (MN-major)
constexpr uint32_t FB_DH1 = FB_H1 + TM * HW * 2;          // dH1 [128 r][128]: A of dW1 (MN-major)
constexpr uint32_t FB_X = FB_DH1 + TM * TH * 2;           // [X | 1 | 0] [128 r][32]: B of dW1 (MN-major)
constexpr uint32_t FB_H2 = FB_X + TM * XW * 2;            // h2 rows (bf16), for dW3
constexpr uint32_t FB_DY = FB_H2 + TM * TH * 2;           // dy [128]
constexpr uint32_t FB_W3 = FB_DY + TM * 4;                // w3 (fp32) [128]
constexpr uint32_t FB_SMEM = FB_W3 + TH * 4;
// requested: more than the tiles use, so that every operand the contractions
// address, read with either stride order, lies inside the CTA's allocation
constexpr uint32_t FB_SMEM_REQ = 225 * 1024;
static_assert(FB_SMEM <= FB_SMEM_REQ && FB_SMEM_REQ <= 227 * 1024,
              "the fused backward's tiles fit one CTA's shared memory");
constexpr uint32_t kBwTmemCols = 512;
constexpr uint32_t kColW2 = 128, kColW1 = 288;

__global__ void __launch_bounds__(kBwThreads, 1) k_mlp_backward_tc(
    TcArgs w, const float* __restrict__ x, const uint16_t* __restrict__ h1, const uint16_t* __restrict__ h2,
    const float* __restrict__ y, const float* __restrict__ tgt, int64_t R, const int32_t* __restrict__ R_dev,
    float* __restrict__ grads, double* __restrict__ loss, int32_t* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar;
  const int t = threadIdx.x, warp = t >> 5;
  const int r = t & (TM - 1), hf = t >> 7, u0 = 64 * hf;  // row of the tile, first unit of this half
  float* w3f = reinterpret_cast<float*>(sm + FB_W3);
  float* s_dy = reinterpret_cast<float*>(sm + FB_DY);
  const uint16_t* s_h2 = reinterpret_cast<const uint16_t*>(sm + FB_H2);
  for (int i = t; i < TH * (TH / 8); i += kBwThreads) {  // B [n = j][k] = W2 [k][j]
    const int n = i % TH, k8 = (i / TH) * 8;
    uint32_t q[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      q[e] = (uint32_t)w.w2[(k8 + 2 * e) * TH + n] | ((uint32_t)w.w2[(k8 + 2 * e + 1) * TH + n] << 16);
    *reinterpret_cast<uint4*>(sm + FB_W2T + core_off(n, k8, SBO_K128)) = make_uint4(q[0], q[1], q[2], q[3]);
  }
  for (int i = t; i < TH; i += kBwThreads) w3f[i] = __uint_as_float((uint32_t)w.w3[i] << 16);
  for (int rr = t; rr < TM; rr += kBwThreads) {  // the constant columns: a one, then zeros (the bias gradients)
    const uint4 one = make_uint4(0x3F80u, 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sm + FB_X + core_off(rr, TI, SBO_X)) = one;
    *reinterpret_cast<uint4*>(sm + FB_X + core_off(rr, TI + 8, SBO_X)) = zero;
    *reinterpret_cast<uint4*>(sm + FB_H1 + core_off(rr, TH, SBO_H)) = one;
    *reinterpret_cast<uint4*>(sm + FB_H1 + core_off(rr, TH + 8, SBO_H)) = zero;
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kBwTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t mbar = smem_u32(&s_mbar);
  const uint32_t base = smem_u32(sm);
  const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;  // TMEM lanes of this warp's rows
  const int64_t Re = R_dev ? (*R_dev > 0 ? (*R_dev < R ? (int64_t)*R_dev : R) : 0) : R;
  const float inv = Re > 0 ? 1.f / (float)Re : 0.f;
  double lsum = 0.0;
  float w3 = 0.f, b3 = 0.f;
  uint32_t phase = 0;
  bool failed = false, pending = false, any = false;
  const int64_t tiles = (R + TM - 1) / TM;
  // The half rows of h2 and h1 (and the row's error) are loaded in one round,
  // and those of the CTA's next tile are issued as soon as the current ones are
  // staged, so they arrive while the tensor cores run (a loop that waited for
  // each pair of loads in turn bounded the kernel).
  uint4 G2[8], G1[8];
  float4 XR[TI / 4];
  float e = 0.f;
  auto load_rows = [&](int64_t tl) {
    const int64_t rw = tl * TM + r;
    const bool in = tl < tiles && rw < R;
#pragma unroll
    for (int q8 = 0; q8 < 8; ++q8) {
      G2[q8] = in ? *reinterpret_cast<const uint4*>(h2 + rw * TH + u0 + 8 * q8) : make_uint4(0u, 0u, 0u, 0u);
      G1[q8] = in ? *reinterpret_cast<const uint4*>(h1 + rw * TH + u0 + 8 * q8) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int k4 = 0; k4 < TI / 4; ++k4)
      XR[k4] = in && hf == 0 ? *reinterpret_cast<const float4*>(x + rw * TI + 4 * k4) : make_float4(0.f, 0.f, 0.f, 0.f);
    e = (tl < tiles && rw < Re) ? y[rw] - tgt[rw] : 0.f;
  };
  load_rows(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const float d = e * inv;
    if (hf == 0) {
      lsum += 0.5 * (double)e * (double)e * (double)inv;
      s_dy[r] = d;
    }
    uint64_t m1 = 0;  // h1 > 0 of this half's 64 units
#pragma unroll
    for (int q8 = 0; q8 < 8; ++q8) {
      const int c8 = u0 + 8 * q8;
      const uint4 g2 = G2[q8], g1 = G1[q8];
      const uint32_t a2[4] = {g2.x, g2.y, g2.z, g2.w}, a1[4] = {g1.x, g1.y, g1.z, g1.w};
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float v0 = __uint_as_float(a2[q] << 16) > 0.f ? d * w3f[c8 + 2 * q] : 0.f;
        const float v1 = __uint_as_float(a2[q] & 0xffff0000u) > 0.f ? d * w3f[c8 + 2 * q + 1] : 0.f;
        pk[q] = pack2(v0, v1);
        const int bit = c8 - u0 + 2 * q;
        if (__uint_as_float(a1[q] << 16) > 0.f) m1 |= 1ull << bit;
        if (__uint_as_float(a1[q] & 0xffff0000u) > 0.f) m1 |= 1ull << (bit + 1);
      }
      *reinterpret_cast<uint4*>(sm + FB_DA + core_off(r, c8, SBO_K128)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      *reinterpret_cast<uint4*>(sm + FB_H1 + core_off(r, c8, SBO_H)) = g1;
      *reinterpret_cast<uint4*>(sm + FB_H2 + (uint32_t)(r * TH + c8) * 2u) = g2;
    }
    if (hf == 0) {  // the row's 16 features, rounded to bf16
#pragma unroll
      for (int k8 = 0; k8 < TI; k8 += 8) {
        const float4 a = XR[k8 / 4], b = XR[k8 / 4 + 1];
        *reinterpret_cast<uint4*>(sm + FB_X + core_off(r, k8, SBO_X)) =
            make_uint4(pack2(a.x, a.y), pack2(a.z, a.w), pack2(b.x, b.y), pack2(b.z, b.w));
      }
    }
    load_rows(tile + gridDim.x);  // the next tile's rows, in flight during this tile's contractions
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // dH1 (before the mask) = dH2 W2
#pragma unroll
      for (int kk = 0; kk < TH / 16; ++kk)
        mma_bf16(tmem, sdesc(base + FB_DA + kk * 256, 128, SBO_K128), sdesc(base + FB_W2T + kk * 256, 128, SBO_K128),
                 kk > 0 ? 1u : 0u);
      commit(mbar);
    }
    {  // dW3, db3 on the CUDA cores while the tensor cores run
      const int u = t & (TH - 1), rb = 64 * hf;
#pragma unroll 8
      for (int q = rb; q < rb + 64; ++q) {
        w3 += s_dy[q] * __uint_as_float((uint32_t)s_h2[q * TH + u] << 16);
        if (u == 0) b3 += s_dy[q];
      }
    }
    if (__syncthreads_or(!wait_parity(mbar, phase))) {
      failed = pending = true;
      break;
    }
    phase ^= 1u;
    fence_after();
    // dh1 = bf16([h1 > 0] D): the row tile of dW1's A
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_addr + (uint32_t)(u0 + c0), v);
      uint32_t pk[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2)
        pk[k / 2] = pack2((m1 >> (c0 + k)) & 1ull ? v[k] : 0.f, (m1 >> (c0 + k + 1)) & 1ull ? v[k + 1] : 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sm + FB_DH1 + core_off(r, u0 + c0 + 8 * q, SBO_K128)) =
            make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
#pragma unroll
      for (int kk = 0; kk < TM / 16; ++kk) {
        const uint32_t acc = (any || kk > 0) ? 1u : 0u;
        // MN-major: LBO steps along K (the rows, 8 at a time), SBO along M / N (8 units)
        mma_bf16_n(tmem + kColW2, sdesc(base + FB_DA + kk * 2 * SBO_K128, SBO_K128, 128),
                   sdesc(base + FB_H1 + kk * 2 * SBO_H, SBO_H, 128), kIdescN2T, acc);
        mma_bf16_n(tmem + kColW1, sdesc(base + FB_DH1 + kk * 2 * SBO_K128, SBO_K128, 128),
                   sdesc(base + FB_X + kk * 2 * SBO_X, SBO_X, 128), kIdescN1T, acc);
      }
      commit(mbar);
    }
    any = true;
    if (__syncthreads_or(!wait_parity(mbar, phase))) {
      failed = pending = true;
      break;
    }
    phase ^= 1u;
    fence_after();
  }
  if (failed) {
    if (t == 0 && status) atomicExch(status, 1);
    if (pending) wait_parity(mbar, phase);
  } else if (any) {
    if (t < TM) {  // row t of the weight-gradient accumulators: hidden unit t
#pragma unroll 1
      for (int c0 = 0; c0 < (int)N2; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_addr + kColW2 + (uint32_t)c0, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int c = c0 + k;
          if (c < TH) atomicAdd(grads + kOffW2 + t * TH + c, v[k]);
          else if (c == TH) atomicAdd(grads + kOffB2 + t, v[k]);
        }
      }
      float v[32];
      tmem_ld32(tmem + lane_addr + kColW1, v);
#pragma unroll
      for (int k = 0; k < TI; ++k) atomicAdd(grads + kOffW1 + t * TI + k, v[k]);
      atomicAdd(grads + kOffB1 + t, v[TI]);
    }
    atomicAdd(grads + kOffW3 + (t & (TH - 1)), w3);
    if ((t & (TH - 1)) == 0) atomicAdd(grads + kOffB3, b3);
  }
  lsum = warp_sum_d(lsum);
  if ((t & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBwTmemCols));
}

// ---------------------------------------------------------------------------
// One training pass (the loss's gradient) with the forward recomputed in the
// same kernel: per 128-row tile, D1 = X W1^T and D2 = H1 W2^T on the tensor
// cores, h1, h2 and y from them in the epilogues, then the backward above
// (dH1 = [H1 > 0] (dH2 W2), dW2 | db2 and dW1 | db1 as contractions over the
// rows).  The activations never leave the SM: the pair of kernels that stores
// h1 and h2 (512 bytes a row) and reads them back moved about 1.7 GB at the
// 200-view size.  256 threads, thread t on row t % 128 and hidden units
// 64 (t / 128) .. + 63; dW3 and db3 (fp32 dy times the bf16 h2, as in the
// backward above) in registers per thread over the whole pass, reduced once.
// TMEM: D1, then dH1, in columns 0-127; dW2 | db2 in 128-271; dW1 | db1 in
// 288-319; D2 in 320-447.  Shared memory holds each operand once, as rows
// (bf16 X, H1, dH2 and dH1 of the tile's 128 rows): the forward's
// contractions read them K-major, the weight gradients (contractions over the
// rows) MN-major through the same core matrices, so no operand is copied
// transposed; X and H1 carry a column of ones for the bias gradients.  The roundings are the
// forward's and the backward's: x, h1, h2, dH2 and dH1 in bf16, fp32 sums; y
// sums its two halves of 64 units and then adds b3.
constexpr uint32_t FT_W2T = 0;                            // W2^T [128 j][128 k] (B of dH1)
constexpr uint32_t FT_W2 = FT_W2T + TH * TH * 2;          // W2 [128 n][128 k] (B of layer 2)
constexpr uint32_t FT_W1 = FT_W2 + TH * TH * 2;           // W1 [128 n][16 k] (B of layer 1)
// the row tiles (XW, HW, SBO_X, SBO_H above)
constexpr uint32_t FT_X = FT_W1 + TH * TI * 2;            // [X | 1 | 0]   [128 r][32]: A of layer 1, B of dW1
constexpr uint32_t FT_H1 = FT_X + TM * XW * 2;            // [H1 | 1 | 0]  [128 r][144]: A of layer 2, B of dW2
constexpr uint32_t FT_DH2 = FT_H1 + TM * HW * 2;          // dH2 [128 r][128]: A of dH1 and of dW2
constexpr uint32_t FT_DH1 = FT_DH2 + TM * TH * 2;         // dH1 [128 r][128]: A of dW1
constexpr uint32_t FT_PAR = FT_DH1 + TM * TH * 2;         // b1, b2, w3 (fp32) [128 each], b3, y halves [2][128]
constexpr uint32_t FT_SMEM = FT_PAR + (3 * TH + 4) * 4 + 2 * TM * 4;
static_assert(FT_SMEM <= 227 * 1024 && 2 * FT_SMEM > 228 * 1024,
              "the training pass's tiles fit one CTA's shared memory, and only one CTA an SM (512 TMEM columns)");
// requested: more than the tiles use, so that every operand the contractions
// address, read with either stride order, lies inside the CTA's allocation
constexpr uint32_t FT_SMEM_REQ = 225 * 1024;
static_assert(FT_SMEM <= FT_SMEM_REQ, "request covers the layout");
constexpr uint32_t kColD2 = 320;

__global__ void __launch_bounds__(kBwThreads, 1) k_mlp_train_tc(
    TcArgs w, const float* __restrict__ x, const float* __restrict__ tgt, int64_t R,
    const int32_t* __restrict__ R_dev, float* __restrict__ y_out, float* __restrict__ grads,
    double* __restrict__ loss, int32_t* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar;
  const int t = threadIdx.x, warp = t >> 5;
  const int r = t & (TM - 1), hf = t >> 7, u0 = 64 * hf;
  float* par = reinterpret_cast<float*>(sm + FT_PAR);  // b1 | b2 | w3 | b3 | y halves
  float* s_yh = par + 3 * TH + 4;
  for (int i = t; i < TH * (TH / 8); i += kBwThreads) {
    const int n = i % TH, k8 = (i / TH) * 8;
    uint32_t q[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      q[e] = (uint32_t)w.w2[(k8 + 2 * e) * TH + n] | ((uint32_t)w.w2[(k8 + 2 * e + 1) * TH + n] << 16);
    *reinterpret_cast<uint4*>(sm + FT_W2T + core_off(n, k8, SBO_K128)) = make_uint4(q[0], q[1], q[2], q[3]);
    *reinterpret_cast<uint4*>(sm + FT_W2 + core_off(n, k8, SBO_K128)) =
        *reinterpret_cast<const uint4*>(w.w2 + n * TH + k8);
  }
  for (int i = t; i < TH * (TI / 8); i += kBwThreads) {
    const int n = i / (TI / 8), k8 = (i % (TI / 8)) * 8;
    *reinterpret_cast<uint4*>(sm + FT_W1 + core_off(n, k8, SBO_K16)) =
        *reinterpret_cast<const uint4*>(w.w1 + n * TI + k8);
  }
  for (int i = t; i < TH; i += kBwThreads) {
    par[i] = w.b1[i];
    par[TH + i] = w.b2[i];
    par[2 * TH + i] = __uint_as_float((uint32_t)w.w3[i] << 16);
  }
  for (int r = t; r < TM; r += kBwThreads) {  // the constant columns: a one, then zeros (the bias gradients)
    const uint4 one = make_uint4(0x3F80u, 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sm + FT_X + core_off(r, TI, SBO_X)) = one;
    *reinterpret_cast<uint4*>(sm + FT_X + core_off(r, TI + 8, SBO_X)) = zero;
    *reinterpret_cast<uint4*>(sm + FT_H1 + core_off(r, TH, SBO_H)) = one;
    *reinterpret_cast<uint4*>(sm + FT_H1 + core_off(r, TH + 8, SBO_H)) = zero;
  }
  if (t == 0) {
    par[3 * TH] = w.b3[0];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kBwTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t mbar = smem_u32(&s_mbar);
  const uint32_t base = smem_u32(sm);
  const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;  // TMEM lanes of this warp's rows
  const int64_t Re = R_dev ? (*R_dev > 0 ? (*R_dev < R ? (int64_t)*R_dev : R) : 0) : R;
  const float inv = Re > 0 ? 1.f / (float)Re : 0.f;
  double lsum = 0.0;
  float w3acc[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) w3acc[k] = 0.f;
  float b3 = 0.f;
  uint32_t phase = 0;
  bool failed = false, pending = false, any = false;
  const int64_t tiles = (R + TM - 1) / TM;
  auto mma_wait = [&]() -> bool {  // every thread: the committed MMAs are complete
    if (__syncthreads_or(!wait_parity(mbar, phase))) return false;
    phase ^= 1u;
    fence_after();
    return true;
  };
  // the x row and target of the CTA's next tile, loaded while this one runs
  float4 XR[TI / 4];
  float tg = 0.f;
  auto load_rows = [&](int64_t tl) {
    const int64_t rw = tl * TM + r;
    const bool in = tl < tiles && rw < R;
#pragma unroll
    for (int k4 = 0; k4 < TI / 4; ++k4)
      XR[k4] = in && hf == 0 ? *reinterpret_cast<const float4*>(x + rw * TI + 4 * k4) : make_float4(0.f, 0.f, 0.f, 0.f);
    tg = (tl < tiles && rw < Re) ? tgt[rw] : 0.f;
  };
  load_rows(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * TM + r;
    const bool valid = row < R, counted = row < Re;
    const float tgv = tg;
    if (hf == 0) {  // the row's 16 features in bf16: X A tile and X^T
      float xv[TI];
#pragma unroll
      for (int k = 0; k < TI; k += 4) {
        const float4 v = XR[k / 4];
        xv[k] = v.x; xv[k + 1] = v.y; xv[k + 2] = v.z; xv[k + 3] = v.w;
      }
#pragma unroll
      for (int k8 = 0; k8 < TI; k8 += 8) {
        const uint32_t p[4] = {pack2(xv[k8], xv[k8 + 1]), pack2(xv[k8 + 2], xv[k8 + 3]),
                               pack2(xv[k8 + 4], xv[k8 + 5]), pack2(xv[k8 + 6], xv[k8 + 7])};
        *reinterpret_cast<uint4*>(sm + FT_X + core_off(r, k8, SBO_X)) = make_uint4(p[0], p[1], p[2], p[3]);
      }
    }
    load_rows(tile + gridDim.x);  // in flight during this tile's contractions
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // layer 1: D1 = X W1^T
      mma_bf16(tmem, sdesc(base + FT_X, 128, SBO_X), sdesc(base + FT_W1, 128, SBO_K16), 0u);
      commit(mbar);
    }
    if (!mma_wait()) {
      failed = pending = true;
      break;
    }
    // h1 = bf16(relu(D1 + b1)): the H1 A tile, [H1^T; 1; 0] and the mask h1 > 0
    uint64_t m1 = 0;
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_addr + (uint32_t)(u0 + c0), v);
      uint32_t pk[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2)
        pk[k / 2] = pack2(fmaxf(v[k] + par[u0 + c0 + k], 0.f), fmaxf(v[k + 1] + par[u0 + c0 + k + 1], 0.f));
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sm + FT_H1 + core_off(r, u0 + c0 + 8 * q, SBO_H)) =
            make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (__uint_as_float(pk[k] << 16) > 0.f) m1 |= 1ull << (c0 + 2 * k);
        if (__uint_as_float(pk[k] & 0xffff0000u) > 0.f) m1 |= 1ull << (c0 + 2 * k + 1);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // layer 2: D2 = H1 W2^T
#pragma unroll
      for (int kk = 0; kk < TH / 16; ++kk)
        mma_bf16(tmem + kColD2, sdesc(base + FT_H1 + kk * 256, 128, SBO_H),
                 sdesc(base + FT_W2 + kk * 256, 128, SBO_K128), kk > 0 ? 1u : 0u);
      commit(mbar);
    }
    if (!mma_wait()) {
      failed = pending = true;
      break;
    }
    // h2 = bf16(relu(D2 + b2)); y = W3 . h2 + b3 from the two halves
    uint32_t h2p[32];
    float acc = 0.f;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_addr + kColD2 + (uint32_t)(u0 + c0), v);
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        const int c = u0 + c0 + k;
        const uint32_t pk = pack2(fmaxf(v[k] + par[TH + c], 0.f), fmaxf(v[k + 1] + par[TH + c + 1], 0.f));
        h2p[(c0 + k) / 2] = pk;
        acc += __uint_as_float(pk << 16) * par[2 * TH + c] + __uint_as_float(pk & 0xffff0000u) * par[2 * TH + c + 1];
      }
    }
    s_yh[hf * TM + r] = acc;
    __syncthreads();
    const float yv = s_yh[r] + s_yh[TM + r] + par[3 * TH];
    if (y_out && valid && hf == 0) y_out[row] = yv;
    const float e = counted ? yv - tgv : 0.f;
    const float d = e * inv;
    if (hf == 0) {
      lsum += 0.5 * (double)e * (double)e * (double)inv;
      b3 += d;
    }
    // dH2 = [h2 > 0] d w3 (bf16): its row tile, the A operand of dH1 and of dW2;
    // dW3 partials d h2
#pragma unroll
    for (int q8 = 0; q8 < 8; ++q8) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 8 * q8 + 2 * q, c = u0 + j;
        const float lo = __uint_as_float(h2p[j / 2] << 16), hi = __uint_as_float(h2p[j / 2] & 0xffff0000u);
        pk[q] = pack2(lo > 0.f ? d * par[2 * TH + c] : 0.f, hi > 0.f ? d * par[2 * TH + c + 1] : 0.f);
        w3acc[j] += d * lo;
        w3acc[j + 1] += d * hi;
      }
      *reinterpret_cast<uint4*>(sm + FT_DH2 + core_off(r, u0 + 8 * q8, SBO_K128)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // dH1 (before the mask) = dH2 W2
#pragma unroll
      for (int kk = 0; kk < TH / 16; ++kk)
        mma_bf16(tmem, sdesc(base + FT_DH2 + kk * 256, 128, SBO_K128), sdesc(base + FT_W2T + kk * 256, 128, SBO_K128),
                 kk > 0 ? 1u : 0u);
      commit(mbar);
    }
    if (!mma_wait()) {
      failed = pending = true;
      break;
    }
    // dh1 = bf16([h1 > 0] D): the row tile of dW1's A
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_addr + (uint32_t)(u0 + c0), v);
      uint32_t pk[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2)
        pk[k / 2] = pack2((m1 >> (c0 + k)) & 1ull ? v[k] : 0.f, (m1 >> (c0 + k + 1)) & 1ull ? v[k + 1] : 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sm + FT_DH1 + core_off(r, u0 + c0 + 8 * q, SBO_K128)) =
            make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // dW2 | db2 and dW1 | db1, accumulated over the CTA's tiles
#pragma unroll
      for (int kk = 0; kk < TM / 16; ++kk) {
        const uint32_t accu = (any || kk > 0) ? 1u : 0u;
        // MN-major: LBO steps along K (the rows, 8 at a time), SBO along M / N (8 units)
        mma_bf16_n(tmem + kColW2, sdesc(base + FT_DH2 + kk * 2 * SBO_K128, SBO_K128, 128),
                   sdesc(base + FT_H1 + kk * 2 * SBO_H, SBO_H, 128), kIdescN2T, accu);
        mma_bf16_n(tmem + kColW1, sdesc(base + FT_DH1 + kk * 2 * SBO_K128, SBO_K128, 128),
                   sdesc(base + FT_X + kk * 2 * SBO_X, SBO_X, 128), kIdescN1T, accu);
      }
      commit(mbar);
    }
    any = true;
    if (!mma_wait()) {
      failed = pending = true;
      break;
    }
  }
  if (failed) {
    if (t == 0 && status) atomicExch(status, 1);
    if (pending) wait_parity(mbar, phase);
  } else if (any) {
    if (t < TM) {  // row t of the weight-gradient accumulators: hidden unit t
#pragma unroll 1
      for (int c0 = 0; c0 < (int)N2; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_addr + kColW2 + (uint32_t)c0, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int c = c0 + k;
          if (c < TH) atomicAdd(grads + kOffW2 + t * TH + c, v[k]);
          else if (c == TH) atomicAdd(grads + kOffB2 + t, v[k]);
        }
      }
      float v[32];
      tmem_ld32(tmem + lane_addr + kColW1, v);
#pragma unroll
      for (int k = 0; k < TI; ++k) atomicAdd(grads + kOffW1 + t * TI + k, v[k]);
      atomicAdd(grads + kOffB1 + t, v[TI]);
    }
    // dW3 and db3: the rows' partials summed over each warp, one atomic per warp and unit
#pragma unroll
    for (int k = 0; k < 64; ++k) {
      const float sum = warp_sum(w3acc[k]);
      if ((t & 31) == 0) atomicAdd(grads + kOffW3 + u0 + k, sum);
    }
    b3 = warp_sum(b3);
    if ((t & 31) == 0 && hf == 0) atomicAdd(grads + kOffB3, b3);
  }
  lsum = warp_sum_d(lsum);
  if ((t & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBwTmemCols));
}
}  // namespace

// Launches k_mlp_backward_tc over the rows (one CTA per SM: its shared
// memory and 512 TMEM columns).
tgs_status launch_mlp_backward_tc(const tgs_mlp* w, const float* x, const uint16_t* h1, const uint16_t* h2,
                                  const float* y, const float* target, int64_t R, const int32_t* R_dev,
                                  float* grads, double* loss, int32_t* status, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch();
  static bool attr[64] = {};
  if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
  if (!attr[dev]) {
    cudaFuncSetAttribute(k_mlp_backward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FB_SMEM_REQ);
    attr[dev] = true;
  }
  const int64_t tiles = (R + TM - 1) / TM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, device_sm_count()));
  k_mlp_backward_tc<<<grid, kBwThreads, FB_SMEM_REQ, s>>>(TcArgs{w->w1, w->w2, w->w3, w->b1, w->b2, w->b3}, x, h1, h2, y,
                                                      target, R, R_dev, grads, loss, status);
  return check_launch();
}

// Launches k_mlp_train_tc over the rows (one CTA per SM: its shared memory
// and 512 TMEM columns).
tgs_status launch_mlp_train_tc(const tgs_mlp* w, const float* x, const float* target, int64_t R,
                               const int32_t* R_dev, float* y, float* grads, double* loss, int32_t* status,
                               cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch();
  static bool attr[64] = {};
  if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
  if (!attr[dev]) {
    cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FT_SMEM_REQ);
    attr[dev] = true;
  }
  const int64_t tiles = (R + TM - 1) / TM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, device_sm_count()));
  k_mlp_train_tc<<<grid, kBwThreads, FT_SMEM_REQ, s>>>(TcArgs{w->w1, w->w2, w->w3, w->b1, w->b2, w->b3}, x, target, R,
                                                   R_dev, y, grads, loss, status);
  return check_launch();
}

}  // namespace tgs

using namespace tgs;

extern "C" tgs_status tgs_mlp_forward_tc(const tgs_mlp* w, int64_t rows, const float* x, float* y, uint16_t* h1,
                                         uint16_t* h2, int32_t* status, tgs_stream stream) {
  if (!w || !w->w1 || !w->w2 || !w->w3 || !w->b1 || !w->b2 || !w->b3 || rows < 0 || (rows > 0 && (!x || !y)))
    return TGS_ERR_INVALID_ARG;
  if (!aligned16(w->w1) || !aligned16(w->w2) || !aligned16(x) || (h1 && !aligned16(h1)) || (h2 && !aligned16(h2)))
    return TGS_ERR_INVALID_ARG;
  if (rows == 0) return TGS_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch();
  static bool attr[64] = {};
  if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
  if (!attr[dev]) {
    cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_REQ);
    attr[dev] = true;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (rows + TM - 1) / TM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 2ll * sms));
  k_mlp_forward_tc<<<grid, kTcThreads, SMEM_REQ, (cudaStream_t)stream>>>(
      TcArgs{w->w1, w->w2, w->w3, w->b1, w->b2, w->b3}, x, rows, y, h1, h2, status, 0);
  return check_launch();
}

extern "C" tgs_status tgs_mlp_tc_wait_drill(int32_t* status, tgs_stream stream) {
  if (!status) return TGS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch();
  static bool attr[64] = {};
  if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
  if (!attr[dev]) {
    cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_REQ);
    attr[dev] = true;
  }
  k_mlp_forward_tc<<<1, kTcThreads, SMEM_REQ, (cudaStream_t)stream>>>(TcArgs{}, nullptr, 0, nullptr, nullptr,
                                                                       nullptr, status, 1);
  return check_launch();
}
