// Sparse forward rasterization and its adjoint (Sec. 3.6, Eq. 1).
//
// One thread block per active tile, one thread per sampled pixel of the tile
// (block size = 32 * ceil(n_pix / 32), so a tile sampled at rate 0.1 runs as
// one warp).  The tile's depth-ordered splat list is staged through shared
// memory in batches of one splat per thread; a block-wide vote ends the walk
// once every pixel has saturated.  The backward replays the same walk in
// reverse from the stored final transmittance, recovering T_k by division,
// and sums each splat's adjoint over the warp's pixels with shuffles before a
// single vector atomic per warp and splat.
#include "tgs_common.cuh"

namespace tgs {

void launch_project_bwd(const tgs_gaussians& g, const tgs_camera& cam, const int32_t* radius, const float* grad2d,
                        const tgs_param_ptrs& grads, uint8_t* touched, int write_untouched, int accumulate,
                        float* row, cudaStream_t s);
bool gaussians_ok(const tgs_gaussians* g);
bool camera_ok(const tgs_camera* c);

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr int kUnroll = 4;  // splats per step of the forward walk
constexpr int kCkptEvery = 32;  // list positions per checkpoint slot (a multiple of kUnroll)

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Splat {
  float2 xy;
  float2 yr;   // the rows [y0, y1] outside which alpha < 1/255 (with a margin)
  float4 co;   // the conic pre-scaled to base-2 exponents: (-a/2, -b, -c/2) log2(e), then the opacity
  float4 rgb;  // r, g, b, (unused)
};

// Staging scale of the conic: with a' = -a log2(e) / 2, b' = -b log2(e) and
// c' = -c log2(e) / 2 the exponent of Eq. 1's Gaussian in base 2 is
// p = a' dx^2 + b' dx dy + c' dy^2 = log2(e) power.
constexpr float kPow2A = -0.5f * kLog2e;
constexpr float kPow2B = -kLog2e;
// back to the conic: a = a' kInvA, b = b' kInvB, c = c' kInvA
constexpr float kInvA = -1.3862943611198906f;  // -2 ln 2
constexpr float kInvB = -0.6931471805599453f;  // -ln 2

// p = log2(e) power at offset (dx, dy) from the splat's centre, with the
// pre-scaled conic: (a' dx + b' dy) dx + c' dy^2 (explicitly rounded, so
// every kernel takes the same decisions for the same splat and pixel).
__device__ __forceinline__ float splat_pow2(const float4& co, float dx, float dy) {
  const float t = __fmaf_rn(co.x, dx, __fmul_rn(co.y, dy));
  return __fmaf_rn(t, dx, __fmul_rn(__fmul_rn(co.z, dy), dy));
}

// alpha of a splat at offset (dx, dy) from its centre; G receives exp(power).
// Returns false when the splat is skipped (power > 0 or alpha < 1/255).
__device__ __forceinline__ bool splat_alpha_p(const float4& co, float dx, float dy, float& alpha, float& G, float& p) {
  p = splat_pow2(co, dx, dy);
  if (p > 0.f) return false;
  G = ex2_approx(p);
  alpha = fminf(kAlphaMax, __fmul_rn(co.w, G));
  return alpha >= kAlphaMin;
}

__device__ __forceinline__ bool splat_alpha(const float4& co, float dx, float dy, float& alpha, float& G) {
  const float p = splat_pow2(co, dx, dy);
  if (p > 0.f) return false;
  G = ex2_approx(p);
  alpha = fminf(kAlphaMax, __fmul_rn(co.w, G));
  return alpha >= kAlphaMin;
}

// The same decision without a branch: alpha and G are computed in every case
// (for power > 0, G may be +inf and alpha 0.99, finite either way), and the
// return value says whether the splat counts.
__device__ __forceinline__ bool splat_alpha_nb(const float4& co, float dx, float dy, float& alpha, float& G) {
  const float p = splat_pow2(co, dx, dy);
  G = ex2_approx(p);
  alpha = fminf(kAlphaMax, __fmul_rn(co.w, G));
  return p <= 0.f && alpha >= kAlphaMin;
}

struct RasterArgs {
  const float2* xy;
  const float4* conic_opac;
  const float* rgb;
  const int2* ranges;
  const int32_t* vals;
  const int32_t* active_tiles;
  const int32_t* n_active;
  const int32_t* pix_off;
  const uint8_t* pix_idx;
  int tiles_x;
  float bg[3];
};

// Rows a splat can reach: alpha >= 1/255 needs power >= -tau with
// tau = ln(255 o), i.e. the ellipse a dx^2 + 2 b dx dy + c dy^2 <= 2 tau,
// whose half-height is sqrt(2 tau a / (a c - b^2)).  The margin (1e-3
// relative + 1e-3 px) covers the rounding of the kernels' own alpha test, so
// a pixel outside [y0, y1] never passes it.  Empty when o <= 1/255.
__device__ __forceinline__ float2 splat_rows(float y, const float4& c) {
  const float tau = logf(255.f * c.w);
  if (!(tau > 0.f)) return make_float2(INFINITY, -INFINITY);
  const float det = c.x * c.z - c.y * c.y;
  if (!(det > 0.f) || !(c.x > 0.f)) return make_float2(-INFINITY, INFINITY);
  const float h = sqrtf(2.f * tau * c.x / det) * 1.001f + 1e-3f;
  return make_float2(y - h, y + h);
}

// A splat's projected record as loaded (loads only: a walk fetches the next
// batch's records into registers and waits on them only when it stages them,
// a whole batch later).
struct SplatRaw {
  float2 xy;
  float4 c;
  float r, g, b;
  int id;
};

__device__ __forceinline__ void fetch_splat(const RasterArgs& a, int id, SplatRaw& w) {
  w.id = id;
  w.xy = a.xy[id];
  w.c = a.conic_opac[id];
  w.r = a.rgb[3 * id];
  w.g = a.rgb[3 * id + 1];
  w.b = a.rgb[3 * id + 2];
}

__device__ __forceinline__ void finish_splat(const SplatRaw& w, Splat& sp) {
  sp.xy = w.xy;
  sp.yr = splat_rows(w.xy.y, w.c);
  sp.co = make_float4(__fmul_rn(w.c.x, kPow2A), __fmul_rn(w.c.y, kPow2B), __fmul_rn(w.c.z, kPow2A), w.c.w);
  sp.rgb = make_float4(w.r, w.g, w.b, __int_as_float(w.id));
}

__device__ __forceinline__ void load_splat(const RasterArgs& a, int k, Splat& sp) {
  SplatRaw w;
  fetch_splat(a, a.vals[k], w);
  finish_splat(w, sp);
}

// The rows [y0, y1] spanned by the sampled pixels of the calling warp
// (sampled pixels are in row-major order, so a warp's pixels form a band).
__device__ __forceinline__ float2 warp_rows(bool has, float py) {
  float lo = has ? py : INFINITY, hi = has ? py : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  return make_float2(lo, hi);
}

// Forward of active tile j (one thread per sampled pixel; sm holds
// blockDim.x splats).
// Checkpoints of the sampled forward for the split backward: slot c (c = 0
// .. n_slots - 1) of pixel s holds (T, C_r, C_g, C_b) in front of tile-list
// position (c + 1) kCkptEvery, at data[c * stride + s]; written by every
// pixel whose walk reaches that position.
struct Ckpt {
  float4* data;
  int n_slots;
  int64_t stride;
  const float* rgb;    // the forward's output (read by the backward)
  int32_t* tile_last;  // [active rank] longest blended run of the tile's pixels (nullable)
};

// SELECT: the blend of each group of kUnroll splats with selects instead of
// branches (more instructions, shorter dependent chains) - the better choice
// when few warps share an SM (a sparse step); with many warps per SM the
// branches' skipped work wins.  Both produce the same bits.
template <bool SELECT>
__device__ __forceinline__ void render_tile_fwd(const RasterArgs& a, int j, Splat* sm, float* __restrict__ out_rgb,
                                                float* __restrict__ out_T, int32_t* __restrict__ out_last,
                                                Ckpt ck = Ckpt{nullptr, 0, 0, nullptr, nullptr}) {
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  const bool has_pix = p0 + (int)threadIdx.x < p1;
  const int s = p0 + threadIdx.x;
  float px = 0.f, py = 0.f;
  if (has_pix) {
    const int l = a.pix_idx[s];
    px = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
    py = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
  }
  const int2 range = a.ranges[j];
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  bool done = !has_pix;
  const int B = blockDim.x;
  const float2 band = warp_rows(has_pix, py);  // splats outside it are skipped by the whole warp
  const int lane = threadIdx.x & 31;
  // the next batch's records are fetched into registers while the current
  // one is blended, and the list entries (ids) of the batch after it
  SplatRaw nxt;
  int idn = 0;
  const int tid = threadIdx.x;
  if (range.x + tid < range.y) fetch_splat(a, a.vals[range.x + tid], nxt);
  if (range.x + B + tid < range.y) idn = a.vals[range.x + B + tid];
  for (int base = range.x; base < range.y; base += B) {
    if (__syncthreads_count(done) == B) break;
    if (base + tid < range.y) finish_splat(nxt, sm[tid]);
    __syncthreads();
    if (base + B + tid < range.y) fetch_splat(a, idn, nxt);
    if (base + 2 * B + tid < range.y) idn = a.vals[base + 2 * B + tid];
    const int cnt = min(B, range.y - base);
    // Runs of kCkptEvery positions (B is a multiple of it), walked by every
    // thread so that the warp's ballot below stays converged: the checkpoint
    // in front of each run, then the run's splats that can reach the warp's
    // rows (a bit mask from one ballot), kUnroll at a time: their alphas do
    // not depend on T, so they are evaluated together and only the blend runs
    // in list order.  The splats left out fail every alpha test of the warp.
    for (int q32 = 0; q32 < cnt; q32 += kCkptEvery) {
      if (ck.data && !done) {
        const int c = (base - range.x + q32) / kCkptEvery - 1;  // state in front of this run
        if (c >= 0 && c < ck.n_slots) ck.data[c * ck.stride + s] = make_float4(T, C0, C1, C2);
      }
      const int qe = min(cnt, q32 + kCkptEvery);
      bool in_l = false;
      if (q32 + lane < qe) {
        const float2 yr = sm[q32 + lane].yr;
        in_l = yr.y >= band.x && yr.x <= band.y;
      }
      unsigned mask = __ballot_sync(0xffffffffu, in_l);
      while (mask && !done) {
        int qq[kUnroll];
        float al[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const bool val = mask != 0u;
          qq[u] = val ? q32 + __ffs(mask) - 1 : q32;
          mask &= mask - 1u;
          const float2 xy = sm[qq[u]].xy;
          float G;
          ok[u] = (SELECT ? splat_alpha_nb(sm[qq[u]].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], G)
                          : splat_alpha(sm[qq[u]].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], G)) &&
                  val;
        }
        if (!SELECT) {
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            if (!ok[u]) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.f, al[u]));
            if (Tn < kTStop) {
              done = true;
              break;
            }
            const float4 rgb = sm[qq[u]].rgb;
            const float w = al[u] * T;
            C0 += w * rgb.x;
            C1 += w * rgb.y;
            C2 += w * rgb.z;
            T = Tn;
            last = base + qq[u] + 1 - range.x;
          }
          continue;
        }
        // the blend without branches: a splat past the stopping one, or
        // skipped, leaves the state as it is
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, al[u]));
          const bool stop = ok[u] && !done && Tn < kTStop;
          const bool take = ok[u] && !done && !stop;
          done = done || stop;
          const float4 rgb = sm[qq[u]].rgb;
          const float w = al[u] * T;
          C0 = take ? C0 + w * rgb.x : C0;
          C1 = take ? C1 + w * rgb.y : C1;
          C2 = take ? C2 + w * rgb.z : C2;
          T = take ? Tn : T;
          last = take ? base + qq[u] + 1 - range.x : last;
        }
      }
    }
  }
  if (has_pix) {
    out_rgb[3 * s] = C0 + T * a.bg[0];
    out_rgb[3 * s + 1] = C1 + T * a.bg[1];
    out_rgb[3 * s + 2] = C2 + T * a.bg[2];
    out_T[s] = T;
    out_last[s] = last;
  }
  if (ck.tile_last) {  // the tile's longest blended run, for the pieces of the backward
    __shared__ int s_tl;
    __syncthreads();
    if (threadIdx.x == 0) s_tl = 0;
    __syncthreads();
    if (last > 0) atomicMax(&s_tl, last);
    __syncthreads();
    if (threadIdx.x == 0) ck.tile_last[j] = s_tl;
  }
}

template <bool SELECT>
__global__ void k_render_fwd(RasterArgs a, float* __restrict__ out_rgb, float* __restrict__ out_T,
                             int32_t* __restrict__ out_last, Ckpt ck) {
  extern __shared__ Splat sm[];
  const int j = blockIdx.x;
  if (j >= *a.n_active) return;
  render_tile_fwd<SELECT>(a, j, sm, out_rgb, out_T, out_last, ck);
}

// The same forward with two threads per sampled pixel: a warp holds 16
// pixels twice, and of every 32-position run the first half (lanes 0-15)
// walks positions 0-15 from the pixel's state, exactly as the walk above,
// while the second half (lanes 16-31) walks positions 16-31 at the same time
// from a local (T, C) = (1, 0), without stopping.  The halves then compose,
// (T, C) -> (T T_b, C + T C_b); where the product comes within 1e-5 of the
// stopping transmittance the second half walks its positions again from the
// composed entry state, with the stop, so every stop and n_last is the
// sequential walk's.  The walk of a run is half as long and the block has
// twice the warps; T and C differ from the sequential walk's by the rounding
// of the composition only.
constexpr float kTStopPairMargin = kTStop * (1.f + 1e-5f);

template <bool SELECT>
__device__ __forceinline__ void pair_walk(const Splat* sm, int q0, unsigned mask, float px, float py, int base_pos,
                                          bool can_stop, float& T, float& C0, float& C1, float& C2, int& last,
                                          bool& done) {
  while (mask && !done) {
    int qq[kUnroll];
    float al[kUnroll];
    bool ok[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool val = mask != 0u;
      qq[u] = val ? q0 + __ffs(mask) - 1 : q0;
      mask &= mask - 1u;
      const float2 xy = sm[qq[u]].xy;
      float G;
      ok[u] = (SELECT ? splat_alpha_nb(sm[qq[u]].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], G)
                      : splat_alpha(sm[qq[u]].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], G)) &&
              val;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const float Tn = __fmul_rn(T, __fsub_rn(1.f, al[u]));
      const bool stop = ok[u] && !done && can_stop && Tn < kTStop;
      const bool take = ok[u] && !done && !stop;
      done = done || stop;
      const float4 rgb = sm[qq[u]].rgb;
      const float w = al[u] * T;
      C0 = take ? C0 + w * rgb.x : C0;
      C1 = take ? C1 + w * rgb.y : C1;
      C2 = take ? C2 + w * rgb.z : C2;
      T = take ? Tn : T;
      last = take ? base_pos + qq[u] + 1 : last;
    }
  }
}

template <bool SELECT>
__device__ __forceinline__ void render_tile_fwd_pair(const RasterArgs& a, int j, Splat* sm,
                                                     float* __restrict__ out_rgb, float* __restrict__ out_T,
                                                     int32_t* __restrict__ out_last, const Ckpt& ck) {
  const unsigned full = 0xffffffffu;
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  const int lane = threadIdx.x & 31, h = lane >> 4;
  const int s = p0 + 16 * (int)(threadIdx.x >> 5) + (lane & 15);
  const bool has_pix = s < p1;
  float px = 0.f, py = 0.f;
  if (has_pix) {
    const int l = a.pix_idx[s];
    px = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
    py = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
  }
  const int2 range = a.ranges[j];
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  bool done = !has_pix;
  const int B = blockDim.x;
  const float2 band = warp_rows(has_pix, py);
  SplatRaw nxt;
  int idn = 0;
  const int tid = threadIdx.x;
  if (range.x + tid < range.y) fetch_splat(a, a.vals[range.x + tid], nxt);
  if (range.x + B + tid < range.y) idn = a.vals[range.x + B + tid];
  for (int base = range.x; base < range.y; base += B) {
    if (__syncthreads_count(done) == B) break;
    if (base + tid < range.y) finish_splat(nxt, sm[tid]);
    __syncthreads();
    if (base + B + tid < range.y) fetch_splat(a, idn, nxt);
    if (base + 2 * B + tid < range.y) idn = a.vals[base + 2 * B + tid];
    const int cnt = min(B, range.y - base);
    const int base_pos = base - range.x;
    for (int q32 = 0; q32 < cnt; q32 += kCkptEvery) {
      if (ck.data && !done && h == 0) {
        const int c = (base_pos + q32) / kCkptEvery - 1;  // state in front of this run
        if (c >= 0 && c < ck.n_slots) ck.data[c * ck.stride + s] = make_float4(T, C0, C1, C2);
      }
      const int qe = min(cnt, q32 + kCkptEvery);
      bool in_l = false;
      if (q32 + lane < qe) {
        const float2 yr = sm[q32 + lane].yr;
        in_l = yr.y >= band.x && yr.x <= band.y;
      }
      const unsigned m32 = __ballot_sync(full, in_l);
      const unsigned hm = h ? (m32 >> 16) : (m32 & 0xFFFFu);
      const int q0 = q32 + 16 * h;
      // half 0: the pixel's state, with the stop; half 1: a local state from (1, 0)
      float Tw = h ? 1.f : T, W0 = h ? 0.f : C0, W1 = h ? 0.f : C1, W2 = h ? 0.f : C2;
      int lw = h ? 0 : last;
      bool dw = done;
      pair_walk<SELECT>(sm, q0, hm, px, py, base_pos, h == 0, Tw, W0, W1, W2, lw, dw);
      __syncwarp();
      const float oT = __shfl_xor_sync(full, Tw, 16), o0 = __shfl_xor_sync(full, W0, 16),
                  o1 = __shfl_xor_sync(full, W1, 16), o2 = __shfl_xor_sync(full, W2, 16);
      const int ol = __shfl_xor_sync(full, lw, 16);
      const bool od = __shfl_xor_sync(full, (int)dw, 16) != 0;
      // A: the first half's state (exact), Bh: the second half's local walk
      const float aT = h ? oT : Tw, a0 = h ? o0 : W0, a1 = h ? o1 : W1, a2 = h ? o2 : W2;
      const int al_ = h ? ol : lw;
      const bool ad = h ? od : dw;
      const float bT = h ? Tw : oT, b0 = h ? W0 : o0, b1 = h ? W1 : o1, b2 = h ? W2 : o2;
      const int bl = h ? lw : ol;
      // stopped in the first half, or nothing blended in the second: the first half's state
      const bool first = ad || bl == 0;
      const float Tc = __fmul_rn(aT, bT);
      // the stop may lie in the second half: it walks its positions again from the exact entry state
      const bool again = !first && Tc < kTStopPairMargin;
      if (__any_sync(full, again)) {  // warp-uniform, so that every lane takes part in the shuffles
        float rT = aT, r0 = a0, r1 = a1, r2 = a2;
        int rl = al_;
        bool rd = false;
        if (h && again) pair_walk<false>(sm, q0, hm, px, py, base_pos, true, rT, r0, r1, r2, rl, rd);
        __syncwarp();
        const int src = (lane & 15) + 16;
        rT = __shfl_sync(full, rT, src);
        r0 = __shfl_sync(full, r0, src);
        r1 = __shfl_sync(full, r1, src);
        r2 = __shfl_sync(full, r2, src);
        rl = __shfl_sync(full, rl, src);
        rd = __shfl_sync(full, (int)rd, src) != 0;
        if (again) {
          T = rT; C0 = r0; C1 = r1; C2 = r2; last = rl; done = rd;
          continue;
        }
      }
      if (first) {
        T = aT; C0 = a0; C1 = a1; C2 = a2; last = al_; done = ad;
      } else {
        T = Tc;
        C0 = a0 + aT * b0;
        C1 = a1 + aT * b1;
        C2 = a2 + aT * b2;
        last = bl;
      }
    }
  }
  if (has_pix && h == 0) {
    out_rgb[3 * s] = C0 + T * a.bg[0];
    out_rgb[3 * s + 1] = C1 + T * a.bg[1];
    out_rgb[3 * s + 2] = C2 + T * a.bg[2];
    out_T[s] = T;
    out_last[s] = last;
  }
  if (ck.tile_last) {
    __shared__ int s_tl;
    __syncthreads();
    if (threadIdx.x == 0) s_tl = 0;
    __syncthreads();
    if (last > 0 && h == 0) atomicMax(&s_tl, last);
    __syncthreads();
    if (threadIdx.x == 0) ck.tile_last[j] = s_tl;
  }
}

template <bool SELECT>
__global__ void k_render_fwd_pair(RasterArgs a, float* __restrict__ out_rgb, float* __restrict__ out_T,
                                  int32_t* __restrict__ out_last, Ckpt ck) {
  extern __shared__ Splat sm[];
  const int j = blockIdx.x;
  if (j >= *a.n_active) return;
  render_tile_fwd_pair<SELECT>(a, j, sm, out_rgb, out_T, out_last, ck);
}

// The same forward with every warp on its own: a warp takes 32 sampled
// pixels of one tile (piece `piece` of tile j; j < 0 for none), stages its
// own 32-splat batches of the tile's list (one per lane, the next batch
// fetched while the current one is blended), walks them for its pixels and
// stops when they have saturated.  Same results as render_tile_fwd (the same
// per-pixel operations in the same order).  Returns the lane's blended count.
template <bool SELECT>
__device__ __forceinline__ int render_tile_fwd_warp(const RasterArgs& a, int j, int piece, Splat* sm,
                                                    float* __restrict__ out_rgb, float* __restrict__ out_T,
                                                    int32_t* __restrict__ out_last, const Ckpt& ck) {
  const int lane = threadIdx.x & 31;
  const int t = j >= 0 ? (a.active_tiles ? a.active_tiles[j] : j) : 0;
  const int p0 = j >= 0 ? a.pix_off[j] : 0, p1 = j >= 0 ? a.pix_off[j + 1] : 0;
  const int s = p0 + 32 * piece + lane;
  const bool has_pix = s < p1;
  float px = 0.f, py = 0.f;
  if (has_pix) {
    const int l = a.pix_idx[s];
    px = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
    py = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
  }
  const int2 range = j >= 0 ? a.ranges[j] : make_int2(0, 0);
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  bool done = !has_pix;
  const float2 band = warp_rows(has_pix, py);
  SplatRaw nxt;
  int idn = 0;
  if (range.x + lane < range.y) fetch_splat(a, a.vals[range.x + lane], nxt);
  if (range.x + kCkptEvery + lane < range.y) idn = a.vals[range.x + kCkptEvery + lane];
  for (int base = range.x; base < range.y; base += kCkptEvery) {
    if (__all_sync(0xffffffffu, done)) break;
    __syncwarp();
    if (base + lane < range.y) finish_splat(nxt, sm[lane]);
    __syncwarp();
    if (base + kCkptEvery + lane < range.y) fetch_splat(a, idn, nxt);
    if (base + 2 * kCkptEvery + lane < range.y) idn = a.vals[base + 2 * kCkptEvery + lane];
    const int cnt = min(kCkptEvery, range.y - base);
    if (ck.data && !done) {
      const int c = (base - range.x) / kCkptEvery - 1;  // state in front of this run
      if (c >= 0 && c < ck.n_slots) ck.data[c * ck.stride + s] = make_float4(T, C0, C1, C2);
    }
    bool in_l = false;
    if (lane < cnt) {
      const float2 yr = sm[lane].yr;
      in_l = yr.y >= band.x && yr.x <= band.y;
    }
    unsigned mask = __ballot_sync(0xffffffffu, in_l);
    while (mask && !done) {
      int qq[kUnroll];
      float al[kUnroll];
      bool ok[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const bool val = mask != 0u;
        qq[u] = val ? __ffs(mask) - 1 : 0;
        mask &= mask - 1u;
        const float2 xy = sm[qq[u]].xy;
        float G;
        ok[u] = (SELECT ? splat_alpha_nb(sm[qq[u]].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], G)
                        : splat_alpha(sm[qq[u]].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], G)) &&
                val;
      }
      if (!SELECT) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          if (!ok[u]) continue;
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, al[u]));
          if (Tn < kTStop) {
            done = true;
            break;
          }
          const float4 rgb = sm[qq[u]].rgb;
          const float w = al[u] * T;
          C0 += w * rgb.x;
          C1 += w * rgb.y;
          C2 += w * rgb.z;
          T = Tn;
          last = base + qq[u] + 1 - range.x;
        }
        continue;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, al[u]));
        const bool stop = ok[u] && !done && Tn < kTStop;
        const bool take = ok[u] && !done && !stop;
        done = done || stop;
        const float4 rgb = sm[qq[u]].rgb;
        const float w = al[u] * T;
        C0 = take ? C0 + w * rgb.x : C0;
        C1 = take ? C1 + w * rgb.y : C1;
        C2 = take ? C2 + w * rgb.z : C2;
        T = take ? Tn : T;
        last = take ? base + qq[u] + 1 - range.x : last;
      }
    }
  }
  if (has_pix) {
    out_rgb[3 * s] = C0 + T * a.bg[0];
    out_rgb[3 * s + 1] = C1 + T * a.bg[1];
    out_rgb[3 * s + 2] = C2 + T * a.bg[2];
    out_T[s] = T;
    out_last[s] = last;
  }
  return last;
}

// Several tiles per block for the warp-independent walk: wpt warps per tile
// (32 sampled pixels each), blockDim.x / (32 wpt) tiles per block, so that
// tiles of few sampled pixels (a warp each at 32 or fewer) still fill 8-warp
// blocks.  The block meets once, at the end, for each tile's longest blended
// run.
template <bool SELECT>
__global__ void __launch_bounds__(256) k_render_fwd_w(RasterArgs a, int wpt, float* __restrict__ out_rgb,
                                                      float* __restrict__ out_T, int32_t* __restrict__ out_last,
                                                      Ckpt ck) {
  __shared__ Splat sm[8][kCkptEvery];
  __shared__ int s_tl[8];
  const int warp = threadIdx.x >> 5;
  const int tpb = (int)(blockDim.x >> 5) / wpt;
  const int lt = warp / wpt, piece = warp - lt * wpt;
  const int n_act = *a.n_active;
  if (blockIdx.x * tpb >= n_act) return;  // the whole block
  const int j = blockIdx.x * tpb + lt < n_act ? blockIdx.x * tpb + lt : -1;
  if (threadIdx.x < 8) s_tl[threadIdx.x] = 0;
  __syncthreads();
  const int last = render_tile_fwd_warp<SELECT>(a, j, piece, sm[warp], out_rgb, out_T, out_last, ck);
  if (ck.tile_last) {  // the tile's longest blended run, for the pieces of the backward
    if (last > 0) atomicMax(&s_tl[lt], last);
    __syncthreads();
    if (j >= 0 && piece == 0 && (threadIdx.x & 31) == 0) ck.tile_last[j] = s_tl[lt];
  }
}

// ---------------------------------------------------------------------------
// Split forward (few active tiles: a sparse step).  One block per active
// tile holds NW groups of G threads, one thread per sampled pixel in each
// group.  In round r, group g walks run r NW + g of the tile's list (the 32
// positions [32 (r NW + g), 32 (r NW + g + 1))) from a local transmittance of
// 1, so the NW runs of a round are walked at once and the tile's walk is NW
// times shorter.  A run walked from T = 1 to local transmittance T_l and
// local colour D_l turns the state (T, C) in front of it into
// (T T_l, C + T D_l); the groups' results are composed per pixel in list
// order through shared memory.  The walk stops in the first run where the
// composed product falls below the stopping transmittance, or whose local
// walk stopped by itself (T_l (1 - alpha) < 1e-4 implies the same for the
// global T <= T_l); that run is walked again by its group from its true entry
// state to find the exact stopping splat.  Checkpoints (the state at the end
// of each run) are written from the composed state, as the sequential walk
// writes them, so the backward is unchanged.  The composition rounds
// differently from the sequential product (one more rounding per run); when
// the product lands within rounding of the stopping value and the re-walk
// does not stop, the walk ends at the end of that run.  Rounds repeat until
// every pixel has stopped or the list ends, so work past the tile's last
// stopping point is bounded by one round.
// ---------------------------------------------------------------------------
constexpr int kLocalStop = 64;  // flag bit beside the run-local last position (0..32)

__device__ __forceinline__ void compose_run(float& T, float& C0, float& C1, float& C2, const float4& e) {
  C0 = __fmaf_rn(T, e.y, C0);
  C1 = __fmaf_rn(T, e.z, C1);
  C2 = __fmaf_rn(T, e.w, C2);
  T = __fmul_rn(T, e.x);
}

template <int NW>
__global__ void k_render_fwd_split(RasterArgs a, float* __restrict__ out_rgb, float* __restrict__ out_T,
                                   int32_t* __restrict__ out_last, Ckpt ck) {
  extern __shared__ float4 smem_f4[];
  __shared__ int s_tl;
  const int j = blockIdx.x;
  if (j >= *a.n_active) return;
  const int G = blockDim.x / NW;
  Splat* sp = reinterpret_cast<Splat*>(smem_f4);           // [NW][32]
  float4* loc = reinterpret_cast<float4*>(sp + NW * 32);   // [NW][G] (T_l, D_l)
  float4* rec = loc + NW * G;                              // [NW][G] state after a stopping run
  int* lastl = reinterpret_cast<int*>(rec + NW * G);       // [NW][G] local last | kLocalStop
  int* rec_last = lastl + NW * G;                          // [NW][G]
  const int g = threadIdx.x / G, i = threadIdx.x - g * G;
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  const bool has_pix = p0 + i < p1;
  const int s = p0 + i;
  float px = 0.f, py = 0.f;
  if (has_pix) {
    const int l = a.pix_idx[s];
    px = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
    py = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
  }
  const int2 range = a.ranges[j];
  const int L = range.y - range.x;
  const int n_runs = (L + kCkptEvery - 1) / kCkptEvery;
  // the running state of pixel i in front of the current round (the same in every group)
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  bool done = !has_pix;
  const Splat* S = sp + 32 * g;
  Splat nxt;
  if (i < 32 && 32 * g + i < L) load_splat(a, range.x + 32 * g + i, nxt);
  for (int r0 = 0; r0 < n_runs; r0 += NW) {
    const int run = r0 + g;
    // the previous round's reads of sp ended before its second barrier
    if (i < 32 && 32 * run + i < L) sp[32 * g + i] = nxt;
    if (__syncthreads_count(done) == (int)blockDim.x) break;
    if (i < 32 && 32 * (run + NW) + i < L) load_splat(a, range.x + 32 * (run + NW) + i, nxt);
    // 1. the group's run from a local T = 1 (alphas of kUnroll splats together, blend with selects)
    const int cnt = min(kCkptEvery, L - 32 * run);
    float Tl = 1.f, D0 = 0.f, D1 = 0.f, D2 = 0.f;
    int ll = 0;
    bool lstop = false;
    if (!done && cnt > 0) {
      for (int q0 = 0; q0 < cnt && !lstop; q0 += kUnroll) {
        float al[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const float2 xy = S[q0 + u].xy;
          float Gv;
          ok[u] = splat_alpha_nb(S[q0 + u].co, __fsub_rn(px, xy.x), __fsub_rn(py, xy.y), al[u], Gv) &&
                  q0 + u < cnt;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const float Tn = __fmul_rn(Tl, __fsub_rn(1.f, al[u]));
          const bool stop = ok[u] && !lstop && Tn < kTStop;
          const bool take = ok[u] && !lstop && !stop;
          lstop = lstop || stop;
          const float4 rgb = S[q0 + u].rgb;
          const float w = al[u] * Tl;
          D0 = take ? D0 + w * rgb.x : D0;
          D1 = take ? D1 + w * rgb.y : D1;
          D2 = take ? D2 + w * rgb.z : D2;
          Tl = take ? Tn : Tl;
          ll = take ? q0 + u + 1 : ll;
        }
      }
    }
    loc[g * G + i] = make_float4(Tl, D0, D1, D2);
    lastl[g * G + i] = ll | (lstop ? kLocalStop : 0);
    __syncthreads();
    // 2. the state in front of this group's run; its checkpoint, or the exact stop inside it
    if (!done && cnt > 0) {
      float T2 = T, E0 = C0, E1 = C1, E2 = C2;
      int l2 = last;
      bool before = false;
      for (int h = 0; h < g; ++h) {
        const float4 e = loc[h * G + i];
        const int lh = lastl[h * G + i];
        if ((lh & kLocalStop) || __fmul_rn(T2, e.x) < kTStop) {
          before = true;
          break;
        }
        compose_run(T2, E0, E1, E2, e);
        if (lh) l2 = 32 * (r0 + h) + lh;
      }
      if (!before) {
        if (lstop || __fmul_rn(T2, Tl) < kTStop) {
          for (int q = 0; q < cnt; ++q) {  // the stopping run again, from its entry state
            const Splat& sq = S[q];
            float al, Gv;
            if (!splat_alpha(sq.co, __fsub_rn(px, sq.xy.x), __fsub_rn(py, sq.xy.y), al, Gv)) continue;
            const float Tn = __fmul_rn(T2, __fsub_rn(1.f, al));
            if (Tn < kTStop) break;
            const float w = al * T2;
            E0 += w * sq.rgb.x;
            E1 += w * sq.rgb.y;
            E2 += w * sq.rgb.z;
            T2 = Tn;
            l2 = 32 * run + q + 1;
          }
          rec[g * G + i] = make_float4(T2, E0, E1, E2);
          rec_last[g * G + i] = l2;
        } else if (ck.data && run < ck.n_slots) {
          compose_run(T2, E0, E1, E2, make_float4(Tl, D0, D1, D2));
          ck.data[run * ck.stride + s] = make_float4(T2, E0, E1, E2);  // in front of position 32 (run + 1)
        }
      }
    }
    __syncthreads();
    // 3. the running state over the whole round (every group the same)
    if (!done) {
#pragma unroll
      for (int h = 0; h < NW; ++h) {
        if (r0 + h >= n_runs) break;
        const float4 e = loc[h * G + i];
        const int lh = lastl[h * G + i];
        if ((lh & kLocalStop) || __fmul_rn(T, e.x) < kTStop) {
          const float4 q = rec[h * G + i];
          T = q.x;
          C0 = q.y;
          C1 = q.z;
          C2 = q.w;
          last = rec_last[h * G + i];
          done = true;
          break;
        }
        compose_run(T, C0, C1, C2, e);
        if (lh) last = 32 * (r0 + h) + lh;
      }
    }
  }
  if (g == 0 && has_pix) {
    out_rgb[3 * s] = C0 + T * a.bg[0];
    out_rgb[3 * s + 1] = C1 + T * a.bg[1];
    out_rgb[3 * s + 2] = C2 + T * a.bg[2];
    out_T[s] = T;
    out_last[s] = last;
  }
  if (ck.tile_last) {
    __syncthreads();
    if (threadIdx.x == 0) s_tl = 0;
    __syncthreads();
    if (g == 0 && last > 0) atomicMax(&s_tl, last);
    __syncthreads();
    if (threadIdx.x == 0) ck.tile_last[j] = s_tl;
  }
}

template <int NW>
size_t split_smem_bytes(int G) {
  return NW * 32 * sizeof(Splat) + (size_t)NW * G * (2 * sizeof(float4) + 2 * sizeof(int));
}

// The adjoints of a splat's centre and conic from the sums over its pixels of
// dL/dpower times dx, dy, dx^2, dx dy, dy^2 (power = -(a dx^2 + c dy^2)/2 -
// b dx dy, dx = px - x): dL/dx = a m1 + b m2, dL/dy = c m2 + b m1,
// dL/da = -m3 / 2, dL/db = -m4, dL/dc = -m5 / 2 (co: the pre-scaled conic).
__device__ __forceinline__ void power_moments_to_grad(const float4& co, float m1, float m2, float m3, float m4,
                                                      float m5, float (&g)[5]) {
  const float A = co.x * kInvA, Bc = co.y * kInvB, Cc = co.z * kInvA;
  g[0] = A * m1 + Bc * m2;
  g[1] = Cc * m2 + Bc * m1;
  g[2] = -0.5f * m3;
  g[3] = -m4;
  g[4] = -0.5f * m5;
}

// Sum of v[0..7] over the warp, scattered: lane l ends with the total of
// v[(l >> 2) & 7] (halving exchanges at distances 16, 8, 4, then a butterfly
// over the last two bits): 9 shuffles instead of 40.
__device__ __forceinline__ float warp_reduce_scatter8(const float (&v)[9], int lane) {
  float a4[4], b2[2];
  {
    const bool up = lane & 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float send = up ? v[k] : v[4 + k];
      const float keep = up ? v[4 + k] : v[k];
      a4[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float send = up ? a4[k] : a4[2 + k];
      const float keep = up ? a4[2 + k] : a4[k];
      b2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  const bool up = lane & 4;
  float c = (up ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, up ? b2[0] : b2[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// Sum of v[0..3] over the warp, scattered: lane l ends with the total of
// v[(l >> 3) & 3] (halving exchanges at distances 16 and 8, then a butterfly
// over the last three bits): 6 shuffles.
__device__ __forceinline__ float warp_reduce_scatter4(const float (&v)[4], int lane) {
  float b2[2];
  {
    const bool up = lane & 16;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float send = up ? v[k] : v[2 + k];
      const float keep = up ? v[2 + k] : v[k];
      b2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  const bool up = lane & 8;
  float c = (up ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, up ? b2[0] : b2[1], 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// Where the backward also accumulates the error back-projection statistics of
// Sec. 3.8 (Eq. 12): the per-pixel error e (from the loss) and the per-
// Gaussian rows (E, W, D, 0) they are added to.
struct StatsK {
  const float* err;
  float4* stats;
};

// Per-splat adjoints of a batch are summed over the block in shared memory
// (acc, 9 floats per batch slot) and flushed once per block and splat with
// vector atomics, instead of once per warp and splat.
__device__ __forceinline__ void render_tile_bwd(const RasterArgs& a, int j, Splat* sm,
                                                const float* __restrict__ T_final, const int32_t* __restrict__ n_last,
                                                const float* __restrict__ dL_drgb, float* __restrict__ grad2d) {
  __shared__ int s_max_last;
  float* acc = reinterpret_cast<float*>(sm + blockDim.x);
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  const bool has_pix = p0 + (int)threadIdx.x < p1;
  const int s = p0 + threadIdx.x;
  float px = 0.f, py = 0.f, T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  int last = 0;
  if (has_pix) {
    const int l = a.pix_idx[s];
    px = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
    py = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
    T = T_final[s];
    last = n_last[s];
    g0 = dL_drgb[3 * s];
    g1 = dL_drgb[3 * s + 1];
    g2 = dL_drgb[3 * s + 2];
  }
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  if (last > 0) atomicMax(&s_max_last, last);
  __syncthreads();
  const int2 range = a.ranges[j];
  const int end = range.x + s_max_last;  // no pixel blended anything past here
  float S0 = a.bg[0], S1 = a.bg[1], S2 = a.bg[2];
  const int B = blockDim.x;
  const int lane = threadIdx.x & 31;
  int warp_last = last;  // the warp skips splats none of its pixels blended
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) warp_last = max(warp_last, __shfl_xor_sync(0xffffffffu, warp_last, o));
  const float2 band = warp_rows(last > 0, py);  // and splats that cannot reach its rows
  // the next batch's records are fetched into registers while the current
  // one is replayed, and the list entries (ids) of the batch after it
  SplatRaw nxt;
  int idn = 0;
  {
    const int k = end - B + (int)threadIdx.x;
    if (end > range.x && k >= range.x) fetch_splat(a, a.vals[k], nxt);
    if (end > range.x && k - B >= range.x) idn = a.vals[k - B];
  }
  for (int top = end; top > range.x; top -= B) {
    const int lo = max(range.x, top - B);
    const int cnt = top - lo;
    __syncthreads();
    // batch [top - B, top) was fetched into slot threadIdx.x - (B - cnt)
    {
      const int k = top - B + (int)threadIdx.x;
      if (k >= range.x) finish_splat(nxt, sm[threadIdx.x - (B - cnt)]);
#pragma unroll
      for (int c = 0; c < 9; ++c) acc[9 * threadIdx.x + c] = 0.f;
    }
    __syncthreads();
    {
      const int k = top - 2 * B + (int)threadIdx.x;
      if (k >= range.x) fetch_splat(a, idn, nxt);
      if (k - B >= range.x) idn = a.vals[k - B];
    }
    const int qmax = min(cnt - 1, range.x + warp_last - 1 - lo);
    for (int q = qmax; q >= 0; --q) {
      const Splat sp = sm[q];
      const int pos = lo + q - range.x;  // position in the tile list
      float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool hit = false;
      if (sp.yr.y < band.x || sp.yr.x > band.y) continue;  // warp-uniform: no pixel of the warp is reached
      if (pos < last) {
        const float dx = __fsub_rn(px, sp.xy.x), dy = __fsub_rn(py, sp.xy.y);
        float alpha, G;
        if (splat_alpha(sp.co, dx, dy, alpha, G)) {
          hit = true;
          T = __fdividef(T, 1.f - alpha);  // transmittance in front of this splat (1 - alpha >= 0.01)
          const float wgt = alpha * T;
          v[6] = wgt * g0;
          v[7] = wgt * g1;
          v[8] = wgt * g2;
          const float e0 = sp.rgb.x - S0, e1 = sp.rgb.y - S1, e2 = sp.rgb.z - S2;
          const float dalpha = T * (e0 * g0 + e1 * g1 + e2 * g2);
          S0 += alpha * e0;  // the light seen behind the splat in front
          S1 += alpha * e1;
          S2 += alpha * e2;
          if (alpha < kAlphaMax) {  // not clamped
            v[5] = dalpha * G;
            const float dpow = dalpha * alpha;
            const float tx = dpow * dx, ty = dpow * dy;
            v[0] = tx;  // the moments of dL/dpower; the conic is applied per splat
            v[1] = ty;
            v[2] = tx * dx;
            v[3] = tx * dy;
            v[4] = ty * dy;
          }
        }
      }
      if (__any_sync(0xffffffffu, hit)) {
        const float r8 = warp_reduce_scatter8(v, lane);
        const float r9 = warp_sum(v[8]);
        if ((lane & 3) == 0) atomicAdd(acc + 9 * q + ((lane >> 2) & 7), r8);
        else if (lane == 1) atomicAdd(acc + 9 * q + 8, r9);
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const float* r = acc + 9 * threadIdx.x;
      if (r[0] != 0.f || r[1] != 0.f || r[2] != 0.f || r[3] != 0.f || r[4] != 0.f || r[5] != 0.f ||
          r[6] != 0.f || r[7] != 0.f || r[8] != 0.f) {
        const Splat& sq = sm[threadIdx.x];
        float* gp = grad2d + 12 * (size_t)__float_as_int(sq.rgb.w);
        float gc[5];
        power_moments_to_grad(sq.co, r[0], r[1], r[2], r[3], r[4], gc);
        red_add_v4(gp, gc[0], gc[1], gc[2], gc[3]);
        red_add_v4(gp + 4, gc[4], r[5], r[6], r[7]);
        atomicAdd(gp + 8, r[8]);
      }
    }
  }
}

__global__ void k_render_bwd(RasterArgs a, const float* __restrict__ T_final, const int32_t* __restrict__ n_last,
                             const float* __restrict__ dL_drgb, float* __restrict__ grad2d) {
  extern __shared__ Splat sm[];
  const int j = blockIdx.x;
  if (j >= *a.n_active) return;
  render_tile_bwd(a, j, sm, T_final, n_last, dL_drgb, grad2d);
}

// Split backward, one warp per piece: piece c of tile j is list positions
// [c E, (c + 1) E) (E = kCkptEvery), or from n_slots E to the end for
// c = n_slots, replayed for every sampled pixel of the tile, PPL pixels per
// lane (pixel p0 + lane + 32 u).  A pixel whose last blended splat lies in
// the piece starts from (T_final, bg); one whose walk goes on past it starts
// from the forward's checkpoint at the piece's back edge, with the light
// from behind recovered as S = (out - C) / T (out = T-weighted colours +
// T_final bg).  The lane first sums its pixels' adjoints of a splat in
// registers, so one warp reduction serves 32 PPL pixels, and the warp's
// totals go straight to the Gaussian's gradient row (two vector atomics and
// one scalar).  Warps never wait on each other: each stages its splats, one
// per lane, in its own slice of shared memory (sm, 32 entries).
//
// STATS: the same replay also sums, per splat, Eq. 12's e w, w and D w over
// the pixels (w = T alpha the compositing weight, e the pixel's error, D the
// conic Mahalanobis distance of the pixel centre) into its statistics row.
template <int PPL, bool STATS>
__device__ __forceinline__ void render_piece_bwd_warp(const RasterArgs& a, int j, int c, Splat* sm,
                                                      const float* __restrict__ T_final,
                                                      const int32_t* __restrict__ n_last,
                                                      const float* __restrict__ dL_drgb,
                                                      float* __restrict__ grad2d, const Ckpt& ck,
                                                      const StatsK st = StatsK{nullptr, nullptr}) {
  constexpr int E = kCkptEvery;
  const int lane = threadIdx.x & 31;
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  int max_last;
  if (ck.tile_last) {
    max_last = ck.tile_last[j];  // from the forward
  } else {
    int m = 0;
#pragma unroll
    for (int u = 0; u < PPL; ++u) {
      const int s = p0 + lane + 32 * u;
      if (s < p1) m = max(m, n_last[s]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    max_last = m;
  }
  const int lo_pos = c * E;
  const int hi_pos = c < ck.n_slots ? min(lo_pos + E, max_last) : max_last;
  if (hi_pos <= lo_pos) return;  // warp-uniform: nothing blended here
  float px[PPL], py[PPL], T[PPL], g0[PPL], g1[PPL], g2[PPL], S0[PPL], S1[PPL], S2[PPL];
  float ep[STATS ? PPL : 1];
  int last[PPL];
  int warp_last = 0;
#pragma unroll
  for (int u = 0; u < PPL; ++u) {
    const int s = p0 + lane + 32 * u;
    last[u] = s < p1 ? n_last[s] : 0;
    if (last[u] <= lo_pos) last[u] = 0;  // this pixel blended nothing in the piece
    px[u] = py[u] = 0.f;
    T[u] = 1.f;
    g0[u] = g1[u] = g2[u] = 0.f;
    if (STATS) ep[u] = last[u] > 0 ? st.err[s] : 0.f;
    S0[u] = a.bg[0];
    S1[u] = a.bg[1];
    S2[u] = a.bg[2];
    if (last[u] > 0) {
      const int l = a.pix_idx[s];
      px[u] = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
      py[u] = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
      g0[u] = dL_drgb[3 * s];
      g1[u] = dL_drgb[3 * s + 1];
      g2[u] = dL_drgb[3 * s + 2];
      if (c < ck.n_slots && last[u] > lo_pos + E) {
        const float4 q = ck.data[c * ck.stride + s];  // in front of position (c + 1) E
        T[u] = q.x;
        const float iT = 1.f / q.x;
        S0[u] = (ck.rgb[3 * s] - q.y) * iT;
        S1[u] = (ck.rgb[3 * s + 1] - q.z) * iT;
        S2[u] = (ck.rgb[3 * s + 2] - q.w) * iT;
        last[u] = lo_pos + E;
      } else {
        T[u] = T_final[s];
      }
    }
    warp_last = max(warp_last, last[u]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) warp_last = max(warp_last, __shfl_xor_sync(0xffffffffu, warp_last, o));
  // slot u of the lanes holds 32 consecutive sampled pixels (row-major): a band of rows; a splat
  // outside a slot's band is skipped for that slot by the whole warp
  float2 band[PPL];
#pragma unroll
  for (int u = 0; u < PPL; ++u) band[u] = warp_rows(last[u] > 0, py[u]);
  const int2 range = a.ranges[j];
  const int first = range.x + lo_pos, end = range.x + min(hi_pos, warp_last);
  for (int top = end; top > first; top -= 32) {
    const int lo = max(first, top - 32);
    __syncwarp();
    if (lo + lane < top) load_splat(a, lo + lane, sm[lane]);
    __syncwarp();
    for (int q = top - lo - 1; q >= 0; --q) {
      const Splat sp = sm[q];
      const int pos = lo + q - range.x;  // position in the tile list
      float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float sv[4] = {0.f, 0.f, 0.f, 0.f};
      bool hit = false;
#pragma unroll
      for (int u = 0; u < PPL; ++u) {
        if (sp.yr.y < band[u].x || sp.yr.x > band[u].y) continue;  // warp-uniform
        if (pos >= last[u]) continue;
        const float dx = __fsub_rn(px[u], sp.xy.x), dy = __fsub_rn(py[u], sp.xy.y);
        float alpha, G, pw;
        if (!splat_alpha_p(sp.co, dx, dy, alpha, G, pw)) continue;
        hit = true;
        T[u] = __fdividef(T[u], 1.f - alpha);  // transmittance in front of this splat (1 - alpha >= 0.01)
        const float wgt = alpha * T[u];
        if (STATS) {
          // a dx^2 + 2 b dx dy + c dy^2 = -2 power = -2 ln(2) p
          const float D = sqrtf(fmaxf(pw * kInvA, 0.f));
          sv[0] += ep[u] * wgt;
          sv[1] += wgt;
          sv[2] += D * wgt;
        }
        v[6] += wgt * g0[u];
        v[7] += wgt * g1[u];
        v[8] += wgt * g2[u];
        const float e0 = sp.rgb.x - S0[u], e1 = sp.rgb.y - S1[u], e2 = sp.rgb.z - S2[u];
        const float dalpha = T[u] * (e0 * g0[u] + e1 * g1[u] + e2 * g2[u]);
        S0[u] += alpha * e0;  // the light seen behind the splat in front
        S1[u] += alpha * e1;
        S2[u] += alpha * e2;
        if (alpha < kAlphaMax) {  // not clamped
          v[5] += dalpha * G;
          const float dpow = dalpha * alpha;
          const float tx = dpow * dx, ty = dpow * dy;
          v[0] += tx;  // the moments of dL/dpower; the conic is applied per splat
          v[1] += ty;
          v[2] += tx * dx;
          v[3] += tx * dy;
          v[4] += ty * dy;
        }
      }
      if (!__any_sync(0xffffffffu, hit)) continue;
      const float r8 = warp_reduce_scatter8(v, lane);  // lane 4 k + (0..3): component k
      const float r9 = warp_sum(v[8]);
      // components 0..3 to lane 0, 4..7 to lane 16
      const float c1 = __shfl_down_sync(0xffffffffu, r8, 4);
      const float c2 = __shfl_down_sync(0xffffffffu, r8, 8);
      const float c3 = __shfl_down_sync(0xffffffffu, r8, 12);
      float* gp = grad2d + 12 * (size_t)__float_as_int(sp.rgb.w);
      if (lane == 0) {
        float gc[5];
        power_moments_to_grad(sp.co, r8, c1, c2, c3, 0.f, gc);
        red_add_v4(gp, gc[0], gc[1], gc[2], gc[3]);
      } else if (lane == 16) {
        red_add_v4(gp + 4, -0.5f * r8, c1, c2, c3);  // dL/dc from the dy^2 moment
      } else if (lane == 1) {
        atomicAdd(gp + 8, r9);
      }
      if (STATS) {
        const float rs = warp_reduce_scatter4(sv, lane);  // lane 8 k + (0..7): statistic k
        const float s1 = __shfl_down_sync(0xffffffffu, rs, 8);
        const float s2 = __shfl_down_sync(0xffffffffu, rs, 16);
        if (lane == 0) red_add_v4(reinterpret_cast<float*>(st.stats + __float_as_int(sp.rgb.w)), rs, s1, s2, 0.f);
      }
    }
  }
}

constexpr int kBwdWarps = 4;  // pieces per block of the one-view split backward

template <int PPL, bool STATS>
__global__ void __launch_bounds__(32 * kBwdWarps, PPL <= 3 ? 7 : 1)
    k_render_bwd_warp(RasterArgs a, const float* __restrict__ T_final, const int32_t* __restrict__ n_last,
                      const float* __restrict__ dL_drgb, float* __restrict__ grad2d, Ckpt ck, StatsK st) {
  __shared__ Splat sm[kBwdWarps][32];
  const int j = blockIdx.x;
  if (j >= *a.n_active) return;
  const int w = threadIdx.x >> 5;
  const int c = blockIdx.y * kBwdWarps + w;
  if (c > ck.n_slots) return;  // warp-uniform; the kernel has no block-wide barrier
  render_piece_bwd_warp<PPL, STATS>(a, j, c, sm[w], T_final, n_last, dL_drgb, grad2d, ck, st);
}

// Error back-projection statistics (Sec. 3.8, Eq. 12): one
// block per active tile, one thread per sampled pixel, walking the tile's
// list front to back up to the pixel's n_last (the forward's stopping
// decision) and recomputing alpha and T as the forward does.  For each splat
// the warp sums (e w, w, D w) over its pixels (w = T alpha, D the conic
// Mahalanobis distance) and one lane adds them to the Gaussian's float4 row.
__global__ void k_error_stats(RasterArgs a, const int32_t* __restrict__ n_last, const float* __restrict__ err_pix,
                              float* __restrict__ stats) {
  extern __shared__ Splat sm[];
  __shared__ int s_max_last;
  const int j = blockIdx.x;
  if (j >= *a.n_active) return;
  const int t = a.active_tiles ? a.active_tiles[j] : j;
  const int p0 = a.pix_off[j], p1 = a.pix_off[j + 1];
  const bool has_pix = p0 + (int)threadIdx.x < p1;
  const int s = p0 + threadIdx.x;
  const int lane = threadIdx.x & 31;
  float px = 0.f, py = 0.f, e = 0.f, T = 1.f;
  int last = 0;
  if (has_pix) {
    const int l = a.pix_idx[s];
    px = (float)((t % a.tiles_x) * TGS_TILE + (l & 15)) + 0.5f;
    py = (float)((t / a.tiles_x) * TGS_TILE + (l >> 4)) + 0.5f;
    e = err_pix[s];
    last = n_last[s];
  }
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  if (last > 0) atomicMax(&s_max_last, last);
  __syncthreads();
  const int2 range = a.ranges[j];
  const int end = range.x + s_max_last;
  const int B = blockDim.x;
  const float2 band = warp_rows(last > 0, py);  // splats that cannot reach the warp's rows are skipped
  for (int base = range.x; base < end; base += B) {
    __syncthreads();  // the previous batch is no longer read
    if (base + (int)threadIdx.x < end) load_splat(a, base + threadIdx.x, sm[threadIdx.x]);
    __syncthreads();
    const int cnt = min(B, end - base);
    for (int q = 0; q < cnt; ++q) {
      const Splat sp = sm[q];
      if (sp.yr.y < band.x || sp.yr.x > band.y) continue;  // warp-uniform
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      bool on = false;
      if (base + q - range.x < last) {
        const float dx = __fsub_rn(px, sp.xy.x), dy = __fsub_rn(py, sp.xy.y);
        float alpha, G;
        if (splat_alpha(sp.co, dx, dy, alpha, G)) {
          const float w = alpha * T;
          // a dx^2 + 2 b dx dy + c dy^2 = -2 power = -2 ln(2) p
          const float qf = splat_pow2(sp.co, dx, dy) * kInvA;
          const float D = sqrtf(fmaxf(qf, 0.f));
          v0 = e * w;
          v1 = w;
          v2 = D * w;
          T = __fmul_rn(T, __fsub_rn(1.f, alpha));  // the forward's transmittance sequence
          on = true;
        }
      }
      if (!__any_sync(0xffffffffu, on)) continue;
      v0 = warp_sum(v0);
      v1 = warp_sum(v1);
      v2 = warp_sum(v2);
      if (lane == 0) red_add_v4(stats + 4 * (size_t)__float_as_int(sp.rgb.w), v0, v1, v2, 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// Several views in one persistent launch: CTAs take (view, tile) items from
// an atomic counter (items of view v are [base[v], base[v+1])) until none
// are left.  There is no waiting on other CTAs, only one atomic per item.
// ---------------------------------------------------------------------------
constexpr int kMaxViews = 16;

struct BatchArgs {
  int n_views;
  int pieces;  // backward items per tile: 1, or checkpoint slots + 1
  int base[kMaxViews + 1];
  RasterArgs a[kMaxViews];
  float* rgb[kMaxViews];
  float* T[kMaxViews];
  int32_t* last[kMaxViews];
  const float* dL[kMaxViews];
  float* grad2d[kMaxViews];
  Ckpt ck[kMaxViews];
  const float* err[kMaxViews];  // per-pixel errors, when the statistics are accumulated
  float4* stats;                // [N] (E, W, D, 0) rows shared by the views
};

__device__ __forceinline__ bool next_item(const BatchArgs& b, int* counter, int* s_item, int& v, int& j) {
  __syncthreads();  // the previous item's shared memory is no longer read
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
  __syncthreads();
  const int item = *s_item;
  if (item >= b.base[b.n_views]) return false;
  v = 0;
  while (item >= b.base[v + 1]) ++v;
  j = item - b.base[v];
  return true;
}

// The same, claiming `step` consecutive items per atomic: the first is
// returned in *first (shared), the caller walks them.
__device__ __forceinline__ bool next_items(const BatchArgs& b, int* counter, int* s_item, int step, int& first) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, step);
  __syncthreads();
  first = *s_item;
  return first < b.base[b.n_views];
}

__device__ __forceinline__ void item_view(const BatchArgs& b, int item, int& v, int& q) {
  v = 0;
  while (item >= b.base[v + 1]) ++v;
  q = item - b.base[v];
}

__global__ void k_render_fwd_batched(BatchArgs b, int* __restrict__ counter) {
  extern __shared__ Splat sm[];
  __shared__ int s_item;
  int v, j;
  while (next_item(b, counter, &s_item, v, j)) {
    if (j < *b.a[v].n_active) render_tile_fwd<false>(b.a[v], j, sm, b.rgb[v], b.T[v], b.last[v], b.ck[v]);
  }
}

// Whole tiles, one item per block (the backward without checkpoints).
__global__ void k_render_bwd_batched(BatchArgs b, int* __restrict__ counter) {
  extern __shared__ Splat sm[];
  __shared__ int s_item;
  int v, q;
  while (next_item(b, counter, &s_item, v, q))
    if (q < *b.a[v].n_active) render_tile_bwd(b.a[v], q, sm, b.T[v], b.last[v], b.dL[v], b.grad2d[v]);
}

// With checkpoints: items are (view, tile, piece) with the pieces of a tile
// consecutive; each warp claims kPieceClaim of them per atomic and replays
// them as the one-view split backward does.
constexpr int kPieceClaim = 4;
constexpr int kBatchBwdWarps = 4;

template <int PPL, bool STATS>
__global__ void __launch_bounds__(32 * kBatchBwdWarps) k_render_bwd_batched_warp(BatchArgs b,
                                                                                int* __restrict__ counter) {
  __shared__ Splat sm[kBatchBwdWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int total = b.base[b.n_views];
  for (;;) {
    int first = 0;
    if (lane == 0) first = atomicAdd(counter, kPieceClaim);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= total) return;
    const int end = min(first + kPieceClaim, total);
    for (int item = first; item < end; ++item) {
      int v, q;
      item_view(b, item, v, q);
      const int j = q / b.pieces, c = q - j * b.pieces;
      if (j >= *b.a[v].n_active) continue;
      render_piece_bwd_warp<PPL, STATS>(b.a[v], j, c, sm[w], b.T[v], b.last[v], b.dL[v], b.grad2d[v], b.ck[v],
                                        StatsK{b.err[v], b.stats});
    }
  }
}

static bool raster_args(const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals,
                        const int32_t* active_tiles, const int32_t* n_active, const int32_t* pix_off,
                        const uint8_t* pix_idx, const tgs_camera* cam, const float* bg, RasterArgs& a) {
  if (!proj || !proj->xy || !proj->conic_opac || !proj->rgb || !tile_ranges || !vals || !n_active || !pix_off ||
      !pix_idx || !camera_ok(cam) || !bg)
    return false;
  if (!aligned8(proj->xy) || !aligned16(proj->conic_opac) || !aligned8(tile_ranges)) return false;
  a.xy = reinterpret_cast<const float2*>(proj->xy);
  a.conic_opac = reinterpret_cast<const float4*>(proj->conic_opac);
  a.rgb = proj->rgb;
  a.ranges = reinterpret_cast<const int2*>(tile_ranges);
  a.vals = vals;
  a.active_tiles = active_tiles;
  a.n_active = n_active;
  a.pix_off = pix_off;
  a.pix_idx = pix_idx;
  a.tiles_x = tiles_x(cam->width);
  a.bg[0] = bg[0];
  a.bg[1] = bg[1];
  a.bg[2] = bg[2];
  return true;
}

static int block_for(int n_pix_max) { return std::min(256, std::max(32, (n_pix_max + 31) / 32 * 32)); }


// Whether the automatic choice may pick the split walk: measured slower than
// the sequential walk at 500k Gaussians, 720 tiles of 85 pixels (0.085-0.089
// against 0.067 ms), so only an explicit setting selects it.
constexpr bool kSplitAuto = false;

// The split forward's group count: 0 = chosen per launch (below), or fixed
// at 1, 2 or 4 by tgs_set_forward_split (tuning and tests).
static int g_fwd_split = 0;

// The automatic choice of the walk with two threads per pixel: for tiles of
// at most 32 sampled pixels in a sparse launch, where one warp per tile
// leaves the GPU short of warps.  Measured at 500k Gaussians, 1280x720, 720
// tiles of 25 pixels: 0.046 ms, against 0.054 for the warp-independent walk
// (eight tiles per block) and 0.064 for one 32-thread block per tile.  At 85
// pixels per tile (0.068 against 0.060) and in launches of several waves
// (3600 tiles of 85 pixels: 0.216 against 0.162) the sequential block walk
// stays faster: the composition and the second half's walk past the stop
// cost more than the shorter chains gain.
static bool pair_walk_auto(int B, bool sparse) { return B == 32 && sparse; }

// Groups per tile of the split forward for a launch of n_active tiles of B
// threads: the largest of 4 and 2 whose blocks all fit on the GPU at once
// (one wave), else 1 (the sequential walk).

static int split_groups(int n_active, int B) {
  const int wp = B / 32;  // 1..8
  const bool nw_ok[2] = {4 * B <= 1024, 2 * B <= 1024};
  if (g_fwd_split == 1 || g_fwd_split == 3 || g_fwd_split == 5) return 1;
  if (g_fwd_split) return (g_fwd_split == 4 && !nw_ok[0]) || (g_fwd_split == 2 && !nw_ok[1]) ? 1 : g_fwd_split;
  if (!kSplitAuto) return 1;
  static int per_sm[64][9][2] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  const int sms = device_sm_count();
  for (int k = 0; k < 2; ++k) {
    const int nw = k == 0 ? 4 : 2;
    if (!nw_ok[k]) continue;
    int& r = per_sm[dev][wp][k];
    if (r == 0) {
      int b = 0;
      if (nw == 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_render_fwd_split<4>, 4 * B, split_smem_bytes<4>(B));
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_render_fwd_split<2>, 2 * B, split_smem_bytes<2>(B));
      r = b > 0 ? b : -1;
    }
    if (r > 0 && (int64_t)n_active <= (int64_t)sms * r) return nw;
  }
  return 1;
}

}  // namespace tgs

using namespace tgs;

// Checkpoint buffer checks: stride covers every sampled pixel slot.
static bool ckpt_of(const tgs_checkpoints* c, int32_t n_active_max, int32_t n_pix_max, const float* rgb, Ckpt& k) {
  k = Ckpt{nullptr, 0, 0, nullptr, nullptr};
  if (!c || c->n_slots <= 0) return true;
  if (!c->data || !aligned16(c->data) || c->stride < (int64_t)n_active_max * n_pix_max) return false;
  k.data = reinterpret_cast<float4*>(c->data);
  k.n_slots = c->n_slots;
  k.stride = c->stride;
  k.rgb = rgb;
  k.tile_last = c->tile_last;
  return true;
}

extern "C" tgs_status tgs_set_forward_split(int32_t groups) {
  if (groups < 0 || groups > 5) return TGS_ERR_INVALID_ARG;
  g_fwd_split = groups;
  return TGS_OK;
}

extern "C" size_t tgs_checkpoint_bytes(int32_t n_active_max, int32_t n_pix_max, int32_t n_slots) {
  if (n_active_max <= 0 || n_pix_max <= 0 || n_slots <= 0) return 0;
  return sizeof(float4) * (size_t)n_slots * (size_t)n_active_max * (size_t)n_pix_max;
}

extern "C" tgs_status tgs_render_sampled(const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals,
                                         const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                                         const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                                         const tgs_camera* cam, const float* bg, float* rgb, float* T_final,
                                         int32_t* n_last, const tgs_checkpoints* ckpt, tgs_stream stream) {
  RasterArgs a;
  if (n_active_max < 0 || n_pix_max < 1 || n_pix_max > 256) return TGS_ERR_INVALID_ARG;
  if (!raster_args(proj, tile_ranges, vals, active_tiles, n_active, pix_off, pix_idx, cam, bg, a))
    return TGS_ERR_INVALID_ARG;
  if (!rgb || !T_final || !n_last) return TGS_ERR_INVALID_ARG;
  Ckpt ck;
  if (!ckpt_of(ckpt, n_active_max, n_pix_max, rgb, ck)) return TGS_ERR_INVALID_ARG;
  if (n_active_max == 0) return TGS_OK;
  const int B = block_for(n_pix_max);
  // sampled training (checkpoints) with few tiles: the split walk, NW groups per tile
  const int nw = ck.data ? split_groups(n_active_max, B) : 1;
  if (nw == 4) {
    k_render_fwd_split<4><<<n_active_max, 4 * B, split_smem_bytes<4>(B), (cudaStream_t)stream>>>(a, rgb, T_final,
                                                                                                 n_last, ck);
    return check_launch();
  }
  if (nw == 2) {
    k_render_fwd_split<2><<<n_active_max, 2 * B, split_smem_bytes<2>(B), (cudaStream_t)stream>>>(a, rgb, T_final,
                                                                                                 n_last, ck);
    return check_launch();
  }
  // selects when the launch gives fewer than 16 warps per SM
  const bool sparse = (int64_t)n_active_max * (B / 32) < 16 * (int64_t)device_sm_count();
  if (g_fwd_split == 5 || (g_fwd_split == 0 && pair_walk_auto(B, sparse))) {  // two threads per pixel
    const int B2 = 32 * ((n_pix_max + 15) / 16);
    if (sparse)
      k_render_fwd_pair<true><<<n_active_max, B2, B2 * sizeof(Splat), (cudaStream_t)stream>>>(a, rgb, T_final, n_last,
                                                                                              ck);
    else
      k_render_fwd_pair<false><<<n_active_max, B2, B2 * sizeof(Splat), (cudaStream_t)stream>>>(a, rgb, T_final,
                                                                                               n_last, ck);
    return check_launch();
  }
  if (g_fwd_split == 3) {
    const int wpt = B / 32, tpb = 8 / wpt;
    const int grid = (n_active_max + tpb - 1) / tpb;
    if (sparse)
      k_render_fwd_w<true><<<grid, 32 * wpt * tpb, 0, (cudaStream_t)stream>>>(a, wpt, rgb, T_final, n_last, ck);
    else
      k_render_fwd_w<false><<<grid, 32 * wpt * tpb, 0, (cudaStream_t)stream>>>(a, wpt, rgb, T_final, n_last, ck);
    return check_launch();
  }
  if (sparse)
    k_render_fwd<true><<<n_active_max, B, B * sizeof(Splat), (cudaStream_t)stream>>>(a, rgb, T_final, n_last, ck);
  else
    k_render_fwd<false><<<n_active_max, B, B * sizeof(Splat), (cudaStream_t)stream>>>(a, rgb, T_final, n_last, ck);
  return check_launch();
}

// The one-view backward; with st.stats set, Eq. 12's statistics of the same
// pixels too (fused into the warp-per-piece replay, or as the separate pass
// after the whole-tile backward).
static tgs_status render_backward_impl(const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals,
                                       const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                                       const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                                       const tgs_camera* cam, const float* bg, const float* T_final,
                                       const int32_t* n_last, const float* dL_drgb, float* grad2d,
                                       int64_t n_gaussians, const tgs_checkpoints* ckpt, StatsK st,
                                       int32_t accumulate_stats, tgs_stream stream) {
  RasterArgs a;
  if (n_gaussians < 0 || n_active_max < 0 || n_pix_max < 1 || n_pix_max > 256) return TGS_ERR_INVALID_ARG;
  if (!raster_args(proj, tile_ranges, vals, active_tiles, n_active, pix_off, pix_idx, cam, bg, a))
    return TGS_ERR_INVALID_ARG;
  if (!T_final || !n_last || !dL_drgb) return TGS_ERR_INVALID_ARG;
  if (n_gaussians > 0 && (!grad2d || !aligned16(grad2d))) return TGS_ERR_INVALID_ARG;
  const bool stats = st.stats != nullptr;
  Ckpt ck;
  if (!ckpt_of(ckpt, n_active_max, n_pix_max, ckpt ? ckpt->rgb : nullptr, ck)) return TGS_ERR_INVALID_ARG;
  if (ck.data && !ck.rgb) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_gaussians == 0) return TGS_OK;
  cudaMemsetAsync(grad2d, 0, sizeof(float) * 12 * (size_t)n_gaussians, s);
  if (stats && !accumulate_stats) cudaMemsetAsync(st.stats, 0, sizeof(float4) * (size_t)n_gaussians, s);
  if (n_active_max > 0) {
    const int B = block_for(n_pix_max);
    const size_t smem = B * (sizeof(Splat) + 9 * sizeof(float));
    if (ck.data) {
      // one warp per piece, kBwdWarps pieces per block, B / 32 pixels per lane
      const dim3 grid(n_active_max, (ck.n_slots + 1 + kBwdWarps - 1) / kBwdWarps);
      switch ((B / 32) * 2 + (stats ? 1 : 0)) {
#define TGS_BWD_WARP(P)                                                                                         \
  case 2 * P: k_render_bwd_warp<P, false><<<grid, 32 * kBwdWarps, 0, s>>>(a, T_final, n_last, dL_drgb, grad2d, \
                                                                         ck, st); break;                       \
  case 2 * P + 1: k_render_bwd_warp<P, true><<<grid, 32 * kBwdWarps, 0, s>>>(a, T_final, n_last, dL_drgb,       \
                                                                            grad2d, ck, st); break;
        TGS_BWD_WARP(1) TGS_BWD_WARP(2) TGS_BWD_WARP(3) TGS_BWD_WARP(4)
        TGS_BWD_WARP(5) TGS_BWD_WARP(6) TGS_BWD_WARP(7) TGS_BWD_WARP(8)
#undef TGS_BWD_WARP
        default: break;
      }
    } else {
      k_render_bwd<<<n_active_max, B, smem, s>>>(a, T_final, n_last, dL_drgb, grad2d);
      if (stats)
        k_error_stats<<<n_active_max, B, B * sizeof(Splat), s>>>(a, n_last, st.err, reinterpret_cast<float*>(st.stats));
    }
  }
  return check_launch();
}

extern "C" tgs_status tgs_render_backward_sampled(const tgs_projected* proj, const int32_t* tile_ranges,
                                                  const int32_t* vals, const int32_t* active_tiles,
                                                  const int32_t* n_active, int32_t n_active_max,
                                                  const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                                                  const tgs_camera* cam, const float* bg, const float* T_final,
                                                  const int32_t* n_last, const float* dL_drgb, float* grad2d,
                                                  int64_t n_gaussians, const tgs_checkpoints* ckpt,
                                                  tgs_stream stream) {
  return render_backward_impl(proj, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                              n_pix_max, cam, bg, T_final, n_last, dL_drgb, grad2d, n_gaussians, ckpt,
                              StatsK{nullptr, nullptr}, 0, stream);
}

extern "C" tgs_status tgs_render_backward_sampled_stats(
    const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals, const int32_t* active_tiles,
    const int32_t* n_active, int32_t n_active_max, const int32_t* pix_off, const uint8_t* pix_idx,
    int32_t n_pix_max, const tgs_camera* cam, const float* bg, const float* T_final, const int32_t* n_last,
    const float* dL_drgb, float* grad2d, int64_t n_gaussians, const tgs_checkpoints* ckpt, const float* err_pix,
    float* stats, int32_t accumulate_stats, tgs_stream stream) {
  if (!err_pix || (n_gaussians > 0 && (!stats || !aligned16(stats)))) return TGS_ERR_INVALID_ARG;
  return render_backward_impl(proj, tile_ranges, vals, active_tiles, n_active, n_active_max, pix_off, pix_idx,
                              n_pix_max, cam, bg, T_final, n_last, dL_drgb, grad2d, n_gaussians, ckpt,
                              StatsK{err_pix, reinterpret_cast<float4*>(stats)}, accumulate_stats, stream);
}

extern "C" tgs_status tgs_error_stats_sampled(const tgs_projected* proj, const int32_t* tile_ranges,
                                              const int32_t* vals, const int32_t* active_tiles,
                                              const int32_t* n_active, int32_t n_active_max, const int32_t* pix_off,
                                              const uint8_t* pix_idx, int32_t n_pix_max, const tgs_camera* cam,
                                              const int32_t* n_last, const float* err_pix, float* stats,
                                              int64_t n_gaussians, int32_t accumulate, tgs_stream stream) {
  RasterArgs a;
  const float bg[3] = {0.f, 0.f, 0.f};
  if (n_gaussians < 0 || n_active_max < 0 || n_pix_max < 1 || n_pix_max > 256) return TGS_ERR_INVALID_ARG;
  if (!raster_args(proj, tile_ranges, vals, active_tiles, n_active, pix_off, pix_idx, cam, bg, a))
    return TGS_ERR_INVALID_ARG;
  if (!n_last || !err_pix) return TGS_ERR_INVALID_ARG;
  if (n_gaussians > 0 && (!stats || !aligned16(stats))) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_gaussians == 0) return TGS_OK;
  if (!accumulate) cudaMemsetAsync(stats, 0, sizeof(float) * 4 * (size_t)n_gaussians, s);
  if (n_active_max > 0) {
    const int B = block_for(n_pix_max);
    k_error_stats<<<n_active_max, B, B * sizeof(Splat), s>>>(a, n_last, err_pix, stats);
  }
  return check_launch();
}

extern "C" tgs_status tgs_backward_sampled(const tgs_gaussians* g, const tgs_camera* cam, const tgs_projected* proj,
                                           const int32_t* tile_ranges, const int32_t* vals,
                                           const int32_t* active_tiles, const int32_t* n_active,
                                           int32_t n_active_max, const int32_t* pix_off, const uint8_t* pix_idx,
                                           int32_t n_pix_max, const float* bg, const float* T_final,
                                           const int32_t* n_last, const float* dL_drgb, float* grad2d,
                                           const tgs_param_ptrs* grads, uint8_t* touched, int32_t write_untouched,
                                           const tgs_checkpoints* ckpt, tgs_stream stream) {
  RasterArgs a;
  if (!gaussians_ok(g) || n_active_max < 0 || n_pix_max < 1 || n_pix_max > 256) return TGS_ERR_INVALID_ARG;
  if (!raster_args(proj, tile_ranges, vals, active_tiles, n_active, pix_off, pix_idx, cam, bg, a))
    return TGS_ERR_INVALID_ARG;
  if (!T_final || !n_last || !dL_drgb || !grads || !proj->radius) return TGS_ERR_INVALID_ARG;
  if (g->n > 0 && (!grad2d || !aligned16(grad2d) || !param_ptrs_ok(grads)))
    return TGS_ERR_INVALID_ARG;
  const tgs_status st = tgs_render_backward_sampled(proj, tile_ranges, vals, active_tiles, n_active, n_active_max,
                                                    pix_off, pix_idx, n_pix_max, cam, bg, T_final, n_last, dL_drgb,
                                                    grad2d, g->n, ckpt, stream);
  if (st != TGS_OK || g->n == 0) return st;
  launch_project_bwd(*g, *cam, proj->radius, grad2d, *grads, touched, write_untouched, 0, nullptr,
                     (cudaStream_t)stream);
  return check_launch();
}

static tgs_status batch_args(const tgs_view_batch* views, int32_t n_views, bool backward, BatchArgs& b, int& B) {
  if (!views || n_views < 1 || n_views > kMaxViews) return TGS_ERR_INVALID_ARG;
  b.n_views = n_views;
  b.stats = nullptr;
  for (int v = 0; v < kMaxViews; ++v) b.err[v] = nullptr;
  b.base[0] = 0;
  B = 32;
  // checkpoints: all views or none, with one slot count
  const int slots = views[0].ckpt.n_slots > 0 ? views[0].ckpt.n_slots : 0;
  b.pieces = backward && slots > 0 ? slots + 1 : 1;
  for (int v = 0; v < n_views; ++v) {
    const tgs_view_batch& w = views[v];
    if (w.n_active_max < 0 || w.n_pix_max < 1 || w.n_pix_max > 256) return TGS_ERR_INVALID_ARG;
    if (!raster_args(&w.proj, w.tile_ranges, w.vals, w.active_tiles, w.n_active, w.pix_off, w.pix_idx, &w.cam,
                     w.bg, b.a[v]))
      return TGS_ERR_INVALID_ARG;
    if (!w.rgb || !w.T_final || !w.n_last) return TGS_ERR_INVALID_ARG;
    if (backward && (!w.dL_drgb || !w.grad2d || !aligned16(w.grad2d) || w.n_gaussians < 0))
      return TGS_ERR_INVALID_ARG;
    b.rgb[v] = w.rgb;
    b.T[v] = w.T_final;
    b.last[v] = w.n_last;
    b.dL[v] = w.dL_drgb;
    b.grad2d[v] = w.grad2d;
    if ((w.ckpt.n_slots > 0 ? w.ckpt.n_slots : 0) != slots) return TGS_ERR_INVALID_ARG;
    if (!ckpt_of(&w.ckpt, w.n_active_max, w.n_pix_max, w.rgb, b.ck[v])) return TGS_ERR_INVALID_ARG;
    if (b.ck[v].data && w.ckpt.rgb && w.ckpt.rgb != w.rgb) return TGS_ERR_INVALID_ARG;
    b.base[v + 1] = b.base[v] + w.n_active_max * (backward ? b.pieces : 1);
    B = std::max(B, block_for(w.n_pix_max));
  }
  return TGS_OK;
}

static int bwd_warp_blocks_per_sm(int ppl) {
  int per_sm = 0;
  const int T = 32 * kBatchBwdWarps;
  switch (ppl) {
#define TGS_OCC(P) \
  case P: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd_batched_warp<P, false>, T, 0); break;
    TGS_OCC(1) TGS_OCC(2) TGS_OCC(3) TGS_OCC(4) TGS_OCC(5) TGS_OCC(6) TGS_OCC(7)
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd_batched_warp<8, false>, T, 0);
#undef TGS_OCC
  }
  return per_sm;
}

extern "C" tgs_status tgs_render_batched_resident(int32_t n_pix_max, int32_t backward, int32_t* ctas) {
  if (!ctas || n_pix_max < 1 || n_pix_max > 256 || backward < 0 || backward > 2) return TGS_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch();
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int B = block_for(n_pix_max);
  if (backward == 2)
    per_sm = bwd_warp_blocks_per_sm(B / 32);
  else if (backward)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd_batched, B,
                                                  B * (sizeof(Splat) + 9 * sizeof(float)));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_fwd_batched, B, B * sizeof(Splat));
  *ctas = sms * per_sm;
  return check_launch();
}

extern "C" tgs_status tgs_render_sampled_batched(const tgs_view_batch* views, int32_t n_views, int32_t grid_ctas,
                                                 int32_t* counter, tgs_stream stream) {
  BatchArgs b;
  int B = 32;
  tgs_status st = batch_args(views, n_views, false, b, B);
  if (st != TGS_OK) return st;
  if (grid_ctas < 1 || !counter) return TGS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  if (b.base[n_views] == 0) return check_launch();
  k_render_fwd_batched<<<grid_ctas, B, B * sizeof(Splat), s>>>(b, counter);
  return check_launch();
}

static tgs_status render_backward_batched_impl(const tgs_view_batch* views, int32_t n_views, int32_t grid_ctas,
                                               int32_t* counter, const float* const* err_pix, float* stats,
                                               int64_t n_stats, int32_t accumulate_stats, tgs_stream stream) {
  BatchArgs b;
  int B = 32;
  tgs_status st = batch_args(views, n_views, true, b, B);
  if (st != TGS_OK) return st;
  if (grid_ctas < 1 || !counter) return TGS_ERR_INVALID_ARG;
  const bool with_stats = err_pix != nullptr;
  b.stats = reinterpret_cast<float4*>(stats);
  for (int v = 0; v < n_views; ++v) {
    b.err[v] = with_stats ? err_pix[v] : nullptr;
    if (with_stats && (!b.err[v] || views[v].n_gaussians > n_stats)) return TGS_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (int v = 0; v < n_views; ++v)
    if (views[v].n_gaussians > 0)
      cudaMemsetAsync(views[v].grad2d, 0, sizeof(float) * 12 * (size_t)views[v].n_gaussians, s);
  if (with_stats && !accumulate_stats && n_stats > 0) cudaMemsetAsync(stats, 0, sizeof(float4) * (size_t)n_stats, s);
  cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  if (b.base[n_views] == 0) return check_launch();
  if (b.pieces == 1) {
    k_render_bwd_batched<<<grid_ctas, B, B * (sizeof(Splat) + 9 * sizeof(float)), s>>>(b, counter);
    // without checkpoints the statistics are the separate pass, view by view
    for (int v = 0; with_stats && v < n_views; ++v)
      if (views[v].n_active_max > 0) {
        const int Bv = block_for(views[v].n_pix_max);
        k_error_stats<<<views[v].n_active_max, Bv, Bv * sizeof(Splat), s>>>(b.a[v], b.last[v], b.err[v], stats);
      }
    return check_launch();
  }
  switch ((B / 32) * 2 + (with_stats ? 1 : 0)) {
#define TGS_BWD_BATCH(P)                                                                                        \
  case 2 * P: k_render_bwd_batched_warp<P, false><<<grid_ctas, 32 * kBatchBwdWarps, 0, s>>>(b, counter); break; \
  case 2 * P + 1: k_render_bwd_batched_warp<P, true><<<grid_ctas, 32 * kBatchBwdWarps, 0, s>>>(b, counter); break;
    TGS_BWD_BATCH(1) TGS_BWD_BATCH(2) TGS_BWD_BATCH(3) TGS_BWD_BATCH(4)
    TGS_BWD_BATCH(5) TGS_BWD_BATCH(6) TGS_BWD_BATCH(7) TGS_BWD_BATCH(8)
#undef TGS_BWD_BATCH
    default: break;
  }
  return check_launch();
}

extern "C" tgs_status tgs_render_backward_batched(const tgs_view_batch* views, int32_t n_views, int32_t grid_ctas,
                                                  int32_t* counter, tgs_stream stream) {
  return render_backward_batched_impl(views, n_views, grid_ctas, counter, nullptr, nullptr, 0, 0, stream);
}

extern "C" tgs_status tgs_render_backward_batched_stats(const tgs_view_batch* views, int32_t n_views,
                                                        int32_t grid_ctas, int32_t* counter,
                                                        const float* const* err_pix, float* stats,
                                                        int64_t n_gaussians, int32_t accumulate_stats,
                                                        tgs_stream stream) {
  if (!err_pix || n_gaussians < 0 || (n_gaussians > 0 && (!stats || !aligned16(stats)))) return TGS_ERR_INVALID_ARG;
  return render_backward_batched_impl(views, n_views, grid_ctas, counter, err_pix, stats, n_gaussians,
                                      accumulate_stats, stream);
}

extern "C" tgs_status tgs_project_backward(const tgs_gaussians* g, const tgs_camera* cam, const tgs_projected* proj,
                                           const float* grad2d, const tgs_param_ptrs* grads, uint8_t* touched,
                                           int32_t write_untouched, int32_t accumulate, float* view_row,
                                           tgs_stream stream) {
  if (!gaussians_ok(g) || !camera_ok(cam) || !proj || !grads) return TGS_ERR_INVALID_ARG;
  if (accumulate && !touched) return TGS_ERR_INVALID_ARG;
  if (view_row && !aligned8(view_row)) return TGS_ERR_INVALID_ARG;
  if (g->n == 0) return TGS_OK;
  if (!proj->radius || !grad2d || !aligned16(grad2d) || !param_ptrs_ok(grads))
    return TGS_ERR_INVALID_ARG;
  launch_project_bwd(*g, *cam, proj->radius, grad2d, *grads, touched, write_untouched, accumulate, view_row,
                     (cudaStream_t)stream);
  return check_launch();
}
