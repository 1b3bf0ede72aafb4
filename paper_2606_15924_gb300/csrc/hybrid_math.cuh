// The per-parameter arithmetic of the moment-damped LM / Adam hybrid update
// (Sec. 3.9, Eq. 14; App. A), shared by the update kernels and the fused
// projection-adjoint-and-update kernel.
#pragma once
#include "tgs_common.cuh"

namespace tgs {

struct OptK {
  float lr[6];
  float b1, b2, eps, eps_lm, ibc1, ibc2;  // ibc: reciprocals of the bias corrections 1 - beta^t
  int mode;
  const int32_t* step_dev;  // when set, bias corrections use this step
};

// Square root and quotient through the SFU approximations (relative error a
// few 1e-7): the update's step sizes need no more, and the IEEE forms cost
// several times the instructions of the moment arithmetic around them.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int D>
__device__ __forceinline__ void lm_block(const float (&g)[D], const float (&m)[D], const float (&v)[D],
                                         const float* __restrict__ rows, int k_rows, int64_t n, int64_t i, int off,
                                         int mode, float eps_lm, float (&out)[D]) {
  if (mode == 1) {
    float jj[D];
#pragma unroll
    for (int a = 0; a < D; ++a) jj[a] = rows ? 0.f : g[a] * g[a];
    for (int r = 0; rows && r < k_rows; ++r) {
      const float* row = rows + ((size_t)r * n + i) * 14 + off;
#pragma unroll
      for (int a = 0; a < D; ++a) jj[a] += row[a] * row[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) out[a] = __fdividef(-m[a], jj[a] + sqrt_approx(v[a]) + eps_lm);
    return;
  }
  // full J^T J: lower triangle, then Cholesky A = L L^T and two triangular solves
  float A[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) A[a][b] = rows ? 0.f : g[a] * g[b];
  for (int r = 0; rows && r < k_rows; ++r) {
    const float* row = rows + ((size_t)r * n + i) * 14 + off;
    float J[D];
#pragma unroll
    for (int a = 0; a < D; ++a) J[a] = row[a];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) A[a][b] += J[a] * J[b];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) A[a][a] += sqrtf(v[a]) + eps_lm;
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      float s = A[a][b];
#pragma unroll
      for (int k = 0; k < b; ++k) s -= A[a][k] * A[b][k];
      if (a == b) A[a][a] = sqrtf(fmaxf(s, 1e-30f));
      else A[a][b] = s / A[b][b];
    }
  }
  float y[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float s = -m[a];
#pragma unroll
    for (int k = 0; k < a; ++k) s -= A[a][k] * y[k];
    y[a] = s / A[a][a];
  }
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    float s = y[a];
#pragma unroll
    for (int k = a + 1; k < D; ++k) s -= A[k][a] * out[k];
    out[a] = s / A[a][a];
  }
}

__device__ __forceinline__ void moments(float g, float& m, float& v, const OptK& o) {
  m = o.b1 * m + (1.f - o.b1) * g;
  v = o.b2 * v + (1.f - o.b2) * g * g;
}

__device__ __forceinline__ float adam_delta(float m, float v, float lr, const OptK& o) {
  return __fdividef(-lr * (m * o.ibc1), sqrt_approx(v * o.ibc2) + o.eps);
}

__device__ __forceinline__ void bias_corrections(OptK& o) {
  if (o.step_dev) {
    const float st = (float)max(1, *o.step_dev);
    o.ibc1 = 1.f / (1.f - powf(o.b1, st));
    o.ibc2 = 1.f / (1.f - powf(o.b2, st));
  }
}

// The geometry LM block (means, log-scales, quaternion: 10 parameters) of
// Gaussian i in registers: the moments (gm, gv) take gradient gg, and the
// parameters gp their step.
template <int MODE>
__device__ __forceinline__ void lm_geo_step(const float (&gg)[10], float (&gp)[10], float (&gm)[10], float (&gv)[10],
                                            const float* __restrict__ rows, int k_rows, int64_t n, int64_t i,
                                            const OptK& o) {
#pragma unroll
  for (int k = 0; k < 10; ++k) moments(gg[k], gm[k], gv[k], o);
  if (MODE == 0) {
#pragma unroll
    for (int k = 0; k < 10; ++k) gp[k] += adam_delta(gm[k], gv[k], o.lr[k < 3 ? 0 : k < 6 ? 1 : 2], o);
  } else {
    float dgeo[10];
    lm_block<10>(gg, gm, gv, rows, k_rows, n, i, 0, MODE, o.eps_lm, dgeo);
#pragma unroll
    for (int k = 0; k < 10; ++k) gp[k] += o.lr[k < 3 ? 0 : k < 6 ? 1 : 2] * dgeo[k];
  }
}

// The appearance LM block (SH DC r g b and the opacity logit) and the first
// higher SH coefficient (the fourth lane of SH float4 0, an Adam step) of
// Gaussian i in registers, from sg (the gradient of SH float4 0) and og
// (opacity logit): parameters (sp, op), moments (smm, om) and (sv, ov).
template <int MODE>
__device__ __forceinline__ void lm_app_step(const float (&sg)[4], float og, float (&sp)[4], float (&smm)[4],
                                            float (&sv)[4], float& op, float& om, float& ov,
                                            const float* __restrict__ rows, int k_rows, int64_t n, int64_t i,
                                            const OptK& o) {
#pragma unroll
  for (int k = 0; k < 4; ++k) moments(sg[k], smm[k], sv[k], o);
  moments(og, om, ov, o);
  if (MODE == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) sp[k] += adam_delta(smm[k], sv[k], o.lr[4], o);
    op += adam_delta(om, ov, o.lr[3], o);
  } else {
    const float ag[4] = {sg[0], sg[1], sg[2], og}, am[4] = {smm[0], smm[1], smm[2], om},
                av[4] = {sv[0], sv[1], sv[2], ov};
    float dapp[4];
    lm_block<4>(ag, am, av, rows, k_rows, n, i, 10, MODE, o.eps_lm, dapp);
#pragma unroll
    for (int k = 0; k < 3; ++k) sp[k] += o.lr[4] * dapp[k];
    op += o.lr[3] * dapp[3];
  }
  sp[3] += adam_delta(smm[3], sv[3], o.lr[5], o);
}

// The geometry LM block of Gaussian i (means, log-scales, quaternion: 10
// parameters) from its gradient gg, read from and written to memory.
template <int MODE>
__device__ __forceinline__ void lm_update_geo(const tgs_param_ptrs& P, const tgs_param_ptrs& M,
                                              const tgs_param_ptrs& V, int64_t n, int64_t i, const float (&gg)[10],
                                              const float* __restrict__ rows, int k_rows, const OptK& o) {
  float gp[10], gm[10], gv[10];
  const GeoW gP = geo_of(P), gM = geo_of(M), gV = geo_of(V);
  {
    const float* a = gP.mean(i);
    const float* b = gM.mean(i);
    const float* c = gV.mean(i);
    const float* d = gP.lsc(i);
    const float* e = gM.lsc(i);
    const float* f = gV.lsc(i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gp[k] = a[k]; gm[k] = b[k]; gv[k] = c[k];
      gp[3 + k] = d[k]; gm[3 + k] = e[k]; gv[3 + k] = f[k];
    }
  }
  {
    const float4 a = *gP.quat(i), c = *gM.quat(i), d = *gV.quat(i);
    gp[6] = a.x; gp[7] = a.y; gp[8] = a.z; gp[9] = a.w;
    gm[6] = c.x; gm[7] = c.y; gm[8] = c.z; gm[9] = c.w;
    gv[6] = d.x; gv[7] = d.y; gv[8] = d.z; gv[9] = d.w;
  }
  lm_geo_step<MODE>(gg, gp, gm, gv, rows, k_rows, n, i, o);
  {
    float* a = gP.mean(i);
    float* b = gM.mean(i);
    float* c = gV.mean(i);
    float* d = gP.lsc(i);
    float* e = gM.lsc(i);
    float* f = gV.lsc(i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a[k] = gp[k]; b[k] = gm[k]; c[k] = gv[k];
      d[k] = gp[3 + k]; e[k] = gm[3 + k]; f[k] = gv[3 + k];
    }
  }
  *gP.quat(i) = make_float4(gp[6], gp[7], gp[8], gp[9]);
  *gM.quat(i) = make_float4(gm[6], gm[7], gm[8], gm[9]);
  *gV.quat(i) = make_float4(gv[6], gv[7], gv[8], gv[9]);
}

// The appearance LM block of Gaussian i and its SH float4 0, read from and
// written to memory.
template <int MODE>
__device__ __forceinline__ void lm_update_app(const tgs_param_ptrs& P, const tgs_param_ptrs& M,
                                              const tgs_param_ptrs& V, int64_t n, int64_t i, const float (&sg)[4],
                                              float og, const float* __restrict__ rows, int k_rows, const OptK& o) {
  const GeoW gP = geo_of(P), gM = geo_of(M), gV = geo_of(V);
  const float4 p0 = reinterpret_cast<const float4*>(P.sh)[12 * i];
  const float4 m0 = reinterpret_cast<const float4*>(M.sh)[12 * i], v0 = reinterpret_cast<const float4*>(V.sh)[12 * i];
  float sp[4] = {p0.x, p0.y, p0.z, p0.w};
  float smm[4] = {m0.x, m0.y, m0.z, m0.w}, sv[4] = {v0.x, v0.y, v0.z, v0.w};
  float op = *gP.opac(i), om = *gM.opac(i), ov = *gV.opac(i);
  lm_app_step<MODE>(sg, og, sp, smm, sv, op, om, ov, rows, k_rows, n, i, o);
  *gP.opac(i) = op; *gM.opac(i) = om; *gV.opac(i) = ov;
  reinterpret_cast<float4*>(P.sh)[12 * i] = make_float4(sp[0], sp[1], sp[2], sp[3]);
  reinterpret_cast<float4*>(M.sh)[12 * i] = make_float4(smm[0], smm[1], smm[2], smm[3]);
  reinterpret_cast<float4*>(V.sh)[12 * i] = make_float4(sv[0], sv[1], sv[2], sv[3]);
}

// Both LM blocks and SH float4 0 of Gaussian i: gradient gg (means,
// log-scales, quaternion), sg (SH float4 0) and og (opacity logit).
template <int MODE>
__device__ __forceinline__ void lm_update_one(const tgs_param_ptrs& P, const tgs_param_ptrs& M,
                                              const tgs_param_ptrs& V, int64_t n, int64_t i, const float (&gg)[10],
                                              const float (&sg)[4], float og, const float* __restrict__ rows,
                                              int k_rows, const OptK& o) {
  lm_update_geo<MODE>(P, M, V, n, i, gg, rows, k_rows, o);
  lm_update_app<MODE>(P, M, V, n, i, sg, og, rows, k_rows, o);
}

// Adam update of Gaussian i's SH float4 k (1..11) from its gradient g.
__device__ __forceinline__ void adam_sh_one(const tgs_param_ptrs& P, const tgs_param_ptrs& M,
                                            const tgs_param_ptrs& V, int64_t i, int k, float4 gq, const OptK& o) {
  const int64_t f = 12 * i + k;
  float4 pp = reinterpret_cast<const float4*>(P.sh)[f];
  float4 mq = reinterpret_cast<const float4*>(M.sh)[f], vq = reinterpret_cast<const float4*>(V.sh)[f];
  moments(gq.x, mq.x, vq.x, o); moments(gq.y, mq.y, vq.y, o);
  moments(gq.z, mq.z, vq.z, o); moments(gq.w, mq.w, vq.w, o);
  pp.x += adam_delta(mq.x, vq.x, o.lr[5], o); pp.y += adam_delta(mq.y, vq.y, o.lr[5], o);
  pp.z += adam_delta(mq.z, vq.z, o.lr[5], o); pp.w += adam_delta(mq.w, vq.w, o.lr[5], o);
  reinterpret_cast<float4*>(P.sh)[f] = pp;
  reinterpret_cast<float4*>(M.sh)[f] = mq;
  reinterpret_cast<float4*>(V.sh)[f] = vq;
}

// OptK from the C-ABI options at host step `step`.
inline OptK make_optk(const tgs_opt* opt, int32_t step, const int32_t* step_dev) {
  OptK o;
  for (int k = 0; k < 6; ++k) o.lr[k] = opt->lr[k];
  o.b1 = opt->beta1; o.b2 = opt->beta2; o.eps = opt->eps_adam; o.eps_lm = opt->eps_lm; o.mode = opt->mode;
  o.step_dev = step_dev;
  o.ibc1 = (float)(1.0 / (1.0 - pow((double)opt->beta1, (double)step)));
  o.ibc2 = (float)(1.0 / (1.0 - pow((double)opt->beta2, (double)step)));
  return o;
}

}  // namespace tgs
