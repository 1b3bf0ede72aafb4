// Error-driven densification and pruning (Sec. 3.8, Eq. 13; Alg. 1 step 11;
// Table 6).  The paper fixes the difficulty scores and says that percentile
// thresholds of them drive densification and pruning; the procedure here is
// the reading the header states.  Every decision is an explicitly rounded
// single-precision operation, so a selection is reproducible bit for bit.
//
// One step: (1) per Gaussian the score, the candidate test and a 32-bit
// ranking key (candidates by descending score, or every Gaussian by
// descending accumulated weight for the final pruning); (2) a stable radix
// sort of (key, index) pairs, so equal keys keep the lower index first;
// (3) the top of the order is marked densified (or the tail pruned);
// (4) an exclusive scan of the per-Gaussian output counts (0, 1 or 2);
// (5) a scatter of the surviving, cloned and split Gaussians and their
// moments to the output arrays in input order.
#include "radix.cuh"
#include "scan.cuh"
#include "tgs_common.cuh"

namespace tgs {

bool gaussians_ok(const tgs_gaussians* g);

constexpr uint32_t kKeyTop = 0x7F800000u;  // bits of +inf: keys of finite non-negative values fall below
constexpr uint32_t kKeyNone = 0xFFFFFFFFu;  // not ranked (after every ranked key)
constexpr float kLogSplit = 0.47000362924573558f;  // ln 1.6: the children's log-scale decrease

__device__ __forceinline__ bool row_nonzero(const float4& a, const float4& b, const float4& c) {
  return a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f || b.x != 0.f || b.y != 0.f || b.z != 0.f ||
         b.w != 0.f || c.x != 0.f;
}

// accum[i] += (|(dL/dx, dL/dy)|, 1) for every Gaussian with a non-zero
// compositing adjoint in this view's grad2d [N,12].
__global__ void k_screen_grad(const float4* __restrict__ grad2d, int64_t n, float2* __restrict__ accum) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = grad2d[3 * i], b = grad2d[3 * i + 1], c = grad2d[3 * i + 2];
  if (!row_nonzero(a, b, c)) return;
  const float norm = __fsqrt_rn(__fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y)));
  float2 q = accum[i];
  q.x = __fadd_rn(q.x, norm);
  q.y = __fadd_rn(q.y, 1.f);
  accum[i] = q;
}

struct DensK {
  float lam_eff, eps, tau_grad, log_split, logit_prune;
  int topk_pm, final_mode, final_pm;
};

// (1) prune flag, ranking key and index of every Gaussian; n_rank counts the
// densification candidates (every Gaussian in the final pruning).
__global__ void k_dens_keys(GeoC geo, const float4* __restrict__ stats,
                            const float2* __restrict__ accum, int64_t n, DensK k, uint8_t* __restrict__ flag,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int32_t* __restrict__ n_rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ranked = false;
  if (i < n) {
    const bool prune = geo.opac(i) < k.logit_prune;
    const float4 st = stats[i];
    uint32_t key = kKeyNone;
    if (k.final_mode) {
      key = kKeyTop - __float_as_uint(st.y);  // every Gaussian by its accumulated weight W
      ranked = true;
    } else {
      const float2 ac = accum[i];
      const float g = __fdiv_rn(ac.x, ac.y > 1.f ? ac.y : 1.f);
      if (!prune && st.y > 0.f && g >= k.tau_grad) {
        const float den = __fadd_rn(st.y, k.eps);
        const float e = __fdiv_rn(st.x, den), d = __fdiv_rn(st.z, den);
        const float s = __fadd_rn(e, __fmul_rn(k.lam_eff, d));  // Eq. 13
        key = kKeyTop - __float_as_uint(s);
        ranked = true;
      }
    }
    flag[i] = prune ? 1 : 0;
    keys[i] = key;
    vals[i] = (uint32_t)i;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, ranked);
  if ((threadIdx.x & 31) == 0 && bal) atomicAdd(n_rank, __popc(bal));
}

// (3) densify the first floor(n_rank topk / 1000) of the order, or (final
// pruning) prune everything past the first floor(n final / 1000).
__global__ void k_dens_mark(const uint32_t* __restrict__ order, int64_t n, const int32_t* __restrict__ n_rank,
                            DensK k, uint8_t* __restrict__ flag) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t i = order[p];
  if (k.final_mode) {
    if (p >= n * k.final_pm / 1000) flag[i] = 1;
  } else if (p < (int64_t)*n_rank * k.topk_pm / 1000) {
    flag[i] |= 2;  // densified (the candidates are never pruned)
  }
}

struct ParamsIn {
  GeoC g;
  const float4* sh;
};

struct ParamsOut {
  GeoW g;
  float4* sh;
};

// Copies row i of one parameter-shaped array set into row o of another.
__device__ __forceinline__ void copy_row(const ParamsIn& a, int64_t i, const ParamsOut& b, int64_t o) {
  const float3 m = a.g.mean(i), l = a.g.lsc(i);
  float* bm = b.g.mean(o);
  float* bl = b.g.lsc(o);
  bm[0] = m.x; bm[1] = m.y; bm[2] = m.z;
  bl[0] = l.x; bl[1] = l.y; bl[2] = l.z;
  *b.g.quat(o) = a.g.quat(i);
  *b.g.opac(o) = a.g.opac(i);
#pragma unroll
  for (int c = 0; c < 12; ++c) b.sh[12 * o + c] = a.sh[12 * i + c];
}

__device__ __forceinline__ void zero_row(const ParamsOut& b, int64_t o) {
  float* bm = b.g.mean(o);
  float* bl = b.g.lsc(o);
#pragma unroll
  for (int c = 0; c < 3; ++c) bm[c] = bl[c] = 0.f;
  *b.g.quat(o) = make_float4(0.f, 0.f, 0.f, 0.f);
  *b.g.opac(o) = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) b.sh[12 * o + c] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// (5) output rows of Gaussian i from offset off[i]: kept (parameters and
// moments copied); cloned (the copy after it, zero moments); split (two
// children, zero moments).  Rows past the capacity are not written.
__global__ void k_dens_scatter(ParamsIn P, ParamsIn M, ParamsIn V, const uint8_t* __restrict__ flag,
                               const int64_t* __restrict__ off, int64_t n, DensK k, ParamsOut PO, ParamsOut MO,
                               ParamsOut VO, int64_t capacity, int64_t* __restrict__ src) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint8_t f = flag[i];
  if (f & 1) return;  // pruned
  const bool dens = (f & 2) != 0;
  const int64_t o = off[i];
  const int copies = dens ? 2 : 1;
  if (o + copies > capacity) return;
  int ax = 0;
  const float3 ls3 = P.g.lsc(i);
  const float lsa[3] = {ls3.x, ls3.y, ls3.z};
  float lmax = lsa[0];
#pragma unroll
  for (int a = 1; a < 3; ++a)
    if (lsa[a] > lmax) {
      lmax = lsa[a];
      ax = a;
    }
  const bool split = dens && lmax > k.log_split;
  for (int q = 0; q < copies; ++q) {
    copy_row(P, i, PO, o + q);
    if (src) src[o + q] = i;
    if (dens) {
      zero_row(MO, o + q);
      zero_row(VO, o + q);
    } else {
      copy_row(M, i, MO, o + q);
      copy_row(V, i, VO, o + q);
    }
  }
  if (dens && !split) {  // the original keeps its moments, the copy starts from zero
    copy_row(M, i, MO, o);
    copy_row(V, i, VO, o);
  }
  if (split) {
    const float4 qr = P.g.quat(i);
    const float inv = rsqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float w = qr.x * inv, x = qr.y * inv, y = qr.z * inv, z = qr.w * inv;
    // column ax of the rotation matrix of (w, x, y, z)
    float col[3];
    if (ax == 0) {
      col[0] = 1.f - 2.f * (y * y + z * z); col[1] = 2.f * (x * y + w * z); col[2] = 2.f * (x * z - w * y);
    } else if (ax == 1) {
      col[0] = 2.f * (x * y - w * z); col[1] = 1.f - 2.f * (x * x + z * z); col[2] = 2.f * (y * z + w * x);
    } else {
      col[0] = 2.f * (x * z + w * y); col[1] = 2.f * (y * z - w * x); col[2] = 1.f - 2.f * (x * x + y * y);
    }
    const float sig = expf(lmax);
    const float3 mu3 = P.g.mean(i);
    const float mu[3] = {mu3.x, mu3.y, mu3.z};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float sgn = q == 0 ? 1.f : -1.f;
      float* om = PO.g.mean(o + q);
      float* ol = PO.g.lsc(o + q);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        om[c] = mu[c] + sgn * sig * col[c];
        ol[c] = lsa[c] - kLogSplit;
      }
    }
  }
}

}  // namespace tgs

using namespace tgs;

namespace {

struct DensWs {
  uint8_t* flag;
  uint32_t *k0, *v0, *k1, *v1;
  RadixScratch rs;
  int32_t* n_rank;
  int64_t* off;
  int64_t* scan_sums;
};

DensWs carve_dens(void* base, int64_t n, size_t* bytes) {
  Carver c(base);
  const size_t m = (size_t)std::max<int64_t>(n, 1);
  DensWs w;
  w.flag = c.take<uint8_t>(m);
  w.k0 = c.take<uint32_t>(m);
  w.v0 = c.take<uint32_t>(m);
  w.k1 = c.take<uint32_t>(m);
  w.v1 = c.take<uint32_t>(m);
  w.rs.hist = c.take<uint32_t>(radix_hist_elems(n));
  w.rs.bin_total = c.take<uint32_t>(RS_BINS);
  w.n_rank = c.take<int32_t>(1);
  w.off = c.take<int64_t>(m);
  w.scan_sums = c.take<int64_t>((size_t)std::max(1, scan_blocks(n)));
  if (bytes) *bytes = c.size();
  return w;
}

ParamsIn in_of(const tgs_param_ptrs& p) {
  return ParamsIn{geo_const(geo_of(p)), reinterpret_cast<const float4*>(p.sh)};
}

ParamsOut out_of(const tgs_param_ptrs& p) { return ParamsOut{geo_of(p), reinterpret_cast<float4*>(p.sh)}; }

}  // namespace

extern "C" tgs_status tgs_accumulate_screen_grad(const float* grad2d, int64_t n, float* accum, tgs_stream stream) {
  if (n < 0 || (n > 0 && (!grad2d || !accum || !aligned16(grad2d) || !aligned8(accum)))) return TGS_ERR_INVALID_ARG;
  if (n == 0) return TGS_OK;
  k_screen_grad<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4*>(grad2d), n, reinterpret_cast<float2*>(accum));
  return check_launch();
}

extern "C" size_t tgs_density_control_workspace_size(int64_t n) {
  size_t b = 0;
  carve_dens(nullptr, n, &b);
  return b;
}

extern "C" tgs_status tgs_density_control(const tgs_gaussians* g, const tgs_param_ptrs* m_in,
                                          const tgs_param_ptrs* v_in, const float* stats, const float* accum,
                                          const tgs_density_params* cfg, const tgs_param_ptrs* g_out,
                                          const tgs_param_ptrs* m_out, const tgs_param_ptrs* v_out,
                                          int64_t capacity, int64_t* n_out, int64_t* src_out, void* workspace,
                                          size_t workspace_bytes, tgs_stream stream) {
  if (!g || !m_in || !v_in || !cfg || !g_out || !m_out || !v_out || !n_out || capacity < 0) return TGS_ERR_INVALID_ARG;
  const int64_t n = g->n;
  if (n < 0 || n > 0x7fffffffLL) return TGS_ERR_INVALID_ARG;
  if (cfg->topk_permille < 0 || cfg->topk_permille > 1000 || cfg->final_permille < 0 ||
      cfg->final_permille > 1000 || (cfg->final_prune != 0 && cfg->final_prune != 1) || !(cfg->eps >= 0.f))
    return TGS_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < tgs_density_control_workspace_size(n)) return TGS_ERR_INVALID_ARG;
  if (n > 0) {
    if (!stats || !accum || !aligned16(stats) || !aligned8(accum)) return TGS_ERR_INVALID_ARG;
    if (!gaussians_ok(g) || !param_ptrs_ok(m_in) || !param_ptrs_ok(v_in)) return TGS_ERR_INVALID_ARG;
    if (capacity > 0 && (!param_ptrs_ok(g_out) || !param_ptrs_ok(m_out) || !param_ptrs_ok(v_out)))
      return TGS_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    cudaMemsetAsync(n_out, 0, sizeof(int64_t), s);
    return check_launch();
  }
  DensWs w = carve_dens(workspace, n, nullptr);
  DensK k{cfg->lambda_eff, cfg->eps, cfg->tau_grad, cfg->log_scale_split, cfg->opacity_logit_prune,
          cfg->topk_permille, cfg->final_prune, cfg->final_permille};
  const int blocks = (int)((n + 255) / 256);
  cudaMemsetAsync(w.n_rank, 0, sizeof(int32_t), s);
  k_dens_keys<<<blocks, 256, 0, s>>>(geo_of(*g), reinterpret_cast<const float4*>(stats),
                                     reinterpret_cast<const float2*>(accum), n, k, w.flag, w.k0, w.v0, w.n_rank);
  const int cur = radix_sort_pairs(w.k0, w.v0, w.k1, w.v1, nullptr, (int32_t)n, 0, 32, w.rs, nullptr, s);
  const uint32_t* order = cur ? w.v1 : w.v0;
  k_dens_mark<<<blocks, 256, 0, s>>>(order, n, w.n_rank, k, w.flag);
  const uint8_t* fl = w.flag;
  int64_t* off = w.off;
  auto load = [=] __device__(int64_t i) -> int64_t { return (fl[i] & 1) ? 0 : ((fl[i] & 2) ? 2 : 1); };
  auto store = [=] __device__(int64_t i, int64_t pre, int64_t) { off[i] = pre; };
  exclusive_scan<int64_t>(load, store, nullptr, n, w.scan_sums, n_out, s);
  if (capacity > 0) {
    const tgs_param_ptrs gin{const_cast<float*>(g->means), const_cast<float*>(g->log_scales),
                             const_cast<float*>(g->quats), const_cast<float*>(g->opacity_logits),
                             const_cast<float*>(g->sh), g->geo_stride};
    k_dens_scatter<<<blocks, 256, 0, s>>>(in_of(gin), in_of(*m_in), in_of(*v_in), w.flag, w.off, n, k,
                                          out_of(*g_out), out_of(*m_out), out_of(*v_out), capacity, src_out);
  }
  return check_launch();
}
