// Moment-damped Levenberg-Marquardt / Adam hybrid update (Sec. 3.9, Eq. 14;
// App. A).  One thread per Gaussian, all state in registers: the 10-parameter
// geometry block and the 4-parameter appearance block each solve
// (J^T J + diag(sqrt(v) + eps)) D = -m (Cholesky in mode 2), the 45 higher SH
// coefficients take a bias-corrected Adam step.  Untouched Gaussians are not
// read or written.
#include "hybrid_math.cuh"

namespace tgs {

// Touched Gaussians appended to a list (order irrelevant: updates are
// independent), one atomic per block.
__global__ void __launch_bounds__(256) k_compact_touched(const uint8_t* __restrict__ touched, int64_t n,
                                                         int32_t* __restrict__ list, int32_t* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = i < n && (!touched || touched[i]);
  const int64_t pos = block_append(on, count);
  if (on) list[pos] = (int32_t)i;
}


// LM blocks (geometry 10, appearance 4) and the first SH float4 (DC colour +
// one higher coefficient) of each touched Gaussian.
template <int MODE>
__global__ void __launch_bounds__(128) k_hybrid_lm(tgs_param_ptrs P, tgs_param_ptrs G, tgs_param_ptrs M,
                                                   tgs_param_ptrs V, int64_t n, const int32_t* __restrict__ list,
                                                   const int32_t* __restrict__ count, const float* __restrict__ rows,
                                                   int k_rows, OptK o) {
  bias_corrections(o);
  const int64_t cnt = *count;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x) {
  const int64_t i = list[q];
  float gg[10];
  const GeoW gG = geo_of(G);
  const float* gm = gG.mean(i);
  const float* gl = gG.lsc(i);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gg[k] = gm[k];
    gg[3 + k] = gl[k];
  }
  const float4 b = *gG.quat(i);
  gg[6] = b.x; gg[7] = b.y; gg[8] = b.z; gg[9] = b.w;
  const float4 g0 = reinterpret_cast<const float4*>(G.sh)[12 * i];
  const float sg[4] = {g0.x, g0.y, g0.z, g0.w};
  lm_update_one<MODE>(P, M, V, n, i, gg, sg, *gG.opac(i), rows, k_rows, o);
  }
}

// Adam on SH float4s 1..11 of each touched Gaussian: one thread per float4,
// eleven consecutive threads per Gaussian (176 contiguous bytes per array).
__global__ void __launch_bounds__(256) k_adam_sh(tgs_param_ptrs P, tgs_param_ptrs G, tgs_param_ptrs M,
                                                 tgs_param_ptrs V, const int32_t* __restrict__ list,
                                                 const int32_t* __restrict__ count, OptK o) {
  bias_corrections(o);
  const int64_t total = (int64_t)*count * 11;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
  const int64_t q = e / 11;
  const int k = 1 + (int)(e - q * 11);
  const int64_t i = list[q];
  adam_sh_one(P, M, V, i, k, reinterpret_cast<const float4*>(G.sh)[12 * i + k], o);
  }
}

}  // namespace tgs

using namespace tgs;

extern "C" size_t tgs_hybrid_step_workspace_size(int64_t n) {
  return align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), 256) + 256;
}

extern "C" tgs_status tgs_hybrid_step(const tgs_param_ptrs* params, const tgs_param_ptrs* grads,
                                      const tgs_param_ptrs* m, const tgs_param_ptrs* v, int64_t n,
                                      const uint8_t* touched, const float* view_rows, int32_t k_rows, int32_t step,
                                      const int32_t* step_dev, const tgs_opt* opt, void* workspace,
                                      size_t workspace_bytes, tgs_stream stream) {
  if (n < 0 || !opt || step < 1 || opt->mode < 0 || opt->mode > 2 || (view_rows && k_rows < 1) ||
      !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f) || n >= INT32_MAX)
    return TGS_ERR_INVALID_ARG;
  if (n == 0) return TGS_OK;
  if (!param_ptrs_ok(params) || !param_ptrs_ok(grads) || !param_ptrs_ok(m) || !param_ptrs_ok(v))
    return TGS_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < tgs_hybrid_step_workspace_size(n)) return TGS_ERR_INVALID_ARG;
  OptK o = make_optk(opt, step, step_dev);
  cudaStream_t s = (cudaStream_t)stream;
  Carver c(workspace);
  int32_t* list = c.take<int32_t>((size_t)n);
  int32_t* count = c.take<int32_t>(1);
  cudaMemsetAsync(count, 0, sizeof(int32_t), s);
  k_compact_touched<<<(int)((n + 255) / 256), 256, 0, s>>>(touched, n, list, count);
  // the touched count lives on the device: grid-stride loops over it with
  // grids of a few waves of the GPU (not one thread per Gaussian)
  const int sms = device_sm_count();
  const int lb = (int)std::min<int64_t>((n + 127) / 128, (int64_t)sms * 16);
  const int sb = (int)std::min<int64_t>((n * 11 + 255) / 256, (int64_t)sms * 16);
  if (o.mode == 0) k_hybrid_lm<0><<<lb, 128, 0, s>>>(*params, *grads, *m, *v, n, list, count, view_rows, k_rows, o);
  else if (o.mode == 1) k_hybrid_lm<1><<<lb, 128, 0, s>>>(*params, *grads, *m, *v, n, list, count, view_rows, k_rows, o);
  else k_hybrid_lm<2><<<lb, 128, 0, s>>>(*params, *grads, *m, *v, n, list, count, view_rows, k_rows, o);
  k_adam_sh<<<sb, 256, 0, s>>>(*params, *grads, *m, *v, list, count, o);
  return check_launch();
}
