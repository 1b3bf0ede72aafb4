// Library-wide C ABI entry points: version, error reporting, device check.
#include "tgs_common.cuh"

namespace tgs {
static thread_local int32_t g_last_cuda_error = 0;
void set_cuda_error(cudaError_t e) { g_last_cuda_error = (int32_t)e; }
int device_sm_count() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev >= 64) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }
  if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  return sms[dev] > 0 ? sms[dev] : 1;
}
}  // namespace tgs

extern "C" const char* tgs_version(void) { return "turbogs-gb300 0.1.0 (sm_103a)"; }

extern "C" int32_t tgs_last_cuda_error(void) { return tgs::g_last_cuda_error; }

extern "C" const char* tgs_status_string(int32_t status) {
  switch (status) {
    case TGS_OK: return "ok";
    case TGS_ERR_INVALID_ARG: return "invalid argument";
    case TGS_ERR_CAPACITY: return "capacity exceeded";
    case TGS_ERR_CUDA: return "CUDA error";
    case TGS_ERR_TIMEOUT: return "device wait timed out";
    case TGS_ERR_DEVICE: return "no usable sm_103 device";
    default: return "unknown status";
  }
}

extern "C" tgs_status tgs_device_check(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    tgs::set_cuda_error(e);
    return TGS_ERR_DEVICE;
  }
  cudaDeviceProp p;
  e = cudaGetDeviceProperties(&p, dev);
  if (e != cudaSuccess) {
    tgs::set_cuda_error(e);
    return TGS_ERR_DEVICE;
  }
  return (p.major == 10 && p.minor == 3) ? TGS_OK : TGS_ERR_DEVICE;
}

// Number of kernel nodes in a captured CUDA graph (cudaGraph_t), -1 on error.
// Lets callers count the kernels one replay launches.
extern "C" int64_t tgs_graph_count_kernels(void* graph) {
  cudaGraph_t g = static_cast<cudaGraph_t>(graph);
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  if (n == 0) return 0;
  cudaGraphNode_t* nodes = new cudaGraphNode_t[n];
  int64_t k = -1;
  if (cudaGraphGetNodes(g, nodes, &n) == cudaSuccess) {
    k = 0;
    for (size_t i = 0; i < n; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
  }
  delete[] nodes;
  return k;
}

namespace {
__global__ void k_advance_counters(int64_t* it, int32_t* step) {
  if (it) *it += 1;
  if (step) *step += 1;
}
}  // namespace

extern "C" tgs_status tgs_advance_counters(int64_t* iter_dev, int32_t* step_dev, tgs_stream stream) {
  if (!iter_dev && !step_dev) return TGS_ERR_INVALID_ARG;
  k_advance_counters<<<1, 1, 0, (cudaStream_t)stream>>>(iter_dev, step_dev);
  return tgs::check_launch();
}
