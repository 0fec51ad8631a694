// Error plumbing, version and the L1 loss term of Eq. 1 / Eq. 2.
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace lgs {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

cudaError_t set_smem_limit(const void* func, int bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> done;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(func);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[func] = bytes;
  return e;
}

// loss += weight * mean|pred - target|, grad = weight * sign(pred - target) / count.
template <typename TT>
__global__ void l1_loss_kernel(const float* __restrict__ pred, const TT* __restrict__ target,
                               int64_t count, float scale, float* __restrict__ grad,
                               float* __restrict__ loss) {
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float d = pred[i] - to_float(target[i]);
    acc += fabsf(d);
    grad[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v * scale);
  }
}

}  // namespace lgs

using namespace lgs;

extern "C" const char* lgs_version(void) { return "lgs 0.1 (sm_103a)"; }

extern "C" const char* lgs_last_error(void) { return g_last_error.c_str(); }

extern "C" int64_t lgs_graph_kernel_nodes(void* graph) {
  clear_error();
  if (!graph) return -1;
  cudaGraph_t g = reinterpret_cast<cudaGraph_t>(graph);
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
  int64_t k = 0;
  for (size_t i = 0; i < n; i++) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) return -1;
    if (t == cudaGraphNodeTypeKernel) k++;
  }
  return k;
}

extern "C" lgs_status lgs_zero(void* dev, size_t bytes, void* stream) {
  clear_error();
  if (bytes == 0) return LGS_OK;
  LGS_CHECK_ARG(dev != nullptr, "null pointer");
  LGS_CHECK_CUDA(cudaMemsetAsync(dev, 0, bytes, as_stream(stream)));
  return LGS_OK;
}

extern "C" lgs_status lgs_l1_loss(const float* pred, const void* target, int target_dtype,
                                  int64_t count, float weight, float* grad, float* loss_dev,
                                  void* stream) {
  clear_error();
  LGS_CHECK_ARG(count >= 0, "count < 0");
  if (count == 0) return LGS_OK;
  LGS_CHECK_ARG(pred && target && grad && loss_dev, "null pointer");
  LGS_CHECK_ARG(target_dtype == LGS_F32 || target_dtype == LGS_BF16, "bad target dtype");
  float scale = weight / (float)count;
  int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 8);
  cudaStream_t s = as_stream(stream);
  if (target_dtype == LGS_F32)
    l1_loss_kernel<float><<<blocks, 256, 0, s>>>(pred, (const float*)target, count, scale, grad,
                                                 loss_dev);
  else
    l1_loss_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(
        pred, (const __nv_bfloat16*)target, count, scale, grad, loss_dev);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
