// gs_render_bwd_static: the render backward for callers that cannot allocate
// device memory.
//
// gs_render_bwd needs a scratch buffer of 32 bytes per (camera, Gaussian) for
// the 2D gradients it accumulates before the projection chain rule, and
// expects the caller to own it.  Some callers cannot provide one: a mapping
// thread with a hard real-time budget must not take the device-wide
// synchronisation that cudaMalloc / cudaFree imply, and some host
// applications forbid a library (and its caller's plug-in code) from owning
// device memory at all.  This entry point uses a fixed scratch array that is
// part of the library's device image instead, so neither the caller nor the
// library allocates anything per call.
//
// The array is a file-scope __device__ symbol of kStaticRecords records
// (16 MiB); every GPU on which the library is loaded holds it until the
// process exits.  Host code cannot use the symbol's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it together
// with the unique ID of the device's current context; that first call should
// therefore come before any stream capture.  A later call in another context
// of the device (after cudaDeviceReset, the array is loaded anew) looks the
// address up again, and should likewise not be the first call inside a
// capture.  Every call shares the array and leaves its last contents behind:
// the wrapped call zeroes the part it uses before accumulating, and two
// calls whose work overlaps on the GPU (different streams, no ordering) race
// on it.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace lgs {

// 524,288 (camera, Gaussian) records of 8 floats: 16 MiB.
constexpr int64_t kStaticRecords = (int64_t)1 << 19;
static constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_static_grad2d[kStaticRecords * LGS_PROJ_STRIDE];

static std::mutex g_static_mu;
static float* g_static_ptr[kMaxDevices];
static unsigned long long g_static_ctx[kMaxDevices];  // context the address belongs to

// Unique ID of the calling thread's current context (0: none is current, or
// the driver entry points are unavailable).
static unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(p);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_static_grad2d on the current device, looked up on the
// first call and again when the device's current context has changed.
static lgs_status static_scratch(float** out) {
  int dev = -1;
  LGS_CHECK_CUDA(cudaGetDevice(&dev));
  LGS_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "device index out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  const unsigned long long ctx = current_context_id();
  if (g_static_ptr[dev] == nullptr || ctx == 0 || ctx != g_static_ctx[dev]) {
    void* p = nullptr;
    LGS_CHECK_CUDA(cudaGetSymbolAddress(&p, g_static_grad2d));  // makes the context current
    g_static_ptr[dev] = static_cast<float*>(p);
    g_static_ctx[dev] = current_context_id();
  }
  *out = g_static_ptr[dev];
  return LGS_OK;
}

}  // namespace lgs

using namespace lgs;

extern "C" int64_t gs_render_bwd_static_capacity(void) { return kStaticRecords; }

extern "C" lgs_status gs_render_bwd_static(
    const float* means, const float* quats, const float* log_scales,
    const float* opacity_logits, const float* proj, const uint32_t* ids,
    const uint32_t* ranges, int64_t n, const lgs_camera* cams_host, int n_cams,
    const void* colors, const void* feats, int feat_dim, int chan_dtype, const float* bg_host,
    const float* T_final, const uint32_t* last, const float* d_rgb, const float* d_depth,
    const float* d_feat, float* d_means, float* d_quats, float* d_log_scales,
    float* d_opacity_logits, float* d_colors, float* d_feats, void* stream) {
  clear_error();
  LGS_CHECK_ARG(n >= 0 && n_cams >= 1 && n_cams <= LGS_MAX_CAMS, "bad n or n_cams");
  LGS_CHECK_ARG((int64_t)n_cams * n <= kStaticRecords,
                "n_cams * n exceeds the static scratch of 524288 (camera, Gaussian) records");
  float* scratch = nullptr;
  lgs_status st = static_scratch(&scratch);
  if (st != LGS_OK) return st;
  return gs_render_bwd(means, quats, log_scales, opacity_logits, proj, ids, ranges, n, cams_host,
                       n_cams, colors, feats, feat_dim, chan_dtype, bg_host, T_final, last, d_rgb,
                       d_depth, d_feat, scratch, d_means, d_quats, d_log_scales, d_opacity_logits,
                       d_colors, d_feats, stream);
}
