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
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should therefore come before any stream capture.  Every call shares
// the array and leaves its last contents behind: the wrapped call zeroes the
// part it uses before accumulating, and two calls whose work overlaps on the
// GPU (different streams, no ordering) race on it.
#include <mutex>

#include "common.cuh"

namespace lgs {

// 524,288 (camera, Gaussian) records of 8 floats: 16 MiB.
constexpr int64_t kStaticRecords = (int64_t)1 << 19;
static constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_static_grad2d[kStaticRecords * LGS_PROJ_STRIDE];

static std::mutex g_static_mu;
static float* g_static_ptr[kMaxDevices];

// Device address of g_static_grad2d on the current device (looked up once).
static lgs_status static_scratch(float** out) {
  int dev = -1;
  LGS_CHECK_CUDA(cudaGetDevice(&dev));
  LGS_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "device index out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev] == nullptr) {
    void* p = nullptr;
    LGS_CHECK_CUDA(cudaGetSymbolAddress(&p, g_static_grad2d));
    g_static_ptr[dev] = static_cast<float*>(p);
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
