// Shared device helpers and host-side argument checking for liblgs.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "lgs.h"

namespace lgs {

// ---------------------------------------------------------------- host errors
void set_error(const std::string& msg);
void clear_error();

#define LGS_CHECK_ARG(cond, msg)                     \
  do {                                               \
    if (!(cond)) {                                   \
      ::lgs::set_error(std::string(__func__) + ": " + (msg)); \
      return LGS_ERR_INVALID;                        \
    }                                                \
  } while (0)

#define LGS_CHECK_CUDA(expr)                                                   \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::lgs::set_error(std::string(__func__) + ": " + cudaGetErrorString(e_)); \
      return LGS_ERR_CUDA;                                                     \
    }                                                                          \
  } while (0)

#define LGS_CHECK_LAUNCH() LGS_CHECK_CUDA(cudaGetLastError())

// Raises a kernel's dynamic shared-memory limit once per process.
cudaError_t set_smem_limit(const void* func, int bytes);

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- constants
// Thresholds of the compositing rule (front-to-back alpha blending of the
// standard 3DGS pipeline that Sec. III-B.1 renders with).
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr int kTile = LGS_TILE;
constexpr int kTilePixels = kTile * kTile;

// Cameras passed by value to kernels (a keyframe window).
struct CamBlock {
  lgs_camera cam[LGS_MAX_CAMS];
};

// ---------------------------------------------------------------- device math
// The compositing decision arithmetic is pinned with explicit round-to-nearest
// intrinsics so the forward and the backward reach bit-identical alphas.
__device__ __forceinline__ float gauss_power(float a, float b, float c, float dx, float dy) {
  // -(a dx^2 + c dy^2)/2 - b dx dy
  float q = __fmul_rn(a, __fmul_rn(dx, dx));
  q = __fmaf_rn(c, __fmul_rn(dy, dy), q);
  float cross = __fmul_rn(b, __fmul_rn(dx, dy));
  return __fmaf_rn(-0.5f, q, -cross);
}

__device__ __forceinline__ float raw_alpha(float o, float power) {
  return __fmul_rn(o, __expf(power));
}

// GELU in its tanh form (Hendrycks & Gimpel): 0.5 x (1 + tanh(u)),
// u = sqrt(2/pi) (x + 0.044715 x^3), with the hardware tanh approximation,
// and its derivative 0.5 (1 + t) + 0.5 x (1 - t^2) sqrt(2/pi) (1 + 0.134145 x^2).
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu_tanh(float x) {
  const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
  return 0.5f * x * (1.f + tanh_approx(u));
}
__device__ __forceinline__ float gelu_tanh_grad(float x) {
  const float x2 = x * x;
  const float t = tanh_approx(0.7978845608028654f * fmaf(0.044715f * x, x2, x));
  return fmaf(0.5f, 1.f + t,
              0.5f * x * (1.f - t * t) * 0.7978845608028654f * fmaf(0.134145f, x2, 1.f));
}

// The same two functions on a pair of values with the packed FP32 pipe
// (FFMA2 / FMUL2 / FADD2: per component identical to the scalar
// round-to-nearest operations), two tanh per pair.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 tanh_approx2(float2 u) {
  return f2(tanh_approx(u.x), tanh_approx(u.y));
}
__device__ __forceinline__ float2 gelu_tanh2(float2 x) {
  constexpr float K = 0.7978845608028654f, KC = 0.7978845608028654f * 0.044715f;
  const float2 x2 = __fmul2_rn(x, x);
  const float2 t = tanh_approx2(__fmul2_rn(x, __ffma2_rn(x2, f2(KC, KC), f2(K, K))));
  const float2 h = __fmul2_rn(x, f2(0.5f, 0.5f));
  return __ffma2_rn(h, t, h);
}
__device__ __forceinline__ float2 gelu_tanh_grad2(float2 x) {
  constexpr float K = 0.7978845608028654f, KC = 0.7978845608028654f * 0.044715f,
                  K3 = 0.7978845608028654f * 0.134145f;
  const float2 x2 = __fmul2_rn(x, x);
  const float2 t = tanh_approx2(__fmul2_rn(x, __ffma2_rn(x2, f2(KC, KC), f2(K, K))));
  const float2 q = __ffma2_rn(x2, f2(K3, K3), f2(K, K));               // K (1 + 3c x^2)
  const float2 s = __ffma2_rn(t, f2(-t.x, -t.y), f2(1.f, 1.f));        // 1 - t^2
  const float2 r = __fmul2_rn(__fmul2_rn(x, f2(0.5f, 0.5f)), s);       // x (1 - t^2) / 2
  return __ffma2_rn(r, q, __ffma2_rn(t, f2(0.5f, 0.5f), f2(0.5f, 0.5f)));
}

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }

}  // namespace lgs
