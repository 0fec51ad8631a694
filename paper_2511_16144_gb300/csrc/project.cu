// EWA projection of 3D Gaussians (forward) and its chain-rule backward.
//
// LEGO-SLAM Sec. III-B.1 renders its language-embedded Gaussians "following
// the standard 3DGS pipeline"; this is that pipeline's projection: camera
// transform, local affine (Jacobian) approximation of the perspective map,
// 2D covariance with a 0.3 px^2 low-pass dilation, its inverse (the conic)
// and the tile rectangle of the support where o exp(power) >= 1/255.
#include <cmath>
#include <string>

#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

// Smallest index of a Gaussian with a non-finite parameter (LGS_ERR_NONFINITE
// of lgs_sync_status); all ones = none.
__device__ unsigned long long g_nonfinite = ~0ull;

struct ProjState {
  float qn[4], qnorm;
  float Rq[9], s[3], M[9], S3[9];
  float t[3];
  float txc, tyc, limx, limy;
  int clampx, clampy;
  float T2[6];    // J R_c
  float S2[3];    // Sigma2 (00, 01, 11) with dilation
  float conic[3];
  float u, v, o;
  bool valid;     // passes depth, determinant and opacity tests
};

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Everything the projection computes for one Gaussian and one camera.
__device__ void project_state(const float* p, const float4 q, const float* ls, float logit,
                              const lgs_camera& cam, ProjState& P) {
  P.valid = false;
  float qq = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  P.qnorm = qq;
  float inv = qq > 0.f ? 1.f / qq : 0.f;
  P.qn[0] = q.x * inv; P.qn[1] = q.y * inv; P.qn[2] = q.z * inv; P.qn[3] = q.w * inv;
  float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
  float* R = P.Rq;
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int k = 0; k < 3; k++) P.s[k] = expf(ls[k]);
#pragma unroll
  for (int j = 0; j < 3; j++)
#pragma unroll
    for (int k = 0; k < 3; k++) P.M[3 * j + k] = R[3 * j + k] * P.s[k];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++)
      P.S3[3 * i + j] = P.M[3 * i] * P.M[3 * j] + P.M[3 * i + 1] * P.M[3 * j + 1] +
                        P.M[3 * i + 2] * P.M[3 * j + 2];
  const float* V = cam.viewmat;
#pragma unroll
  for (int i = 0; i < 3; i++)
    P.t[i] = V[4 * i] * p[0] + V[4 * i + 1] * p[1] + V[4 * i + 2] * p[2] + V[4 * i + 3];
  P.o = sigmoidf_(logit);
  float tz = P.t[2];
  if (!(tz > cam.znear) || !(qq > 0.f)) return;

  float W = (float)cam.width, H = (float)cam.height;
  float lox = (-0.15f * W - cam.cx) / cam.fx, hix = (1.15f * W - cam.cx) / cam.fx;
  float loy = (-0.15f * H - cam.cy) / cam.fy, hiy = (1.15f * H - cam.cy) / cam.fy;
  float rx = P.t[0] / tz, ry = P.t[1] / tz;
  P.clampx = rx < lox ? -1 : (rx > hix ? 1 : 0);
  P.clampy = ry < loy ? -1 : (ry > hiy ? 1 : 0);
  P.limx = P.clampx < 0 ? lox : hix;
  P.limy = P.clampy < 0 ? loy : hiy;
  P.txc = (P.clampx ? P.limx : rx) * tz;
  P.tyc = (P.clampy ? P.limy : ry) * tz;
  float J00 = cam.fx / tz, J02 = -cam.fx * P.txc / (tz * tz);
  float J11 = cam.fy / tz, J12 = -cam.fy * P.tyc / (tz * tz);
#pragma unroll
  for (int j = 0; j < 3; j++) {
    P.T2[j] = J00 * V[j] + J02 * V[8 + j];
    P.T2[3 + j] = J11 * V[4 + j] + J12 * V[8 + j];
  }
  float A[6];  // T2 S3 (2x3)
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 3; j++)
      A[3 * i + j] = P.T2[3 * i] * P.S3[j] + P.T2[3 * i + 1] * P.S3[3 + j] +
                     P.T2[3 * i + 2] * P.S3[6 + j];
  float s00 = A[0] * P.T2[0] + A[1] * P.T2[1] + A[2] * P.T2[2];
  float s01 = A[0] * P.T2[3] + A[1] * P.T2[4] + A[2] * P.T2[5];
  float s11 = A[3] * P.T2[3] + A[4] * P.T2[4] + A[5] * P.T2[5];
  P.S2[0] = s00 + kDilation;
  P.S2[1] = s01;
  P.S2[2] = s11 + kDilation;
  float det = P.S2[0] * P.S2[2] - P.S2[1] * P.S2[1];
  if (!(det > 0.f)) return;
  float idet = 1.f / det;
  P.conic[0] = P.S2[2] * idet;
  P.conic[1] = -P.S2[1] * idet;
  P.conic[2] = P.S2[0] * idet;
  P.u = cam.fx * P.t[0] / tz + cam.cx;
  P.v = cam.fy * P.t[1] / tz + cam.cy;
  if (!(P.o >= kAlphaMin)) return;
  P.valid = true;
}

// Tile rectangle of the support; false when it misses the image.
__device__ bool support_rect(const ProjState& P, const lgs_camera& cam, ushort4& rect) {
  float m = 0.5f * (P.S2[0] + P.S2[2]);
  float hd = 0.5f * (P.S2[0] - P.S2[2]);
  float lam = m + sqrtf(hd * hd + P.S2[1] * P.S2[1]);
  float e = sqrtf(2.f * logf(255.f * P.o) * lam);
  float r = e * (1.f + 1e-5f) + 1e-3f;
  float W1 = (float)(cam.width - 1), H1 = (float)(cam.height - 1);
  float x0 = fmaxf(ceilf(P.u - r - 0.5f), 0.f), x1 = fminf(floorf(P.u + r - 0.5f), W1);
  float y0 = fmaxf(ceilf(P.v - r - 0.5f), 0.f), y1 = fminf(floorf(P.v + r - 0.5f), H1);
  if (!(x0 <= x1) || !(y0 <= y1)) return false;
  rect.x = (unsigned short)((int)x0 / kTile);
  rect.y = (unsigned short)((int)y0 / kTile);
  rect.z = (unsigned short)((int)x1 / kTile + 1);
  rect.w = (unsigned short)((int)y1 / kTile + 1);
  return true;
}

__global__ void project_kernel(const float* __restrict__ means, const float4* __restrict__ quats,
                               const float* __restrict__ log_scales,
                               const float* __restrict__ logits, int64_t n, CamBlock cams,
                               float4* __restrict__ proj, ushort4* __restrict__ rect) {
  int c = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const lgs_camera& cam = cams.cam[c];
    float p[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float ls[3] = {log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2]};
    const float4 q = quats[i];
    const float lg = logits[i];
    const bool finite = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(ls[0]) &&
                        isfinite(ls[1]) && isfinite(ls[2]) && isfinite(q.x) && isfinite(q.y) &&
                        isfinite(q.z) && isfinite(q.w) && isfinite(lg);
    if (!finite && c == 0) atomicMin(&g_nonfinite, (unsigned long long)i);
    ProjState P;
    project_state(p, q, ls, lg, cam, P);
    ushort4 r = make_ushort4(0, 0, 0, 0);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (finite && P.valid && support_rect(P, cam, r)) {
      a = make_float4(P.u, P.v, P.conic[0], P.conic[1]);
      // the cutoff of the tile test: a pixel with o e^power >= 1/255 has
      // q = -2 power <= 2 ln(255 o); the margin covers the FP32 rounding of
      // q here and in the renderer (power, exponential)
      const float cut = fmaf(2.f * logf(255.f * P.o), 1.001f, 1e-2f);
      b = make_float4(P.conic[2], P.o, P.t[2], cut);
    } else {
      r = make_ushort4(0, 0, 0, 0);
    }
    int64_t k = (int64_t)c * n + i;
    proj[2 * k] = a;
    proj[2 * k + 1] = b;
    rect[k] = r;
  }
}

// Chain rule from the 2D gradients g7 = d(u, v, a, b, c, o, tz) of one
// (camera, Gaussian) to the parameters (accumulated into the outputs).
// The camera-space part of the projection backward: from the 2D gradient
// record g7 = d(u, v, a, b, c, o, t_z) to dS3 (world 3D covariance), dJ (the
// full 2x3 gradient of the EWA Jacobian J, row-major) and dt (camera-space
// mean).
__device__ __forceinline__ void camera_backward(const ProjState& P, const lgs_camera& cam,
                                                const float* g7, float* dS3, float* dJ,
                                                float& dt0, float& dt1, float& dt2) {
  float du = g7[0], dv = g7[1], da = g7[2], db = g7[3], dc = g7[4], dz = g7[6];
  float tx = P.t[0], ty = P.t[1], tz = P.t[2];
  float fx = cam.fx, fy = cam.fy;
  const float* V = cam.viewmat;
  // conic = Sigma2^-1: dSigma2 = -Q G Q, G = [[da, db/2], [db/2, dc]]
  float Q00 = P.conic[0], Q01 = P.conic[1], Q11 = P.conic[2];
  float G01 = 0.5f * db;
  float QG00 = Q00 * da + Q01 * G01, QG01 = Q00 * G01 + Q01 * dc;
  float QG10 = Q01 * da + Q11 * G01, QG11 = Q01 * G01 + Q11 * dc;
  float dS00 = -(QG00 * Q00 + QG01 * Q01);
  float dS01 = -(QG00 * Q01 + QG01 * Q11);
  float dS11 = -(QG10 * Q01 + QG11 * Q11);
  // Sigma2 = T Sigma3 T^T: dSigma3 = T^T dS T, dT = 2 dS T Sigma3
  const float* T = P.T2;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++)
      dS3[3 * i + j] = T[i] * (dS00 * T[j] + dS01 * T[3 + j]) +
                       T[3 + i] * (dS01 * T[j] + dS11 * T[3 + j]);
  float TS[6];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 3; j++)
      TS[3 * i + j] = T[3 * i] * P.S3[j] + T[3 * i + 1] * P.S3[3 + j] + T[3 * i + 2] * P.S3[6 + j];
  float dT[6];
#pragma unroll
  for (int j = 0; j < 3; j++) {
    dT[j] = 2.f * (dS00 * TS[j] + dS01 * TS[3 + j]);
    dT[3 + j] = 2.f * (dS01 * TS[j] + dS11 * TS[3 + j]);
  }
  // T = J R_c: dJ = dT R_c^T
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      dJ[3 * k + b] = dT[3 * k] * V[4 * b] + dT[3 * k + 1] * V[4 * b + 1] +
                      dT[3 * k + 2] * V[4 * b + 2];
  const float dJ00 = dJ[0], dJ02 = dJ[2], dJ11 = dJ[4], dJ12 = dJ[5];
  float itz = 1.f / tz, itz2 = itz * itz;
  dt0 = 0.f;
  dt1 = 0.f;
  dt2 = 0.f;
  dt2 += -dJ00 * fx * itz2 + dJ02 * 2.f * fx * P.txc * itz2 * itz;
  if (P.clampx) dt2 += -dJ02 * fx * P.limx * itz2;
  else dt0 += -dJ02 * fx * itz2;
  dt2 += -dJ11 * fy * itz2 + dJ12 * 2.f * fy * P.tyc * itz2 * itz;
  if (P.clampy) dt2 += -dJ12 * fy * P.limy * itz2;
  else dt1 += -dJ12 * fy * itz2;
  // u = fx tx/tz + cx, v = fy ty/tz + cy, depth = tz
  dt0 += du * fx * itz;
  dt1 += dv * fy * itz;
  dt2 += -(du * fx * tx + dv * fy * ty) * itz2 + dz;
}

__device__ void project_backward(const ProjState& P, const lgs_camera& cam, const float* g7,
                                 float* dmean, float* dquat, float* dls, float& dlogit) {
  const float* V = cam.viewmat;
  float dS3[9], dJ[6], dt0, dt1, dt2;
  camera_backward(P, cam, g7, dS3, dJ, dt0, dt1, dt2);
  dlogit += g7[5] * P.o * (1.f - P.o);
  // t = R_c p + t_c
#pragma unroll
  for (int j = 0; j < 3; j++) dmean[j] += V[j] * dt0 + V[4 + j] * dt1 + V[8 + j] * dt2;
  // Sigma3 = M M^T with M = R S: dM = 2 dSigma3 M
  float dM[9];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++)
      dM[3 * i + j] = 2.f * (dS3[3 * i] * P.M[j] + dS3[3 * i + 1] * P.M[3 + j] +
                             dS3[3 * i + 2] * P.M[6 + j]);
  float dR[9];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float ds = dM[k] * P.Rq[k] + dM[3 + k] * P.Rq[3 + k] + dM[6 + k] * P.Rq[6 + k];
    dls[k] += ds * P.s[k];
#pragma unroll
    for (int j = 0; j < 3; j++) dR[3 * j + k] = dM[3 * j + k] * P.s[k];
  }
  float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
  float dq[4];
  dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                 w * dR[7] - 2.f * x * dR[8]);
  dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                 z * dR[7] - 2.f * y * dR[8]);
  dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                 y * dR[5] + x * dR[6] + y * dR[7]);
  float dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
  float iq = 1.f / P.qnorm;
#pragma unroll
  for (int i = 0; i < 4; i++) dquat[i] += (dq[i] - P.qn[i] * dot) * iq;
}

// One thread per Gaussian, summing the chain rule over cameras.
__global__ void project_bwd_kernel(const float* __restrict__ means, const float4* __restrict__ quats,
                                   const float* __restrict__ log_scales,
                                   const float* __restrict__ logits, int64_t n, int n_cams,
                                   CamBlock cams, const float4* __restrict__ grad2d,
                                   float* __restrict__ d_means, float* __restrict__ d_quats,
                                   float* __restrict__ d_log_scales, float* __restrict__ d_logits) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float dm[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f}, dl[3] = {0.f, 0.f, 0.f};
    float dlg = 0.f;
    bool any = false;
    float p[3], ls[3];
    float4 q;
    for (int c = 0; c < n_cams; c++) {
      int64_t k = (int64_t)c * n + i;
      float4 g0 = grad2d[2 * k], g1 = grad2d[2 * k + 1];
      if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f &&
          g1.y == 0.f && g1.z == 0.f)
        continue;
      if (!any) {
        p[0] = means[3 * i]; p[1] = means[3 * i + 1]; p[2] = means[3 * i + 2];
        ls[0] = log_scales[3 * i]; ls[1] = log_scales[3 * i + 1]; ls[2] = log_scales[3 * i + 2];
        q = quats[i];
        any = true;
      }
      ProjState P;
      project_state(p, q, ls, logits[i], cams.cam[c], P);
      if (!P.valid) continue;
      float g7[7] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z};
      project_backward(P, cams.cam[c], g7, dm, dq, dl, dlg);
    }
    if (!any) continue;
    for (int j = 0; j < 3; j++) d_means[3 * i + j] += dm[j];
    for (int j = 0; j < 4; j++) d_quats[4 * i + j] += dq[j];
    for (int j = 0; j < 3; j++) d_log_scales[3 * i + j] += dl[j];
    d_logits[i] += dlg;
  }
}

lgs_status launch_project_bwd(const float* means, const float* quats, const float* log_scales,
                              const float* logits, int64_t n, int n_cams, const CamBlock& cams,
                              const float* grad2d, float* d_means, float* d_quats,
                              float* d_log_scales, float* d_logits, cudaStream_t s) {
  if (n == 0) return LGS_OK;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  project_bwd_kernel<<<blocks, 256, 0, s>>>(means, (const float4*)quats, log_scales, logits, n,
                                            n_cams, cams, (const float4*)grad2d, d_means,
                                            d_quats, d_log_scales, d_logits);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

// Camera pose gradient: a left perturbation T <- exp(xi^) T of camera c's
// world->camera transform, xi = (rho, phi), moves each camera-space mean to
// t + phi x t + rho and turns J R_c into J (I + phi^) R_c, so per Gaussian
// dL/drho += dL/dt and dL/dphi += t x dL/dt + (A21 - A12, A02 - A20, A10 - A01)
// with A = J^T dJ.  One thread per (Gaussian, camera); a block sums its six
// values and adds them to d_pose[c] once.
__global__ void __launch_bounds__(256)
pose_grad_kernel(const float* __restrict__ means, const float4* __restrict__ quats,
                 const float* __restrict__ log_scales, const float* __restrict__ logits,
                 int64_t n, CamBlock cams, const float4* __restrict__ grad2d,
                 float* __restrict__ d_pose) {
  __shared__ float red[8][6];
  const int c = blockIdx.y;
  const lgs_camera& cam = cams.cam[c];
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = (int64_t)c * n + i;
    const float4 g0 = grad2d[2 * k], g1 = grad2d[2 * k + 1];
    if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f &&
        g1.y == 0.f && g1.z == 0.f)
      continue;
    const float p[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    const float ls[3] = {log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2]};
    ProjState P;
    project_state(p, quats[i], ls, logits[i], cam, P);
    if (!P.valid) continue;
    const float g7[7] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z};
    float dS3[9], dJ[6], dt0, dt1, dt2;
    camera_backward(P, cam, g7, dS3, dJ, dt0, dt1, dt2);
    const float tz = P.t[2], itz = 1.f / tz;
    const float J00 = cam.fx * itz, J02 = -cam.fx * P.txc * itz * itz;
    const float J11 = cam.fy * itz, J12 = -cam.fy * P.tyc * itz * itz;
    const float A01 = J00 * dJ[1], A02 = J00 * dJ[2];
    const float A10 = J11 * dJ[3], A12 = J11 * dJ[5];
    const float A20 = J02 * dJ[0] + J12 * dJ[3], A21 = J02 * dJ[1] + J12 * dJ[4];
    const float tx = P.t[0], ty = P.t[1];
    acc[0] += dt0;
    acc[1] += dt1;
    acc[2] += dt2;
    acc[3] += ty * dt2 - tz * dt1 + A21 - A12;
    acc[4] += tz * dt0 - tx * dt2 + A02 - A20;
    acc[5] += tx * dt1 - ty * dt0 + A10 - A01;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 6; j++) {
    float v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = 0.f;
    for (int w = 0; w < 8; w++) v += red[w][threadIdx.x];
    if (v != 0.f) atomicAdd(d_pose + 6 * c + threadIdx.x, v);
  }
}

lgs_status fill_cams(const lgs_camera* cams_host, int n_cams, CamBlock& cb) {
  LGS_CHECK_ARG(cams_host != nullptr, "cams_host is null");
  LGS_CHECK_ARG(n_cams >= 1 && n_cams <= LGS_MAX_CAMS, "n_cams out of range");
  for (int c = 0; c < n_cams; c++) {
    const lgs_camera& k = cams_host[c];
    bool finite = std::isfinite(k.fx) && std::isfinite(k.fy) && std::isfinite(k.cx) &&
                  std::isfinite(k.cy) && std::isfinite(k.znear);
    for (int j = 0; j < 12; j++) finite = finite && std::isfinite(k.viewmat[j]);
    if (!finite) {
      set_error(std::string(__func__) + ": camera " + std::to_string(c) +
                " has a non-finite value");
      return LGS_ERR_NONFINITE;
    }
    LGS_CHECK_ARG(k.width > 0 && k.height > 0 && k.width <= 65535 * kTile &&
                      k.height <= 65535 * kTile,
                  "bad image size");
    LGS_CHECK_ARG(k.fx > 0.f && k.fy > 0.f && k.znear > 0.f, "bad intrinsics");
    cb.cam[c] = k;
  }
  return LGS_OK;
}

unsigned long long nonfinite_word(bool clear) {
  unsigned long long v = ~0ull, none = ~0ull;
  if (cudaMemcpyFromSymbol(&v, g_nonfinite, sizeof(v)) != cudaSuccess) return ~0ull;
  if (clear && v != none) cudaMemcpyToSymbol(g_nonfinite, &none, sizeof(none));
  return v;
}

}  // namespace lgs

using namespace lgs;

extern "C" lgs_status gs_project(const float* means, const float* quats, const float* log_scales,
                                 const float* opacity_logits, int64_t n,
                                 const lgs_camera* cams_host, int n_cams, float* proj,
                                 uint16_t* rect, void* stream) {
  clear_error();
  LGS_CHECK_ARG(n >= 0 && n < (int64_t)1 << 32, "n out of range");
  CamBlock cb;
  lgs_status st = fill_cams(cams_host, n_cams, cb);
  if (st != LGS_OK) return st;
  if (n == 0) return LGS_OK;
  LGS_CHECK_ARG(means && quats && log_scales && opacity_logits && proj && rect, "null pointer");
  LGS_CHECK_ARG(aligned(quats, 16) && aligned(proj, 16) && aligned(rect, 8), "misaligned pointer");
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), n_cams);
  project_kernel<<<grid, 256, 0, as_stream(stream)>>>(means, (const float4*)quats, log_scales,
                                                      opacity_logits, n, cb, (float4*)proj,
                                                      (ushort4*)rect);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

extern "C" lgs_status gs_pose_grad(const float* means, const float* quats, const float* log_scales,
                                   const float* opacity_logits, int64_t n,
                                   const lgs_camera* cams_host, int n_cams, const float* grad2d,
                                   float* d_pose, void* stream) {
  clear_error();
  LGS_CHECK_ARG(n >= 0 && n < (int64_t)1 << 32, "n out of range");
  CamBlock cb;
  lgs_status st = fill_cams(cams_host, n_cams, cb);
  if (st != LGS_OK) return st;
  LGS_CHECK_ARG(d_pose, "d_pose is null");
  cudaStream_t s = as_stream(stream);
  LGS_CHECK_CUDA(cudaMemsetAsync(d_pose, 0, sizeof(float) * 6 * (size_t)n_cams, s));
  if (n == 0) return LGS_OK;
  LGS_CHECK_ARG(means && quats && log_scales && opacity_logits && grad2d, "null pointer");
  LGS_CHECK_ARG(aligned(quats, 16) && aligned(grad2d, 16), "misaligned pointer");
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 152 * 4), n_cams);
  pose_grad_kernel<<<grid, 256, 0, s>>>(means, (const float4*)quats, log_scales, opacity_logits,
                                        n, cb, (const float4*)grad2d, d_pose);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
