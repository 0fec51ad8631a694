// D-SSIM term of the photometric loss (LEGO-SLAM Sec. III-B.3: L_rgb combines
// an L1 and a D-SSIM term between the rendered and the observed image).
//
// SSIM per colour channel with an 11 x 11 Gaussian window (sigma 1.5,
// normalised), the images zero outside their borders, C1 = 0.01^2,
// C2 = 0.03^2:  mu = G * x, s_x^2 = G * x^2 - mu_x^2, s_xy = G * xy - mu_x mu_y,
// SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)).
// loss += weight (1 - mean SSIM).  Its gradient: with s = -weight / N per
// pixel and channel, b = dL/ds_x^2, c = dL/ds_xy and a = dL/dmu_x - 2 mu_x b -
// mu_y c, dL/dx = G * a + 2 x (G * b) + y (G * c).
//
// Two kernels over 16 x 16 output tiles, each staging a 26 x 26 halo patch in
// shared memory and filtering separably (rows, then columns): the forward
// forms the five window sums, SSIM and the (a, b, c) maps; the backward
// filters (a, b, c) and forms the gradient.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace lgs {

namespace {

constexpr int kT = 16;            // output tile edge
constexpr int kR = 5;             // window radius
constexpr int kP = kT + 2 * kR;   // halo'd patch edge
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;

struct Img {
  int n, h, w;
};

// normalised Gaussian taps, passed by value
struct Win {
  float g[2 * kR + 1];
};

// Loads channel ch of `nmaps` [n,H,W,3] maps into smem patches (zero outside).
template <int NMAPS>
__device__ __forceinline__ void load_patch(const float* const* maps, const Img& im, int img, int ch,
                                           int x0, int y0, float (*patch)[kP * kP]) {
  for (int e = threadIdx.x; e < kP * kP; e += blockDim.x) {
    const int px = x0 - kR + e % kP, py = y0 - kR + e / kP;
    const bool in = px >= 0 && py >= 0 && px < im.w && py < im.h;
    const int64_t o = ((((int64_t)img * im.h + (in ? py : 0)) * im.w + (in ? px : 0)) * 3) + ch;
#pragma unroll
    for (int m = 0; m < NMAPS; m++) patch[m][e] = in ? maps[m][o] : 0.f;
  }
}

__global__ void __launch_bounds__(256)
ssim_fwd_kernel(const float* __restrict__ x, const float* __restrict__ y, Img im, Win win, float s,
                float* __restrict__ amap, float* __restrict__ bmap, float* __restrict__ cmap,
                float weight, float inv_n, float* __restrict__ loss) {
  __shared__ float patch[2][kP * kP];
  __shared__ float rows[5][kP * kT];
  __shared__ float red[8];
  const int tiles_x = (im.w + kT - 1) / kT, tiles_y = (im.h + kT - 1) / kT;
  const int img = blockIdx.x / (tiles_x * tiles_y);
  const int t = blockIdx.x - img * tiles_x * tiles_y;
  const int x0 = (t % tiles_x) * kT, y0 = (t / tiles_x) * kT;
  const int lx = threadIdx.x % kT, ly = threadIdx.x / kT;
  const int px = x0 + lx, py = y0 + ly;
  const bool inside = px < im.w && py < im.h;
  const float* maps[2] = {x, y};
  float part = 0.f;
  for (int ch = 0; ch < 3; ch++) {
    __syncthreads();
    load_patch<2>(maps, im, img, ch, x0, y0, patch);
    __syncthreads();
    // rows: kP rows x kT output columns, five sums each
    for (int e = threadIdx.x; e < kP * kT; e += blockDim.x) {
      const int r = e / kT, cx = e % kT;
      float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; k++) {
        const float a = patch[0][r * kP + cx + k], b = patch[1][r * kP + cx + k], g = win.g[k];
        mx = fmaf(g, a, mx);
        my = fmaf(g, b, my);
        xx = fmaf(g, a * a, xx);
        yy = fmaf(g, b * b, yy);
        xy = fmaf(g, a * b, xy);
      }
      rows[0][e] = mx; rows[1][e] = my; rows[2][e] = xx; rows[3][e] = yy; rows[4][e] = xy;
    }
    __syncthreads();
    float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; k++) {
      const int e = (ly + k) * kT + lx;
      const float g = win.g[k];
      mx = fmaf(g, rows[0][e], mx);
      my = fmaf(g, rows[1][e], my);
      xx = fmaf(g, rows[2][e], xx);
      yy = fmaf(g, rows[3][e], yy);
      xy = fmaf(g, rows[4][e], xy);
    }
    if (inside) {
      const float vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
      const float a1 = 2.f * mx * my + kC1, a2 = 2.f * cxy + kC2;
      const float b1 = mx * mx + my * my + kC1, b2 = vx + vy + kC2;
      const float ib = 1.f / (b1 * b2);
      const float ssim = a1 * a2 * ib;
      part += 1.f - ssim;
      const float dmx = s * (2.f * my * a2 * ib - 2.f * mx * ssim / b1);
      const float b = -s * ssim / b2;
      const float c = s * 2.f * a1 * ib;
      const int64_t o = ((((int64_t)img * im.h + py) * im.w + px) * 3) + ch;
      amap[o] = dmx - 2.f * mx * b - my * c;
      bmap[o] = b;
      cmap[o] = c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int w = 0; w < 8; w++) v += red[w];
    atomicAdd(loss, weight * inv_n * v);
  }
}

__global__ void __launch_bounds__(256)
ssim_bwd_kernel(const float* __restrict__ x, const float* __restrict__ y, Img im, Win win,
                const float* __restrict__ amap, const float* __restrict__ bmap,
                const float* __restrict__ cmap, float* __restrict__ grad) {
  __shared__ float patch[3][kP * kP];
  __shared__ float rows[3][kP * kT];
  const int tiles_x = (im.w + kT - 1) / kT, tiles_y = (im.h + kT - 1) / kT;
  const int img = blockIdx.x / (tiles_x * tiles_y);
  const int t = blockIdx.x - img * tiles_x * tiles_y;
  const int x0 = (t % tiles_x) * kT, y0 = (t / tiles_x) * kT;
  const int lx = threadIdx.x % kT, ly = threadIdx.x / kT;
  const int px = x0 + lx, py = y0 + ly;
  const bool inside = px < im.w && py < im.h;
  const float* maps[3] = {amap, bmap, cmap};
  for (int ch = 0; ch < 3; ch++) {
    __syncthreads();
    load_patch<3>(maps, im, img, ch, x0, y0, patch);
    __syncthreads();
    for (int e = threadIdx.x; e < kP * kT; e += blockDim.x) {
      const int r = e / kT, cx = e % kT;
      float sa = 0.f, sb = 0.f, sc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; k++) {
        const float g = win.g[k];
        const int q = r * kP + cx + k;
        sa = fmaf(g, patch[0][q], sa);
        sb = fmaf(g, patch[1][q], sb);
        sc = fmaf(g, patch[2][q], sc);
      }
      rows[0][e] = sa; rows[1][e] = sb; rows[2][e] = sc;
    }
    __syncthreads();
    if (inside) {
      float ga = 0.f, gb = 0.f, gc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; k++) {
        const int e = (ly + k) * kT + lx;
        const float g = win.g[k];
        ga = fmaf(g, rows[0][e], ga);
        gb = fmaf(g, rows[1][e], gb);
        gc = fmaf(g, rows[2][e], gc);
      }
      const int64_t o = ((((int64_t)img * im.h + py) * im.w + px) * 3) + ch;
      grad[o] += ga + 2.f * x[o] * gb + y[o] * gc;
    }
  }
}

Win window() {
  Win w;
  double g[2 * kR + 1], sum = 0;
  for (int k = 0; k <= 2 * kR; k++) sum += g[k] = std::exp(-(k - kR) * (k - kR) / (2.0 * 1.5 * 1.5));
  for (int k = 0; k <= 2 * kR; k++) w.g[k] = (float)(g[k] / sum);
  return w;
}

}  // namespace
}  // namespace lgs

using namespace lgs;

extern "C" size_t lgs_dssim_workspace(int n_img, int height, int width) {
  if (n_img < 0 || height < 0 || width < 0) return 0;
  return 3 * sizeof(float) * 3 * (size_t)n_img * height * width;
}

extern "C" lgs_status lgs_dssim_loss(const float* pred, const float* target, int n_img,
                                     int height, int width, float weight, float* grad,
                                     float* loss_dev, void* workspace, size_t workspace_bytes,
                                     void* stream) {
  clear_error();
  LGS_CHECK_ARG(n_img >= 0 && height >= 0 && width >= 0, "negative size");
  LGS_CHECK_ARG((int64_t)n_img * height * width < ((int64_t)1 << 31), "image too large");
  const int64_t npx = (int64_t)n_img * height * width;
  if (npx == 0) return LGS_OK;
  LGS_CHECK_ARG(pred && target && grad && loss_dev && workspace, "null pointer");
  LGS_CHECK_ARG(aligned(workspace, 4) && aligned(pred, 4) && aligned(target, 4) && aligned(grad, 4),
                "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= lgs_dssim_workspace(n_img, height, width), "workspace too small");
  const Win win = window();
  float* amap = (float*)workspace;
  float* bmap = amap + 3 * npx;
  float* cmap = bmap + 3 * npx;
  const Img im{n_img, height, width};
  const int64_t blocks =
      (int64_t)n_img * ((width + kT - 1) / kT) * ((height + kT - 1) / kT);
  const float inv_n = (float)(1.0 / (3.0 * (double)npx));
  cudaStream_t s = as_stream(stream);
  ssim_fwd_kernel<<<(unsigned)blocks, 256, 0, s>>>(pred, target, im, win, -weight * inv_n, amap,
                                                   bmap, cmap, weight, inv_n, loss_dev);
  ssim_bwd_kernel<<<(unsigned)blocks, 256, 0, s>>>(pred, target, im, win, amap, bmap, cmap, grad);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
