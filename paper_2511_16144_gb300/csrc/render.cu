// Tile rasteriser: front-to-back alpha compositing of RGB, depth and a
// D-channel language feature (forward) and its reverse-order backward.
//
// LEGO-SLAM Sec. III-B.1 renders the RGB image and the feature map
// F_render from the language-embedded Gaussians "following the standard
// 3DGS pipeline"; Sec. III-B.3 (Eq. 1-2) optimises the map through them.
//
// Layout: one CTA of 256 threads per 16x16 tile (one thread per pixel) and
// per feature chunk of FC channels; the first chunk also carries RGB and
// depth.  A D = 16 map is one chunk of 20 channels; the plain 512-channel
// path runs 16 chunks of 32 in parallel, each recomputing alpha.
//
// Forward: batches of 256 sorted instances are staged in shared memory (one
// coalesced gather per thread), every pixel walks the batch, and the CTA
// stops as soon as all its pixels have hit the T < 1e-4 stop.
//
// Backward: each pixel walks its instances back to front from `last`,
// recovering T by division from T_final.  dL/dalpha_i = T_i (x_i . g) -
// S_i / (1 - alpha_i) needs only the running scalar S (suffix sum of
// w_k (x_k . g) plus T_final (bg . g)).  Per batch of 16 instances every
// pixel records its blend weight w and dpower = alpha dL/dalpha (0 when the
// 0.99 clamp is active) in shared memory; the warp then transposes the
// reduction so each lane sums, for one instance, w * g over 16 pixels
// (colour / depth / feature gradients) and the spatial moments of dpower
// (sum, x, y, x^2, xy, y^2) from which the 2D-mean, conic and opacity
// gradients follow in closed form.  Lane pairs combine with one shuffle,
// warps with shared-memory atomics, and the CTA issues one vector atomic
// per (tile, instance) to global memory.
#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

constexpr int kThreads = 256;
constexpr int kFwdBatch = 256;
constexpr int kBwdBatch = 16;

struct RasterArgs {
  const float4* proj;
  const uint32_t* ids;
  const uint2* ranges;
  int64_t n;
  int tiles_x, tiles_y, width, height, D;
  const void* colors;
  const void* feats;
  float bg0, bg1, bg2;
  float* rgb;
  float* depth;
  float* feat;
  float* T_final;
  uint32_t* last;
  uint32_t* n_contrib;
  const float* d_rgb;
  const float* d_depth;
  const float* d_feat;
  float4* grad2d;
  float* d_colors;
  float* d_feats;
};

template <typename TC, int FC>
__device__ __forceinline__ void load_feats(const TC* __restrict__ src, float* dst);

template <>
__device__ __forceinline__ void load_feats<float, 8>(const float* __restrict__ src, float* dst) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < 2; q++) reinterpret_cast<float4*>(dst)[q] = s4[q];
}
template <>
__device__ __forceinline__ void load_feats<float, 16>(const float* __restrict__ src, float* dst) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < 4; q++) reinterpret_cast<float4*>(dst)[q] = s4[q];
}
template <>
__device__ __forceinline__ void load_feats<float, 32>(const float* __restrict__ src, float* dst) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < 8; q++) reinterpret_cast<float4*>(dst)[q] = s4[q];
}
template <int FC>
__device__ __forceinline__ void load_bf16_feats(const __nv_bfloat16* __restrict__ src, float* dst) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int q = 0; q < FC / 8; q++) {
    uint4 u = s4[q];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float2 f = __bfloat1622float2(h[k]);
      dst[8 * q + 2 * k] = f.x;
      dst[8 * q + 2 * k + 1] = f.y;
    }
  }
}
template <>
__device__ __forceinline__ void load_feats<__nv_bfloat16, 8>(const __nv_bfloat16* __restrict__ src,
                                                             float* dst) {
  load_bf16_feats<8>(src, dst);
}
template <>
__device__ __forceinline__ void load_feats<__nv_bfloat16, 16>(const __nv_bfloat16* __restrict__ src,
                                                              float* dst) {
  load_bf16_feats<16>(src, dst);
}
template <>
__device__ __forceinline__ void load_feats<__nv_bfloat16, 32>(const __nv_bfloat16* __restrict__ src,
                                                              float* dst) {
  load_bf16_feats<32>(src, dst);
}

// Stages one instance's geometry and channels (RGB, depth first when RGB).
template <int FC, typename TC, bool RGB>
__device__ __forceinline__ void stage_instance(const RasterArgs& A, int64_t projbase, uint32_t g,
                                               int f0, float2& xy, float4& co, float* ch) {
  const float4* rec = A.proj + 2 * (projbase + g);
  float4 r0 = rec[0], r1 = rec[1];
  xy = make_float2(r0.x, r0.y);
  co = make_float4(r0.z, r0.w, r1.x, r1.y);
  if (RGB) {
    const TC* c = reinterpret_cast<const TC*>(A.colors) + 3 * (int64_t)g;
    ch[0] = to_float(c[0]);
    ch[1] = to_float(c[1]);
    ch[2] = to_float(c[2]);
    ch[3] = r1.z;
  }
  load_feats<TC, FC>(reinterpret_cast<const TC*>(A.feats) + (int64_t)g * A.D + f0,
                     ch + (RGB ? 4 : 0));
}

template <int FC, bool RGB>
constexpr int nchan() { return FC + (RGB ? 4 : 0); }

template <int FC, bool RGB>
constexpr size_t fwd_smem() {
  return kFwdBatch * (sizeof(float4) + sizeof(float2) + sizeof(float) * nchan<FC, RGB>());
}

template <int FC, typename TC, bool RGB>
__global__ void __launch_bounds__(kThreads, FC <= 16 ? 4 : 1) render_fwd_kernel(RasterArgs A, int chunk_base) {
  constexpr int NCH = nchan<FC, RGB>();
  extern __shared__ float4 smem4[];
  float4* s_co = smem4;
  float2* s_xy = reinterpret_cast<float2*>(s_co + kFwdBatch);
  float* s_ch = reinterpret_cast<float*>(s_xy + kFwdBatch);

  const int tile = blockIdx.x;
  const int f0 = (chunk_base + blockIdx.y) * FC;
  const int tiles = A.tiles_x * A.tiles_y;
  const int cam = tile / tiles, t = tile - cam * tiles;
  const int tx = t % A.tiles_x, ty = t / A.tiles_x;
  const int px = tx * kTile + (threadIdx.x & 15), py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < A.width && py < A.height;
  const float pxc = px + 0.5f, pyc = py + 0.5f;
  const uint2 range = A.ranges[tile];
  const int64_t projbase = (int64_t)cam * A.n;

  float acc[NCH];
#pragma unroll
  for (int k = 0; k < NCH; k++) acc[k] = 0.f;
  float T = 1.f;
  uint32_t lastpos = 0, count = 0;
  bool done = !inside;

  for (uint32_t b0 = range.x; b0 < range.y; b0 += kFwdBatch) {
    if (__syncthreads_count(done) == kThreads) break;
    const int nb = (int)((range.y - b0) < (uint32_t)kFwdBatch ? (range.y - b0) : (uint32_t)kFwdBatch);
    if ((int)threadIdx.x < nb) {
      uint32_t g = A.ids[b0 + threadIdx.x];
      stage_instance<FC, TC, RGB>(A, projbase, g, f0, s_xy[threadIdx.x], s_co[threadIdx.x],
                                  s_ch + threadIdx.x * NCH);
    }
    __syncthreads();
    if (!done) {
      for (int j = 0; j < nb; j++) {
        const float2 xy = s_xy[j];
        const float4 co = s_co[j];
        const float power = gauss_power(co.x, co.y, co.z, xy.x - pxc, xy.y - pyc);
        if (power > 0.f) continue;
        const float alpha = fminf(kAlphaMax, raw_alpha(co.w, power));
        if (alpha < kAlphaMin) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
        if (Tn < kTStop) {
          done = true;
          break;
        }
        const float w = __fmul_rn(alpha, T);
        const float4* c4 = reinterpret_cast<const float4*>(s_ch + j * NCH);
        const float2 ww = f2(w, w);
#pragma unroll
        for (int q = 0; q < NCH / 4; q++) {  // packed FP32 pairs (FFMA2)
          const float4 v = c4[q];
          const float2 a0 = __ffma2_rn(ww, f2(v.x, v.y), f2(acc[4 * q], acc[4 * q + 1]));
          const float2 a1 = __ffma2_rn(ww, f2(v.z, v.w), f2(acc[4 * q + 2], acc[4 * q + 3]));
          acc[4 * q + 0] = a0.x;
          acc[4 * q + 1] = a0.y;
          acc[4 * q + 2] = a1.x;
          acc[4 * q + 3] = a1.y;
        }
        T = Tn;
        lastpos = b0 - range.x + j + 1;
        count++;
      }
    }
  }
  if (!inside) return;
  const int64_t pix = ((int64_t)cam * A.height + py) * A.width + px;
  if (RGB) {
    A.rgb[3 * pix + 0] = acc[0] + T * A.bg0;
    A.rgb[3 * pix + 1] = acc[1] + T * A.bg1;
    A.rgb[3 * pix + 2] = acc[2] + T * A.bg2;
    A.depth[pix] = acc[3];
    A.T_final[pix] = T;
    A.last[pix] = lastpos;
    if (A.n_contrib) A.n_contrib[pix] = count;
  }
  float4* out = reinterpret_cast<float4*>(A.feat + pix * A.D + f0);
#pragma unroll
  for (int q = 0; q < FC / 4; q++)
    out[q] = make_float4(acc[(RGB ? 4 : 0) + 4 * q], acc[(RGB ? 4 : 0) + 4 * q + 1],
                         acc[(RGB ? 4 : 0) + 4 * q + 2], acc[(RGB ? 4 : 0) + 4 * q + 3]);
}

// ------------------------------------------------------------------ backward

template <int FC, bool RGB>
struct BwdSmem {
  static constexpr int NCH = nchan<FC, RGB>();
  static constexpr int NV = NCH + 6;          // channel sums + 6 spatial moments
  static constexpr int GROUP = 16 * NCH + 4;  // one 16-pixel tile row of upstream gradients
  static constexpr int WROW = 33;
  static constexpr size_t g_off = 0;
  static constexpr size_t w_off = g_off + sizeof(float) * 16 * GROUP;
  static constexpr size_t p_off = w_off + sizeof(float) * 8 * kBwdBatch * WROW;
  // two batch buffers (sums, channels, conic + opacity, means, ids): the
  // next batch is staged while the current one is written out
  static constexpr size_t st_off = p_off + sizeof(float) * 8 * kBwdBatch * WROW;
  static constexpr size_t acc_off = 0;
  static constexpr size_t ch_off = acc_off + sizeof(float) * kBwdBatch * NV;
  static constexpr size_t co_off = (ch_off + sizeof(float) * kBwdBatch * NCH + 15) / 16 * 16;
  static constexpr size_t xy_off = co_off + sizeof(float4) * kBwdBatch;
  static constexpr size_t gid_off = xy_off + sizeof(float2) * kBwdBatch;
  static constexpr size_t stage = (gid_off + sizeof(uint32_t) * kBwdBatch + 15) / 16 * 16;
  static constexpr size_t total = st_off + 2 * stage + 16;
};

template <int FC, typename TC, bool RGB>
__global__ void __launch_bounds__(kThreads, FC <= 16 ? 3 : 2)
render_bwd_kernel(RasterArgs A, int chunk_base) {
  using L = BwdSmem<FC, RGB>;
  constexpr int NCH = L::NCH, NV = L::NV, B = kBwdBatch;
  extern __shared__ float4 smem4[];
  char* sm = reinterpret_cast<char*>(smem4);
  float* s_g = reinterpret_cast<float*>(sm + L::g_off);
  float* s_w = reinterpret_cast<float*>(sm + L::w_off);
  float* s_p = reinterpret_cast<float*>(sm + L::p_off);
  __shared__ uint32_t s_maxlast;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.x;
  const int f0 = (chunk_base + blockIdx.y) * FC;
  const int tiles = A.tiles_x * A.tiles_y;
  const int cam = tile / tiles, t = tile - cam * tiles;
  const int tx = t % A.tiles_x, ty = t / A.tiles_x;
  const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool inside = px < A.width && py < A.height;
  const float pxc = px + 0.5f, pyc = py + 0.5f;
  const uint2 range = A.ranges[tile];
  const int64_t projbase = (int64_t)cam * A.n;
  const int64_t pix = ((int64_t)cam * A.height + py) * A.width + px;

  // upstream gradients of this pixel, in registers and in shared memory
  float g[NCH];
#pragma unroll
  for (int k = 0; k < NCH; k++) g[k] = 0.f;
  float T = 1.f, S = 0.f;
  uint32_t my_last = 0;
  if (inside) {
    if (RGB) {
      g[0] = A.d_rgb[3 * pix];
      g[1] = A.d_rgb[3 * pix + 1];
      g[2] = A.d_rgb[3 * pix + 2];
      g[3] = A.d_depth[pix];
    }
    const float4* df = reinterpret_cast<const float4*>(A.d_feat + pix * A.D + f0);
#pragma unroll
    for (int q = 0; q < FC / 4; q++) {
      float4 v = df[q];
      g[(RGB ? 4 : 0) + 4 * q + 0] = v.x;
      g[(RGB ? 4 : 0) + 4 * q + 1] = v.y;
      g[(RGB ? 4 : 0) + 4 * q + 2] = v.z;
      g[(RGB ? 4 : 0) + 4 * q + 3] = v.w;
    }
    T = A.T_final[pix];
    my_last = A.last[pix];
    if (RGB) S = T * (A.bg0 * g[0] + A.bg1 * g[1] + A.bg2 * g[2]);
  }
  {
    float* row = s_g + ly * L::GROUP + lx * NCH;
#pragma unroll
    for (int k = 0; k < NCH; k++) row[k] = g[k];
  }
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (my_last) atomicMax(&s_maxlast, my_last);
  __syncthreads();
  const int blk_last = (int)s_maxlast;

  // batch buffer `buf`: sums, channels, conic + opacity, means, Gaussian ids
  auto stage_at = [&](int buf) { return sm + L::st_off + (size_t)buf * L::stage; };
  // zero the sums of buffer `buf` and stage the batch [lo, hi) into it
  auto stage_batch = [&](int buf, int lo, int hi) {
    char* st = stage_at(buf);
    float* acc = reinterpret_cast<float*>(st + L::acc_off);
    for (int i = threadIdx.x; i < B * NV; i += kThreads) acc[i] = 0.f;
    if ((int)threadIdx.x < hi - lo) {
      const uint32_t gid = A.ids[range.x + lo + threadIdx.x];
      reinterpret_cast<uint32_t*>(st + L::gid_off)[threadIdx.x] = gid;
      stage_instance<FC, TC, RGB>(A, projbase, gid, f0,
                                  reinterpret_cast<float2*>(st + L::xy_off)[threadIdx.x],
                                  reinterpret_cast<float4*>(st + L::co_off)[threadIdx.x],
                                  reinterpret_cast<float*>(st + L::ch_off) + threadIdx.x * NCH);
    }
  };
  if (blk_last > 0) stage_batch(0, max(blk_last - B, 0), blk_last);
  __syncthreads();

  int buf = 0;
  for (int hi = blk_last; hi > 0; hi -= B, buf ^= 1) {
    const int lo = max(hi - B, 0), nb = hi - lo;
    char* st = stage_at(buf);
    float* s_acc = reinterpret_cast<float*>(st + L::acc_off);
    const float* s_ch = reinterpret_cast<const float*>(st + L::ch_off);
    const float4* s_co = reinterpret_cast<const float4*>(st + L::co_off);
    const float2* s_xy = reinterpret_cast<const float2*>(st + L::xy_off);
    const uint32_t* s_gid = reinterpret_cast<const uint32_t*>(st + L::gid_off);

    // phase 1: per pixel, back to front through the batch (a warp whose
    // pixels all end before this batch has nothing to add to it)
    float* wrow = s_w + warp * B * L::WROW;
    float* prow = s_p + warp * B * L::WROW;
    const bool warp_active = __any_sync(0xffffffffu, (uint32_t)lo < my_last);
    if (warp_active)
    for (int j = nb - 1; j >= 0; j--) {
      float w = 0.f, dp = 0.f;
      if ((uint32_t)(lo + j) < my_last) {
        const float2 xy = s_xy[j];
        const float4 co = s_co[j];
        const float power = gauss_power(co.x, co.y, co.z, xy.x - pxc, xy.y - pyc);
        if (power <= 0.f) {
          const float araw = raw_alpha(co.w, power);
          const float alpha = fminf(kAlphaMax, araw);
          if (alpha >= kAlphaMin) {
            // fast reciprocal: T only enters gradient values here, never a decision
            const float inv = __fdividef(1.f, __fsub_rn(1.f, alpha));
            const float Tj = T * inv;
            w = alpha * Tj;
            const float4* c4 = reinterpret_cast<const float4*>(s_ch + j * NCH);
            float2 x2 = f2(0.f, 0.f), y2 = f2(0.f, 0.f);  // two packed partial sums
#pragma unroll
            for (int q = 0; q < NCH / 4; q++) {
              const float4 v = c4[q];
              x2 = __ffma2_rn(f2(v.x, v.y), f2(g[4 * q], g[4 * q + 1]), x2);
              y2 = __ffma2_rn(f2(v.z, v.w), f2(g[4 * q + 2], g[4 * q + 3]), y2);
            }
            const float2 xy2 = __fadd2_rn(x2, y2);
            const float xg = xy2.x + xy2.y;
            const float dal = Tj * xg - S * inv;
            S = fmaf(w, xg, S);
            T = Tj;
            if (araw < kAlphaMax) dp = dal * alpha;
          }
        }
      }
      wrow[j * L::WROW + lane] = w;
      prow[j * L::WROW + lane] = dp;
    }
    __syncwarp();

    // phase 2: lane (j, h) reduces instance j over the warp's tile row h
    if (warp_active) {
      const int j = lane & 15, h = lane >> 4;
      const float* wr = wrow + j * L::WROW + 16 * h;
      const float* pr = prow + j * L::WROW + 16 * h;
      const float* gr = s_g + (2 * warp + h) * L::GROUP;
      float cs[NCH];
#pragma unroll
      for (int k = 0; k < NCH; k++) cs[k] = 0.f;
      float S0 = 0.f, Sx = 0.f, Sxx = 0.f;
#pragma unroll 4
      for (int k = 0; k < 16; k++) {
        const float wv = wr[k], pv = pr[k];
        const float4* g4 = reinterpret_cast<const float4*>(gr + k * NCH);
        const float2 w2 = f2(wv, wv);
#pragma unroll
        for (int q = 0; q < NCH / 4; q++) {  // packed FP32 pairs (FFMA2)
          const float4 v = g4[q];
          const float2 a0 = __ffma2_rn(w2, f2(v.x, v.y), f2(cs[4 * q], cs[4 * q + 1]));
          const float2 a1 = __ffma2_rn(w2, f2(v.z, v.w), f2(cs[4 * q + 2], cs[4 * q + 3]));
          cs[4 * q + 0] = a0.x;
          cs[4 * q + 1] = a0.y;
          cs[4 * q + 2] = a1.x;
          cs[4 * q + 3] = a1.y;
        }
        const float xl = (float)k + 0.5f;
        S0 += pv;
        Sx = fmaf(pv, xl, Sx);
        Sxx = fmaf(pv, xl * xl, Sxx);
      }
      const float yl = (float)(2 * warp + h) + 0.5f;
      float vals[NV];
#pragma unroll
      for (int k = 0; k < NCH; k++) vals[k] = cs[k];
      vals[NCH + 0] = S0;
      vals[NCH + 1] = Sx;
      vals[NCH + 2] = yl * S0;
      vals[NCH + 3] = Sxx;
      vals[NCH + 4] = yl * Sx;
      vals[NCH + 5] = yl * yl * S0;
      // lane h keeps half h of the values and adds its partner's copy
      float keep[NV / 2];
#pragma unroll
      for (int v = 0; v < NV / 2; v++) {
        const float a = vals[v], b = vals[NV / 2 + v];
        const float send = h ? a : b;
        keep[v] = (h ? b : a) + __shfl_xor_sync(0xffffffffu, send, 16);
      }
      if (j < nb) {
        float* dst = s_acc + j * NV + h * (NV / 2);
#pragma unroll
        for (int v = 0; v < NV / 2; v++) atomicAdd(dst + v, keep[v]);
      }
    }
    __syncthreads();  // the batch's sums are complete

    // the next batch goes into the other buffer, whose last readers (phase 3
    // of the batch before this one) finished before the previous barrier
    if (hi - B > 0) stage_batch(buf ^ 1, max(hi - 2 * B, 0), hi - B);

    // phase 3: one global update per (tile, instance)
    if ((int)threadIdx.x < nb) {
      const int j = threadIdx.x;
      const float* a = s_acc + j * NV;
      const float S0 = a[NCH], Sx = a[NCH + 1], Sy = a[NCH + 2], Sxx = a[NCH + 3],
                  Sxy = a[NCH + 4], Syy = a[NCH + 5];
      const float2 xy = s_xy[j];
      const float4 co = s_co[j];
      const float U = xy.x - (float)(tx * kTile), V = xy.y - (float)(ty * kTile);
      const float Sdx = U * S0 - Sx, Sdy = V * S0 - Sy;
      const float Sdxx = U * U * S0 - 2.f * U * Sx + Sxx;
      const float Sdxy = U * V * S0 - U * Sy - V * Sx + Sxy;
      const float Sdyy = V * V * S0 - 2.f * V * Sy + Syy;
      const float du = -(co.x * Sdx + co.y * Sdy);
      const float dv = -(co.z * Sdy + co.y * Sdx);
      const float dz = RGB ? a[3] : 0.f;
      float4* dst = A.grad2d + 2 * (projbase + s_gid[j]);
      atomicAdd(dst, make_float4(du, dv, -0.5f * Sdxx, -Sdxy));
      atomicAdd(dst + 1, make_float4(-0.5f * Sdyy, S0 / co.w, dz, 0.f));
    }
    constexpr int NQ = FC / 4;
    constexpr int PER = (RGB ? 3 : 0) + NQ;
    for (int i = threadIdx.x; i < nb * PER; i += kThreads) {
      const int j = i / PER, r = i - j * PER;
      const float* a = s_acc + j * NV;
      const int64_t gid = s_gid[j];
      if (RGB && r < 3) {
        atomicAdd(A.d_colors + 3 * gid + r, a[r]);
      } else {
        const int q = r - (RGB ? 3 : 0);
        const float* src = a + (RGB ? 4 : 0) + 4 * q;
        atomicAdd(reinterpret_cast<float4*>(A.d_feats + gid * A.D + f0) + q,
                  make_float4(src[0], src[1], src[2], src[3]));
      }
    }
    __syncthreads();  // the next batch is staged; this one has been read
  }
}

// ------------------------------------------------------------------ launch

template <typename K>
static cudaError_t prepare(K kernel, size_t smem) {
  return set_smem_limit(reinterpret_cast<const void*>(kernel), (int)smem);
}

template <int FC, typename TC>
static lgs_status launch_fwd(const RasterArgs& A, int ntile, int nchunks, cudaStream_t s) {
  constexpr size_t sm0 = fwd_smem<FC, true>(), sm1 = fwd_smem<FC, false>();
  LGS_CHECK_CUDA(prepare(render_fwd_kernel<FC, TC, true>, sm0));
  render_fwd_kernel<FC, TC, true><<<dim3(ntile, 1), kThreads, sm0, s>>>(A, 0);
  LGS_CHECK_LAUNCH();
  if (nchunks > 1) {
    LGS_CHECK_CUDA(prepare(render_fwd_kernel<FC, TC, false>, sm1));
    render_fwd_kernel<FC, TC, false><<<dim3(ntile, nchunks - 1), kThreads, sm1, s>>>(A, 1);
    LGS_CHECK_LAUNCH();
  }
  return LGS_OK;
}

template <int FC, typename TC>
static lgs_status launch_bwd(const RasterArgs& A, int ntile, int nchunks, cudaStream_t s) {
  constexpr size_t sm0 = BwdSmem<FC, true>::total, sm1 = BwdSmem<FC, false>::total;
  LGS_CHECK_CUDA(prepare(render_bwd_kernel<FC, TC, true>, sm0));
  render_bwd_kernel<FC, TC, true><<<dim3(ntile, 1), kThreads, sm0, s>>>(A, 0);
  LGS_CHECK_LAUNCH();
  if (nchunks > 1) {
    LGS_CHECK_CUDA(prepare(render_bwd_kernel<FC, TC, false>, sm1));
    render_bwd_kernel<FC, TC, false><<<dim3(ntile, nchunks - 1), kThreads, sm1, s>>>(A, 1);
    LGS_CHECK_LAUNCH();
  }
  return LGS_OK;
}

// Shared argument checks; fills the geometry part of RasterArgs.
static lgs_status common_args(const float* proj, const uint32_t* ids, const uint32_t* ranges,
                              int64_t n, const lgs_camera* cams_host, int n_cams,
                              const void* colors, const void* feats, int feat_dim,
                              int chan_dtype, const float* bg_host, RasterArgs& A, int& ntile) {
  LGS_CHECK_ARG(n >= 0 && n < ((int64_t)1 << 31), "n out of range");
  LGS_CHECK_ARG(cams_host && n_cams >= 1 && n_cams <= LGS_MAX_CAMS, "bad cameras");
  LGS_CHECK_ARG(feat_dim >= 8 && feat_dim % 8 == 0 && feat_dim <= 4096,
                "feat_dim must be a multiple of 8 in [8, 4096]");
  LGS_CHECK_ARG(chan_dtype == LGS_F32 || chan_dtype == LGS_BF16, "bad channel dtype");
  LGS_CHECK_ARG(ranges && bg_host, "null pointer");
  LGS_CHECK_ARG(n == 0 || (proj && ids && colors && feats), "null pointer");
  LGS_CHECK_ARG(aligned(proj, 16) && aligned(feats, 16) && aligned(ranges, 8),
                "misaligned pointer");
  int W = cams_host[0].width, H = cams_host[0].height;
  for (int c = 1; c < n_cams; c++)
    LGS_CHECK_ARG(cams_host[c].width == W && cams_host[c].height == H,
                  "cameras of one launch must share the image size");
  LGS_CHECK_ARG(W > 0 && H > 0, "bad image size");
  A.proj = (const float4*)proj;
  A.ids = ids;
  A.ranges = (const uint2*)ranges;
  A.n = n;
  A.width = W;
  A.height = H;
  A.tiles_x = (W + kTile - 1) / kTile;
  A.tiles_y = (H + kTile - 1) / kTile;
  A.D = feat_dim;
  A.colors = colors;
  A.feats = feats;
  A.bg0 = bg_host[0];
  A.bg1 = bg_host[1];
  A.bg2 = bg_host[2];
  ntile = n_cams * A.tiles_x * A.tiles_y;
  return LGS_OK;
}

}  // namespace lgs

using namespace lgs;

extern "C" lgs_status gs_render_fwd(const float* proj, const uint32_t* ids, const uint32_t* ranges,
                                    int64_t n, const lgs_camera* cams_host, int n_cams,
                                    const void* colors, const void* feats, int feat_dim,
                                    int chan_dtype, const float* bg_host, float* rgb,
                                    float* depth, float* feat, float* T_final, uint32_t* last,
                                    uint32_t* n_contrib_opt, void* stream) {
  clear_error();
  RasterArgs A = {};
  int ntile = 0;
  lgs_status st = common_args(proj, ids, ranges, n, cams_host, n_cams, colors, feats, feat_dim,
                              chan_dtype, bg_host, A, ntile);
  if (st != LGS_OK) return st;
  LGS_CHECK_ARG(rgb && depth && feat && T_final && last, "null output");
  LGS_CHECK_ARG(aligned(feat, 16), "feat must be 16-byte aligned");
  A.rgb = rgb;
  A.depth = depth;
  A.feat = feat;
  A.T_final = T_final;
  A.last = last;
  A.n_contrib = n_contrib_opt;
  cudaStream_t s = as_stream(stream);
  const bool bf = chan_dtype == LGS_BF16;
  // channel chunk FC: 16 for the compact features, else the widest of 32 /
  // 16 / 8 that divides feat_dim
  if (feat_dim == 16)
    return bf ? launch_fwd<16, __nv_bfloat16>(A, ntile, 1, s) : launch_fwd<16, float>(A, ntile, 1, s);
  if (feat_dim % 32 == 0)
    return bf ? launch_fwd<32, __nv_bfloat16>(A, ntile, feat_dim / 32, s)
              : launch_fwd<32, float>(A, ntile, feat_dim / 32, s);
  if (feat_dim % 16 == 0)
    return bf ? launch_fwd<16, __nv_bfloat16>(A, ntile, feat_dim / 16, s)
              : launch_fwd<16, float>(A, ntile, feat_dim / 16, s);
  return bf ? launch_fwd<8, __nv_bfloat16>(A, ntile, feat_dim / 8, s)
            : launch_fwd<8, float>(A, ntile, feat_dim / 8, s);
}

extern "C" lgs_status gs_render_bwd(const float* means, const float* quats,
                                    const float* log_scales, const float* opacity_logits,
                                    const float* proj, const uint32_t* ids,
                                    const uint32_t* ranges, int64_t n,
                                    const lgs_camera* cams_host, int n_cams, const void* colors,
                                    const void* feats, int feat_dim, int chan_dtype,
                                    const float* bg_host, const float* T_final,
                                    const uint32_t* last, const float* d_rgb,
                                    const float* d_depth, const float* d_feat, float* grad2d,
                                    float* d_means, float* d_quats, float* d_log_scales,
                                    float* d_opacity_logits, float* d_colors, float* d_feats,
                                    void* stream) {
  clear_error();
  RasterArgs A = {};
  int ntile = 0;
  lgs_status st = common_args(proj, ids, ranges, n, cams_host, n_cams, colors, feats, feat_dim,
                              chan_dtype, bg_host, A, ntile);
  if (st != LGS_OK) return st;
  CamBlock cb;
  st = fill_cams(cams_host, n_cams, cb);
  if (st != LGS_OK) return st;
  LGS_CHECK_ARG(T_final && last && d_rgb && d_depth && d_feat, "null input");
  LGS_CHECK_ARG(n == 0 || (means && quats && log_scales && opacity_logits && grad2d && d_means &&
                           d_quats && d_log_scales && d_opacity_logits && d_colors && d_feats),
                "null output");
  LGS_CHECK_ARG(aligned(d_feat, 16) && aligned(grad2d, 16) && aligned(d_feats, 16) &&
                    aligned(quats, 16),
                "misaligned pointer");
  if (n == 0) return LGS_OK;
  cudaStream_t s = as_stream(stream);
  LGS_CHECK_CUDA(cudaMemsetAsync(grad2d, 0, sizeof(float) * LGS_PROJ_STRIDE * (size_t)n_cams * n, s));
  A.T_final = const_cast<float*>(T_final);
  A.last = const_cast<uint32_t*>(last);
  A.d_rgb = d_rgb;
  A.d_depth = d_depth;
  A.d_feat = d_feat;
  A.grad2d = (float4*)grad2d;
  A.d_colors = d_colors;
  A.d_feats = d_feats;
  const bool bf = chan_dtype == LGS_BF16;
  if (feat_dim == 16)
    st = bf ? launch_bwd<16, __nv_bfloat16>(A, ntile, 1, s) : launch_bwd<16, float>(A, ntile, 1, s);
  else if (feat_dim % 32 == 0)
    st = bf ? launch_bwd<32, __nv_bfloat16>(A, ntile, feat_dim / 32, s)
            : launch_bwd<32, float>(A, ntile, feat_dim / 32, s);
  else if (feat_dim % 16 == 0)
    st = bf ? launch_bwd<16, __nv_bfloat16>(A, ntile, feat_dim / 16, s)
            : launch_bwd<16, float>(A, ntile, feat_dim / 16, s);
  else
    st = bf ? launch_bwd<8, __nv_bfloat16>(A, ntile, feat_dim / 8, s)
            : launch_bwd<8, float>(A, ntile, feat_dim / 8, s);
  if (st != LGS_OK) return st;
  return launch_project_bwd(means, quats, log_scales, opacity_logits, n, n_cams, cb, grad2d,
                            d_means, d_quats, d_log_scales, d_opacity_logits, s);
}
