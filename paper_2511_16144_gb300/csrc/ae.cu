// Scene-adaptive autoencoder on the tensor cores (tcgen05, TMEM accumulators).
//
// LEGO-SLAM Sec. IV-A.2: encoder E_phi and decoder D_theta are stacks of 1x1
// convolutions -- the same MLP applied to every pixel -- compressing the
// extractor's high-dimensional features to 16 channels.  They are pretrained
// as an autoencoder; Sec. III-B.3 Eq. 2 distils the rendered 16-d map through
// the frozen decoder with an L1 loss; Sec. III-B.4 Eq. 3 adapts the encoder
// alone with an L1 loss against the rendered map.
//
// Widths 512-256-128-64-16 and the mirrored decoder, GELU (tanh form) on hidden layers,
// bias everywhere (layers 0-3 encoder, 4-7 decoder).  GEMMs take BF16
// operands and accumulate in FP32 in tensor memory; activations between
// layers are BF16.
//
// Kernels
//   layer_kernel<NT, KC>: out[P, N] = epilogue(A[P, K] . W[N, K]^T) for one
//     128-row tile per CTA, K streamed in chunks of KC through two stages into
//     the canonical K-major layout -- by 3-D TMA loads from one thread for
//     BF16 operands, by cp.async from every thread (converting) for an FP32
//     A; one thread issues the MMAs, all 128 threads run the epilogue from
//     TMEM (thread = row).  The encoder has its own fused kernel
//     (ae_encode_fused.cu), the map step's decoder distillation too
//     (ae_fused.cu).
//     Epilogues: bias+GELU (+ pre-activation), linear, GELU'-gated backward,
//     and the fused losses (L1 against a target, or L2 + (1 - cos)) that
//     also emit the output gradient.
//   dw_kernel<KT>: the partial dW[N, K] = sum_p G[p, n] X[p, k] over one
//     pixel range, and the partial bias gradient sum_p G[p, n], in the same
//     launch; the pixel dimension is the MMA's K, so G and X as stored are
//     MN-major operands that TMA loads land without a transpose.  Each CTA
//     stores its partial tile to its own slice of the workspace (no atomics).
//   adam_all kernel: sums every element's partials in a fixed order (slice
//     0, 1, ...), stores the gradient and takes the Adam step, for every
//     layer in one launch; the training step is therefore bit-reproducible.
//   pack_all kernel (SIMT; one launch for every layer).
#include <algorithm>
#include <cstring>
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "tc05.cuh"

namespace lgs {

constexpr int kAeLayers = LGS_AE_LAYERS;
constexpr int kAeWidths[9] = {512, 256, 128, 64, 16, 64, 128, 256, 512};
constexpr uint32_t kSpinLimit = 1u << 22;  // polls before a wait gives up

__device__ unsigned g_ae_error;  // 1: a bounded wait gave up; 4: shared memory misaligned

enum Epi : int {
  EPI_GELU = 0,      // out = gelu(acc + b) (bf16), pre = acc + b (bf16, optional)
  EPI_LIN_F32 = 1,   // out = acc + b (f32)
  EPI_LIN_BF16 = 2,  // out = acc + b (bf16)
  EPI_DGELU = 3,     // out = acc * gelu'(pre_in) (bf16)
  EPI_DX_F32 = 4,    // out = acc (f32)
  EPI_DX_BF16 = 5,   // out = acc (bf16)
  EPI_L1_BF16T = 6,  // y = acc + b; loss += s|y - t|; out = s sign(y - t) (bf16); t bf16
  EPI_L1_F32T = 7,   // same with an f32 target
  EPI_RECON = 8,     // y = acc + b vs x: loss += s (mean (y-x)^2 + 1 - cos); out = dL/dy
  EPI_ARGMIN = 9     // closest codeword: argmin_n (b_n - 2 acc_n) -> out_u32, hist[n] += 1
};

struct LayerArgs {
  const void* A;
  int a_f32;
  const __nv_bfloat16* W;
  const float* bias;
  int64_t P;
  int K, N;
  int epi;
  __nv_bfloat16* out_bf;
  float* out_f32;
  __nv_bfloat16* pre_out;
  const __nv_bfloat16* pre_in;
  const void* target;
  float scale;
  float* loss;
  uint32_t* out_u32;
  uint32_t* hist;
};

__device__ __forceinline__ float gelu_f(float x) { return gelu_tanh(x); }
__device__ __forceinline__ float gelu_grad_f(float x) { return gelu_tanh_grad(x); }

__device__ __forceinline__ void store_bf16x32(__nv_bfloat16* dst, const float* v, int n) {
  // n = 16 or 32 values to a 16-byte aligned destination
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (q * 8 >= n) break;
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; k++) h[k] = __floats2bfloat162_rn(v[8 * q + 2 * k], v[8 * q + 2 * k + 1]);
    reinterpret_cast<uint4*>(dst)[q] = u;
  }
}

__device__ __forceinline__ void load_bf16x32(const __nv_bfloat16* src, float* v, int n) {
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (q * 8 >= n) break;
    uint4 u = reinterpret_cast<const uint4*>(src)[q];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float2 f = __bfloat1622float2(h[k]);
      v[8 * q + 2 * k] = f.x;
      v[8 * q + 2 * k + 1] = f.y;
    }
  }
}

__device__ __forceinline__ void report_timeout() { atomicOr(&g_ae_error, 1u); }

constexpr int kLayerThreads = 256;  // 8 warps: producer / MMA lanes, then all run the epilogue

template <int NT, int KC>
struct LayerSmem {
  static constexpr int A_BYTES = 128 * KC * 2;
  static constexpr int B_BYTES = NT * KC * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr size_t total = 2 * STAGE + 64;
  static constexpr uint32_t TCOLS = NT < 32 ? 32 : NT;
  static constexpr int BROWS = NT > 256 ? 256 : NT;  // weight rows per TMA box
};

// The 16-byte piece `chunk` (0-7) of row r in a 128-byte swizzled box: the
// pieces of each row are permuted by XOR with r % 8.
__device__ __forceinline__ uint32_t sw128_piece(int r, int chunk) {
  return (uint32_t)(r * 128 + ((chunk ^ (r & 7)) << 4));
}

// tmap / omap: the target and the output of EPI_RECON as 128-byte swizzle
// maps with 64-column x 128-row boxes (unused by the other epilogues).
template <int NT, int KC>
__global__ void __launch_bounds__(kLayerThreads, 2) layer_kernel(const __grid_constant__ LayerArgs a,
                                                      const __grid_constant__ CUtensorMap amap,
                                                      const __grid_constant__ CUtensorMap bmap,
                                                      const __grid_constant__ CUtensorMap tmap,
                                                      const __grid_constant__ CUtensorMap omap) {
  using L = LayerSmem<NT, KC>;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * L::STAGE);   // [2] MMAs of a stage done
  uint64_t* full = mbar + 2;                                          // [2] TMA data of a stage in
  uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 2);
  uint64_t* xbar = reinterpret_cast<uint64_t*>(sm + 2 * L::STAGE + 40);  // EPI_RECON target in
  uint64_t* dbar = xbar + 1;  // a give-up waits here for the MMAs already issued
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * 128;
  const int n0 = blockIdx.y * NT;
  const int K = a.K;
  // the 128-byte swizzle of the TMA path repeats every 1 KB from the stage base
  if (tc::smem_addr(sm) & 1023u) {
    if (tid == 0) atomicOr(&g_ae_error, 4u);
    return;
  }
  if (warp == 0) tc::tmem_alloc(tslot, L::TCOLS);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::mbar_init(xbar, 1);
    tc::mbar_init(dbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;
  int issued = 0;  // K-chunks whose TMA loads thread 0 issued

  const int nk = K / KC;
  constexpr uint32_t SBO = KC * 16;
  if (!a.a_f32) {
    // BF16 A: thread 0 streams A and W chunks by TMA, thread 32 issues the
    // MMAs; the stages are handed over by mbarriers, no block barrier in the
    // loop.  KC = 64: one 2-D box per operand in the 128-byte swizzle layout
    // (rows of 128 B); KC = 16: 3-D boxes that land as 2 blocks of rows x 16
    // bytes (K-adjacent core matrices rows * 16 bytes apart).
    const uint32_t sbase = tc::smem_addr(sm);
    if (tid == 0) {
      for (int kc = 0; kc < nk && ok; kc++) {
        const int s = kc & 1;
        if (kc >= 2 && !tc::mbar_wait(&mbar[s], ((kc - 2) >> 1) & 1, kSpinLimit)) {
          ok = false;
          break;
        }
        const uint32_t st = sbase + s * L::STAGE;
        tc::mbar_expect_tx(&full[s], L::STAGE);
        if constexpr (KC == 64) {
          tc::tma_load_2d(st, &amap, kc * 64, (int)row0, &full[s]);
#pragma unroll
          for (int h = 0; h < NT / L::BROWS; h++)
            tc::tma_load_2d(st + L::A_BYTES + h * L::BROWS * 128, &bmap, kc * 64, n0 + h * L::BROWS,
                        &full[s]);
        } else {
          tc::tma_load_3d(st, &amap, 0, (int)row0, kc * (KC / 8), &full[s]);
#pragma unroll
          for (int h = 0; h < NT / L::BROWS; h++)
            tc::tma_load_3d(st + L::A_BYTES + h * L::BROWS * KC * 2, &bmap, 0, n0 + h * L::BROWS,
                        kc * (KC / 8), &full[s]);
        }
        issued = kc + 1;
      }
    } else if (tid == 32) {
      for (int kc = 0; kc < nk && ok; kc++) {
        const int s = kc & 1;
        if (!tc::mbar_wait(&full[s], (kc >> 1) & 1, kSpinLimit)) {
          ok = false;
          break;
        }
        tc::fence_after();
        const uint32_t sa_u = sbase + s * L::STAGE, sb_u = sa_u + L::A_BYTES;
#pragma unroll
        for (int j = 0; j < KC / 16; j++) {
          const uint64_t ad = KC == 64 ? tc::sdesc_sw128(sa_u + j * 32)
                                       : tc::sdesc(sa_u + j * 2 * 2048, 2048, 128);
#pragma unroll
          for (int h = 0; h < NT / L::BROWS; h++) {
            const uint64_t bd =
                KC == 64 ? tc::sdesc_sw128(sb_u + h * L::BROWS * 128 + j * 32)
                         : tc::sdesc(sb_u + h * L::BROWS * KC * 2 + j * 2 * L::BROWS * 16,
                                     L::BROWS * 16, 128);
            tc::mma_bf16(tmem + h * 256, ad, bd, tc::idesc_bf16(128, L::BROWS), (kc | j) != 0);
          }
        }
        tc::commit(&mbar[s]);
      }
    }
  } else {
  // FP32 A (converted to BF16 while staged): every thread copies with
  // cp.async, K-chunk kc into stage kc & 1 (A: 128 rows x KC, B: NT x KC)
  auto load_chunk = [&](int kc) {
    const int s = kc & 1;
    uint8_t* sa = sm + s * L::STAGE;
    uint8_t* sb = sa + L::A_BYTES;
    const uint32_t sa_u = tc::smem_addr(sa), sb_u = tc::smem_addr(sb);
    constexpr int APIECES = 128 * (KC / 8);
    for (int i = tid; i < APIECES; i += kLayerThreads) {
      const int r = i / (KC / 8), c = i % (KC / 8);
      const int64_t p = row0 + r;
      const bool valid = p < a.P;
      const int64_t pc = valid ? p : 0;
      const uint32_t off = tc::core_offset(r, c, KC);
      if (a.a_f32) {
        const float4* src = reinterpret_cast<const float4*>(
            reinterpret_cast<const float*>(a.A) + pc * K + kc * KC + c * 8);
        float4 f0 = valid ? src[0] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 f1 = valid ? src[1] : make_float4(0.f, 0.f, 0.f, 0.f);
        uint4 u;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
        h[0] = __floats2bfloat162_rn(f0.x, f0.y);
        h[1] = __floats2bfloat162_rn(f0.z, f0.w);
        h[2] = __floats2bfloat162_rn(f1.x, f1.y);
        h[3] = __floats2bfloat162_rn(f1.z, f1.w);
        *reinterpret_cast<uint4*>(sa + off) = u;
      } else {
        const __nv_bfloat16* src =
            reinterpret_cast<const __nv_bfloat16*>(a.A) + pc * K + kc * KC + c * 8;
        tc::cp_async16_zfill(sa_u + off, src, valid);
      }
    }
    constexpr int BPIECES = NT * (KC / 8);
    for (int i = tid; i < BPIECES; i += kLayerThreads) {
      const int r = i / (KC / 8), c = i % (KC / 8);
      const __nv_bfloat16* src = a.W + (int64_t)(n0 + r) * K + kc * KC + c * 8;
      tc::cp_async16(sb_u + tc::core_offset(r, c, KC), src);
    }
    tc::cp_async_commit();
  };
  // chunk kc + 1 is in flight while chunk kc waits for its data and its MMAs
  load_chunk(0);
  for (int kc = 0; kc < nk; kc++) {
    const int s = kc & 1;
    if (kc + 1 < nk) {
      // stage (kc + 1) & 1 is free once the MMAs of chunk kc - 1 are done;
      // every thread polls and the block agrees before anyone moves on
      const bool freed = kc < 1 || tc::mbar_wait(&mbar[s ^ 1], ((kc - 1) >> 1) & 1, kSpinLimit);
      if (!__syncthreads_and(freed)) {
        ok = false;
        break;
      }
      load_chunk(kc + 1);
      tc::cp_async_wait_group<1>();
    } else {
      tc::cp_async_wait_all();
    }
    tc::fence_async_smem();
    __syncthreads();
    const uint32_t sa_u = tc::smem_addr(sm + s * L::STAGE), sb_u = sa_u + L::A_BYTES;
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int j = 0; j < KC / 16; j++) {
        const uint64_t ad = tc::sdesc(sa_u + j * 256, 128, SBO);
#pragma unroll
        for (int h = 0; h < (NT > 256 ? NT / 256 : 1); h++) {
          constexpr int NM = NT > 256 ? 256 : NT;
          const uint64_t bd = tc::sdesc(sb_u + h * (NM / 8) * SBO + j * 256, 128, SBO);
          tc::mma_bf16(tmem + h * 256, ad, bd, tc::idesc_bf16(128, NM), (kc | j) != 0);
        }
      }
      tc::commit(&mbar[s]);
    }
  }
  }
  ok = __syncthreads_and(ok);
  if (ok) ok = __syncthreads_and(tc::mbar_wait(&mbar[(nk - 1) & 1], ((nk - 1) >> 1) & 1, kSpinLimit));
  if (!ok) {
    if (tid == 0) report_timeout();
    // before the CTA leaves: its copies in flight land (at most the last two
    // chunks' TMA loads; every thread's cp.async groups) and the MMAs issued
    // so far finish, each wait bounded again
    if (a.a_f32) {
      tc::cp_async_wait_all();
    } else if (tid == 0) {
      for (int c = issued > 2 ? issued - 2 : 0; c < issued; c++)
        tc::mbar_wait(&full[c & 1], (c >> 1) & 1, kSpinLimit);
    }
    if (tid == (a.a_f32 ? 0 : 32)) {
      tc::commit(dbar);
      tc::mbar_wait(dbar, 0, kSpinLimit);
    }
  } else {
    tc::fence_after();
    // ---------------------------------------------------------- epilogue
    // Warps w and w + 4 read TMEM lane quadrant w % 4 (thread = row) and
    // split the columns: half h = w / 4 takes [h NT / 2, (h + 1) NT / 2)
    // (h = 0 takes all of them when NT < 64).  The drained stages hold the
    // bias slice (bytes 0-2047), the per-row partials the two halves
    // exchange (2048-6143) and, for EPI_RECON, the target tile (from 8192).
    static_assert(2 * L::STAGE >= 6144, "epilogue scratch does not fit");
    const int q = warp & 3, h = warp >> 2;
    const int r = q * 32 + lane;
    const int64_t p = row0 + r;
    const bool valid = p < a.P;
    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16);
    constexpr int CW = NT < 32 ? 16 : 32;
    constexpr bool kSplit = NT >= 64;
    const int cbeg = kSplit ? h * (NT / 2) : 0;
    const int cend = kSplit ? cbeg + NT / 2 : (h == 0 ? NT : 0);
    float* sbias = reinterpret_cast<float*>(sm);
    float4* sx4 = reinterpret_cast<float4*>(sm + 2048);
    if (a.bias) {
      for (int i = tid; i < NT; i += kLayerThreads) sbias[i] = a.bias[n0 + i];
      __syncthreads();
    }
    // the bias of columns c0 .. c0 + CW - 1 (one broadcast 16-byte read per 4)
    auto bias_of = [&](int c0, float* bb) {
#pragma unroll
      for (int i = 0; i < CW / 4; i++) {
        const float4 t = reinterpret_cast<const float4*>(sbias + c0)[i];
        bb[4 * i] = t.x;
        bb[4 * i + 1] = t.y;
        bb[4 * i + 2] = t.z;
        bb[4 * i + 3] = t.w;
      }
    };
    float lsum = 0.f;
    if (a.epi == EPI_ARGMIN) {
      // |x - c_n|^2 - |x|^2 = |c_n|^2 - 2 x.c_n with |c_n|^2 in the bias;
      // columns in increasing order, strict < keeps the lower index on ties
      float best = INFINITY;
      uint32_t bi = 0;
      for (int c0 = cbeg; c0 < cend; c0 += CW) {
        float v[32], bb[32];
        if (CW == 32) tc::tmem_ld32(tb + c0, v);
        else tc::tmem_ld16(tb + c0, v);
        bias_of(c0, bb);
#pragma unroll
        for (int i = 0; i < CW; i++) {
          const float sc = fmaf(-2.f, v[i], bb[i]);
          if (sc < best) {
            best = sc;
            bi = (uint32_t)(n0 + c0 + i);
          }
        }
      }
      // the upper half hands its best over; the lower half wins ties
      float* xb = reinterpret_cast<float*>(sx4);
      uint32_t* xi = reinterpret_cast<uint32_t*>(xb + 128);
      if (kSplit && h == 1) {
        xb[r] = best;
        xi[r] = bi;
      }
      __syncthreads();
      if (h == 0) {
        if (kSplit && xb[r] < best) {
          best = xb[r];
          bi = xi[r];
        }
        if (valid && a.out_u32) a.out_u32[p] = bi;
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? bi : (0x80000000u | lane));
        if (valid && a.hist && lane == __ffs(peers) - 1) atomicAdd(a.hist + bi, (uint32_t)__popc(peers));
      }
    } else if (a.epi == EPI_RECON) {
      if constexpr (NT == 512 && 2 * L::STAGE >= 8192 + 128 * 512 * 2) {
        // The target tile [128 x 512] lands in the free stages by eight TMA
        // loads of 64 columns (16 KB each, rows of 128 B with the 128-byte
        // swizzle, so the 16-byte pieces of the rows a warp reads together
        // fall in distinct banks); dL/dy replaces it in place and leaves by
        // eight TMA stores through the same swizzle.
        const uint32_t sx = tc::smem_addr(sm) + 8192;
        if (tid == 0) {
          tc::mbar_expect_tx(xbar, 128 * 512 * 2);
#pragma unroll
          for (int b = 0; b < 8; b++) tc::tma_load_2d(sx + b * 16384, &tmap, 64 * b, (int)row0, xbar);
        }
        const bool landed = tc::mbar_wait(xbar, 0, kSpinLimit);
        if (__syncthreads_and(landed)) {
          uint8_t* xt = sm + 8192;
          // columns c0 .. c0 + 31 of row r, as 32 floats
          auto load_x = [&](int c0, float* x) {
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
              const uint4 u = *reinterpret_cast<const uint4*>(
                  xt + (c0 >> 6) * 16384 + sw128_piece(r, ((c0 & 63) >> 3) + q4));
              const __nv_bfloat162* hh = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
              for (int k = 0; k < 4; k++) {
                const float2 f = __bfloat1622float2(hh[k]);
                x[8 * q4 + 2 * k] = f.x;
                x[8 * q4 + 2 * k + 1] = f.y;
              }
            }
          };
          // pass 1: row statistics of y against x = target, per half
          float sdd = 0.f, syx = 0.f, syy = 0.f, sxx = 0.f;
          for (int c0 = cbeg; c0 < cend; c0 += 32) {
            float v[32], x[32], bb[32];
            tc::tmem_ld32(tb + c0, v);
            load_x(c0, x);
            bias_of(c0, bb);
#pragma unroll
            for (int i = 0; i < 32; i++) {
              const float y = v[i] + bb[i];
              const float d = y - x[i];
              sdd = fmaf(d, d, sdd);
              syx = fmaf(y, x[i], syx);
              syy = fmaf(y, y, syy);
              sxx = fmaf(x[i], x[i], sxx);
            }
          }
          sx4[h * 128 + r] = make_float4(sdd, syx, syy, sxx);
          __syncthreads();
          const float4 s0 = sx4[r], s1 = sx4[128 + r];
          sdd = s0.x + s1.x;
          syx = s0.y + s1.y;
          syy = s0.z + s1.z;
          sxx = s0.w + s1.w;
          const float invN = 1.f / (float)a.N;
          const float ny = sqrtf(syy), nx = sqrtf(sxx);
          const float inv = 1.f / fmaxf(ny * nx, 1e-30f);
          const float cosv = syx * inv;
          if (valid && h == 0) lsum = a.scale * (sdd * invN + 1.f - cosv);
          const float iy2 = 1.f / fmaxf(syy, 1e-30f);
          // pass 2: dL/dy = s (2 (y - x)/N - (x/(|y||x|) - cos y/|y|^2))
          const float c2 = 2.f * invN * a.scale, cx = a.scale * inv, cy = a.scale * cosv * iy2;
          for (int c0 = cbeg; c0 < cend; c0 += 32) {
            float v[32], x[32], bb[32];
            tc::tmem_ld32(tb + c0, v);
            load_x(c0, x);
            bias_of(c0, bb);
#pragma unroll
            for (int i = 0; i < 32; i++) {
              const float y = v[i] + bb[i];
              v[i] = fmaf(c2, y - x[i], fmaf(cy, y, -cx * x[i]));
            }
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
              uint4 u;
              __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
              for (int k = 0; k < 4; k++)
                hh[k] = __floats2bfloat162_rn(v[8 * q4 + 2 * k], v[8 * q4 + 2 * k + 1]);
              *reinterpret_cast<uint4*>(xt + (c0 >> 6) * 16384 +
                                        sw128_piece(r, ((c0 & 63) >> 3) + q4)) = u;
            }
          }
          tc::fence_async_smem();
          __syncthreads();
          if (tid == 0) {
#pragma unroll
            for (int b = 0; b < 8; b++) tc::tma_store_2d(&omap, 64 * b, (int)row0, sx + b * 16384);
            tc::bulk_wait_read();
          }
        } else if (tid == 0) {
          report_timeout();
          if (!landed) tc::mbar_wait(xbar, 0, kSpinLimit);  // let the target loads land
        }
      }
    } else {
      for (int c0 = cbeg; c0 < cend; c0 += CW) {
        float v[32], bb[32];
        if (CW == 32) tc::tmem_ld32(tb + c0, v);
        else tc::tmem_ld16(tb + c0, v);
        if (!valid) continue;
        const int n = n0 + c0;
        const int64_t o = p * a.N + n;
        switch (a.epi) {
          case EPI_GELU: {
            bias_of(c0, bb);
#pragma unroll
            for (int i = 0; i < CW; i++) v[i] += bb[i];
            if (a.pre_out) store_bf16x32(a.pre_out + o, v, CW);
#pragma unroll
            for (int i = 0; i < CW; i++) v[i] = gelu_f(v[i]);
            store_bf16x32(a.out_bf + o, v, CW);
            break;
          }
          case EPI_LIN_F32:
          case EPI_LIN_BF16: {
            bias_of(c0, bb);
#pragma unroll
            for (int i = 0; i < CW; i++) v[i] += bb[i];
            if (a.epi == EPI_LIN_BF16) {
              store_bf16x32(a.out_bf + o, v, CW);
            } else {
#pragma unroll
              for (int q4 = 0; q4 < CW / 4; q4++)
                reinterpret_cast<float4*>(a.out_f32 + o)[q4] =
                    make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
            }
            break;
          }
          case EPI_DGELU: {
            float pr[32];
            load_bf16x32(a.pre_in + o, pr, CW);
#pragma unroll
            for (int i = 0; i < CW; i++) v[i] *= gelu_grad_f(pr[i]);
            store_bf16x32(a.out_bf + o, v, CW);
            break;
          }
          case EPI_DX_F32: {
#pragma unroll
            for (int q4 = 0; q4 < CW / 4; q4++)
              reinterpret_cast<float4*>(a.out_f32 + o)[q4] =
                  make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
            break;
          }
          case EPI_DX_BF16:
            store_bf16x32(a.out_bf + o, v, CW);
            break;
          case EPI_L1_BF16T:
          case EPI_L1_F32T: {
            float t[32];
            bias_of(c0, bb);
            if (a.epi == EPI_L1_BF16T) {
              load_bf16x32(reinterpret_cast<const __nv_bfloat16*>(a.target) + o, t, CW);
            } else {
#pragma unroll
              for (int i = 0; i < CW; i++) t[i] = reinterpret_cast<const float*>(a.target)[o + i];
            }
#pragma unroll
            for (int i = 0; i < CW; i++) {
              const float d = v[i] + bb[i] - t[i];
              lsum += fabsf(d);
              v[i] = d > 0.f ? a.scale : (d < 0.f ? -a.scale : 0.f);
            }
            store_bf16x32(a.out_bf + o, v, CW);
            break;
          }
          default:
            break;
        }
      }
      if (a.epi == EPI_L1_BF16T || a.epi == EPI_L1_F32T) lsum *= a.scale;
    }
    if (a.loss) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      if (lane == 0 && lsum != 0.f) atomicAdd(a.loss, lsum);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::TCOLS);
}

// ------------------------------------------------------------------ dW

struct DwArgs {
  int64_t P;
  int N, K;
  int chunks_per_cta;      // 64-pixel chunks per CTA
  int a_tx, b_tx;          // bytes one stage's G and X loads deliver
  float* part;             // [splits][N][K]: CTA z's partial dW in slice z (overwritten)
  float* dbpart;           // [splits][N]: its partial column sums of G, or null
};

// Shared memory of dw_kernel: a ring of stages, each one 64-pixel chunk of
// G (128 features) and X (KT features) as the TMA lands them, MN-major
// operands whose K is the pixel: with 64 or more features, 64-feature boxes
// in the 128-byte swizzle layout (64 pixel rows of 128 B per box, boxes
// 8 KB apart); with fewer, 8-feature groups of 64 pixels x 16 bytes.  Then
// a 512-byte block of BF16 ones for the bias sums and the barriers.
template <int KT>
struct DwSmem {
  static constexpr int PC = 64;                  // pixels per stage
  static constexpr int A_BYTES = 128 * PC * 2;   // G^T: up to 16 groups x 64 pixels x 16 B
  static constexpr int B_BYTES = KT * PC * 2;    // X^T: KT / 8 groups
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int S = (196608 / STAGE) < 8 ? (196608 / STAGE) : 8;
  static constexpr int ONES = S * STAGE;
  static constexpr int BAR = ONES + 512;         // full[S], empty[S], done, drain, TMEM slot
  static constexpr size_t total = BAR + (2 * S + 2) * 8 + 16;
  // dW in columns [0, KT), the bias sums in [KT, KT + 16)
  static constexpr uint32_t TCOLS = KT + 16 <= 32 ? 32 : KT + 16 <= 64 ? 64 : KT + 16 <= 128 ? 128
                                  : KT + 16 <= 256 ? 256 : 512;
};

// part[z][n0 .. n0 + 127][k0 .. k0 + KT) = sum_p G[p, n] X[p, k] over the
// pixel range of split z = blockIdx.z, and (k-tile 0, dbpart given)
// dbpart[z][n] = sum_p G[p, n].  The pixel is the MMA's K: both operands are
// MN-major (G and X as stored, rows = pixels), so the TMA loads them without
// a transpose; the bias sums are one more N = 16 MMA of G^T against a block
// of ones.  Thread 0 streams the stages, thread 32 issues the MMAs; all 128
// threads store the tile (thread = row) to the CTA's own slice, so the sum
// over splits is left to a fixed-order pass.
// GSW: G in the swizzled layout (N >= 64); X is swizzled when KT >= 64.
template <int KT, bool GSW>
__global__ void __launch_bounds__(128, 1) dw_kernel(const __grid_constant__ DwArgs a,
                                                   const __grid_constant__ CUtensorMap gmap,
                                                   const __grid_constant__ CUtensorMap xmap) {
  using L = DwSmem<KT>;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L::BAR);
  uint64_t* empty = full + L::S;
  uint64_t* done = empty + L::S;
  uint64_t* dbar = done + 1;  // a give-up waits here for the MMAs already issued
  uint32_t* tslot = reinterpret_cast<uint32_t*>(dbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * 128, k0 = blockIdx.y * KT;
  const bool bias = a.dbpart != nullptr && blockIdx.y == 0;
  const int64_t pbeg = (int64_t)blockIdx.z * a.chunks_per_cta * L::PC;
  const int64_t pend = min(a.P, pbeg + (int64_t)a.chunks_per_cta * L::PC);
  const int nchunks = pend > pbeg ? (int)((pend - pbeg + L::PC - 1) / L::PC) : 0;
  constexpr bool XSW = KT >= 64;
  if ((GSW || XSW) && (tc::smem_addr(sm) & 1023u)) {  // the swizzle repeats every 1 KB
    if (tid == 0) atomicOr(&g_ae_error, 4u);
    return;
  }
  if (warp == 0) tc::tmem_alloc(tslot, L::TCOLS);
  if (tid == 0) {
    for (int i = 0; i < 2 * L::S + 2; i++) tc::mbar_init(&full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) reinterpret_cast<uint4*>(sm + L::ONES)[tid] = make_uint4(0x3F803F80u, 0x3F803F80u,
                                                                        0x3F803F80u, 0x3F803F80u);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t sbase = tc::smem_addr(sm);
  bool ok = true;
  int issued = 0;  // chunks whose TMA loads thread 0 issued
  if (tid == 0) {
    for (int ch = 0; ch < nchunks && ok; ch++) {
      const int s = ch % L::S;
      if (ch >= L::S && !tc::mbar_wait(&empty[s], (uint32_t)(ch / L::S - 1) & 1, kSpinLimit)) {
        ok = false;
        break;
      }
      const uint32_t st = sbase + s * L::STAGE;
      const int p0 = (int)(pbeg + (int64_t)ch * L::PC);
      tc::mbar_expect_tx(&full[s], (uint32_t)(a.a_tx + a.b_tx));
      if constexpr (GSW) {
        for (int b = 0; b < 2 && n0 + 64 * b < a.N; b++)
          tc::tma_load_2d(st + b * 8192, &gmap, n0 + 64 * b, p0, &full[s]);
      } else {
        tc::tma_load_3d(st, &gmap, 0, p0, n0 / 8, &full[s]);
      }
      if constexpr (XSW) {
#pragma unroll
        for (int b = 0; b < KT / 64; b++)
          tc::tma_load_2d(st + L::A_BYTES + b * 8192, &xmap, k0 + 64 * b, p0, &full[s]);
      } else {
        tc::tma_load_3d(st + L::A_BYTES, &xmap, 0, p0, k0 / 8, &full[s]);
      }
      issued = ch + 1;
    }
  } else if (tid == 32) {
    // MN-major A and B (bits 15 and 16).  Swizzled: 64-feature atoms 8 KB
    // apart (LBO), 8-pixel groups 1 KB apart (SBO), a K-step of 16 pixels
    // is 2 KB; unswizzled: K-adjacent core matrices (the next 8 pixels)
    // 128 B apart (LBO), MN-adjacent ones (the next 8 features) 1 KB (SBO).
    constexpr uint32_t kMN = (1u << 15) | (1u << 16);
    constexpr uint64_t kSw = (uint64_t)2 << 61;
    const uint64_t ones = tc::sdesc(sbase + L::ONES, 128, 256);
    for (int ch = 0; ch < nchunks && ok; ch++) {
      const int s = ch % L::S;
      if (!tc::mbar_wait(&full[s], (uint32_t)(ch / L::S) & 1, kSpinLimit)) {
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t sa = sbase + s * L::STAGE, sb = sa + L::A_BYTES;
#pragma unroll
      for (int j = 0; j < L::PC / 16; j++) {
        const uint64_t ad = GSW ? tc::sdesc(sa + j * 2048, 8192, 1024) | kSw
                                : tc::sdesc(sa + j * 256, 128, L::PC * 16);
        const uint64_t bd = XSW ? tc::sdesc(sb + j * 2048, 8192, 1024) | kSw
                                : tc::sdesc(sb + j * 256, 128, L::PC * 16);
        tc::mma_bf16(tmem, ad, bd, tc::idesc_bf16(128, KT) | kMN, (ch | j) != 0);
        if (bias) tc::mma_bf16(tmem + KT, ad, ones, tc::idesc_bf16(128, 16) | (1u << 15), (ch | j) != 0);
      }
      tc::commit(&empty[s]);
    }
    if (ok && nchunks > 0) tc::commit(done);
  }
  ok = __syncthreads_and(ok);
  if (ok && nchunks > 0) ok = __syncthreads_and(tc::mbar_wait(done, 0, kSpinLimit));
  if (!ok) {
    if (tid == 0) {
      report_timeout();
      // the loads still in flight (at most one ring's worth) land first
      for (int c = issued > L::S ? issued - L::S : 0; c < issued; c++)
        tc::mbar_wait(&full[c % L::S], (uint32_t)(c / L::S) & 1, kSpinLimit);
    } else if (tid == 32) {  // and the MMAs issued so far finish
      tc::commit(dbar);
      tc::mbar_wait(dbar, 0, kSpinLimit);
    }
  } else {
    // the launch gives every split at least one chunk; an empty one stores zeros
    const int n = n0 + warp * 32 + lane;
    const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16);
    float* prow = a.part + ((int64_t)blockIdx.z * a.N + n) * a.K + k0;
    if (nchunks > 0) tc::fence_after();
    constexpr int CW = KT < 32 ? 16 : 32;
    for (int c0 = 0; c0 < KT; c0 += CW) {
      float v[32];
      if (nchunks > 0) {
        if (CW == 32) tc::tmem_ld32(tb + c0, v);
        else tc::tmem_ld16(tb + c0, v);
      } else {
#pragma unroll
        for (int q = 0; q < 32; q++) v[q] = 0.f;
      }
      if (n < a.N) {
        float4* dst = reinterpret_cast<float4*>(prow + c0);
#pragma unroll
        for (int q = 0; q < CW / 4; q++)
          dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
    if (bias) {
      float v[32];
      if (nchunks > 0) tc::tmem_ld16(tb + KT, v);
      else v[0] = 0.f;
      if (n < a.N) a.dbpart[(int64_t)blockIdx.z * a.N + n] = v[0];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L::TCOLS);
}


// Adam on up to 2 * kAeLayers parameter tensors in one launch: segment j
// holds elements [start[j], start[j + 1]) of the concatenation.  Its
// gradient is the sum of splits[j] partial slices (part[j], slice z at
// z * len), added in slice order (0, 1, ...) and stored to g[j] as well.
struct AdamSegs {
  float* w[2 * kAeLayers];
  float* m[2 * kAeLayers];
  float* v[2 * kAeLayers];
  float* g[2 * kAeLayers];
  const float* part[2 * kAeLayers];
  int splits[2 * kAeLayers];
  int64_t start[2 * kAeLayers + 1];
  int n;
};
__global__ void adam_all_kernel(const __grid_constant__ AdamSegs S, float lr, float bc1, float bc2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int64_t total = S.start[S.n];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int j = 0;
    while (S.start[j + 1] <= e) j++;
    const int64_t i = e - S.start[j], len = S.start[j + 1] - S.start[j];
    const float* pp = S.part[j] + i;
    const int nz = S.splits[j];
    float gi = 0.f;
    int z = 0;
    for (; z + 8 <= nz; z += 8) {  // eight loads in flight, added in slice order
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; u++) t[u] = pp[(int64_t)(z + u) * len];
#pragma unroll
      for (int u = 0; u < 8; u++) gi += t[u];
    }
    for (; z < nz; z++) gi += pp[(int64_t)z * len];
    S.g[j][i] = gi;
    const float mi = b1 * S.m[j][i] + (1.f - b1) * gi;
    const float vi = b2 * S.v[j][i] + (1.f - b2) * gi * gi;
    S.m[j][i] = mi;
    S.v[j][i] = vi;
    S.w[j][i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// BF16 copies W and W^T of up to kAeLayers layers in one launch.
struct PackSegs {
  const float* W[kAeLayers];
  __nv_bfloat16* Wb[kAeLayers];
  __nv_bfloat16* Wt[kAeLayers];
  int N[kAeLayers], K[kAeLayers];
  int64_t start[kAeLayers + 1];
  int n;
};
__global__ void pack_all_kernel(const __grid_constant__ PackSegs S) {
  const int64_t total = S.start[S.n];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int j = 0;
    while (S.start[j + 1] <= e) j++;
    const int64_t i = e - S.start[j];
    const int K = S.K[j], N = S.N[j];
    const int n = (int)(i / K), k = (int)(i % K);
    const __nv_bfloat16 b = __float2bfloat16_rn(S.W[j][i]);
    S.Wb[j][i] = b;
    S.Wt[j][(int64_t)k * N + n] = b;
  }
}

// ------------------------------------------------------------------ host side

template <int NT, int KC>
static lgs_status launch_layer_t(const LayerArgs& a, cudaStream_t s) {
  using L = LayerSmem<NT, KC>;
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(layer_kernel<NT, KC>), (int)L::total));
  CUtensorMap amap, bmap, tmap, omap;
  std::memset(&amap, 0, sizeof(amap));
  std::memset(&bmap, 0, sizeof(bmap));
  std::memset(&tmap, 0, sizeof(tmap));
  std::memset(&omap, 0, sizeof(omap));
  if (!a.a_f32) {  // A [P, K] and W [N, K] as K-major chunks of KC columns
    const bool made = KC == 64 ? make_swizzled_map(&amap, a.A, a.P, a.K, 64, 128) &&
                                     make_swizzled_map(&bmap, a.W, a.N, a.K, 64, L::BROWS)
                               : make_kmajor_map(&amap, a.A, a.P, a.K, 128, KC / 8) &&
                                     make_kmajor_map(&bmap, a.W, a.N, a.K, L::BROWS, KC / 8);
    if (!made) return LGS_ERR_CUDA;
  }
  if (a.epi == EPI_RECON) {  // whole 512-wide rows, staged in the two stages
    if (NT != 512 || a.N != 512 || 2 * L::STAGE < 8192 + 128 * 512 * 2) {
      set_error("the reconstruction loss needs 512-wide rows and K >= 64");
      return LGS_ERR_INVALID;
    }
    if (!make_swizzled_map(&tmap, a.target, a.P, 512, 64, 128) ||
        !make_swizzled_map(&omap, a.out_bf, a.P, 512, 64, 128))
      return LGS_ERR_CUDA;
  }
  dim3 grid((unsigned)((a.P + 127) / 128), a.N / NT);
  layer_kernel<NT, KC><<<grid, kLayerThreads, L::total, s>>>(a, amap, bmap, tmap, omap);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

static lgs_status launch_layer(const LayerArgs& a, cudaStream_t s) {
  if (a.P == 0) return LGS_OK;
  const bool k16 = a.K == 16;
  switch (a.N) {
    case 16: return k16 ? launch_layer_t<16, 16>(a, s) : launch_layer_t<16, 64>(a, s);
    case 64: return k16 ? launch_layer_t<64, 16>(a, s) : launch_layer_t<64, 64>(a, s);
    case 128: return k16 ? launch_layer_t<128, 16>(a, s) : launch_layer_t<128, 64>(a, s);
    case 256: return k16 ? launch_layer_t<256, 16>(a, s) : launch_layer_t<256, 64>(a, s);
    case 512: return k16 ? launch_layer_t<512, 16>(a, s) : launch_layer_t<512, 64>(a, s);
    default: set_error("unsupported layer width"); return LGS_ERR_INVALID;
  }
}

// How dw_kernel splits one layer's weight gradient: 128-feature row tiles,
// KT-feature column tiles, and the pixel chunks (64 pixels) cut into `splits`
// ranges of chunks_per_cta, so that the grid holds about one CTA per SM.
// Every split gets at least one chunk.  The workspace holds one partial
// [N, K] slice (and [N] bias slice) per split.
struct DwPlan {
  int KT, ntile, ktile, chunks_per_cta;
  int64_t splits;
};
static DwPlan dw_plan(int64_t P, int N, int K) {
  DwPlan d;
  d.KT = K == 16 ? 16 : K == 64 ? 64 : K == 128 ? 128 : 256;
  d.ntile = (N + 127) / 128;
  d.ktile = K / d.KT;
  const int64_t chunks = std::max<int64_t>(1, (P + 63) / 64);
  int64_t splits = std::max<int64_t>(1, sm_count() / (d.ntile * d.ktile));
  splits = std::min<int64_t>(splits, chunks);
  d.chunks_per_cta = (int)((chunks + splits - 1) / splits);
  d.splits = (chunks + d.chunks_per_cta - 1) / d.chunks_per_cta;
  return d;
}

template <int KT, bool GSW>
static lgs_status launch_dw_t(const __nv_bfloat16* G, const __nv_bfloat16* X, DwArgs a,
                              cudaStream_t s) {
  using L = DwSmem<KT>;
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(dw_kernel<KT, GSW>), (int)L::total));
  // G [P, N] and X [P, K], pixels as rows (rows past P read as zero): with 64
  // or more features, 64-feature x 64-pixel boxes in the 128-byte swizzle;
  // otherwise viewed as [features / 8][P][8] and loaded as g blocks of
  // 64 pixels x 16 bytes
  const int ga = std::min(16, a.N / 8), gb = KT / 8;
  CUtensorMap gmap, xmap;
  const bool made = (GSW ? make_swizzled_map(&gmap, G, a.P, a.N, 64, L::PC)
                         : make_kmajor_map(&gmap, G, a.P, a.N, L::PC, ga)) &&
                    (KT >= 64 ? make_swizzled_map(&xmap, X, a.P, a.K, 64, L::PC)
                              : make_kmajor_map(&xmap, X, a.P, a.K, L::PC, gb));
  if (!made) return LGS_ERR_CUDA;
  a.a_tx = ga * L::PC * 16;  // both layouts: min(128, N) features x 64 pixels
  a.b_tx = gb * L::PC * 16;
  static_assert(L::PC == 64, "dw_plan counts 64-pixel chunks");
  const DwPlan d = dw_plan(a.P, a.N, a.K);
  a.chunks_per_cta = d.chunks_per_cta;
  dw_kernel<KT, GSW><<<dim3(d.ntile, d.ktile, (unsigned)d.splits), 128, L::total, s>>>(a, gmap,
                                                                                      xmap);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

// The partials of dW = G^T X and db = colsum(G) for one layer, in one
// launch: dw_plan(P, N, K).splits slices of [N, K] in part and of [N] in
// dbpart.
static lgs_status launch_dw(const __nv_bfloat16* G, const __nv_bfloat16* X, int64_t P, int N,
                            int K, float* part, float* dbpart, cudaStream_t s) {
  if (P == 0) return LGS_OK;
  DwArgs a{P, N, K, 0, 0, 0, part, dbpart};
  // G in the swizzled layout when each 128-feature tile is one or two
  // whole 64-feature boxes (N = 64 or a multiple of 128)
  if (N == 64 || N % 128 == 0) {
    if (K == 16) return launch_dw_t<16, true>(G, X, a, s);
    if (K == 64) return launch_dw_t<64, true>(G, X, a, s);
    if (K == 128) return launch_dw_t<128, true>(G, X, a, s);
    return launch_dw_t<256, true>(G, X, a, s);  // K = 256 or 512 (two column tiles)
  }
  if (K == 16) return launch_dw_t<16, false>(G, X, a, s);
  if (K == 64) return launch_dw_t<64, false>(G, X, a, s);
  if (K == 128) return launch_dw_t<128, false>(G, X, a, s);
  return launch_dw_t<256, false>(G, X, a, s);
}

static LayerArgs layer(const void* A, bool a_f32, const uint16_t* W, const float* b, int64_t P,
                       int K, int N, int epi) {
  LayerArgs a = {};
  a.A = A;
  a.a_f32 = a_f32 ? 1 : 0;
  a.W = reinterpret_cast<const __nv_bfloat16*>(W);
  a.bias = b;
  a.P = P;
  a.K = K;
  a.N = N;
  a.epi = epi;
  return a;
}

// Workspace carving (bf16 activation buffers, f32 partials; 256-byte aligned).
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  __nv_bfloat16* bf(int64_t P, int w) {
    __nv_bfloat16* p = base ? reinterpret_cast<__nv_bfloat16*>(base + off) : nullptr;
    off += ((size_t)P * w * 2 + 255) & ~(size_t)255;
    return p;
  }
  float* f32(int64_t count) {
    float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += ((size_t)count * 4 + 255) & ~(size_t)255;
    return p;
  }
};

// The fused encoder keeps its activations on chip: only the packed weights.
static void* carve_encode(Carver& c) { return c.bf(1, (int)(encode_pack_bytes() / 2)); }

struct DecodeBufs {
  __nv_bfloat16* a[3];
  void* pack;
};
// The packed weight units first, at offset 0 whatever P (ae_decode_pack
// writes them there), then the layer-by-layer activations.
static void carve_decode(Carver& c, int64_t P, DecodeBufs& B) {
  B.pack = c.bf(1, (int)(decode_pack_bytes() / 2));
  const int w[3] = {64, 128, 256};
  for (int i = 0; i < 3; i++) B.a[i] = c.bf(P, w[i]);
}

struct TrainBufs {
  __nv_bfloat16* act[8];   // output of layer l (post-activation; z for l = 3)
  __nv_bfloat16* pre[8];   // pre-activation of hidden layers
  __nv_bfloat16* grad[8];  // gradient w.r.t. the output of layer l (after GELU')
  float* wpart[8];         // dw_plan(...).splits partial weight gradients of layer l
  float* bpart[8];         // and its partial bias gradients
  int splits[8];
};
static void carve_train(Carver& c, int64_t P, TrainBufs& B) {
  for (int l = 0; l < kAeLayers; l++) {
    const int w = kAeWidths[l + 1];
    B.act[l] = c.bf(P, w);
    B.pre[l] = c.bf(P, w);
    B.grad[l] = c.bf(P, w);
  }
  for (int l = 0; l < kAeLayers; l++) {
    const int K = kAeWidths[l], N = kAeWidths[l + 1];
    const DwPlan d = dw_plan(P, N, K);
    B.splits[l] = (int)d.splits;
    B.wpart[l] = c.f32(d.splits * N * K);
    B.bpart[l] = c.f32(d.splits * N);
  }
}

static lgs_status check_weights(const lgs_ae_weights* w, int first, int last) {
  LGS_CHECK_ARG(w != nullptr, "weights are null");
  for (int l = first; l <= last; l++) {
    LGS_CHECK_ARG(w->W[l] && w->Wt[l] && w->b[l], "null weight pointer");
    LGS_CHECK_ARG(aligned(w->W[l], 16) && aligned(w->Wt[l], 16), "weights must be 16-byte aligned");
  }
  return LGS_OK;
}

}  // namespace lgs

using namespace lgs;

extern "C" size_t ae_workspace_bytes(int64_t P, int what) {
  if (P < 0) return 0;
  Carver c(nullptr);
  if (what == LGS_AE_ENCODE) {
    carve_encode(c);
  } else if (what == LGS_AE_DECODE) {
    DecodeBufs B;
    carve_decode(c, P, B);
  } else if (what == LGS_AE_TRAIN) {
    TrainBufs B;
    carve_train(c, P, B);
  } else {
    return 0;
  }
  return c.off + 256;
}

extern "C" lgs_status ae_encode(const lgs_ae_weights* w, const uint16_t* x, int64_t P, float* z,
                                void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  LGS_CHECK_ARG(P >= 0, "P < 0");
  lgs_status st = check_weights(w, 0, 3);
  if (st != LGS_OK) return st;
  if (P == 0) return LGS_OK;
  LGS_CHECK_ARG(x && z && workspace, "null pointer");
  LGS_CHECK_ARG(aligned(x, 16) && aligned(z, 16) && aligned(workspace, 256), "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= ae_workspace_bytes(P, LGS_AE_ENCODE), "workspace too small");
  cudaStream_t s = as_stream(stream);
  Carver c(workspace);
  void* pack = carve_encode(c);
  return launch_encode_fused(w, x, P, z, pack, s);
}

extern "C" lgs_status ae_decode(const lgs_ae_weights* w, const float* z, int64_t P,
                                const uint16_t* target, float weight, float* loss_dev, float* dz,
                                float* y_opt, void* workspace, size_t workspace_bytes,
                                void* stream) {
  clear_error();
  LGS_CHECK_ARG(P >= 0, "P < 0");
  lgs_status st = check_weights(w, 4, 7);
  if (st != LGS_OK) return st;
  if (P == 0) return LGS_OK;
  LGS_CHECK_ARG(z && workspace, "null pointer");
  LGS_CHECK_ARG(target || y_opt, "nothing to compute: give a target or y_opt");
  LGS_CHECK_ARG(!target || (loss_dev && dz), "a target needs loss_dev and dz");
  LGS_CHECK_ARG(aligned(z, 16) && aligned(workspace, 256) && aligned(target, 32) &&
                    aligned(dz, 16) && aligned(y_opt, 16),
                "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= ae_workspace_bytes(P, LGS_AE_DECODE), "workspace too small");
  cudaStream_t s = as_stream(stream);
  Carver c(workspace);
  DecodeBufs B;
  carve_decode(c, P, B);
  LayerArgs a;
  if (y_opt) {  // inference: layer by layer, activations through the workspace
    a = layer(z, true, w->W[4], w->b[4], P, 16, 64, EPI_GELU); a.out_bf = B.a[0];
    if ((st = launch_layer(a, s)) != LGS_OK) return st;
    a = layer(B.a[0], false, w->W[5], w->b[5], P, 64, 128, EPI_GELU); a.out_bf = B.a[1];
    if ((st = launch_layer(a, s)) != LGS_OK) return st;
    a = layer(B.a[1], false, w->W[6], w->b[6], P, 128, 256, EPI_GELU); a.out_bf = B.a[2];
    if ((st = launch_layer(a, s)) != LGS_OK) return st;
    a = layer(B.a[2], false, w->W[7], w->b[7], P, 256, 512, EPI_LIN_F32); a.out_f32 = y_opt;
    if ((st = launch_layer(a, s)) != LGS_OK) return st;
  }
  if (!target) return LGS_OK;
  // Eq. 2: decoder forward, L1 against F_gt and the gradient back to
  // F_render in one persistent kernel (nothing but dz leaves the chip)
  return launch_decode_fused(w, z, P, target, weight, loss_dev, dz, B.pack, false, s);
}

extern "C" lgs_status ae_decode_pack(const lgs_ae_weights* w, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  clear_error();
  lgs_status st = check_weights(w, 4, 7);
  if (st != LGS_OK) return st;
  LGS_CHECK_ARG(workspace != nullptr, "null pointer");
  LGS_CHECK_ARG(aligned(workspace, 256), "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= decode_pack_bytes(), "workspace too small");
  return launch_decode_pack(w, workspace, as_stream(stream));
}

extern "C" lgs_status ae_decode_packed(const lgs_ae_weights* w, const float* z, int64_t P,
                                       const uint16_t* target, float weight, float* loss_dev,
                                       float* dz, void* workspace, size_t workspace_bytes,
                                       void* stream) {
  clear_error();
  LGS_CHECK_ARG(P >= 0, "P < 0");
  lgs_status st = check_weights(w, 4, 7);
  if (st != LGS_OK) return st;
  if (P == 0) return LGS_OK;
  LGS_CHECK_ARG(z && workspace && target && loss_dev && dz, "null pointer");
  LGS_CHECK_ARG(aligned(z, 16) && aligned(workspace, 256) && aligned(target, 32) &&
                    aligned(dz, 16),
                "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= ae_workspace_bytes(P, LGS_AE_DECODE), "workspace too small");
  Carver c(workspace);
  DecodeBufs B;
  carve_decode(c, P, B);
  return launch_decode_fused(w, z, P, target, weight, loss_dev, dz, B.pack, true,
                             as_stream(stream));
}

extern "C" lgs_status ae_pack(lgs_ae_state* st_, int first, int last, void* stream) {
  clear_error();
  LGS_CHECK_ARG(st_ && first >= 0 && last < kAeLayers && first <= last, "bad arguments");
  cudaStream_t s = as_stream(stream);
  PackSegs S;
  S.n = 0;
  S.start[0] = 0;
  for (int l = first; l <= last; l++) {
    LGS_CHECK_ARG(st_->W[l] && st_->Wbf[l] && st_->Wtbf[l], "null weight pointer");
    const int j = S.n++;
    S.W[j] = st_->W[l];
    S.Wb[j] = reinterpret_cast<__nv_bfloat16*>(st_->Wbf[l]);
    S.Wt[j] = reinterpret_cast<__nv_bfloat16*>(st_->Wtbf[l]);
    S.K[j] = kAeWidths[l];
    S.N[j] = kAeWidths[l + 1];
    S.start[j + 1] = S.start[j] + (int64_t)S.N[j] * S.K[j];
  }
  pack_all_kernel<<<(unsigned)std::min<int64_t>((S.start[S.n] + 255) / 256, 152 * 8), 256, 0, s>>>(S);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

extern "C" lgs_status ae_train_step(lgs_ae_state* st_, const uint16_t* x, const float* target,
                                    int64_t P, int mode, float lr, float* loss_dev,
                                    void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  LGS_CHECK_ARG(st_ != nullptr, "state is null");
  LGS_CHECK_ARG(mode == LGS_AE_RECON || mode == LGS_AE_ENC_ADAPT, "bad mode");
  LGS_CHECK_ARG(P > 0, "P must be positive");
  LGS_CHECK_ARG(x && loss_dev && workspace, "null pointer");
  LGS_CHECK_ARG(mode == LGS_AE_RECON || target, "ENC_ADAPT needs the rendered target");
  LGS_CHECK_ARG(aligned(x, 16) && aligned(workspace, 256) && aligned(target, 16),
                "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= ae_workspace_bytes(P, LGS_AE_TRAIN), "workspace too small");
  const int last = mode == LGS_AE_RECON ? 7 : 3;
  for (int l = 0; l <= last; l++)
    LGS_CHECK_ARG(st_->W[l] && st_->b[l] && st_->mW[l] && st_->vW[l] && st_->mb[l] && st_->vb[l] &&
                      st_->gW[l] && st_->gb[l] && st_->Wbf[l] && st_->Wtbf[l],
                  "null state pointer");
  for (int l = 0; l <= last; l++)  // TMA loads of the BF16 copies
    LGS_CHECK_ARG(aligned(st_->Wbf[l], 16) && aligned(st_->Wtbf[l], 16),
                  "misaligned state pointer");
  cudaStream_t s = as_stream(stream);
  Carver c(workspace);
  TrainBufs B;
  carve_train(c, P, B);
  auto W = [&](int l) { return st_->Wbf[l]; };
  auto Wt = [&](int l) { return st_->Wtbf[l]; };
  lgs_status st;
  // forward, keeping every layer's input and pre-activation
  const void* in = x;
  for (int l = 0; l <= 3; l++) {
    const int K = kAeWidths[l], N = kAeWidths[l + 1];
    LayerArgs a;
    if (l < 3) {
      a = layer(in, false, W(l), st_->b[l], P, K, N, EPI_GELU);
      a.out_bf = B.act[l];
      a.pre_out = B.pre[l];
    } else if (mode == LGS_AE_RECON) {
      a = layer(in, false, W(l), st_->b[l], P, K, N, EPI_LIN_BF16);
      a.out_bf = B.act[l];
    } else {
      // Eq. 3: L1(E(F_gt), F_render), gradient w.r.t. z straight out of the epilogue
      a = layer(in, false, W(l), st_->b[l], P, K, N, EPI_L1_F32T);
      a.out_bf = B.grad[3];
      a.target = target;
      a.scale = 1.f / ((float)P * 16.f);
      a.loss = loss_dev;
    }
    if ((st = launch_layer(a, s)) != LGS_OK) return st;
    in = B.act[l];
  }
  if (mode == LGS_AE_RECON) {
    for (int l = 4; l <= 7; l++) {
      const int K = kAeWidths[l], N = kAeWidths[l + 1];
      LayerArgs a;
      if (l < 7) {
        a = layer(B.act[l - 1], false, W(l), st_->b[l], P, K, N, EPI_GELU);
        a.out_bf = B.act[l];
        a.pre_out = B.pre[l];
      } else {
        a = layer(B.act[6], false, W(7), st_->b[7], P, K, N, EPI_RECON);
        a.out_bf = B.grad[7];
        a.target = x;
        a.scale = 1.f / (float)P;
        a.loss = loss_dev;
      }
      if ((st = launch_layer(a, s)) != LGS_OK) return st;
    }
  }
  // backward: dW_l = grad_l^T input_l, grad_{l-1} = (grad_l W_l) * gelu'(pre_{l-1})
  for (int l = last; l >= 0; l--) {
    const int K = kAeWidths[l], N = kAeWidths[l + 1];
    const __nv_bfloat16* input = l == 0 ? reinterpret_cast<const __nv_bfloat16*>(x) : B.act[l - 1];
    if ((st = launch_dw(B.grad[l], input, P, N, K, B.wpart[l], B.bpart[l], s)) != LGS_OK)
      return st;
    if (l == 0) break;
    LayerArgs a;
    if (l == 4) {  // below the linear latent: no GELU
      a = layer(B.grad[l], false, Wt(l), nullptr, P, N, K, EPI_DX_BF16);
    } else {
      a = layer(B.grad[l], false, Wt(l), nullptr, P, N, K, EPI_DGELU);
      a.pre_in = B.pre[l - 1];
    }
    a.out_bf = B.grad[l - 1];
    if ((st = launch_layer(a, s)) != LGS_OK) return st;
  }
  // Adam on FP32 master weights, then refresh the BF16 copies
  st_->step += 1;
  const float bc1 = 1.f - powf(0.9f, (float)st_->step);
  const float bc2 = 1.f - powf(0.999f, (float)st_->step);
  AdamSegs A;
  A.n = 0;
  A.start[0] = 0;
  for (int l = 0; l <= last; l++) {
    const int64_t nw = (int64_t)kAeWidths[l] * kAeWidths[l + 1], nb = kAeWidths[l + 1];
    for (int wb = 0; wb < 2; wb++) {
      const int j = A.n++;
      A.w[j] = wb ? st_->b[l] : st_->W[l];
      A.m[j] = wb ? st_->mb[l] : st_->mW[l];
      A.v[j] = wb ? st_->vb[l] : st_->vW[l];
      A.g[j] = wb ? st_->gb[l] : st_->gW[l];
      A.part[j] = wb ? B.bpart[l] : B.wpart[l];
      A.splits[j] = B.splits[l];
      A.start[j + 1] = A.start[j] + (wb ? nb : nw);
    }
  }
  adam_all_kernel<<<(unsigned)std::min<int64_t>((A.start[A.n] + 255) / 256, 152 * 8), 256, 0, s>>>(
      A, lr, bc1, bc2);
  LGS_CHECK_LAUNCH();
  return ae_pack(st_, 0, last, stream);
}

namespace lgs {
namespace {
// |c_n|^2 of every BF16 codeword, summed left to right in FP32.
__global__ void codeword_norms_kernel(const __nv_bfloat16* __restrict__ cb, int K, int D,
                                      float* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < D; j++) {
      const float v = __bfloat162float(cb[(int64_t)k * D + j]);
      s = fmaf(v, v, s);
    }
    out[k] = s;
  }
}
}  // namespace
}  // namespace lgs

extern "C" size_t lgs_codebook_workspace(int K) { return K > 0 ? 4 * (size_t)K : 0; }

extern "C" lgs_status lgs_codebook_assign(const uint16_t* x, int64_t P, int D,
                                          const uint16_t* codebook, int K, uint32_t* assign_opt,
                                          uint32_t* hist, void* workspace, size_t workspace_bytes,
                                          void* stream) {
  clear_error();
  LGS_CHECK_ARG(P >= 0 && P < ((int64_t)1 << 31), "P out of range");
  LGS_CHECK_ARG(D == 16 || (D >= 64 && D % 64 == 0 && D <= 4096), "D must be 16 or a multiple of 64");
  LGS_CHECK_ARG(K == 16 || K == 64 || K == 128 || K == 256 || K == 512,
                "codebook size must be 16, 64, 128, 256 or 512");
  LGS_CHECK_ARG(codebook && hist && workspace, "null pointer");
  LGS_CHECK_ARG(P == 0 || x, "null pointer");
  LGS_CHECK_ARG(aligned(x, 16) && aligned(codebook, 16) && aligned(workspace, 4),
                "misaligned pointer");
  LGS_CHECK_ARG(workspace_bytes >= lgs_codebook_workspace(K), "workspace too small");
  if (P == 0) return LGS_OK;
  cudaStream_t s = as_stream(stream);
  float* cnorm = (float*)workspace;
  codeword_norms_kernel<<<(K + 127) / 128, 128, 0, s>>>((const __nv_bfloat16*)codebook, K, D, cnorm);
  LayerArgs a = {};
  a.A = x;
  a.W = (const __nv_bfloat16*)codebook;
  a.bias = cnorm;
  a.P = P;
  a.K = D;
  a.N = K;
  a.epi = EPI_ARGMIN;
  a.out_u32 = assign_opt;
  a.hist = hist;
  return launch_layer(a, s);
}

// The timeout bit word of lgs_device_error; clear: also reset every part.
static lgs_status wait_error_word(bool clear, unsigned* word) {
  unsigned v = 0, zero = 0;
  LGS_CHECK_CUDA(cudaMemcpyFromSymbol(&v, g_ae_error, sizeof(v)));
  if (clear && v) LGS_CHECK_CUDA(cudaMemcpyToSymbol(g_ae_error, &zero, sizeof(zero)));
  *word = v | (fused_error_word(clear) << 4) | (sort_error_word(clear) << 8) |
          (encode_error_word(clear) << 12);
  return LGS_OK;
}

extern "C" lgs_status lgs_device_error(int* code) {
  clear_error();
  LGS_CHECK_ARG(code != nullptr, "code is null");
  unsigned v = 0;
  const lgs_status st = wait_error_word(true, &v);
  if (st != LGS_OK) return st;
  *code = (int)v;
  return LGS_OK;
}

extern "C" lgs_status lgs_sync_status(void* stream, int64_t* detail) {
  clear_error();
  if (detail) *detail = 0;
  LGS_CHECK_CUDA(cudaStreamSynchronize(as_stream(stream)));
  // the records are read with synchronous copies: every kernel that can
  // write them and was enqueued on `stream` has finished
  const unsigned long long nf = nonfinite_word(false);
  if (nf != ~0ull) {
    nonfinite_word(true);
    if (detail) *detail = (int64_t)nf;
    set_error("lgs_sync_status: non-finite parameter of Gaussian " + std::to_string(nf));
    return LGS_ERR_NONFINITE;
  }
  const unsigned long long k = capacity_word(false);
  if (k != 0) {
    capacity_word(true);
    if (detail) *detail = (int64_t)k;
    set_error("lgs_sync_status: gs_bin_sort needed capacity " + std::to_string(k));
    return LGS_ERR_CAPACITY;
  }
  unsigned w = 0;
  lgs_status st = wait_error_word(false, &w);
  if (st != LGS_OK) return st;
  if (w != 0) {
    if ((st = wait_error_word(true, &w)) != LGS_OK) return st;
    if (detail) *detail = (int64_t)w;
    set_error("lgs_sync_status: a bounded wait gave up (sites " + std::to_string(w) + ")");
    return LGS_ERR_TIMEOUT;
  }
  return LGS_OK;
}
