// Language loop signature (LEGO-SLAM Sec. III-D) and compact-space query
// relevance (Sec. I).
//
// A keyframe's signature is the histogram of its language features' closest
// codewords (lgs_codebook_assign, a tensor-core GEMM with an argmin
// epilogue); loop candidates are the spatially close past keyframes whose
// signature's cosine similarity exceeds tau_hist, the two most similar first.
// A text query is projected into the compact space by the encoder and
// compared with the map's features by cosine similarity.
#include <algorithm>

#include "common.cuh"

namespace lgs {

namespace {

// cos(h, hs[m]) for every stored histogram, one warp per histogram.
__global__ void hist_cosine_kernel(const uint32_t* __restrict__ h, const uint32_t* __restrict__ hs,
                                   int M, int K, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= M) return;
  float dot = 0.f, na = 0.f, nb = 0.f;
  for (int k = lane; k < K; k += 32) {
    const float a = (float)h[k], b = (float)hs[(int64_t)m * K + k];
    dot = fmaf(a, b, dot);
    na = fmaf(a, a, na);
    nb = fmaf(b, b, nb);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dot += __shfl_xor_sync(0xffffffffu, dot, o);
    na += __shfl_xor_sync(0xffffffffu, na, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  if (lane == 0) {
    const float den = sqrtf(na) * sqrtf(nb);
    out[m] = den > 0.f ? dot / den : 0.f;
  }
}

// Up to `top` candidates: similarity above tau and camera centre within
// radius, most similar first, ties to the lower index; -1 pads.  One block.
__global__ void __launch_bounds__(256)
loop_candidates_kernel(const float* __restrict__ sim, const float* __restrict__ centres, int M,
                       float cx, float cy, float cz, float tau, float r2, int top,
                       int* __restrict__ out) {
  __shared__ float bs[8];
  __shared__ int bi[8];
  __shared__ int chosen[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < top; t++) {
    float best = -INFINITY;
    int idx = -1;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      bool taken = false;
      for (int u = 0; u < t; u++) taken |= chosen[u] == m;
      const float dx = centres[3 * m] - cx, dy = centres[3 * m + 1] - cy,
                  dz = centres[3 * m + 2] - cz;
      const float s = sim[m];
      if (taken || !(s > tau) || !(dx * dx + dy * dy + dz * dz < r2)) continue;
      if (s > best || (s == best && m < idx)) {
        best = s;
        idx = m;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (oi >= 0 && (idx < 0 || ob > best || (ob == best && oi < idx))) {
        best = ob;
        idx = oi;
      }
    }
    if (lane == 0) {
      bs[warp] = best;
      bi[warp] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = -INFINITY;
      int i = -1;
      for (int w = 0; w < 8; w++)
        if (bi[w] >= 0 && (i < 0 || bs[w] > b || (bs[w] == b && bi[w] < i))) {
          b = bs[w];
          i = bi[w];
        }
      chosen[t] = i;
      out[t] = i;
    }
    __syncthreads();
  }
}

constexpr int kMaxQueries = 64;
constexpr int kMaxQueryDim = 64;

// out[m, j] = cos(f_m, q_j); queries and their norms staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
query_kernel(const T* __restrict__ feats, int64_t M, int D, const float* __restrict__ queries,
             int Q, float* __restrict__ out) {
  __shared__ float sq[kMaxQueries * kMaxQueryDim];
  __shared__ float qn[kMaxQueries];
  for (int e = threadIdx.x; e < Q * D; e += blockDim.x) sq[e] = queries[e];
  __syncthreads();
  for (int j = threadIdx.x; j < Q; j += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < D; k++) s = fmaf(sq[j * D + k], sq[j * D + k], s);
    qn[j] = sqrtf(s);
  }
  __syncthreads();
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    float f[kMaxQueryDim];
    float nf = 0.f;
#pragma unroll 8
    for (int k = 0; k < D; k++) {
      f[k] = to_float(feats[m * D + k]);
      nf = fmaf(f[k], f[k], nf);
    }
    nf = sqrtf(nf);
    for (int j = 0; j < Q; j++) {
      float dot = 0.f;
#pragma unroll 8
      for (int k = 0; k < D; k++) dot = fmaf(f[k], sq[j * D + k], dot);
      const float den = nf * qn[j];
      out[m * Q + j] = den > 0.f ? dot / den : 0.f;
    }
  }
}

}  // namespace
}  // namespace lgs

using namespace lgs;

extern "C" lgs_status lgs_hist_cosine(const uint32_t* hist, const uint32_t* hists, int M, int K,
                                      float* out, void* stream) {
  clear_error();
  LGS_CHECK_ARG(M >= 0 && K >= 1, "bad sizes");
  if (M == 0) return LGS_OK;
  LGS_CHECK_ARG(hist && hists && out, "null pointer");
  hist_cosine_kernel<<<(M + 7) / 8, 256, 0, as_stream(stream)>>>(hist, hists, M, K, out);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

extern "C" lgs_status lgs_loop_candidates(const float* sim, const float* centres, int M,
                                          const float* cur_centre_host, float tau_hist,
                                          float radius, int top, int* out, void* stream) {
  clear_error();
  LGS_CHECK_ARG(M >= 0 && top >= 1 && top <= 8, "top must be in [1, 8]");
  LGS_CHECK_ARG(cur_centre_host && out, "null pointer");
  LGS_CHECK_ARG(M == 0 || (sim && centres), "null pointer");
  LGS_CHECK_ARG(radius >= 0.f, "negative radius");
  loop_candidates_kernel<<<1, 256, 0, as_stream(stream)>>>(
      sim, centres, M, cur_centre_host[0], cur_centre_host[1], cur_centre_host[2], tau_hist,
      radius * radius, top, out);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

extern "C" lgs_status gs_query_relevance(const void* feats, int feat_dtype, int64_t M, int D,
                                         const float* queries, int Q, float* out, void* stream) {
  clear_error();
  LGS_CHECK_ARG(M >= 0 && D >= 1 && D <= kMaxQueryDim, "D must be in [1, 64]");
  LGS_CHECK_ARG(Q >= 1 && Q <= kMaxQueries, "Q must be in [1, 64]");
  LGS_CHECK_ARG(Q * D <= kMaxQueries * kMaxQueryDim, "too many query values");
  LGS_CHECK_ARG(feat_dtype == LGS_F32 || feat_dtype == LGS_BF16, "feat_dtype must be F32 or BF16");
  if (M == 0) return LGS_OK;
  LGS_CHECK_ARG(feats && queries && out, "null pointer");
  const int blocks = (int)std::min<int64_t>((M + 255) / 256, 152 * 8);
  cudaStream_t s = as_stream(stream);
  if (feat_dtype == LGS_F32)
    query_kernel<float><<<blocks, 256, 0, s>>>((const float*)feats, M, D, queries, Q, out);
  else
    query_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)feats, M, D, queries,
                                                       Q, out);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
