// Language-guided Gaussian pruning (LEGO-SLAM Sec. III-C, Eq. 4) unioned
// with the geometric criteria, and order-preserving compaction of the kept
// Gaussians.
//
// Eq. 4: each Gaussian G_i examines its K nearest neighbours in 3D; a
// neighbour G_j is redundant when d(p_i, p_j) < tau_dist and the cosine of
// their compact language features exceeds tau_sim.  Only neighbours within
// tau_dist can satisfy the rule, so the neighbour search runs on a uniform
// grid of cells just wider than tau_dist: the Gaussians are radix-sorted by
// cell, and every query scans the 3 x 3 rows of three consecutive cells
// around its own (each row one contiguous run of the sorted order).  Where
// the grid has at most 8 cells per Gaussian a table holds each cell's first
// sorted position, filled from the sorted keys, and a row's run is two loads;
// a cell the table leaves open (one inside a gap of more than kFillRun empty
// cells, or every cell of a larger grid) is found by binary search.  A query keeps the 16 nearest candidates in registers
// (ranked by squared distance, then index), then tests its first K for
// similarity and marks those it outranks (higher opacity logit, or equal
// logit and lower index).
//
// Every decision is a float comparison turned into a mask bit, so the
// arithmetic is spelled out with round-to-nearest intrinsics in a fixed
// order (no fused multiply-add): dx = x_j - x_i, d2 = (dx dx + dy dy) + dz dz,
// d = sqrt(d2) < tau_dist; |f| = sqrt of the sequential sum of f_k f_k;
// sim = (sequential sum of f_ik f_jk) / (|f_i| |f_j|), 0 for a zero norm.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

namespace {

constexpr int kKnnMax = 16;
constexpr int kPruneMaxDim = 64;
constexpr int kCellsPerGaussian = 8;  // the largest grid the start table covers
constexpr int kFillRun = 16;          // the longest run of cells one thread fills
constexpr uint32_t kOpen = 0xffffffffu;

struct Grid {
  float lo[3];
  float inv_cell;
  uint32_t g[3];
};

__device__ __forceinline__ uint32_t cell_coord(float x, float lo, float inv, uint32_t g) {
  // clamped, so Gaussians outside the bounds land in the border cells
  const float u = floorf(__fmul_rn(__fsub_rn(x, lo), inv));
  return (uint32_t)fminf(fmaxf(u, 0.f), (float)(g - 1));
}

template <typename T>
__device__ __forceinline__ float feat_at(const T* f, int64_t i, int d, int k);
template <>
__device__ __forceinline__ float feat_at<float>(const float* f, int64_t i, int d, int k) {
  return f[(int64_t)d * i + k];
}
template <>
__device__ __forceinline__ float feat_at<__nv_bfloat16>(const __nv_bfloat16* f, int64_t i, int d,
                                                         int k) {
  return __bfloat162float(f[(int64_t)d * i + k]);
}

// Cell key and index per Gaussian; geometric bit into the mask; feature norm.
template <typename T>
__global__ void prune_prep_kernel(const float* __restrict__ means, const float* __restrict__ logits,
                                  const float* __restrict__ log_scales, const T* __restrict__ feats,
                                  int d, int64_t n, Grid grid, float thr_logit, float thr_logscale,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                  float* __restrict__ norms, uint8_t* __restrict__ mask) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
    const uint32_t cx = cell_coord(x, grid.lo[0], grid.inv_cell, grid.g[0]);
    const uint32_t cy = cell_coord(y, grid.lo[1], grid.inv_cell, grid.g[1]);
    const uint32_t cz = cell_coord(z, grid.lo[2], grid.inv_cell, grid.g[2]);
    keys[i] = (cz * grid.g[1] + cy) * grid.g[0] + cx;
    vals[i] = (uint32_t)i;
    float s = 0.f;
    for (int k = 0; k < d; k++) {
      const float v = feat_at(feats, i, d, k);
      s = __fadd_rn(s, __fmul_rn(v, v));
    }
    norms[i] = __fsqrt_rn(s);
    const float ls = fmaxf(fmaxf(log_scales[3 * i], log_scales[3 * i + 1]), log_scales[3 * i + 2]);
    mask[i] = (logits[i] < thr_logit || ls > thr_logscale) ? 1 : 0;
  }
}

// Sorted copies of (x, y, z, logit) next to the sorted cell keys.
__global__ void prune_gather_kernel(const float* __restrict__ means,
                                    const float* __restrict__ logits,
                                    const uint32_t* __restrict__ order, int64_t n,
                                    float4* __restrict__ sp) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = order[t];
    // an index out of range only follows a sort whose look-back gave up
    // (LGS_ERR_TIMEOUT): park it at infinity, where it has no neighbours
    sp[t] = i < n ? make_float4(means[3 * (int64_t)i], means[3 * (int64_t)i + 1],
                                means[3 * (int64_t)i + 2], logits[i])
                  : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
  }
}

// First position in the sorted keys with key >= k.
__device__ __forceinline__ int64_t lower_bound(const uint32_t* __restrict__ keys, int64_t n,
                                               uint32_t k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// start[c] = the first sorted position with key >= c, for c in [0, cells]:
// position t (t = n stands for the end) fills the cells after its
// predecessor's key up to its own.  A run longer than kFillRun stays open
// (kOpen, set beforehand), as does anything after keys out of order or out of
// range (only a sort that gave up leaves those).
__global__ void cell_start_kernel(const uint32_t* __restrict__ skey, int64_t n, uint32_t cells,
                                  uint32_t* __restrict__ start) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t prev = t > 0 ? (int64_t)skey[t - 1] : -1;
    const int64_t key = t < n ? (int64_t)skey[t] : (int64_t)cells;
    const int64_t cur = key < (int64_t)cells ? key : (int64_t)cells;
    if (cur - prev > kFillRun) continue;
    for (int64_t c = prev + 1; c <= cur; c++) start[c] = (uint32_t)t;
  }
}

__device__ __forceinline__ int64_t run_start(const uint32_t* __restrict__ start,
                                             const uint32_t* __restrict__ keys, int64_t n,
                                             uint32_t c) {
  const uint32_t v = start ? start[c] : kOpen;
  return v != kOpen ? (int64_t)v : lower_bound(keys, n, c);
}

__device__ __forceinline__ bool closer(float d2, uint32_t j, float e2, uint32_t ej) {
  return d2 < e2 || (d2 == e2 && j < ej);
}

// sequential sum over k of f_ik f_jk, whole rows fetched as 16-byte vectors
// when every row starts on a 16-byte boundary (vec), else one element at a time
template <typename T>
__device__ __forceinline__ float row_dot(const T* __restrict__ f, uint32_t i, uint32_t j, int d,
                                         bool vec);
template <>
__device__ __forceinline__ float row_dot<float>(const float* __restrict__ f, uint32_t i,
                                                uint32_t j, int d, bool vec) {
  float dot = 0.f;
  if (vec) {
    const float4* a = (const float4*)(f + (int64_t)d * i);
    const float4* b = (const float4*)(f + (int64_t)d * j);
    for (int c = 0; c < d / 4; c++) {
      const float4 x = a[c], y = b[c];
      dot = __fadd_rn(dot, __fmul_rn(x.x, y.x));
      dot = __fadd_rn(dot, __fmul_rn(x.y, y.y));
      dot = __fadd_rn(dot, __fmul_rn(x.z, y.z));
      dot = __fadd_rn(dot, __fmul_rn(x.w, y.w));
    }
    return dot;
  }
  for (int k = 0; k < d; k++)
    dot = __fadd_rn(dot, __fmul_rn(feat_at(f, i, d, k), feat_at(f, j, d, k)));
  return dot;
}
template <>
__device__ __forceinline__ float row_dot<__nv_bfloat16>(const __nv_bfloat16* __restrict__ f,
                                                        uint32_t i, uint32_t j, int d, bool vec) {
  float dot = 0.f;
  if (vec) {
    const uint4* a = (const uint4*)(f + (int64_t)d * i);
    const uint4* b = (const uint4*)(f + (int64_t)d * j);
    for (int c = 0; c < d / 8; c++) {
      const uint4 x = a[c], y = b[c];
      const uint32_t xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int w = 0; w < 4; w++) {  // element 2w in the low half, 2w + 1 in the high half
        dot = __fadd_rn(dot, __fmul_rn(__uint_as_float(xs[w] << 16), __uint_as_float(ys[w] << 16)));
        dot = __fadd_rn(dot, __fmul_rn(__uint_as_float(xs[w] & 0xffff0000u),
                                       __uint_as_float(ys[w] & 0xffff0000u)));
      }
    }
    return dot;
  }
  for (int k = 0; k < d; k++)
    dot = __fadd_rn(dot, __fmul_rn(feat_at(f, i, d, k), feat_at(f, j, d, k)));
  return dot;
}

// KM: the length of the nearest-candidate list, at least K
template <typename T, int KM>
__global__ void __launch_bounds__(128)
    prune_knn_kernel(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sidx,
                     const float4* __restrict__ sp, int64_t n, Grid grid, int K, float tau,
                     float tau_sim, const T* __restrict__ feats, int d, bool vec,
                     const float* __restrict__ norms, const float* __restrict__ logits,
                     const uint32_t* __restrict__ start, uint8_t* __restrict__ redundant) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sidx[t];
    if (i >= n) continue;  // see prune_gather_kernel
    const float4 pi = sp[t];
    const uint32_t key = skey[t];
    const uint32_t cx = key % grid.g[0];
    const uint32_t cy = (key / grid.g[0]) % grid.g[1];
    const uint32_t cz = key / (grid.g[0] * grid.g[1]);
    float bd[KM];
    uint32_t bj[KM];
#pragma unroll
    for (int s = 0; s < KM; s++) {
      bd[s] = INFINITY;
      bj[s] = 0xffffffffu;
    }
    const uint32_t x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < grid.g[0] ? cx + 1 : cx;
    for (int dz = -1; dz <= 1; dz++) {
      const int64_t zz = (int64_t)cz + dz;
      if (zz < 0 || zz >= grid.g[2]) continue;
      for (int dy = -1; dy <= 1; dy++) {
        const int64_t yy = (int64_t)cy + dy;
        if (yy < 0 || yy >= grid.g[1]) continue;
        const uint32_t row = ((uint32_t)zz * grid.g[1] + (uint32_t)yy) * grid.g[0];
        const int64_t a = run_start(start, skey, n, row + x0);
        const int64_t b = run_start(start, skey, n, row + x1 + 1);
        for (int64_t u = a; u < b; u++) {
          if (u == t) continue;
          const float4 pj = sp[u];
          const float dx = __fsub_rn(pj.x, pi.x), dy2 = __fsub_rn(pj.y, pi.y),
                      dz2 = __fsub_rn(pj.z, pi.z);
          const float d2 =
              __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy2, dy2)), __fmul_rn(dz2, dz2));
          if (!(__fsqrt_rn(d2) < tau)) continue;
          const uint32_t j = sidx[u];
          if (j >= n || !closer(d2, j, bd[KM - 1], bj[KM - 1])) continue;
          // insert into the sorted list: e[s-1] <= new < e[s]
#pragma unroll
          for (int s = KM - 1; s > 0; s--) {
            const bool up = closer(d2, j, bd[s - 1], bj[s - 1]);
            const bool here = !up && closer(d2, j, bd[s], bj[s]);
            const float nd = up ? bd[s - 1] : (here ? d2 : bd[s]);
            const uint32_t nj = up ? bj[s - 1] : (here ? j : bj[s]);
            bd[s] = nd;
            bj[s] = nj;
          }
          if (closer(d2, j, bd[0], bj[0])) {
            bd[0] = d2;
            bj[0] = j;
          }
        }
      }
    }
    const float ni = norms[i];
    const float li = pi.w;
#pragma unroll
    for (int s = 0; s < KM; s++) {
      if (s >= K || bj[s] == 0xffffffffu) break;
      const uint32_t j = bj[s];
      const float lj = logits[j];
      if (!(li > lj || (li == lj && i < j))) continue;  // G_i is not the one to keep
      const float dot = row_dot(feats, i, j, d, vec);
      const float nn = __fmul_rn(ni, norms[j]);
      const float sim = nn > 0.f ? __fdiv_rn(dot, nn) : 0.f;
      if (sim > tau_sim) redundant[j] = 1;  // every writer stores the same byte
    }
  }
}

// mask |= redundant << 1, and the number pruned.
__global__ void prune_final_kernel(const uint8_t* __restrict__ redundant, int64_t n,
                                   uint8_t* __restrict__ mask, unsigned long long* count) {
  unsigned c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t m = (uint8_t)(mask[i] | (redundant[i] << 1));
    mask[i] = m;
    c += m != 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// ---------------------------------------------------------------- compaction

constexpr int kScanBlock = 1024;

// Kept Gaussians per block of kScanBlock.
__global__ void __launch_bounds__(256) keep_count_kernel(const uint8_t* __restrict__ mask,
                                                         int64_t n, uint32_t* __restrict__ bcount) {
  __shared__ uint32_t ws[8];
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
  uint32_t c = 0;
  for (int k = threadIdx.x; k < kScanBlock; k += 256) {
    const int64_t i = b0 + k;
    c += (i < n && mask[i] == 0) ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; w++) t += ws[w];
    bcount[blockIdx.x] = t;
  }
}

// Exclusive scan of the block counts in one CTA; total into n_kept.
__global__ void __launch_bounds__(1024) keep_scan_kernel(const uint32_t* __restrict__ bcount,
                                                         int64_t nb, uint64_t* __restrict__ boff,
                                                         int64_t* n_kept) {
  __shared__ uint64_t ws[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
    const int64_t b = c0 + threadIdx.x;
    const uint64_t v = b < nb ? bcount[b] : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      ws[lane] = w;
    }
    __syncthreads();
    const uint64_t incl = x + (warp > 0 ? ws[warp - 1] : 0) + carry;
    if (b < nb) boff[b] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_kept = (int64_t)carry;
}

// new_index[i] = rank of G_i among the kept ones, or 0xffffffff if pruned.
__global__ void __launch_bounds__(256) keep_index_kernel(const uint8_t* __restrict__ mask,
                                                         int64_t n,
                                                         const uint64_t* __restrict__ boff,
                                                         uint32_t* __restrict__ new_index) {
  __shared__ uint32_t ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
  uint64_t base = boff[blockIdx.x];
  for (int k0 = 0; k0 < kScanBlock; k0 += 256) {
    const int64_t i = b0 + k0 + threadIdx.x;
    const bool keep = i < n && mask[i] == 0;
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) ws[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, tot = 0;
    for (int w = 0; w < 8; w++) {
      before += w < warp ? ws[w] : 0u;
      tot += ws[w];
    }
    if (i < n)
      new_index[i] = keep ? (uint32_t)(base + before + __popc(bal & ((1u << lane) - 1u)))
                          : 0xffffffffu;
    base += tot;
    __syncthreads();
  }
}

// dst[new_index[i]] = src[i] for the kept rows, one word per thread.
template <typename W>
__global__ void gather_rows_kernel(const W* __restrict__ src, int64_t n, int words,
                                   const uint32_t* __restrict__ new_index, W* __restrict__ dst) {
  const int64_t total = n * words;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / words;
    const uint32_t o = new_index[i];
    if (o != 0xffffffffu) dst[(int64_t)o * words + (e - i * words)] = src[e];
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PruneLayout {
  size_t k0, k1, v0, v1, sp, norms, red, start, sort, total;
};

PruneLayout prune_layout(int64_t n) {
  PruneLayout L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o += align256(b > 0 ? b : 1); return at; };
  L.k0 = take(4 * n); L.k1 = take(4 * n); L.v0 = take(4 * n); L.v1 = take(4 * n);
  L.sp = take(16 * n); L.norms = take(4 * n); L.red = take(n);
  L.start = take(4 * (kCellsPerGaussian * (size_t)n + 1));
  L.sort = take(sort_pairs_scratch(n));
  L.total = o;
  return L;
}

int grid_for(int64_t n, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 16));
}

template <typename T>
void launch_prune(const float* means, const float* logits, const float* log_scales,
                  const void* feats, int d, int64_t n, const lgs_prune_params& P, const Grid& g,
                  uint64_t cells, int nbits, float thr_logit, float thr_logscale, uint8_t* mask,
                  int64_t* n_pruned, char* ws, const PruneLayout& L, cudaStream_t s) {
  uint32_t *k0 = (uint32_t*)(ws + L.k0), *k1 = (uint32_t*)(ws + L.k1);
  uint32_t *v0 = (uint32_t*)(ws + L.v0), *v1 = (uint32_t*)(ws + L.v1);
  float4* sp = (float4*)(ws + L.sp);
  float* norms = (float*)(ws + L.norms);
  uint8_t* red = (uint8_t*)(ws + L.red);
  const T* f = (const T*)feats;
  prune_prep_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(means, logits, log_scales, f, d, n, g,
                                                        thr_logit, thr_logscale, k0, v0, norms,
                                                        mask);
  if (sort_pairs(k0, v0, k1, v1, n, nbits, ws + L.sort, s)) {
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  prune_gather_kernel<<<grid_for(n, 256), 256, 0, s>>>(means, logits, v0, n, sp);
  cudaMemsetAsync(red, 0, (size_t)n, s);
  uint32_t* start = nullptr;
  if (cells <= (uint64_t)kCellsPerGaussian * (uint64_t)n) {
    start = (uint32_t*)(ws + L.start);
    cudaMemsetAsync(start, 0xff, 4 * (size_t)(cells + 1), s);
    cell_start_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(k0, n, (uint32_t)cells, start);
  }
  const bool vec = d % (int)(16 / sizeof(T)) == 0 && ((uintptr_t)feats & 15) == 0;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, (n + 127) / 128);
  if (P.k <= 8)
    prune_knn_kernel<T, 8><<<blocks, 128, 0, s>>>(k0, v0, sp, n, g, P.k, P.tau_dist, P.tau_sim,
                                                   f, d, vec, norms, logits, start, red);
  else
    prune_knn_kernel<T, kKnnMax><<<blocks, 128, 0, s>>>(k0, v0, sp, n, g, P.k, P.tau_dist,
                                                         P.tau_sim, f, d, vec, norms, logits,
                                                         start, red);
  prune_final_kernel<<<grid_for(n, 256), 256, 0, s>>>(red, n, mask,
                                                      (unsigned long long*)n_pruned);
}

}  // namespace
}  // namespace lgs

using namespace lgs;

extern "C" size_t gs_prune_workspace(int64_t n) {
  if (n < 0) return 0;
  return prune_layout(n).total;
}

extern "C" lgs_status gs_prune(const float* means, const float* opacity_logits,
                               const float* log_scales, const void* feats, int feat_dim,
                               int feat_dtype, int64_t n, const lgs_prune_params* params,
                               uint8_t* mask, int64_t* n_pruned_dev, void* workspace,
                               size_t workspace_bytes, void* stream) {
  clear_error();
  LGS_CHECK_ARG(params, "params is null");
  const lgs_prune_params P = *params;
  LGS_CHECK_ARG(n >= 0 && n < ((int64_t)1 << 31), "n out of range");
  LGS_CHECK_ARG(feat_dim >= 1 && feat_dim <= kPruneMaxDim, "feat_dim must be in [1, 64]");
  LGS_CHECK_ARG(feat_dtype == LGS_F32 || feat_dtype == LGS_BF16, "feat_dtype must be F32 or BF16");
  LGS_CHECK_ARG(P.k >= 1 && P.k <= kKnnMax, "k must be in [1, 16]");
  LGS_CHECK_ARG(std::isfinite(P.tau_dist) && P.tau_dist > 0.f, "tau_dist must be positive");
  LGS_CHECK_ARG(!std::isnan(P.tau_sim), "tau_sim is NaN");
  LGS_CHECK_ARG(P.min_opacity >= 0.f && P.min_opacity < 1.f, "min_opacity must be in [0, 1)");
  LGS_CHECK_ARG(P.max_scale > 0.f, "max_scale must be positive (+inf disables it)");
  LGS_CHECK_ARG(n_pruned_dev && workspace, "null pointer");
  LGS_CHECK_ARG(n == 0 || (means && opacity_logits && log_scales && feats && mask),
                "null pointer");
  LGS_CHECK_ARG(aligned(workspace, 256), "workspace must be 256-byte aligned");
  LGS_CHECK_ARG(aligned(means, 4) && aligned(opacity_logits, 4) && aligned(log_scales, 4) &&
                    aligned(feats, feat_dtype == LGS_F32 ? 4 : 2),
                "misaligned pointer");
  // grid of cells 5 % wider than tau_dist: two Gaussians closer than tau_dist
  // then sit in the same or adjacent cells even after float rounding of the
  // cell coordinates (at most 2^16 cells per axis keeps that rounding below
  // 0.02 cell)
  const double cell = (double)P.tau_dist * 1.05;
  uint64_t total = 1;
  Grid g;
  for (int a = 0; a < 3; a++) {
    LGS_CHECK_ARG(std::isfinite(P.lo[a]) && std::isfinite(P.hi[a]) && P.hi[a] >= P.lo[a],
                  "bounds must be finite with hi >= lo");
    const double cells = std::floor(((double)P.hi[a] - (double)P.lo[a]) / cell) + 1.0;
    LGS_CHECK_ARG(cells <= 65536.0, "more than 2^16 grid cells along an axis: raise tau_dist");
    g.lo[a] = P.lo[a];
    g.g[a] = (uint32_t)cells;
    total *= g.g[a];
  }
  LGS_CHECK_ARG(total < (1ull << 32), "grid has 2^32 cells or more: raise tau_dist");
  g.inv_cell = (float)(1.0 / cell);
  int nbits = 1;
  while (nbits < 32 && (1ull << nbits) < total) nbits++;
  const PruneLayout L = prune_layout(n);
  LGS_CHECK_ARG(workspace_bytes >= L.total, "workspace too small");
  // the geometric thresholds on the log scale, rounded to float once
  const float thr_logit = P.min_opacity > 0.f
                              ? (float)std::log((double)P.min_opacity / (1.0 - P.min_opacity))
                              : -INFINITY;
  const float thr_logscale = std::isfinite(P.max_scale) ? (float)std::log((double)P.max_scale)
                                                        : INFINITY;
  cudaStream_t s = as_stream(stream);
  LGS_CHECK_CUDA(cudaMemsetAsync(n_pruned_dev, 0, sizeof(int64_t), s));
  if (n == 0) return LGS_OK;
  if (feat_dtype == LGS_F32)
    launch_prune<float>(means, opacity_logits, log_scales, feats, feat_dim, n, P, g, total,
                        nbits, thr_logit, thr_logscale, mask, n_pruned_dev, (char*)workspace, L,
                        s);
  else
    launch_prune<__nv_bfloat16>(means, opacity_logits, log_scales, feats, feat_dim, n, P, g,
                                total, nbits, thr_logit, thr_logscale, mask, n_pruned_dev,
                                (char*)workspace, L, s);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

extern "C" size_t gs_compact_workspace(int64_t n) {
  if (n < 0) return 0;
  const int64_t nb = std::max<int64_t>(1, (n + kScanBlock - 1) / kScanBlock);
  return align256(4 * (size_t)nb) + align256(8 * (size_t)nb);
}

extern "C" lgs_status gs_compact_index(const uint8_t* mask, int64_t n, uint32_t* new_index,
                                       int64_t* n_kept_dev, void* workspace,
                                       size_t workspace_bytes, void* stream) {
  clear_error();
  LGS_CHECK_ARG(n >= 0 && n < ((int64_t)1 << 32) - 1, "n out of range");
  LGS_CHECK_ARG(n_kept_dev && workspace, "null pointer");
  LGS_CHECK_ARG(n == 0 || (mask && new_index), "null pointer");
  LGS_CHECK_ARG(aligned(workspace, 256), "workspace must be 256-byte aligned");
  LGS_CHECK_ARG(workspace_bytes >= gs_compact_workspace(n), "workspace too small");
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    LGS_CHECK_CUDA(cudaMemsetAsync(n_kept_dev, 0, sizeof(int64_t), s));
    return LGS_OK;
  }
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  uint32_t* bcount = (uint32_t*)workspace;
  uint64_t* boff = (uint64_t*)((char*)workspace + align256(4 * (size_t)nb));
  keep_count_kernel<<<(unsigned)nb, 256, 0, s>>>(mask, n, bcount);
  keep_scan_kernel<<<1, 1024, 0, s>>>(bcount, nb, boff, n_kept_dev);
  keep_index_kernel<<<(unsigned)nb, 256, 0, s>>>(mask, n, boff, new_index);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

extern "C" lgs_status gs_gather_rows(const void* src, int64_t n, int row_bytes,
                                     const uint32_t* new_index, void* dst, void* stream) {
  clear_error();
  LGS_CHECK_ARG(n >= 0 && n < ((int64_t)1 << 32) - 1, "n out of range");
  LGS_CHECK_ARG(row_bytes > 0 && row_bytes % 2 == 0, "row_bytes must be a positive multiple of 2");
  LGS_CHECK_ARG(n == 0 || (src && dst && new_index), "null pointer");
  const bool wide = row_bytes % 4 == 0;
  LGS_CHECK_ARG(aligned(src, wide ? 4 : 2) && aligned(dst, wide ? 4 : 2), "misaligned rows");
  if (n == 0) return LGS_OK;
  cudaStream_t s = as_stream(stream);
  if (wide) {
    const int words = row_bytes / 4;
    gather_rows_kernel<uint32_t><<<grid_for(n * words, 256), 256, 0, s>>>(
        (const uint32_t*)src, n, words, new_index, (uint32_t*)dst);
  } else {
    const int words = row_bytes / 2;
    gather_rows_kernel<uint16_t><<<grid_for(n * words, 256), 256, 0, s>>>(
        (const uint16_t*)src, n, words, new_index, (uint16_t*)dst);
  }
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
