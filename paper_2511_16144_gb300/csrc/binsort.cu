// 16x16 tile binning with a depth-keyed stable LSD radix sort.
//
// The ordering is the one front-to-back alpha compositing (LEGO-SLAM
// Sec. III-B.1, standard 3DGS pipeline) needs inside every tile: instances
// keyed by (camera, tile, float depth bits), ties by Gaussian index.
//
// Instead of sorting 64-bit keys over all instances, the sort is split in
// two stable stages that give the same total order with less traffic:
//   1. sort the n_cams * n (camera, Gaussian) items by depth bits (4 passes
//      of 8 bits over C*N items), then stably by camera (one pass if C > 1);
//   2. emit one (camera*tiles + tile, Gaussian) pair per covered tile in that
//      order and stably sort the pairs by tile (ceil(log2(C*tiles)) bits,
//      at most 8 per pass).
// Stability makes equal tiles keep depth order and equal depths keep index
// order, which is exactly a stable sort of the 64-bit keys.
#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // items per block and pass
constexpr int kRadix = 256;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int64_t item_count(const int64_t* n_dev, int64_t n_host) {
  return n_dev ? *n_dev : n_host;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum in three launches: per-chunk sums, a one-block scan of
// those sums, and a per-chunk rescan with the carried offset.

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = w;
  }
  __syncthreads();
  T before = warp > 0 ? warp_tot[warp - 1] : T(0);
  total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

template <typename Tin, typename Tout>
__global__ void scan_reduce_kernel(const Tin* __restrict__ in, int64_t n, Tout* __restrict__ part) {
  __shared__ Tout wt[32];
  int64_t base = (int64_t)blockIdx.x * kScanChunk;
  Tout s = 0;
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += (Tout)in[i];
  }
  Tout tot;
  block_exclusive_scan<Tout>(s, wt, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_partials_kernel(T* __restrict__ part, int64_t nb, T* __restrict__ total_out) {
  __shared__ T wt[32];
  T carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    int64_t i = b0 + threadIdx.x;
    T v = i < nb ? part[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(v, wt, tot);
    if (i < nb) part[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <typename Tin, typename Tout>
__global__ void scan_apply_kernel(const Tin* in, Tout* out, int64_t n,
                                  const Tout* __restrict__ part) {
  __shared__ Tout buf[kScanChunk];
  __shared__ Tout wt[32];
  int64_t base = (int64_t)blockIdx.x * kScanChunk;
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    buf[k * kScanThreads + threadIdx.x] = i < n ? (Tout)in[i] : Tout(0);
  }
  __syncthreads();
  Tout loc[kScanItems];
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    loc[k] = s;
    s += buf[threadIdx.x * kScanItems + k];
  }
  Tout tot;
  Tout ex = block_exclusive_scan<Tout>(s, wt, tot) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) buf[threadIdx.x * kScanItems + k] = ex + loc[k];
  __syncthreads();
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) out[i] = buf[k * kScanThreads + threadIdx.x];
  }
}

template <typename Tin, typename Tout>
static void exclusive_scan(const Tin* in, Tout* out, int64_t n, Tout* part, Tout* total,
                           cudaStream_t s) {
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  if (nb == 0) nb = 1;
  scan_reduce_kernel<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part);
  scan_partials_kernel<Tout><<<1, 1024, 0, s>>>(part, nb, total);
  scan_apply_kernel<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part);
}

static int64_t scan_partials_len(int64_t n) { return (n + kScanChunk - 1) / kScanChunk + 1; }

// ------------------------------------------------------------------ radix pass
// Per pass: per-block digit histograms (digit-major, so one exclusive scan
// gives every block's output offset per digit), then a stable scatter that
// ranks keys inside each warp with match_any, orders them by digit in shared
// memory and writes each digit's run contiguously.

__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint32_t* __restrict__ keys, const int64_t* n_dev, int64_t n_host,
                  int shift, uint32_t mask, uint32_t* __restrict__ counts, int nblocks) {
  __shared__ uint32_t h[kSortThreads / 32][kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += kSortThreads)
    (&h[0][0])[i] = 0;
  __syncthreads();
  int64_t n = item_count(n_dev, n_host);
  int64_t base = (int64_t)blockIdx.x * kSortTile + warp * (32 * kSortItems);
#pragma unroll
  for (int r = 0; r < kSortItems; r++) {
    int64_t idx = base + r * 32 + lane;
    bool valid = idx < n;
    uint32_t d = valid ? (keys[idx] >> shift) & mask : (uint32_t)(kRadix + lane);
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == __ffs(peers) - 1) h[warp][d] += __popc(peers);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; w++) s += h[w][d];
    counts[(int64_t)d * nblocks + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                     uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                     const int64_t* n_dev, int64_t n_host, int shift, uint32_t mask,
                     const uint32_t* __restrict__ offsets, int nblocks) {
  __shared__ uint32_t wcnt[kSortThreads / 32][kRadix];
  __shared__ uint32_t dstart[kRadix];
  __shared__ uint32_t wt[32];
  __shared__ uint32_t sk[kSortTile], sv[kSortTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += kSortThreads)
    (&wcnt[0][0])[i] = 0;
  __syncthreads();
  int64_t n = item_count(n_dev, n_host);
  int64_t blk0 = (int64_t)blockIdx.x * kSortTile;
  if (blk0 >= n) return;
  int64_t base = blk0 + warp * (32 * kSortItems);
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kSortItems; r++) {
    int64_t idx = base + r * 32 + lane;
    bool valid = idx < n;
    key[r] = valid ? kin[idx] : 0u;
    val[r] = valid ? vin[idx] : 0u;
    uint32_t d = valid ? (key[r] >> shift) & mask : (uint32_t)(kRadix + lane);
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t prior = valid ? wcnt[warp][d] : 0u;
    rank[r] = prior + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = prior + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive offsets across warps, then across digits
  uint32_t tot = 0;
  if (threadIdx.x < kRadix) {
    int d = threadIdx.x;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; w++) {
      uint32_t t = wcnt[w][d];
      wcnt[w][d] = tot;
      tot += t;
    }
  }
  uint32_t all;
  uint32_t ex = block_exclusive_scan<uint32_t>(tot, wt, all);
  if (threadIdx.x < kRadix) dstart[threadIdx.x] = ex;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; r++) {
    int64_t idx = base + r * 32 + lane;
    if (idx < n) {
      uint32_t d = (key[r] >> shift) & mask;
      uint32_t pos = dstart[d] + wcnt[warp][d] + rank[r];
      sk[pos] = key[r];
      sv[pos] = val[r];
    }
  }
  __syncthreads();
  int m = (int)((n - blk0) < (int64_t)kSortTile ? (n - blk0) : (int64_t)kSortTile);
  for (int j = threadIdx.x; j < m; j += kSortThreads) {
    uint32_t k = sk[j];
    uint32_t d = (k >> shift) & mask;
    uint32_t o = offsets[(int64_t)d * nblocks + blockIdx.x] + (uint32_t)j - dstart[d];
    kout[o] = k;
    vout[o] = sv[j];
  }
}

struct SortBufs {
  uint32_t* counts;   // [kRadix * nblocks]
  uint32_t* part;     // scan partials
};

// Stable LSD sort of (key, val) pairs on bits [0, nbits); ping-pongs between
// (k0, v0) and (k1, v1).  Returns true when the result ended in (k1, v1).
static bool radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                       const int64_t* n_dev, int64_t n_max, int nbits, const SortBufs& b,
                       cudaStream_t s) {
  int nblocks = (int)((n_max + kSortTile - 1) / kSortTile);
  if (nblocks == 0) return false;
  bool flipped = false;
  for (int shift = 0; shift < nbits; shift += 8) {
    int bits = std::min(8, nbits - shift);
    uint32_t mask = (1u << bits) - 1u;
    radix_hist_kernel<<<nblocks, kSortThreads, 0, s>>>(k0, n_dev, n_max, shift, mask, b.counts,
                                                       nblocks);
    exclusive_scan<uint32_t, uint32_t>(b.counts, b.counts, (int64_t)kRadix * nblocks, b.part,
                                       (uint32_t*)nullptr, s);
    radix_scatter_kernel<<<nblocks, kSortThreads, 0, s>>>(k0, v0, k1, v1, n_dev, n_max, shift,
                                                          mask, b.counts, nblocks);
    std::swap(k0, k1);
    std::swap(v0, v1);
    flipped = !flipped;
  }
  return flipped;
}

static int sort_passes(int nbits) { return (nbits + 7) / 8; }

// ------------------------------------------------------------------ binning kernels

__global__ void depth_keys_kernel(const float4* __restrict__ proj, const ushort4* __restrict__ rect,
                                  int64_t m, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    ushort4 r = rect[i];
    bool vis = r.z > r.x && r.w > r.y;
    keys[i] = vis ? __float_as_uint(proj[2 * i + 1].z) : 0xffffffffu;
    vals[i] = (uint32_t)i;
  }
}

__global__ void camera_keys_kernel(const uint32_t* __restrict__ vals, int64_t m, uint32_t n,
                                   uint32_t* __restrict__ keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = vals[i] / n;
}

__global__ void tile_count_kernel(const uint32_t* __restrict__ order,
                                  const ushort4* __restrict__ rect, int64_t m,
                                  uint32_t* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    ushort4 r = rect[order[i]];
    cnt[i] = (r.z > r.x && r.w > r.y) ? (uint32_t)(r.z - r.x) * (uint32_t)(r.w - r.y) : 0u;
  }
}

// K and the number of instances to sort (K, or 0 when K exceeds capacity).
__global__ void finish_count_kernel(const uint64_t* __restrict__ total, int64_t capacity,
                                    int64_t* __restrict__ k_out, int64_t* __restrict__ sort_n) {
  uint64_t k = *total;
  *k_out = (int64_t)k;
  *sort_n = (int64_t)k <= capacity ? (int64_t)k : 0;
}

__global__ void emit_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
                            const uint64_t* __restrict__ offs, int64_t m, uint32_t n,
                            int tiles_x, uint32_t tiles, const int64_t* __restrict__ sort_n,
                            uint32_t* __restrict__ tkey, uint32_t* __restrict__ tval) {
  if (*sort_n == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t item = order[i];
    ushort4 r = rect[item];
    if (!(r.z > r.x && r.w > r.y)) continue;
    uint32_t c = item / n, g = item - c * n;
    uint64_t o = offs[i];
    for (int ty = r.y; ty < r.w; ty++)
      for (int tx = r.x; tx < r.z; tx++) {
        tkey[o] = c * tiles + (uint32_t)(ty * tiles_x + tx);
        tval[o] = g;
        o++;
      }
  }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ tkey, const int64_t* __restrict__ sort_n,
                              uint2* __restrict__ ranges) {
  int64_t k = *sort_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t t = tkey[i];
    if (i == 0 || tkey[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == k - 1 || tkey[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

__global__ void keys_kernel(const uint32_t* __restrict__ tkey, const uint32_t* __restrict__ ids,
                            const float4* __restrict__ proj, const int64_t* __restrict__ sort_n,
                            uint32_t n, uint32_t tiles, uint64_t* __restrict__ keys) {
  int64_t k = *sort_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t t = tkey[i];
    uint32_t c = t / tiles;
    float z = proj[2 * ((int64_t)c * n + ids[i]) + 1].z;
    keys[i] = ((uint64_t)t << 32) | __float_as_uint(z);
  }
}

// ------------------------------------------------------------------ workspace

struct Layout {
  size_t dk0, dk1, dv0, dv1, cnt, offs, tk0, tk1, tv, counts, part, part64, scal, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout layout(int64_t n, int n_cams, int64_t capacity) {
  Layout L;
  int64_t m = (int64_t)n_cams * n;
  int64_t nmax = std::max<int64_t>(m, capacity);
  int64_t nblocks = (nmax + kSortTile - 1) / kSortTile;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += align256(bytes); return at; };
  L.dk0 = take(4 * m); L.dk1 = take(4 * m); L.dv0 = take(4 * m); L.dv1 = take(4 * m);
  L.cnt = take(4 * m);
  L.offs = take(8 * (m + 1));
  L.tk0 = take(4 * capacity); L.tk1 = take(4 * capacity); L.tv = take(4 * capacity);
  L.counts = take(4 * (size_t)kRadix * std::max<int64_t>(nblocks, 1));
  L.part = take(4 * scan_partials_len((int64_t)kRadix * std::max<int64_t>(nblocks, 1)));
  L.part64 = take(8 * scan_partials_len(m + 1));
  L.scal = take(8 * 4);
  L.total = o;
  return L;
}

static int grid_for(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 152 * 16)); }

}  // namespace lgs

using namespace lgs;

extern "C" size_t gs_bin_sort_workspace(int64_t n, int n_cams, int tiles_x, int tiles_y,
                                        int64_t capacity) {
  (void)tiles_x;
  (void)tiles_y;
  if (n < 0 || n_cams < 1 || capacity < 0) return 0;
  return layout(n, n_cams, capacity).total;
}

extern "C" lgs_status gs_bin_sort(const float* proj, const uint16_t* rect, int64_t n, int n_cams,
                                  int tiles_x, int tiles_y, int64_t capacity, uint32_t* ids,
                                  uint32_t* ranges, uint64_t* keys_opt, int64_t* n_instances_dev,
                                  void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  LGS_CHECK_ARG(n >= 0 && n < ((int64_t)1 << 31), "n out of range");
  LGS_CHECK_ARG(n_cams >= 1 && n_cams <= LGS_MAX_CAMS, "n_cams out of range");
  LGS_CHECK_ARG(tiles_x >= 1 && tiles_y >= 1 && tiles_x <= 65535 && tiles_y <= 65535,
                "bad tile grid");
  LGS_CHECK_ARG(capacity >= 0 && capacity < ((int64_t)1 << 32), "capacity out of range");
  LGS_CHECK_ARG(ranges && n_instances_dev && workspace, "null pointer");
  LGS_CHECK_ARG(n == 0 || (proj && rect), "null pointer");
  LGS_CHECK_ARG(capacity == 0 || ids, "ids is null");
  LGS_CHECK_ARG(aligned(workspace, 256), "workspace must be 256-byte aligned");
  LGS_CHECK_ARG(n == 0 || (aligned(proj, 16) && aligned(rect, 8)), "misaligned pointer");
  const int64_t m = (int64_t)n_cams * n;
  const uint32_t tiles = (uint32_t)tiles_x * (uint32_t)tiles_y;
  LGS_CHECK_ARG((uint64_t)tiles * (uint64_t)n_cams < (1ull << 32), "too many tiles");
  Layout L = layout(n, n_cams, capacity);
  LGS_CHECK_ARG(workspace_bytes >= L.total, "workspace too small");
  cudaStream_t s = as_stream(stream);
  char* ws = (char*)workspace;
  auto U32 = [&](size_t off) { return (uint32_t*)(ws + off); };
  int64_t* scal = (int64_t*)(ws + L.scal);
  int64_t* sort_n = scal;
  SortBufs sb{U32(L.counts), U32(L.part)};

  LGS_CHECK_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_cams * tiles, s));
  if (m == 0) {
    LGS_CHECK_CUDA(cudaMemsetAsync(n_instances_dev, 0, sizeof(int64_t), s));
    return LGS_OK;
  }
  // 1. (camera, Gaussian) items by depth, then stably by camera
  uint32_t *dk0 = U32(L.dk0), *dk1 = U32(L.dk1), *dv0 = U32(L.dv0), *dv1 = U32(L.dv1);
  depth_keys_kernel<<<grid_for(m), 256, 0, s>>>((const float4*)proj, (const ushort4*)rect, m,
                                                dk0, dv0);
  if (radix_sort(dk0, dv0, dk1, dv1, nullptr, m, 32, sb, s)) {
    std::swap(dk0, dk1);
    std::swap(dv0, dv1);
  }
  if (n_cams > 1) {
    camera_keys_kernel<<<grid_for(m), 256, 0, s>>>(dv0, m, (uint32_t)n, dk0);
    int cbits = 32 - __builtin_clz((unsigned)(n_cams - 1));
    if (radix_sort(dk0, dv0, dk1, dv1, nullptr, m, cbits, sb, s)) {
      std::swap(dk0, dk1);
      std::swap(dv0, dv1);
    }
  }
  const uint32_t* order = dv0;
  // 2. instance counts and offsets
  uint32_t* cnt = U32(L.cnt);
  uint64_t* offs = (uint64_t*)(ws + L.offs);
  tile_count_kernel<<<grid_for(m), 256, 0, s>>>(order, (const ushort4*)rect, m, cnt);
  exclusive_scan<uint32_t, uint64_t>(cnt, offs, m, (uint64_t*)(ws + L.part64), offs + m, s);
  finish_count_kernel<<<1, 1, 0, s>>>(offs + m, capacity, n_instances_dev, sort_n);
  LGS_CHECK_LAUNCH();
  if (capacity == 0) return LGS_OK;
  // 3. emit (tile, Gaussian) pairs and sort them stably by tile
  int tbits = 1;
  while (tbits < 32 && ((uint64_t)1 << tbits) < (uint64_t)n_cams * tiles) tbits++;
  bool odd = sort_passes(tbits) & 1;
  uint32_t *tk0 = U32(L.tk0), *tk1 = U32(L.tk1);
  uint32_t* tv0 = odd ? U32(L.tv) : ids;   // the last pass lands in ids
  uint32_t* tv1 = odd ? ids : U32(L.tv);
  emit_kernel<<<grid_for(m), 256, 0, s>>>(order, (const ushort4*)rect, offs, m, (uint32_t)n,
                                          tiles_x, tiles, sort_n, tk0, tv0);
  bool flipped = radix_sort(tk0, tv0, tk1, tv1, sort_n, capacity, tbits, sb, s);
  const uint32_t* tkey = flipped ? tk1 : tk0;
  // 4. per-tile ranges and (optionally) the 64-bit keys
  ranges_kernel<<<grid_for(capacity), 256, 0, s>>>(tkey, sort_n, (uint2*)ranges);
  if (keys_opt)
    keys_kernel<<<grid_for(capacity), 256, 0, s>>>(tkey, ids, (const float4*)proj, sort_n,
                                                   (uint32_t)n, tiles, keys_opt);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
