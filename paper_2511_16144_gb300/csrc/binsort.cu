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
//
// Each radix pass is one kernel ("onesweep"): blocks take tile numbers in
// launch order from an atomic counter, rank their 4096 keys per digit inside
// the block, publish their per-digit counts, and find the counts of all
// earlier tiles by decoupled look-back (walking back over published
// aggregates until an inclusive prefix is found).  One histogram kernel per
// sort gives every pass's global digit offsets.  The instance offsets come
// from a single-pass look-back scan.  Spins are bounded: a wait that gives
// up sets the device error word instead of hanging.
#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

constexpr int kOsThreads = 256;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;  // keys per onesweep tile
// smaller tiles for short key sequences, so that a pass spreads over all SMs
constexpr int kOsItemsSmall = 4;
constexpr int64_t kOsSmallMax = 1 << 20;
constexpr int kRadix = 256;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kValMask = (1u << 30) - 1;
constexpr uint64_t kFlag64Agg = 1ull << 62, kFlag64Inc = 2ull << 62,
                   kVal64Mask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kPassesMax = 8;  // 4 depth + 1 camera + up to 3 tile

__device__ unsigned g_sort_error;  // a look-back gave up

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int64_t item_count(const int64_t* n_dev, int64_t n_host) {
  return n_dev ? *n_dev : n_host;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Sum of the published counts of tiles j, j-1, ... back to (and including)
// the nearest inclusive prefix; `col` points at tile 0's entry and
// consecutive tiles are `stride` words apart.  Loads 16 predecessors per
// round so a long chain of aggregates costs few dependent round trips.
constexpr int kLookAhead = 16;
__device__ __forceinline__ uint32_t look_back(const uint32_t* col, int64_t stride, int64_t j) {
  uint32_t prefix = 0, spins = 0;
  while (j >= 0) {
    uint32_t v[kLookAhead];
#pragma unroll
    for (int q = 0; q < kLookAhead; q++)
      v[q] = (j - q >= 0) ? ld_relaxed(col + (j - q) * stride) : kFlagInc;
    int q = 0;
    bool done = false;
#pragma unroll
    for (int k = 0; k < kLookAhead; k++) {
      if (q == k) {
        const uint32_t flag = v[k] & ~kValMask;
        if (flag != 0) {
          prefix += v[k] & kValMask;
          if (flag == kFlagInc) done = true;
          else q++;
        }
      }
    }
    if (done) break;
    j -= q;
    if (q < kLookAhead && ++spins > kSpinLimit) {  // stalled on an unpublished tile
      atomicOr(&g_sort_error, 1u);
      break;
    }
  }
  return prefix;
}

__device__ __forceinline__ uint64_t look_back64(const uint64_t* col, int64_t j) {
  uint64_t prefix = 0;
  uint32_t spins = 0;
  while (j >= 0) {
    uint64_t v[kLookAhead];
#pragma unroll
    for (int q = 0; q < kLookAhead; q++)
      v[q] = (j - q >= 0) ? ld_relaxed64(col + (j - q)) : kFlag64Inc;
    int q = 0;
    bool done = false;
#pragma unroll
    for (int k = 0; k < kLookAhead; k++) {
      if (q == k) {
        const uint64_t flag = v[k] & ~kVal64Mask;
        if (flag != 0) {
          prefix += v[k] & kVal64Mask;
          if (flag == kFlag64Inc) done = true;
          else q++;
        }
      }
    }
    if (done) break;
    j -= q;
    if (q < kLookAhead && ++spins > kSpinLimit) {
      atomicOr(&g_sort_error, 2u);
      break;
    }
  }
  return prefix;
}

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

// ------------------------------------------------------------------ histogram

struct HistPasses {
  int n;
  int shift[4];
  uint32_t mask[4];
};

// Global digit histograms of up to four passes in one read of the keys.
__global__ void __launch_bounds__(256) hist_kernel(const uint32_t* __restrict__ keys,
                                                   const int64_t* n_dev, int64_t n_host,
                                                   HistPasses hp, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[4][kRadix];
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 4 * kRadix; i += 256) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = item_count(n_dev, n_host);
  const int64_t stride = (int64_t)gridDim.x * 256;
  for (int64_t b = (int64_t)blockIdx.x * 256; b < n; b += stride) {
    const int64_t idx = b + threadIdx.x;
    const bool valid = idx < n;
    const uint32_t k = valid ? keys[idx] : 0u;
    for (int p = 0; p < hp.n; p++) {
      const uint32_t d = valid ? (k >> hp.shift[p]) & hp.mask[p] : (uint32_t)(kRadix + lane);
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < hp.n * kRadix; i += 256) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(ghist + i, c);
  }
}

// Digit histograms of up to four passes of the key sequence produced by a
// kernel, accumulated in that kernel while it writes the keys: every lane of
// the warp calls hist_add the same number of times (valid marks real keys),
// then the block adds its counts to the global histograms.
__device__ __forceinline__ void hist_add(uint32_t (*h)[kRadix], const HistPasses& hp, uint32_t k,
                                         bool valid) {
  const int lane = threadIdx.x & 31;
  for (int p = 0; p < hp.n; p++) {
    const uint32_t d = valid ? (k >> hp.shift[p]) & hp.mask[p] : (uint32_t)(kRadix + lane);
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
  }
}

__device__ __forceinline__ void hist_flush(const uint32_t (*h)[kRadix], const HistPasses& hp,
                                           uint32_t* __restrict__ ghist) {
  __syncthreads();
  for (int i = threadIdx.x; i < hp.n * kRadix; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(ghist + i, c);
  }
}

__device__ __forceinline__ void hist_clear(uint32_t (*h)[kRadix]) {
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
}

static HistPasses hist_passes(int nbits) {
  HistPasses hp{(nbits + 7) / 8, {0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int p = 0; p < hp.n; p++) {
    hp.shift[p] = 8 * p;
    const int bits = nbits - 8 * p < 8 ? nbits - 8 * p : 8;
    hp.mask[p] = (1u << bits) - 1u;
  }
  return hp;
}

// ------------------------------------------------------------------ onesweep pass

template <int ITEMS>
__global__ void __launch_bounds__(kOsThreads)
onesweep_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const int64_t* n_dev,
                int64_t n_host, int shift, uint32_t mask, const uint32_t* __restrict__ ghist,
                uint32_t* status, uint32_t* counter) {
  __shared__ uint32_t wcnt[kOsThreads / 32][kRadix];
  __shared__ uint32_t dstart[kRadix];
  __shared__ uint32_t goff[kRadix];
  __shared__ uint32_t wt[32];
  __shared__ uint32_t sk[(kOsThreads * ITEMS)], sv[(kOsThreads * ITEMS)];
  __shared__ uint32_t s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kOsThreads / 32) * kRadix; i += kOsThreads)
    (&wcnt[0][0])[i] = 0;
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t n = item_count(n_dev, n_host);
  const int64_t blk0 = (int64_t)tile * (kOsThreads * ITEMS);
  if (blk0 >= n) return;
  const int64_t base = blk0 + warp * (32 * ITEMS);
  uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < ITEMS; r++) {  // all loads in flight before any ranking
    const int64_t idx = base + r * 32 + lane;
    key[r] = idx < n ? kin[idx] : 0u;
    val[r] = idx < n ? vin[idx] : 0u;
  }
#pragma unroll
  for (int r = 0; r < ITEMS; r++) {
    const int64_t idx = base + r * 32 + lane;
    const bool valid = idx < n;
    const uint32_t d = valid ? (key[r] >> shift) & mask : (uint32_t)(kRadix + lane);
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t prior = valid ? wcnt[warp][d] : 0u;
    rank[r] = prior + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = prior + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int d = threadIdx.x;  // one digit per thread
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kOsThreads / 32; w++) {
    const uint32_t t = wcnt[w][d];
    wcnt[w][d] = tot;
    tot += t;
  }
  uint32_t all;
  dstart[d] = block_exclusive_scan<uint32_t>(tot, wt, all);
  const uint32_t gbase = block_exclusive_scan<uint32_t>(ghist[d], wt, all);
  // decoupled look-back over the earlier tiles' published counts of digit d
  uint32_t* st = status + (size_t)tile * kRadix;
  uint32_t prefix = 0;
  if (tile == 0) {
    st_relaxed(st + d, tot | kFlagInc);
  } else {
    st_relaxed(st + d, tot | kFlagAgg);
    prefix = look_back(status + d, kRadix, (int64_t)tile - 1);
    st_relaxed(st + d, (prefix + tot) | kFlagInc);
  }
  goff[d] = gbase + prefix;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; r++) {
    const int64_t idx = base + r * 32 + lane;
    if (idx < n) {
      const uint32_t dd = (key[r] >> shift) & mask;
      const uint32_t pos = dstart[dd] + wcnt[warp][dd] + rank[r];
      sk[pos] = key[r];
      sv[pos] = val[r];
    }
  }
  __syncthreads();
  const int m = (int)((n - blk0) < (int64_t)(kOsThreads * ITEMS) ? (n - blk0) : (int64_t)(kOsThreads * ITEMS));
  for (int j = threadIdx.x; j < m; j += kOsThreads) {
    const uint32_t k = sk[j];
    const uint32_t dd = (k >> shift) & mask;
    const uint32_t o = goff[dd] + (uint32_t)j - dstart[dd];
    kout[o] = k;
    vout[o] = sv[j];
  }
}

// ------------------------------------------------------------------ binning kernels

// Depth keys of the (camera, Gaussian) items (all ones when invisible), and
// the digit histograms of the depth sort's passes.
__global__ void __launch_bounds__(256)
depth_keys_kernel(const float4* __restrict__ proj, const ushort4* __restrict__ rect, int64_t m,
                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, HistPasses hp,
                  uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[4][kRadix];
  hist_clear(h);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < m; b += stride) {
    const int64_t i = b + threadIdx.x;
    const bool valid = i < m;
    uint32_t k = 0;
    if (valid) {
      const ushort4 r = rect[i];
      const bool vis = r.z > r.x && r.w > r.y;
      k = vis ? __float_as_uint(proj[2 * i + 1].z) : 0xffffffffu;
      keys[i] = k;
      vals[i] = (uint32_t)i;
    }
    hist_add(h, hp, k, valid);
  }
  hist_flush(h, hp, ghist);
}

__global__ void camera_keys_kernel(const uint32_t* __restrict__ vals, int64_t m, uint32_t n,
                                   uint32_t* __restrict__ keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = vals[i] / n;
}

// Exclusive prefix of the covered-tile counts of the depth-ordered items
// (single pass, decoupled look-back per 4096-item tile); the last tile also
// writes K, and the number to sort (K, or 0 when K exceeds capacity).
constexpr int kEmitSlots = 2048;  // instance slots per emission block

__global__ void __launch_bounds__(256)
count_scan_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect, int64_t m,
                  uint64_t* __restrict__ offs, int64_t capacity, int64_t* __restrict__ k_out,
                  int64_t* __restrict__ sort_n, uint64_t* status, uint32_t* counter,
                  uint32_t* __restrict__ bstart) {
  __shared__ uint64_t wt[32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t blk0 = (int64_t)tile * kOsTile;
  if (blk0 >= m) return;
  const int64_t i0 = blk0 + (int64_t)threadIdx.x * kOsItems;
  uint32_t c[kOsItems];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kOsItems; k++) {
    const int64_t i = i0 + k;
    c[k] = 0;
    if (i < m) {
      const ushort4 r = rect[order[i]];
      if (r.z > r.x && r.w > r.y) c[k] = (uint32_t)(r.z - r.x) * (uint32_t)(r.w - r.y);
    }
    sum += c[k];
  }
  uint64_t total;
  const uint64_t ex = block_exclusive_scan<uint64_t>(sum, wt, total);
  if (threadIdx.x == 0) {
    uint64_t prefix = 0;
    if (tile == 0) {
      st_relaxed64(status, total | kFlag64Inc);
    } else {
      st_relaxed64(status + tile, total | kFlag64Agg);
      prefix = look_back64(status, (int64_t)tile - 1);
      st_relaxed64(status + tile, (prefix + total) | kFlag64Inc);
    }
    s_prefix = prefix;
    if (blk0 + kOsTile >= m) {  // the last tile
      const uint64_t k = prefix + total;
      offs[m] = k;
      *k_out = (int64_t)k;
      *sort_n = (int64_t)k <= capacity ? (int64_t)k : 0;
    }
  }
  __syncthreads();
  uint64_t run = s_prefix + ex;
  const uint64_t nblk = ((uint64_t)capacity + kEmitSlots - 1) / kEmitSlots;
#pragma unroll
  for (int k = 0; k < kOsItems; k++) {
    const int64_t i = i0 + k;
    if (i < m) {
      offs[i] = run;
      // the item holding the first slot of every emission block in its range
      for (uint64_t b = (run + kEmitSlots - 1) / kEmitSlots; b < nblk && b * kEmitSlots < run + c[k];
           b++)
        bstart[b] = (uint32_t)i;
    }
    run += c[k];
  }
}

// One thread per instance slot: slot o belongs to the depth-ordered item i
// with offs[i] <= o < offs[i+1].  The offset scan recorded the item holding
// each block's first slot, so a block knows its bracket of items at once;
// when the bracket spans at most 2049 items (always, unless invisible items
// of one camera sit between) it is staged in shared memory and every thread
// binary-searches it, otherwise threads search the bracket in global memory.
// Writes are coalesced and the work is balanced however many tiles a
// Gaussian covers.
constexpr int kEmitThreads = 256;
constexpr int kEmitPer = kEmitSlots / kEmitThreads;

// Last index i in [lo, hi) with a[i] <= o, given a[lo] <= o < a[hi].
template <typename A>
__device__ __forceinline__ int64_t last_le(const A& a, int64_t lo, int64_t hi, uint64_t o) {
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a(mid) <= o) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
            const uint64_t* __restrict__ offs, const uint32_t* __restrict__ bstart, int64_t m,
            uint32_t n, int tiles_x, uint32_t tiles, uint32_t n_tiles_all,
            const int64_t* __restrict__ sort_n, uint32_t* __restrict__ tkey,
            uint32_t* __restrict__ tval, HistPasses hp, uint32_t* __restrict__ ghist) {
  __shared__ uint64_t s_off[kEmitSlots + 2];
  __shared__ uint32_t hst[4][kRadix];
  const int64_t K = *sort_n;
  const int64_t o0 = (int64_t)blockIdx.x * kEmitSlots;
  if (o0 >= K) return;
  hist_clear(hst);
  const int64_t o1 = o0 + kEmitSlots < K ? o0 + kEmitSlots : K;
  const int64_t lo = bstart[blockIdx.x];
  const int64_t hi = o1 < K ? (int64_t)bstart[blockIdx.x + 1] : m - 1;  // holds slot o1 - 1
  const int64_t span = hi - lo + 1;
  const bool staged = span <= kEmitSlots + 1;
  if (staged)
    for (int64_t j = threadIdx.x; j <= span; j += kEmitThreads) s_off[j] = offs[lo + j];
  __syncthreads();
  auto g = [&](int64_t i) { return offs[i]; };
  auto sm = [&](int64_t i) { return s_off[i]; };
  for (int r = 0; r < kEmitPer; r++) {  // every lane runs every round (histograms)
    const int64_t o = o0 + (int64_t)r * kEmitThreads + threadIdx.x;
    bool valid = o < o1;
    uint32_t key = 0;
    if (valid) {
      const int64_t i = staged ? lo + last_le(sm, 0, span, (uint64_t)o)
                               : last_le(g, lo, hi + 1, (uint64_t)o);
      const uint32_t item = order[i];
      const ushort4 rc = rect[item];
      const uint32_t w = (uint32_t)(rc.z - rc.x), h = (uint32_t)(rc.w - rc.y);
      const uint64_t local = (uint64_t)o - offs[i];
      if (rc.z <= rc.x || rc.w <= rc.y || local >= (uint64_t)w * h) {
        valid = false;  // cannot happen
      } else {
        const uint32_t ty = rc.y + (uint32_t)local / w, tx = rc.x + (uint32_t)local % w;
        const uint32_t c = item / n;
        key = c * tiles + ty * (uint32_t)tiles_x + tx;
        if (key >= n_tiles_all) {
          valid = false;  // cannot happen
        } else {
          tkey[o] = key;
          tval[o] = item - c * n;
        }
      }
    }
    hist_add(hst, hp, key, valid);
  }
  hist_flush(hst, hp, ghist);
}

__global__ void ranges_kernel(const uint32_t* __restrict__ tkey, const int64_t* __restrict__ sort_n,
                              uint32_t n_tiles_all, uint2* __restrict__ ranges) {
  int64_t k = *sort_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t t = tkey[i];
    if (t >= n_tiles_all) continue;
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

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static int64_t tiles_of(int64_t n) { return (n + kOsTile - 1) / kOsTile; }
// keys per onesweep tile for a sort of at most n_max keys, and the tile count
static int os_items(int64_t n_max) { return n_max <= kOsSmallMax ? kOsItemsSmall : kOsItems; }
static int64_t os_tiles(int64_t n_max) {
  const int64_t t = (int64_t)kOsThreads * os_items(n_max);
  return std::max<int64_t>(1, (n_max + t - 1) / t);
}

struct Layout {
  size_t dk0, dk1, dv0, dv1, offs, bstart, tk0, tk1, tv;
  size_t zero_begin, ghist, counters, status[kPassesMax], scan_status, scal, zero_end;
  size_t total;
};

static Layout layout(int64_t n, int n_cams, int64_t capacity) {
  Layout L;
  const int64_t m = (int64_t)n_cams * n;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += align256(bytes); return at; };
  L.dk0 = take(4 * m); L.dk1 = take(4 * m); L.dv0 = take(4 * m); L.dv1 = take(4 * m);
  L.offs = take(8 * (m + 1));
  L.bstart = take(4 * ((capacity + kEmitSlots - 1) / kEmitSlots + 1));
  L.tk0 = take(4 * capacity); L.tk1 = take(4 * capacity); L.tv = take(4 * capacity);
  L.zero_begin = o;
  L.ghist = take(4 * kPassesMax * kRadix);
  L.counters = take(4 * (kPassesMax + 1));
  for (int p = 0; p < kPassesMax; p++)
    L.status[p] = take(4 * (size_t)kRadix * os_tiles(p < 5 ? m : capacity));
  L.scan_status = take(8 * std::max<int64_t>(1, tiles_of(m)));
  L.scal = take(8 * 4);
  L.zero_end = o;
  L.total = o;
  return L;
}

static int grid_for(int64_t m) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 152 * 16));
}

// Stable LSD sort of (key, val) on key bits [0, nbits) with onesweep passes
// of <= 8 bits.  ghist: 4 x kRadix digit counts, counters: one tile counter
// per pass, status[p]: kRadix look-back words per tile of pass p; all zeroed
// by the caller.  Returns true when the result ended in (k1, v1).
static bool onesweep_passes(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                            const int64_t* n_dev, int64_t n_max, int nbits, uint32_t* ghist,
                            uint32_t* counters, uint32_t* const* status, cudaStream_t s,
                            bool hist_done = false) {
  const int npass = (nbits + 7) / 8;
  const HistPasses hp = hist_passes(nbits);
  const int64_t ntile = os_tiles(n_max);
  if (!hist_done)  // else the producer of the keys has filled ghist
    hist_kernel<<<(unsigned)std::min<int64_t>(ntile * 2, 152 * 4), 256, 0, s>>>(k0, n_dev, n_max,
                                                                             hp, ghist);
  const bool small = os_items(n_max) == kOsItemsSmall;
  bool flipped = false;
  for (int p = 0; p < npass; p++) {
    if (small)
      onesweep_kernel<kOsItemsSmall><<<(unsigned)ntile, kOsThreads, 0, s>>>(
          k0, v0, k1, v1, n_dev, n_max, hp.shift[p], hp.mask[p], ghist + p * kRadix, status[p],
          counters + p);
    else
      onesweep_kernel<kOsItems><<<(unsigned)ntile, kOsThreads, 0, s>>>(
          k0, v0, k1, v1, n_dev, n_max, hp.shift[p], hp.mask[p], ghist + p * kRadix, status[p],
          counters + p);
    std::swap(k0, k1);
    std::swap(v0, v1);
    flipped = !flipped;
  }
  return flipped;
}

static bool onesweep_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                          const int64_t* n_dev, int64_t n_max, int nbits, int pass0,
                          const Layout& L, char* ws, cudaStream_t s, bool hist_done = false) {
  uint32_t* status[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int p = 0; p < 4 && pass0 + p < kPassesMax; p++)
    status[p] = (uint32_t*)(ws + L.status[pass0 + p]);
  return onesweep_passes(k0, v0, k1, v1, n_dev, n_max, nbits,
                         (uint32_t*)(ws + L.ghist) + pass0 * kRadix,
                         (uint32_t*)(ws + L.counters) + pass0, status, s, hist_done);
}

size_t sort_pairs_scratch(int64_t n) {
  const size_t per = align256(4 * (size_t)kRadix * os_tiles(n));
  return align256(4 * 4 * kRadix) + align256(4 * 4) + 4 * per;
}

bool sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int nbits,
                void* scratch, cudaStream_t s) {
  char* ws = (char*)scratch;
  const size_t per = align256(4 * (size_t)kRadix * os_tiles(n));
  uint32_t* ghist = (uint32_t*)ws;
  uint32_t* counters = (uint32_t*)(ws + align256(4 * 4 * kRadix));
  char* st0 = ws + align256(4 * 4 * kRadix) + align256(4 * 4);
  uint32_t* status[4];
  for (int p = 0; p < 4; p++) status[p] = (uint32_t*)(st0 + p * per);
  cudaMemsetAsync(scratch, 0, sort_pairs_scratch(n), s);
  if (n == 0 || nbits < 1) return false;
  return onesweep_passes(k0, v0, k1, v1, nullptr, n, std::min(nbits, 32), ghist, counters, status,
                         s);
}

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
  LGS_CHECK_ARG(capacity >= 0 && capacity < ((int64_t)1 << 30), "capacity out of range");
  LGS_CHECK_ARG((int64_t)n_cams * n < ((int64_t)1 << 30), "n_cams * n out of range");
  LGS_CHECK_ARG(ranges && n_instances_dev && workspace, "null pointer");
  LGS_CHECK_ARG(n == 0 || (proj && rect), "null pointer");
  LGS_CHECK_ARG(capacity == 0 || ids, "ids is null");
  LGS_CHECK_ARG(aligned(workspace, 256), "workspace must be 256-byte aligned");
  LGS_CHECK_ARG(n == 0 || (aligned(proj, 16) && aligned(rect, 8)), "misaligned pointer");
  const int64_t m = (int64_t)n_cams * n;
  const uint32_t tiles = (uint32_t)tiles_x * (uint32_t)tiles_y;
  // the tile sort has at most three 8-bit passes
  LGS_CHECK_ARG((uint64_t)tiles * (uint64_t)n_cams <= (1ull << 24), "too many tiles");
  Layout L = layout(n, n_cams, capacity);
  LGS_CHECK_ARG(workspace_bytes >= L.total, "workspace too small");
  cudaStream_t s = as_stream(stream);
  char* ws = (char*)workspace;
  auto U32 = [&](size_t off) { return (uint32_t*)(ws + off); };
  int64_t* sort_n = (int64_t*)(ws + L.scal);

  LGS_CHECK_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_cams * tiles, s));
  if (m == 0) {
    LGS_CHECK_CUDA(cudaMemsetAsync(n_instances_dev, 0, sizeof(int64_t), s));
    return LGS_OK;
  }
  LGS_CHECK_CUDA(cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_end - L.zero_begin, s));
  // 1. (camera, Gaussian) items by depth, then stably by camera
  uint32_t *dk0 = U32(L.dk0), *dk1 = U32(L.dk1), *dv0 = U32(L.dv0), *dv1 = U32(L.dv1);
  depth_keys_kernel<<<grid_for(m), 256, 0, s>>>((const float4*)proj, (const ushort4*)rect, m,
                                                dk0, dv0, hist_passes(32), U32(L.ghist));
  if (onesweep_sort(dk0, dv0, dk1, dv1, nullptr, m, 32, 0, L, ws, s, true)) {
    std::swap(dk0, dk1);
    std::swap(dv0, dv1);
  }
  if (n_cams > 1) {
    camera_keys_kernel<<<grid_for(m), 256, 0, s>>>(dv0, m, (uint32_t)n, dk0);
    const int cbits = 32 - __builtin_clz((unsigned)(n_cams - 1));
    if (onesweep_sort(dk0, dv0, dk1, dv1, nullptr, m, cbits, 4, L, ws, s)) {
      std::swap(dk0, dk1);
      std::swap(dv0, dv1);
    }
  }
  const uint32_t* order = dv0;
  // 2. instance offsets of the depth-ordered items, K and the sort count
  uint64_t* offs = (uint64_t*)(ws + L.offs);
  count_scan_kernel<<<(unsigned)std::max<int64_t>(1, tiles_of(m)), 256, 0, s>>>(
      order, (const ushort4*)rect, m, offs, capacity, n_instances_dev, sort_n,
      (uint64_t*)(ws + L.scan_status), U32(L.counters) + kPassesMax, U32(L.bstart));
  LGS_CHECK_LAUNCH();
  if (capacity == 0) return LGS_OK;
  // 3. emit (tile, Gaussian) pairs and sort them stably by tile
  int tbits = 1;
  while (tbits < 32 && ((uint64_t)1 << tbits) < (uint64_t)n_cams * tiles) tbits++;
  const bool odd = ((tbits + 7) / 8) & 1;
  uint32_t *tk0 = U32(L.tk0), *tk1 = U32(L.tk1);
  uint32_t* tv0 = odd ? U32(L.tv) : ids;  // the last pass lands in ids
  uint32_t* tv1 = odd ? ids : U32(L.tv);
  emit_kernel<<<(unsigned)std::max<int64_t>(1, (capacity + kEmitSlots - 1) / kEmitSlots),
                kEmitThreads, 0, s>>>(order, (const ushort4*)rect, offs, U32(L.bstart), m,
                                      (uint32_t)n, tiles_x, tiles, (uint32_t)n_cams * tiles,
                                      sort_n, tk0, tv0, hist_passes(tbits),
                                      U32(L.ghist) + 5 * kRadix);
  const bool flipped =
      onesweep_sort(tk0, tv0, tk1, tv1, sort_n, capacity, tbits, 5, L, ws, s, true);
  const uint32_t* tkey = flipped ? tk1 : tk0;
  // 4. per-tile ranges and (optionally) the 64-bit keys
  ranges_kernel<<<grid_for(capacity), 256, 0, s>>>(tkey, sort_n, (uint32_t)n_cams * tiles,
                                                    (uint2*)ranges);
  if (keys_opt)
    keys_kernel<<<grid_for(capacity), 256, 0, s>>>(tkey, ids, (const float4*)proj, sort_n,
                                                   (uint32_t)n, tiles, keys_opt);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

namespace lgs {
unsigned sort_error_word() {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_sort_error, sizeof(v)) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_sort_error, &zero, sizeof(zero));
  return v;
}
}  // namespace lgs
