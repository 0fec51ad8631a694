// Stable LSD radix sort of (key, value) pairs: the cell sort of the pruning
// neighbour grid.
//
// Each pass of up to 8 bits is one kernel ("onesweep"): blocks take tile
// numbers in launch order from an atomic counter, rank their keys per digit
// inside the block, publish their per-digit counts, and find the counts of
// all earlier tiles by decoupled look-back (walking back over published
// aggregates until an inclusive prefix is found).  One histogram kernel per
// sort gives every pass's global digit offsets.  Spins are bounded: a wait
// that gives up sets the device error word instead of hanging, and the block
// goes on with the counts it has, which are never more than the true prefix,
// so every store stays in bounds (a later pass that reads the resulting
// unordered keys guards its stores the same way).
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

constexpr int kOsThreads = 256;
constexpr int kOsItems = 16;
// smaller tiles for short key sequences, so that a pass spreads over all SMs
constexpr int kOsItemsSmall = 4;
constexpr int64_t kOsSmallMax = 1 << 20;
constexpr int kRadix = 256;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kValMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;  // default polling rounds before a look-back gives up
static std::atomic<uint32_t> g_spin_limit{kSpinLimit};  // lgs_set_sort_wait_limit

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
// Sum of the published counts of tiles j, j-1, ... back to (and including)
// the nearest inclusive prefix; `col` points at tile 0's entry and
// consecutive tiles are `stride` words apart.  Loads 16 predecessors per
// round so a long chain of aggregates costs few dependent round trips.
constexpr int kLookAhead = 16;
__device__ __forceinline__ uint32_t look_back(const uint32_t* col, int64_t stride, int64_t j,
                                              uint32_t spin_limit) {
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
    if (q < kLookAhead && ++spins > spin_limit) {  // stalled on an unpublished tile
      atomicOr(&g_sort_error, 1u);
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
                uint32_t* status, uint32_t* counter, uint32_t spin_limit) {
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
    prefix = look_back(status + d, kRadix, (int64_t)tile - 1, spin_limit);
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
    if (o < n) {  // always, unless an earlier look-back gave up (keys then unordered)
      kout[o] = k;
      vout[o] = sv[j];
    }
  }
}

// ------------------------------------------------------------------ workspace

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// keys per onesweep tile for a sort of at most n_max keys, and the tile count
static int os_items(int64_t n_max) { return n_max <= kOsSmallMax ? kOsItemsSmall : kOsItems; }
static int64_t os_tiles(int64_t n_max) {
  const int64_t t = (int64_t)kOsThreads * os_items(n_max);
  return std::max<int64_t>(1, (n_max + t - 1) / t);
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
  const uint32_t spin = g_spin_limit.load(std::memory_order_relaxed);
  bool flipped = false;
  for (int p = 0; p < npass; p++) {
    if (small)
      onesweep_kernel<kOsItemsSmall><<<(unsigned)ntile, kOsThreads, 0, s>>>(
          k0, v0, k1, v1, n_dev, n_max, hp.shift[p], hp.mask[p], ghist + p * kRadix, status[p],
          counters + p, spin);
    else
      onesweep_kernel<kOsItems><<<(unsigned)ntile, kOsThreads, 0, s>>>(
          k0, v0, k1, v1, n_dev, n_max, hp.shift[p], hp.mask[p], ghist + p * kRadix, status[p],
          counters + p, spin);
    std::swap(k0, k1);
    std::swap(v0, v1);
    flipped = !flipped;
  }
  return flipped;
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

namespace lgs {
unsigned sort_error_word(bool clear) {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_sort_error, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) cudaMemcpyToSymbol(g_sort_error, &zero, sizeof(zero));
  return v;
}
}  // namespace lgs

extern "C" void lgs_set_sort_wait_limit(int64_t polls) {
  const uint32_t v = polls <= 0 ? lgs::kSpinLimit
                                : (uint32_t)std::min<int64_t>(polls, (int64_t)0xffffffff);
  lgs::g_spin_limit.store(v, std::memory_order_relaxed);
}
