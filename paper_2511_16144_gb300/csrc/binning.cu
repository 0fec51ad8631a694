// 16x16 tile binning: every (camera, Gaussian) item emits one instance per
// tile of its support rect that its ellipse q(d) <= cut reaches (tile_hit),
// and each tile's instances are ordered by
// depth, ties by Gaussian index -- the front-to-back order alpha compositing
// needs (LEGO-SLAM Sec. III-B.1, the standard 3DGS pipeline).  The result is
// the same as a stable sort of the keys ((camera * tiles + tile) << 32) |
// bits(depth) in emission order.
//
// Because every tile's segment can be sorted on its own, there is no global
// sort:
//   1. count the instances of every tile (shared-memory histograms per
//      block of contiguous items when a camera's tiles fit, else global
//      atomics) and the total K, keeping for every rect of at most 32 tiles
//      the mask of the tiles it hits;
//   2. one block scans the counts into segment starts, writes the ranges and
//      the write cursors (all ranges stay (0, 0) when K > capacity);
//   3. every item appends (depth bits, index) to each of its tiles' segments
//      (a block reserves one range per tile, then fills it with shared-
//      memory atomics; the order inside a segment is arbitrary), the small
//      rects from their masks;
//   Both passes spread the (item, tile) pairs of each group of 256 items
//   evenly over the block's threads.
//   4. one block per tile sorts its segment's 64-bit (depth bits, index)
//      keys with a stable LSD radix sort in shared memory and writes the
//      Gaussian indices: 256-thread blocks with eight keys a thread take the
//      segments of up to 2,048 keys (48 registers, five blocks per SM), with
//      sixteen keys a thread those of up to 4,096, 1024-thread blocks the
//      longer ones (listed by step 2) up to 12,288 keys, and chunk by chunk
//      from global memory beyond.
// Depths are positive floats, so their bit patterns order like the values.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace lgs {

// Largest instance count a call needed beyond its capacity (LGS_ERR_CAPACITY
// of lgs_sync_status); 0 = none.
__device__ unsigned long long g_capacity_k;

namespace {

constexpr int kSegSmall = 2048;        // keys a 256-thread block sorts with 8 keys a thread
constexpr int kSegMax = 4096;          // keys a 256-thread block sorts in shared memory
constexpr int kSegThreads = 256;
constexpr int kLargeThreads = 1024;    // blocks for the longer segments
constexpr int kLargeItems = 12;        // keys per thread: 12,288 in shared memory
constexpr int kLargeBlocks = 2 * 152;  // persistent grid over the list of long segments
constexpr int kSmemTiles = 32768;      // per-block tile tables (4 B each) up to this many tiles
constexpr int kItemThreads = 256;      // threads (and items per group) of the count and emit passes
constexpr int kItemBlocks = 4 * 152;   // blocks of the count and emit passes
constexpr int kMaskTiles = 32;         // rects of at most this many tiles keep a hit mask
constexpr int kScanThreads = 1024;

__device__ __forceinline__ bool rect_empty(const ushort4& r) { return r.z <= r.x || r.w <= r.y; }

// The ellipse of a visible projected record as the tile test reads it: mean,
// conic (a, b, c), the reciprocals of a and c (IEEE, once per record), the
// cutoff, and the depth (the emitted key).  r0 = (u, v, a, b), r1 = (c, o,
// tz, cut); a, c > 0.
struct Ell {
  float u, v, a, b, c, ia, ic, cut, tz;
};
__device__ __forceinline__ Ell ell_of(const float4& r0, const float4& r1) {
  return Ell{r0.x, r0.y, r0.z, r0.w, r1.x, __frcp_rn(r0.z), __frcp_rn(r1.x), r1.w, r1.z};
}

// Whether the ellipse q(d) = a dx^2 + 2 b dx dy + c dy^2 <= cut, d = (u - x,
// v - y), meets the pixel-centre square [16 tx + 0.5, 16 tx + 15.5] x
// [16 ty + 0.5, 16 ty + 15.5] of tile (tx, ty): zero if the mean is inside,
// else the smallest q over the four edges, each a 1-D quadratic whose
// minimiser (-b X / c on an edge dx = X, -b Y / a on an edge dy = Y, taken
// as a product with the reciprocal) is clamped to the edge.  FP32 with a
// fixed order of round-to-nearest operations (no contraction), so the
// oracle takes the same decision bit for bit.
__device__ __forceinline__ bool tile_hit(const Ell& E, uint32_t tx, uint32_t ty) {
  const float xa = (float)(16u * tx) + 0.5f, xb = (float)(16u * tx) + 15.5f;
  const float ya = (float)(16u * ty) + 0.5f, yb = (float)(16u * ty) + 15.5f;
  const float dx0 = __fsub_rn(E.u, xb), dx1 = __fsub_rn(E.u, xa);
  const float dy0 = __fsub_rn(E.v, yb), dy1 = __fsub_rn(E.v, ya);
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
  const float b2 = __fmul_rn(2.f, E.b);
  auto q = [&](float X, float Y) {
    return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(E.a, X), X), __fmul_rn(__fmul_rn(b2, X), Y)),
                     __fmul_rn(__fmul_rn(E.c, Y), Y));
  };
  float best = INFINITY;
#pragma unroll
  for (int e = 0; e < 2; e++) {
    const float X = e ? dx1 : dx0;
    const float Y = fminf(fmaxf(__fmul_rn(-__fmul_rn(E.b, X), E.ic), dy0), dy1);
    best = fminf(best, q(X, Y));
  }
#pragma unroll
  for (int e = 0; e < 2; e++) {
    const float Y = e ? dy1 : dy0;
    const float X = fminf(fmaxf(__fmul_rn(-__fmul_rn(E.b, Y), E.ia), dx0), dx1);
    best = fminf(best, q(X, Y));
  }
  return best <= E.cut;
}

// One group of kItemThreads consecutive items staged in shared memory for
// the block-wide pair expansion: each item's ellipse record, rect origin and
// width in tiles, rect area, hit mask, and the group's running pair counts.
struct GroupSmem {
  float4 e0[kItemThreads];      // u, v, a, b
  float4 e1[kItemThreads];      // c, 1/a, 1/c, cut
  float tz[kItemThreads];       // depth (the emitted key)
  uint32_t incl[kItemThreads];  // pairs of the items up to and including this one
  uint32_t xy[kItemThreads];    // rect origin: x | y << 16
  uint32_t w[kItemThreads];     // rect width in tiles
  uint32_t area[kItemThreads];  // rect tiles
  uint32_t mask[kItemThreads];  // hit bits over the rect tiles (rects of at most kMaskTiles)
  uint32_t wsum[kItemThreads / 32];
};

__device__ __forceinline__ Ell staged_ell(const GroupSmem& S, int k) {
  const float4 a = S.e0[k], b = S.e1[k];
  return Ell{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, S.tz[k]};
}

// idx = q w + r for idx < 2^20: a product with the reciprocal of w, then one
// exact integer correction (the product's error is below one).
__device__ __forceinline__ void tile_of(uint32_t idx, uint32_t w, uint32_t area, uint32_t& q,
                                        uint32_t& r) {
  if (area >= (1u << 20)) {
    q = idx / w;
    r = idx - q * w;
    return;
  }
  q = (uint32_t)__fmul_rn((float)idx, __frcp_rn((float)w));
  int32_t rr = (int32_t)idx - (int32_t)(q * w);
  if (rr < 0) {
    q--;
    rr += (int32_t)w;
  } else if (rr >= (int32_t)w) {
    q++;
    rr -= (int32_t)w;
  }
  r = (uint32_t)rr;
}

// Position of the r-th set bit (from 0) of m; m has more than r set bits.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r) {
  uint32_t pos = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const uint32_t c = __popc(m & ((1u << s) - 1u));
    if (r >= c) {
      r -= c;
      pos += s;
      m >>= s;
    }
  }
  return pos;
}

// Visits the pairs of the items [i0, i1), group by group of kItemThreads
// items: every thread stages its item (stage(slot, i, area) returns the
// item's pair count), the block scans the counts, and the pairs of the whole
// group are spread evenly over the block's threads, each finding its item by
// a binary search over the running counts -- so a splat over hundreds of
// tiles is shared by all warps instead of holding one back.  pair(slot, p,
// active, i) (pair p of item i) runs on every thread in every round (active false past the
// group's last pair, so that warp votes see converged warps); done(slot, i)
// runs once per item after its group.
template <typename Stage, typename Pair, typename Done>
__device__ __forceinline__ void expand_items(const float4* __restrict__ proj,
                                             const ushort4* __restrict__ rect, int64_t i0,
                                             int64_t i1, GroupSmem& S, Stage&& stage, Pair&& pair,
                                             Done&& done) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  ushort4 rn = make_ushort4(0, 0, 0, 0);
  if (i0 + tid < i1) rn = rect[i0 + tid];
  for (int64_t g = i0; g < i1; g += kItemThreads) {
    const int64_t i = g + tid;
    const ushort4 r = rn;
    rn = make_ushort4(0, 0, 0, 0);  // the next group's rects are in flight meanwhile
    if (i + kItemThreads < i1) rn = rect[i + kItemThreads];
    const uint32_t w = r.z > r.x ? (uint32_t)(r.z - r.x) : 0u;
    const uint32_t area = r.w > r.y ? w * (uint32_t)(r.w - r.y) : 0u;
    uint32_t work = 0;
    if (area) {  // (rects past i1 are empty)
      const float4 r0 = proj[2 * i], r1 = proj[2 * i + 1];
      S.e0[tid] = r0;
      S.e1[tid] = make_float4(r1.x, __frcp_rn(r0.z), __frcp_rn(r1.x), r1.w);
      S.tz[tid] = r1.z;
      S.xy[tid] = (uint32_t)r.x | ((uint32_t)r.y << 16);
      S.w[tid] = w;
      S.area[tid] = area;
      work = stage(tid, i, area);
    }
    uint32_t incl = work;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) S.wsum[warp] = incl;
    __syncthreads();
    uint32_t off = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kItemThreads / 32; q++) {
      const uint32_t v = S.wsum[q];
      off += q < warp ? v : 0u;
      total += v;
    }
    S.incl[tid] = incl + off;
    __syncthreads();
    for (uint32_t j0 = 0; j0 < total; j0 += kItemThreads) {
      const uint32_t j = j0 + (uint32_t)tid;
      const bool active = j < total;
      int k = 0;
      uint32_t p = 0;
      if (active) {  // the first item whose running count exceeds j
#pragma unroll
        for (int step = kItemThreads / 2; step > 0; step >>= 1)
          if (S.incl[k + step - 1] <= j) k += step;
        p = j - (k ? S.incl[k - 1] : 0u);
      }
      pair(k, p, active, g + k);
    }
    __syncthreads();  // the group's tables are read; the next group may restage them
    if (i < i1) done(tid, i);
  }
}

// Items of block b, camera by camera: for camera c, chunk b of that
// camera's n items [c n, (c + 1) n).  A block's per-tile tables so cover few
// tiles densely, and all blocks emit into the tiles of one camera at a time:
// the segments being filled stay within L2, which merges the scattered
// 8-byte writes into whole sectors before they reach DRAM.
__device__ __forceinline__ void cam_chunk(uint32_t n, uint32_t c, int64_t& i0, int64_t& i1) {
  const int64_t per = ((int64_t)n + gridDim.x - 1) / gridDim.x;
  const int64_t a = (int64_t)blockIdx.x * per;
  i0 = (int64_t)c * n + (a < (int64_t)n ? a : (int64_t)n);
  i1 = (int64_t)c * n + (a + per < (int64_t)n ? a + per : (int64_t)n);
}

// 1. per-tile instance counts, K, and the hit masks of the small rects.
__global__ void __launch_bounds__(kItemThreads)
tile_count_kernel(const float4* __restrict__ proj, const ushort4* __restrict__ rect, int64_t m,
                  uint32_t n, int tiles_x, uint32_t tiles, bool local,
                  uint32_t* __restrict__ counts, uint32_t* __restrict__ block_counts,
                  uint32_t* __restrict__ masks, unsigned long long* __restrict__ total) {
  __shared__ GroupSmem S;
  extern __shared__ uint32_t s_cnt[];  // this camera's tiles, when they fit
  const int lane = threadIdx.x & 31;
  unsigned long long k = 0;
  const uint32_t n_cams = (uint32_t)(m / n);
  for (uint32_t c = 0; c < n_cams; c++) {
    if (local) {
      for (uint32_t t = threadIdx.x; t < tiles; t += blockDim.x) s_cnt[t] = 0;
      __syncthreads();
    }
    int64_t i0, i1;
    cam_chunk(n, c, i0, i1);
    const uint32_t base = c * tiles;
    expand_items(
        proj, rect, i0, i1, S,
        [&](int slot, int64_t, uint32_t area) {
          S.mask[slot] = 0;
          return area;
        },
        [&](int slot, uint32_t p, bool active, int64_t) {
          bool hit = false;
          uint32_t area = 0;
          if (active) {
            area = S.area[slot];
            uint32_t qy, qx;
            tile_of(p, S.w[slot], area, qy, qx);
            const uint32_t xy = S.xy[slot];
            const uint32_t tx = (xy & 0xffffu) + qx, ty = (xy >> 16) + qy;
            hit = tile_hit(staged_ell(S, slot), tx, ty);
            if (hit) {
              const uint32_t tt = ty * (uint32_t)tiles_x + tx;
              if (local) atomicAdd(&s_cnt[tt], 1u);
              else atomicAdd(&counts[base + tt], 1u);
              k++;
            }
          }
          // the lanes holding a small rect's pairs are consecutive: the first
          // of them ORs the run's hit bits into the rect's mask
          const uint32_t bal = __ballot_sync(0xffffffffu, hit);
          if (active && area <= (uint32_t)kMaskTiles && (p == 0 || lane == 0)) {
            const uint32_t run = min(32u - (uint32_t)lane, area - p);
            const uint32_t bits = (bal >> lane) & (run == 32 ? 0xffffffffu : (1u << run) - 1u);
            if (bits) atomicOr(&S.mask[slot], bits << p);
          }
        },
        [&](int slot, int64_t i) { masks[i] = S.mask[slot]; });
    if (local) {  // this block's column of the [tile][block] counts, and the totals
      __syncthreads();
      for (uint32_t t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint32_t v = s_cnt[t];
        block_counts[(size_t)(base + t) * gridDim.x + blockIdx.x] = v;
        if (v) atomicAdd(&counts[base + t], v);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  if (lane == 0 && k) atomicAdd(total, k);
}

// 2. exclusive scan of the counts (one block): ranges, cursors, K.
__global__ void __launch_bounds__(kScanThreads)
tile_scan_kernel(const uint32_t* __restrict__ counts, uint32_t n_tiles_all,
                 const unsigned long long* __restrict__ total, int64_t capacity,
                 uint2* __restrict__ ranges, uint32_t* __restrict__ cursor,
                 int64_t* __restrict__ n_instances, int64_t* __restrict__ sort_n,
                 uint32_t* __restrict__ long_tiles, uint32_t* __restrict__ n_long) {
  __shared__ uint32_t ws[32];
  __shared__ uint32_t carry;
  const int64_t K = (int64_t)*total;
  const bool fits = K <= capacity;
  if (threadIdx.x == 0) {
    carry = 0;
    *n_instances = K;
    *sort_n = fits ? K : 0;
    if (!fits) atomicMax(&g_capacity_k, (unsigned long long)K);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t c0 = 0; c0 < n_tiles_all; c0 += kScanThreads) {
    const uint32_t t = c0 + threadIdx.x;
    const uint32_t v = t < n_tiles_all ? counts[t] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      ws[lane] = w;
    }
    __syncthreads();
    const uint32_t incl = carry + (warp > 0 ? ws[warp - 1] : 0u) + x;
    if (t < n_tiles_all) {
      const uint32_t start = incl - v;
      ranges[t] = fits && v ? make_uint2(start, incl) : make_uint2(0u, 0u);
      cursor[t] = start;
      if (fits && v > (uint32_t)kSegMax) long_tiles[atomicAdd(n_long, 1u)] = t;
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = incl;
    __syncthreads();
  }
}

// 2b. where each block's instances of each tile start: the tile's start plus
// the counts of the blocks before it (one warp per tile, a warp scan over
// the blocks in order).
__global__ void __launch_bounds__(256)
block_base_kernel(const uint32_t* __restrict__ block_counts, int nblocks, uint32_t n_tiles_all,
                  const uint32_t* __restrict__ cursor, const int64_t* __restrict__ sort_n,
                  uint32_t* __restrict__ block_base) {
  if (*sort_n == 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= n_tiles_all) return;
  const uint32_t* col = block_counts + (size_t)t * nblocks;
  uint32_t* out = block_base + (size_t)t * nblocks;
  uint32_t run = cursor[t];
  for (int b0 = 0; b0 < nblocks; b0 += 256) {  // eight loads in flight, then eight scans
    uint32_t c[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int b = b0 + 32 * k + lane;
      c[k] = b < nblocks ? col[b] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int b = b0 + 32 * k + lane;
      uint32_t x = c[k];
#pragma unroll
      for (int q = 1; q < 32; q <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, q);
        if (lane >= q) x += y;
      }
      if (b < nblocks) out[b] = run + x - c[k];
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
}

// 3. append (depth bits, Gaussian index) to every covered tile's segment:
// the small rects walk the set bits of their hit masks, the others repeat
// the tile test.  With the tile tables in shared memory a block starts from
// its own bases (block_base row) and places its instances with shared-
// memory atomics; otherwise every instance reserves its slot with a global
// atomic.
__global__ void __launch_bounds__(kItemThreads)
tile_emit_kernel(const float4* __restrict__ proj, const ushort4* __restrict__ rect, int64_t m,
                 uint32_t n, int tiles_x, uint32_t tiles, bool local,
                 const int64_t* __restrict__ sort_n, const uint32_t* __restrict__ block_base,
                 const uint32_t* __restrict__ masks, uint32_t* __restrict__ cursor,
                 unsigned long long* __restrict__ seg) {
  __shared__ GroupSmem S;
  extern __shared__ uint32_t s_cur[];  // [tiles] next slot of this block in this camera
  if (*sort_n == 0) return;  // nothing fits (or nothing visible)
  const uint32_t n_cams = (uint32_t)(m / n);
  for (uint32_t c = 0; c < n_cams; c++) {
    const uint32_t base = c * tiles;
    if (local) {
      for (uint32_t t = threadIdx.x; t < tiles; t += blockDim.x)
        s_cur[t] = block_base[(size_t)(base + t) * gridDim.x + blockIdx.x];
      __syncthreads();
    }
    int64_t i0, i1;
    cam_chunk(n, c, i0, i1);
    const int64_t item0 = (int64_t)c * n;
    expand_items(
        proj, rect, i0, i1, S,
        [&](int slot, int64_t i, uint32_t area) {
          if (area > (uint32_t)kMaskTiles) return area;
          const uint32_t mk = masks[i];
          S.mask[slot] = mk;
          return (uint32_t)__popc(mk);
        },
        [&](int slot, uint32_t p, bool active, int64_t i) {
          if (!active) return;
          const uint32_t area = S.area[slot];
          const bool small = area <= (uint32_t)kMaskTiles;
          uint32_t qy, qx;
          tile_of(small ? nth_set_bit(S.mask[slot], p) : p, S.w[slot], area, qy, qx);
          const uint32_t xy = S.xy[slot];
          const uint32_t tx = (xy & 0xffffu) + qx, ty = (xy >> 16) + qy;
          const Ell E = staged_ell(S, slot);
          if (small || tile_hit(E, tx, ty)) {
            const uint32_t t = base + ty * (uint32_t)tiles_x + tx;
            const uint32_t pos = local ? atomicAdd(&s_cur[t - base], 1u) : atomicAdd(&cursor[t], 1u);
            seg[pos] = ((unsigned long long)__float_as_uint(E.tz) << 32) | (uint32_t)(i - item0);
          }
        },
        [](int, int64_t) {});
    if (local) __syncthreads();  // the cursors are reloaded for the next camera
  }
}

__device__ __forceinline__ uint32_t lane_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// The lanes of a converged warp whose NB-bit digit equals this lane's: one
// ballot per bit (short fixed-latency votes instead of a match instruction).
template <int NB>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < NB; b++) {
    const bool on = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, on);
    peers &= on ? bal : ~bal;
  }
  return peers;
}

// 4. each segment of 64-bit (depth bits, index) keys is sorted by one block:
// a stable LSD radix sort, 8 bits a pass, skipping the digits all keys share;
// each warp holds R consecutive runs of 32 keys, ranks them per digit with
// per-bit ballots in position order, and a per-digit scan over the warps
// places them.  Segments of up to kSegMax keys are sorted by 256-thread
// blocks, one per tile (eight or sixteen keys a thread); longer ones by
// 1024-thread blocks that take them from a list (up to 12,288 keys in shared
// memory), and the rare segment beyond that the same way from global memory.
template <int T, int I>
struct SegSmem {
  static constexpr int W = T / 32;
  static constexpr int G = W / 8;  // groups of 8 warps (T = 256 G threads)
  static constexpr int MAXK = T * I;
  unsigned long long sk[T * I];
  uint16_t wcnt[W][256];  // counts, then offsets (<= MAXK < 2^16)
  uint32_t gsum[G][256];  // per digit, the count of each group of 8 warps
  uint32_t dstart[256];
  uint32_t wsum[8];
  unsigned long long s_or[W], s_and[W], s_max[W];
};
// Equal depths in a sorted segment form runs that are ordered by index in
// place when no run is longer than this; otherwise the segment is sorted
// again on all eight digits.
constexpr int kRunMax = 32;
static_assert(kSegMax < 65536 && kLargeThreads * kLargeItems < 65536, "wcnt is 16-bit");

// Segments longer than a block's shared memory: the same stable LSD radix
// sort with the keys in global memory (ping-pong between the segment and its
// scratch copy, both L2-resident).  Each pass counts the digit over the whole
// segment, then scatters it MAXK keys at a time in position order: within a
// chunk the warps rank their keys as above, and running per-digit offsets
// carry over from chunk to chunk, which keeps the pass stable.
template <int T, int I>
__device__ __noinline__ void big_segment_sort(unsigned long long* src, unsigned long long* dst,
                                              uint32_t cnt, uint32_t tile,
                                              uint32_t* __restrict__ ids,
                                              uint64_t* __restrict__ keys_opt, SegSmem<T, I>& S) {
  constexpr int W = T / 32, CH = T * I;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* hist = reinterpret_cast<uint32_t*>(S.sk);  // [256] digit counts of the segment
  uint32_t* run = hist + 256;                          // [256] next output slot of each digit
  unsigned long long o = 0, a = ~0ull;
  for (uint32_t i = threadIdx.x; i < cnt; i += T) {
    o |= src[i];
    a &= src[i];
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    o |= __shfl_xor_sync(0xffffffffu, o, d);
    a &= __shfl_xor_sync(0xffffffffu, a, d);
  }
  if (lane == 0) {
    S.s_or[warp] = o;
    S.s_and[warp] = a;
  }
  __syncthreads();
  unsigned long long oo = 0, aa = ~0ull;
  for (int w = 0; w < W; w++) {
    oo |= S.s_or[w];
    aa &= S.s_and[w];
  }
  const unsigned long long diff = oo ^ aa;
  auto pass = [&](int shift) {
    if (((diff >> shift) & 0xffull) == 0) return;  // uniform over the block
    for (int d = threadIdx.x; d < 256; d += T) hist[d] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cnt; i += T)
      atomicAdd(&hist[(uint32_t)(src[i] >> shift) & 0xffu], 1u);
    __syncthreads();
    if (threadIdx.x < 256) {  // exclusive scan of the digit counts
      const uint32_t v = hist[threadIdx.x];
      uint32_t x = v;
#pragma unroll
      for (int q = 1; q < 32; q <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, q);
        if (lane >= q) x += y;
      }
      if (lane == 31) S.wsum[warp] = x;
      run[threadIdx.x] = x - v;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t add = 0;
      for (int w = 0; w < warp; w++) add += S.wsum[w];
      run[threadIdx.x] += add;
    }
    __syncthreads();
    for (uint32_t c0 = 0; c0 < cnt; c0 += CH) {
      for (int i = threadIdx.x; i < W * 256; i += T) (&S.wcnt[0][0])[i] = 0;
      __syncthreads();
      const uint32_t base = c0 + (uint32_t)warp * 32u * I;
      unsigned long long key[I];
      uint32_t rank[I];
#pragma unroll
      for (int r = 0; r < I; r++) {
        const uint32_t p = base + r * 32 + lane;
        const bool valid = p < cnt;
        key[r] = valid ? src[p] : 0ull;
        const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & 0xffu : 256u + lane;
        const uint32_t peers = digit_peers<9>(d);  // lanes past the end stay alone
        const uint32_t prior = valid ? S.wcnt[warp][d] : 0u;
        rank[r] = prior + __popc(peers & lane_lt());
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) S.wcnt[warp][d] = (uint16_t)(prior + __popc(peers));
        __syncwarp();
      }
      __syncthreads();
      if (threadIdx.x < 256) {  // per digit: this chunk's warps in order
        const int d = threadIdx.x;
        uint32_t tot = 0;
        for (int w = 0; w < W; w++) {
          const uint32_t c = S.wcnt[w][d];
          S.wcnt[w][d] = (uint16_t)tot;
          tot += c;
        }
        S.dstart[d] = tot;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < I; r++) {
        const uint32_t p = base + r * 32 + lane;
        if (p < cnt) {
          const uint32_t d = (uint32_t)(key[r] >> shift) & 0xffu;
          dst[run[d] + S.wcnt[warp][d] + rank[r]] = key[r];
        }
      }
      __syncthreads();
      if (threadIdx.x < 256) run[threadIdx.x] += S.dstart[threadIdx.x];
      __syncthreads();
    }
    unsigned long long* t = src;
    src = dst;
    dst = t;
    __syncthreads();
  };
  for (int sh = 32; sh < 64; sh += 8) pass(sh);  // depth digits
  bool tie = false;
  for (uint32_t i = threadIdx.x + 1; i < cnt; i += T)
    tie |= (src[i] >> 32) == (src[i - 1] >> 32);
  if (__syncthreads_or(tie))
    for (int sh = 0; sh < 64; sh += 8) pass(sh);  // equal depths: order by index too
  for (uint32_t i = threadIdx.x; i < cnt; i += T) {
    const unsigned long long key = src[i];
    ids[i] = (uint32_t)key;
    if (keys_opt) keys_opt[i] = ((uint64_t)tile << 32) | (key >> 32);
  }
}

// One segment of cnt <= T * I keys (seg[0, cnt)), sorted in shared memory;
// writes the Gaussian indices (and the keys) of the sorted order.
template <int T, int I>
__device__ void smem_segment_sort(const unsigned long long* __restrict__ seg, uint32_t cnt,
                                  uint32_t tile, uint32_t* __restrict__ ids,
                                  uint64_t* __restrict__ keys_opt, SegSmem<T, I>& S) {
  constexpr int W = T / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = (int)((cnt + T - 1) / T);
  const uint32_t base = (uint32_t)warp * 32u * (uint32_t)R;  // this warp's first position
  unsigned long long key[I];
  unsigned long long o = 0, a = ~0ull, mx = 0;
#pragma unroll
  for (int r = 0; r < I; r++) {
    const uint32_t p = base + r * 32 + lane;
    key[r] = 0;
    if (r < R && p < cnt) {
      key[r] = seg[p];
      o |= key[r];
      a &= key[r];
      mx = key[r] > mx ? key[r] : mx;
    }
  }
  // bits that differ between the keys: only those digits need a pass
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    o |= __shfl_xor_sync(0xffffffffu, o, d);
    a &= __shfl_xor_sync(0xffffffffu, a, d);
    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, d);
    mx = m2 > mx ? m2 : mx;
  }
  if (lane == 0) {
    S.s_or[warp] = o;
    S.s_and[warp] = a;
    S.s_max[warp] = mx;
  }
  __syncthreads();
  unsigned long long diff = 0, kmax = 0;
  {
    unsigned long long oo = 0, aa = ~0ull;
    for (int w = 0; w < W; w++) {
      oo |= S.s_or[w];
      aa &= S.s_and[w];
      kmax = S.s_max[w] > kmax ? S.s_max[w] : kmax;
    }
    diff = oo ^ aa;
  }
  // slots past the segment hold copies of the largest key: they share every
  // skipped digit with the real keys and, being later in position, stay
  // behind the real copy in a stable sort
#pragma unroll
  for (int r = 0; r < I; r++)
    if (!(r < R && base + r * 32 + lane < cnt)) key[r] = kmax;
  // one stable pass on the 8-bit digit at `shift` (skipped when every key
  // has the same digit there)
  auto pass = [&](int shift) {
    if (((diff >> shift) & 0xffull) == 0) return;  // uniform over the block
    for (int i = threadIdx.x; i < W * 256; i += T) (&S.wcnt[0][0])[i] = 0;
    __syncthreads();
    uint32_t rank[I];
#pragma unroll
    for (int r = 0; r < I; r++) {
      if (r < R) {  // uniform over the block
        const uint32_t d = (uint32_t)(key[r] >> shift) & 0xffu;
        const uint32_t peers = digit_peers<8>(d);
        const uint32_t prior = S.wcnt[warp][d];
        rank[r] = prior + __popc(peers & lane_lt());
        __syncwarp();
        if (lane == __ffs(peers) - 1) S.wcnt[warp][d] = (uint16_t)(prior + __popc(peers));
        __syncwarp();
      }
    }
    __syncthreads();
    // per digit: warps in order -- thread (d, g) takes the 8 warps of group
    // g, then the groups' offsets are added -- then digits in order
    constexpr int G = SegSmem<T, I>::G;
    static_assert(T == 256 * G, "one thread per (digit, group of 8 warps)");
    uint32_t tot = 0;
    {
      const int d = threadIdx.x & 255, gg = threadIdx.x >> 8;
      for (int w = 8 * gg; w < 8 * gg + 8; w++) {
        const uint32_t c = S.wcnt[w][d];
        S.wcnt[w][d] = (uint16_t)tot;
        tot += c;
      }
      if (G > 1) S.gsum[gg][d] = tot;
    }
    if (G > 1) {
      __syncthreads();
      const int d = threadIdx.x & 255, gg = threadIdx.x >> 8;
      uint32_t off = 0;
      for (int q = 0; q < gg; q++) off += S.gsum[q][d];
      if (off)
        for (int w = 8 * gg; w < 8 * gg + 8; w++) S.wcnt[w][d] = (uint16_t)(S.wcnt[w][d] + off);
      if (gg == 0)
        for (int q = 1; q < G; q++) tot += S.gsum[q][d];
    }
    if (threadIdx.x < 256) {
      const int d = threadIdx.x;
      uint32_t x = tot;
#pragma unroll
      for (int q = 1; q < 32; q <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, q);
        if (lane >= q) x += y;
      }
      if (lane == 31) S.wsum[warp] = x;
      S.dstart[d] = x - tot;  // exclusive within this warp's 32 digits
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t add = 0;
      for (int w = 0; w < warp; w++) add += S.wsum[w];
      S.dstart[threadIdx.x] += add;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < I; r++)
      if (r < R) {
        const uint32_t d = (uint32_t)(key[r] >> shift) & 0xffu;
        S.sk[S.dstart[d] + S.wcnt[warp][d] + rank[r]] = key[r];
      }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < I; r++)
      if (r < R) key[r] = S.sk[base + r * 32 + lane];
    __syncthreads();
  };
  // the depth digits alone order the keys unless two share a depth: each run
  // of equal depths (contiguous now, in emission order) is then put in index
  // order in place by the thread that holds its first key (an insertion sort
  // of the full keys), unless some run is longer than kRunMax, in which case
  // the segment is sorted again on all eight digits (index ones first)
  for (int sh = 32; sh < 64; sh += 8) pass(sh);
#pragma unroll
  for (int r = 0; r < I; r++)  // the current order (also when no pass ran)
    if (r < R) S.sk[base + r * 32 + lane] = key[r];
  __syncthreads();
  bool tie = false, long_run = false;
#pragma unroll
  for (int r = 0; r < I; r++) {
    const uint32_t p = base + r * 32 + lane;
    if (!(r < R && p < cnt)) continue;
    const uint32_t dz = (uint32_t)(key[r] >> 32);
    const bool first = p == 0 || (uint32_t)(S.sk[p - 1] >> 32) != dz;
    if (!first || p + 1 >= cnt || (uint32_t)(S.sk[p + 1] >> 32) != dz) continue;
    // a run starts at p: only its depth bits are read by other threads, and
    // those stay put while it is reordered
    tie = true;
    uint32_t e = p + 1;
    while (e < cnt && e - p <= (uint32_t)kRunMax && (uint32_t)(S.sk[e] >> 32) == dz) e++;
    if (e - p > (uint32_t)kRunMax) {
      long_run = true;
      continue;
    }
    for (uint32_t i = p + 1; i < e; i++) {
      const unsigned long long v = S.sk[i];
      uint32_t j = i;
      for (; j > p && S.sk[j - 1] > v; j--) S.sk[j] = S.sk[j - 1];
      S.sk[j] = v;
    }
  }
  if (__syncthreads_or(long_run)) {
    for (int sh = 0; sh < 64; sh += 8) pass(sh);
  } else if (__syncthreads_or(tie)) {
#pragma unroll
    for (int r = 0; r < I; r++)
      if (r < R) key[r] = S.sk[base + r * 32 + lane];
  }
#pragma unroll
  for (int r = 0; r < I; r++) {
    const uint32_t p = base + r * 32 + lane;
    if (r < R && p < cnt) {
      ids[p] = (uint32_t)key[r];
      if (keys_opt) keys_opt[p] = ((uint64_t)tile << 32) | (key[r] >> 32);
    }
  }
}

// 4a. tiles of at most kSegSmall instances, one 256-thread block each with
// eight keys a thread (most tiles; few registers, so many blocks per SM).
__global__ void __launch_bounds__(kSegThreads, 5)
tile_sort_kernel(const uint2* __restrict__ ranges, const unsigned long long* __restrict__ seg,
                 uint32_t* __restrict__ ids, uint64_t* __restrict__ keys_opt) {
  using SS = SegSmem<kSegThreads, kSegSmall / kSegThreads>;
  extern __shared__ __align__(16) unsigned char seg_smem[];
  SS& S = *reinterpret_cast<SS*>(seg_smem);
  const uint32_t tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  const uint32_t cnt = rg.y - rg.x;
  if (cnt == 0 || cnt > (uint32_t)kSegSmall) return;
  smem_segment_sort<kSegThreads, kSegSmall / kSegThreads>(seg + rg.x, cnt, tile, ids + rg.x,
                                                           keys_opt ? keys_opt + rg.x : nullptr, S);
}

// 4b. the tiles of kSegSmall + 1 to kSegMax instances: 256-thread blocks with
// sixteen keys a thread, one per tile.
__global__ void __launch_bounds__(kSegThreads, 3)
tile_sort_mid_kernel(const uint2* __restrict__ ranges, const unsigned long long* __restrict__ seg,
                     uint32_t* __restrict__ ids, uint64_t* __restrict__ keys_opt) {
  using SS = SegSmem<kSegThreads, kSegMax / kSegThreads>;
  extern __shared__ __align__(16) unsigned char seg_smem[];
  SS& S = *reinterpret_cast<SS*>(seg_smem);
  const uint32_t tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  const uint32_t cnt = rg.y - rg.x;
  if (cnt <= (uint32_t)kSegSmall || cnt > (uint32_t)kSegMax) return;
  smem_segment_sort<kSegThreads, kSegMax / kSegThreads>(seg + rg.x, cnt, tile, ids + rg.x,
                                                         keys_opt ? keys_opt + rg.x : nullptr, S);
}

// 4c. the tiles with more than kSegMax instances, from the list tile_scan
// made: up to 12,288 keys in shared memory, beyond that from global memory.
__global__ void __launch_bounds__(kLargeThreads, 1)
tile_sort_large_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ long_tiles,
                       const uint32_t* __restrict__ n_long, unsigned long long* __restrict__ seg,
                       unsigned long long* __restrict__ scratch, uint32_t* __restrict__ ids,
                       uint64_t* __restrict__ keys_opt) {
  using SS = SegSmem<kLargeThreads, kLargeItems>;
  extern __shared__ __align__(16) unsigned char seg_smem[];
  SS& S = *reinterpret_cast<SS*>(seg_smem);
  const uint32_t nl = *n_long;
  for (uint32_t i = blockIdx.x; i < nl; i += gridDim.x) {
    const uint32_t tile = long_tiles[i];
    const uint2 rg = ranges[tile];
    const uint32_t cnt = rg.y - rg.x;
    if (cnt <= (uint32_t)SS::MAXK)
      smem_segment_sort<kLargeThreads, kLargeItems>(seg + rg.x, cnt, tile, ids + rg.x,
                                                    keys_opt ? keys_opt + rg.x : nullptr, S);
    else
      big_segment_sort<kLargeThreads, kLargeItems>(seg + rg.x, scratch + rg.x, cnt, tile,
                                                   ids + rg.x, keys_opt ? keys_opt + rg.x : nullptr,
                                                   S);
    __syncthreads();  // the shared tables are reused by the next tile
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BinLayout {
  size_t counts, cursor, total, n_long, sort_n, zero_end, block_counts, block_base, masks,
      long_tiles, seg, scratch, size;
  bool local;  // per-block tile tables in shared memory
};

// The per-block tables cover one camera's tiles at a time in shared memory;
// their [tile][block] copies in the workspace are kept below 64 M entries.
bool block_tables(uint64_t tiles, uint64_t n_tiles_all) {
  return tiles <= (uint64_t)kSmemTiles && n_tiles_all * kItemBlocks <= (1ull << 26);
}

BinLayout bin_layout(uint64_t m, uint64_t tiles, uint64_t n_tiles_all, int64_t capacity) {
  BinLayout L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o += align256(b > 0 ? b : 1); return at; };
  L.counts = take(4 * n_tiles_all);
  L.total = take(8);
  L.n_long = take(4);
  L.zero_end = o;  // counts, total and the long-tile count start at zero
  L.sort_n = take(8);
  L.cursor = take(4 * n_tiles_all);
  L.local = block_tables(tiles, n_tiles_all);
  L.block_counts = take(L.local ? 4 * (size_t)kItemBlocks * n_tiles_all : 0);
  L.block_base = take(L.local ? 4 * (size_t)kItemBlocks * n_tiles_all : 0);
  L.masks = take(4 * m);
  L.long_tiles = take(4 * n_tiles_all);
  L.seg = take(8 * (size_t)capacity);
  L.scratch = take(8 * (size_t)capacity);
  L.size = o;
  return L;
}

// Blocks of the count and emit passes: every block takes a chunk of each
// camera's n items.
int grid_items(int64_t n) {
  return (int)std::max<int64_t>(
      1, std::min<int64_t>((n + kItemThreads - 1) / kItemThreads, kItemBlocks));
}

}  // namespace

unsigned long long capacity_word(bool clear) {
  unsigned long long v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_capacity_k, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) cudaMemcpyToSymbol(g_capacity_k, &zero, sizeof(zero));
  return v;
}

}  // namespace lgs

using namespace lgs;

extern "C" size_t gs_bin_sort_workspace(int64_t n, int n_cams, int tiles_x, int tiles_y,
                                        int64_t capacity) {
  if (n < 0 || n_cams < 1 || capacity < 0 || tiles_x < 1 || tiles_y < 1) return 0;
  const uint64_t tiles = (uint64_t)tiles_x * (uint64_t)tiles_y;
  return bin_layout((uint64_t)n_cams * (uint64_t)n, tiles, (uint64_t)n_cams * tiles, capacity).size;
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
  LGS_CHECK_ARG((uint64_t)tiles * (uint64_t)n_cams <= (1ull << 24), "too many tiles");
  const uint32_t n_tiles_all = (uint32_t)n_cams * tiles;
  const BinLayout L = bin_layout((uint64_t)m, tiles, n_tiles_all, capacity);
  LGS_CHECK_ARG(workspace_bytes >= L.size, "workspace too small");
  cudaStream_t s = as_stream(stream);
  char* ws = (char*)workspace;
  LGS_CHECK_CUDA(cudaMemsetAsync(ws, 0, L.zero_end, s));
  if (m == 0) {
    LGS_CHECK_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_tiles_all, s));
    LGS_CHECK_CUDA(cudaMemsetAsync(n_instances_dev, 0, sizeof(int64_t), s));
    return LGS_OK;
  }
  uint32_t* counts = (uint32_t*)(ws + L.counts);
  uint32_t* cursor = (uint32_t*)(ws + L.cursor);
  unsigned long long* total = (unsigned long long*)(ws + L.total);
  int64_t* sort_n = (int64_t*)(ws + L.sort_n);
  unsigned long long* seg = (unsigned long long*)(ws + L.seg);
  const bool local = L.local;
  const size_t cnt_smem = local ? 4 * (size_t)tiles : 0;
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(tile_count_kernel), 4 * kSmemTiles));
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(tile_emit_kernel), 4 * kSmemTiles));
  uint32_t* block_counts = (uint32_t*)(ws + L.block_counts);
  uint32_t* block_base = (uint32_t*)(ws + L.block_base);
  uint32_t* masks = (uint32_t*)(ws + L.masks);
  const int nblk = grid_items(n);
  tile_count_kernel<<<nblk, kItemThreads, cnt_smem, s>>>((const float4*)proj, (const ushort4*)rect,
                                                         m, (uint32_t)n, tiles_x, tiles, local,
                                                         counts, block_counts, masks, total);
  uint32_t* long_tiles = (uint32_t*)(ws + L.long_tiles);
  uint32_t* n_long = (uint32_t*)(ws + L.n_long);
  tile_scan_kernel<<<1, kScanThreads, 0, s>>>(counts, n_tiles_all, total, capacity,
                                              (uint2*)ranges, cursor, n_instances_dev, sort_n,
                                              long_tiles, n_long);
  if (capacity == 0) {
    LGS_CHECK_LAUNCH();
    return LGS_OK;
  }
  if (local)
    block_base_kernel<<<(n_tiles_all + 7) / 8, 256, 0, s>>>(block_counts, nblk, n_tiles_all,
                                                          cursor, sort_n, block_base);
  tile_emit_kernel<<<nblk, kItemThreads, cnt_smem, s>>>((const float4*)proj, (const ushort4*)rect,
                                                        m, (uint32_t)n, tiles_x, tiles, local,
                                                        sort_n, block_base, masks, cursor, seg);
  using SmallSmem = SegSmem<kSegThreads, kSegSmall / kSegThreads>;
  using MidSmem = SegSmem<kSegThreads, kSegMax / kSegThreads>;
  using LargeSmem = SegSmem<kLargeThreads, kLargeItems>;
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(tile_sort_kernel),
                                (int)sizeof(SmallSmem)));
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(tile_sort_large_kernel),
                                (int)sizeof(LargeSmem)));
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(tile_sort_mid_kernel),
                                (int)sizeof(MidSmem)));
  tile_sort_kernel<<<n_tiles_all, kSegThreads, sizeof(SmallSmem), s>>>((const uint2*)ranges, seg,
                                                                       ids, keys_opt);
  tile_sort_mid_kernel<<<n_tiles_all, kSegThreads, sizeof(MidSmem), s>>>((const uint2*)ranges,
                                                                         seg, ids, keys_opt);
  tile_sort_large_kernel<<<std::min<uint32_t>(n_tiles_all, kLargeBlocks), kLargeThreads,
                           sizeof(LargeSmem), s>>>((const uint2*)ranges, long_tiles, n_long, seg,
                                                   (unsigned long long*)(ws + L.scratch), ids,
                                                   keys_opt);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}
