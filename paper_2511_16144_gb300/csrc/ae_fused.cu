// Fused feature distillation through the frozen decoder (LEGO-SLAM
// Sec. III-B.3, Eq. 2): y = D_theta(F_render), loss += w mean|y - F_gt| and
// dF_render = dL/dF_render, for 128-pixel tiles that never leave the chip.
//
// D_theta is 16 -> 64 -> 128 -> 256 -> 512 with GELU (tanh form) after the first three
// layers.  Per tile the CTA runs, on the tensor cores (BF16 operands, FP32
// accumulators in tensor memory):
//   F1..F3  forward hidden layers, activations kept in shared memory (BF16);
//   F4/B1   the 512-wide output in eight 64-column chunks: each chunk's
//           epilogue forms dy = w sign(y - F_gt) / (P 512) and immediately
//           feeds dh3 += dy_chunk W7_chunk, so y and dy never reach memory
//           (dy goes back into tensor memory, double-buffered, as the A
//           operand of that product);
//           B1 reads the chunk's W7 units that F4 used, still in the ring, as
//           an MN-major operand (W7 is streamed once per tile, W7^T never);
//   R3..R1  the pre-activations are recomputed instead of stored (this keeps
//           the working set in shared memory);
//   B2..B4  dh2 = (dh3 * gelu'(pre3)) W6, dh1 = (dh2 * gelu'(pre2)) W5,
//           dz = (dh1 * gelu'(pre1)) W4.
// Consecutive tiles of a CTA overlap: the backward hidden layers of tile t
// (R3, B2..B4, accumulators in TMEM columns 0-255) interleave with the
// forward hidden layers of tile t+1 (F1..F3, columns 256-511), so the tensor
// core works on one tile while the epilogue warps work on the other.  z is
// double-buffered for this.  The output epilogue reads F_gt with one 32-byte
// load per lane (its row's 16 columns of the chunk, one sector) a chunk ahead.
// Warps 0-15 are the epilogue (TMEM -> registers -> shared memory, or back to
// TMEM for dy and d1; warps w, w + 4, w + 8, w + 12 share TMEM lane quadrant
// w % 4 and split the columns in quarters), warp 16 issues the MMAs, warps 17
// and 18 stream the weights as 35 pre-packed units (<= 16 KB each, already in
// the tensor-core's canonical layout) through a 6-stage ring with bulk TMA
// copies.  Every wait is bounded.
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tc05.cuh"

namespace lgs {

namespace {

constexpr int kUnits = 35;
constexpr int kStages = 6;
constexpr uint32_t kStageBytes = 16384;
constexpr uint32_t kLimit = 1u << 22;

// shared-memory map (bytes)
constexpr uint32_t SM_Z = 0;         // 2 x (128 x 16 bf16): z of this tile and the next
constexpr uint32_t SM_H1 = 8192;     // 128 x 64   (h1)
constexpr uint32_t SM_H2 = 24576;    // 128 x 128  (h2, later d2)
constexpr uint32_t SM_H3 = 57344;    // 128 x 256  (h3, later d3)
constexpr uint32_t SM_ST = 122880;   // kStages x 16 KB weight ring
constexpr uint32_t SM_BAR = SM_ST + kStages * kStageBytes;

// tensor-memory columns of the BF16 A operands the epilogue stores there:
// the two dy chunk buffers (free during the output phase, whose forward
// chunks use 256-383 and B1 0-255) and d1 (pre2's columns, read by E6 before)
constexpr uint32_t TM_DY = 384;      // 2 x 32 columns (128 x 64 BF16 each)
constexpr uint32_t TM_D1 = 128;      // 32 columns

// weight matrices of the decoder: forward W (out x in) and transposed Wt
enum Mat { W4 = 0, W5, W6, W7, T4, T5, T6, T7 };
constexpr int kCols[8] = {16, 64, 128, 256, 64, 128, 256, 512};

struct Unit {
  int mat, row0, rows, col0, kc;
};

// The 35 weight units of one tile, in the order the MMAs consume them.
std::vector<Unit> schedule() {
  std::vector<Unit> U;
  auto add = [&](int m, int r0, int rows, int c0, int kc) { U.push_back({m, r0, rows, c0, kc}); };
  add(W4, 0, 64, 0, 16);                                                   // F1
  add(W5, 0, 128, 0, 64);                                                  // F2
  for (int k = 0; k < 4; k++) add(W6, 0, 256, 32 * k, 32);                // F3 (N = 256)
  // F4: eight 64-column output chunks of two K-halves each (64 x 128); the
  // backward product B1 of a chunk reads the same two units again, as an
  // MN-major operand, so W7 is streamed once and W7^T not at all
  for (int c = 0; c < 8; c++)
    for (int u = 0; u < 2; u++) add(W7, 64 * c, 64, 128 * u, 128);
  for (int k = 0; k < 4; k++) add(W6, 0, 256, 32 * k, 32);                // R3 (N = 256)
  for (int k = 0; k < 4; k++) add(T6, 0, 128, 64 * k, 64);               // B2
  add(W5, 0, 128, 0, 64);                                                  // R2
  for (int k = 0; k < 2; k++) add(T5, 0, 64, 64 * k, 64);                // B3
  add(W4, 0, 64, 0, 16);                                                   // R1
  add(T4, 0, 16, 0, 64);                                                   // B4
  return U;
}

struct PackArgs {
  const __nv_bfloat16* mats[8];
  int ld[8];
  Unit units[kUnits];
  uint32_t off[kUnits];
  uint32_t piece0[kUnits + 1];
  uint8_t* pack;
};

// Writes every unit as [rows/8][kc/8][8][8] bf16 core matrices.
__global__ void pack_units_kernel(PackArgs a) {
  const uint32_t total = a.piece0[kUnits];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int u = 0;
    while (a.piece0[u + 1] <= i) u++;
    const Unit U = a.units[u];
    const uint32_t j = i - a.piece0[u];
    const int per_row = U.kc / 8;
    const int r = (int)(j / per_row), c = (int)(j % per_row);
    const __nv_bfloat16* src = a.mats[U.mat] + (int64_t)(U.row0 + r) * a.ld[U.mat] + U.col0 + 8 * c;
    *reinterpret_cast<uint4*>(a.pack + a.off[u] + tc::core_offset(r, c, U.kc)) =
        *reinterpret_cast<const uint4*>(src);
  }
}

struct FusedArgs {
  const uint8_t* pack;
  uint32_t off[kUnits];
  uint32_t bytes[kUnits];
  const float* b4;
  const float* b5;
  const float* b6;
  const float* b7;
  const float* z;
  const __nv_bfloat16* target;
  float* dz;
  int64_t P;
  float scale;
  float* loss;
};

// 16 or 32 consecutive columns of row r as BF16 into an activation tile of
// width kw starting at column col (a multiple of 8).
template <int NV>
__device__ __forceinline__ void put_row(uint8_t* tile, int r, int col, int kw, const float* v) {
#pragma unroll
  for (int q = 0; q < NV / 8; q++) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; k++) h[k] = __floats2bfloat162_rn(v[8 * q + 2 * k], v[8 * q + 2 * k + 1]);
    *reinterpret_cast<uint4*>(tile + tc::core_offset(r, col / 8 + q, kw)) = u;
  }
}

__device__ unsigned g_fused_error;

// -x and -y of a BF16 pair (x in the low half) as floats: the BF16 bits moved
// to the top of the FP32 word with the sign flipped (exact, as is -t itself)
__device__ __forceinline__ float2 neg_bf16x2(__nv_bfloat162 h) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(&h);
  return f2(__uint_as_float((w << 16) ^ 0x80000000u),
            __uint_as_float((w & 0xffff0000u) ^ 0x80000000u));
}

constexpr int kEpiWarps = 16;
constexpr int kProducers = 2;                          // warps streaming the weight units
constexpr int kFusedThreads = (kEpiWarps + 1 + kProducers) * 32;  // + the MMA warp
// barriers: full[kStages], empty[kStages], accH, accT, opH, opT, ybar[2], dyrdy[2],
// drain, the slice barriers sh2[2], sh3[4], sd2[2], sd3[4], then the TMEM slot
constexpr uint32_t kBarBytes = (2 * kStages + 21) * 8 + 4;
constexpr uint32_t SM_BIAS = SM_BAR + 512;             // b4 | b5 | b6 | b7 (960 floats)
constexpr uint32_t SM_ALL = SM_BIAS + 960 * 4;
static_assert(kBarBytes <= SM_BIAS - SM_BAR, "barrier block overlaps the biases");
static_assert(SM_ALL <= 232448, "shared-memory map exceeds 227 KB");
static_assert(SM_H3 + 128 * 256 * 2 <= SM_ST, "h3 overlaps the ring");

// Weight units per tile in stream order.  Units 0-5 are the forward hidden
// layers (F1, F2, F3), 6-21 the output layer (F4, its units read again by
// B1), 22-25 R3, 26-30 B2 and R2, 31-33 B3 and R1, 34 B4.  The first tile of a
// CTA starts with 0-5; every tile then streams 6-30, 31-33, 34, with the next
// tile's F1 (0), F2 (1) and F3 (2-5) slotted in after 30, 33 and 34.
__device__ __forceinline__ int stream_count(bool first, bool next) {
  return (first ? 6 : 0) + 29 + (next ? 6 : 0);
}
__device__ __forceinline__ int stream_unit(bool first, bool next, int j) {
  if (first) {
    if (j < 6) return j;
    j -= 6;
  }
  if (j < 25) return 6 + j;                 // 6..30
  j -= 25;
  if (next) {
    if (j == 0) return 0;                   // F1 of the next tile
    if (j <= 3) return 30 + j;              // 31..33
    if (j == 4) return 1;                   // F2 of the next tile
    if (j == 5) return 34;
    return j - 4;                           // 2..5: F3 of the next tile
  }
  return j < 3 ? 31 + j : 34;
}

__global__ void __launch_bounds__(kFusedThreads, 1)
decode_fused_kernel(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + SM_BAR);
  uint64_t* empty = full + kStages;
  uint64_t* accH = full + 2 * kStages;  // MMA -> epilogue: a forward hidden layer is done
  uint64_t* accT = accH + 1;            // MMA -> epilogue: a backward group is done
  uint64_t* opH = accT + 1;             // epilogue -> MMA: z / h1 / h2 / h3 staged
  uint64_t* opT = opH + 1;              // epilogue -> MMA: d1 written / dz read
  uint64_t* ybar = opT + 1;             // [2] output chunk ready in TMEM buffer c & 1
  // [2] epilogue -> MMA: dy chunk c written, on dyrdy[c & 1].  Two barriers,
  // because a warp may finish chunk c + 1 before a slower one has finished
  // chunk c (nothing else holds it back: the dy buffers alternate), and on
  // one barrier its second arrival would complete chunk c's phase early.  It
  // cannot reach chunk c + 2, whose output F4 c + 2 issues only after every
  // warp's chunk c, so each barrier sees one arrival per warp and phase.
  uint64_t* dyrdy = ybar + 2;
  uint64_t* drain = dyrdy + 2;          // a give-up waits here for the MMAs already issued
  // epilogue -> MMA, one phase per tile: 64-column slice s of h2 / h3 / d2 / d3
  // written (the next GEMM's K-slices start as soon as theirs are in)
  uint64_t* sh2 = drain + 1;            // [2]
  uint64_t* sh3 = sh2 + 2;              // [4]
  uint64_t* sd2 = sh3 + 4;              // [2]
  uint64_t* sd3 = sd2 + 2;              // [4]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sd3 + 4);
  float* sb = reinterpret_cast<float*>(sm + SM_BIAS);
  const float* sb4 = sb;
  const float* sb5 = sb + 64;
  const float* sb6 = sb + 192;
  const float* sb7 = sb + 448;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (a.P + 127) / 128;
  for (int i = tid; i < 960; i += kFusedThreads)
    sb[i] = i < 64 ? a.b4[i] : i < 192 ? a.b5[i - 64] : i < 448 ? a.b6[i - 192] : a.b7[i - 448];
  if (warp == 0) tc::tmem_alloc(tslot, 512);
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(accH, 1);
    tc::mbar_init(accT, 1);
    tc::mbar_init(opH, kEpiWarps);
    tc::mbar_init(opT, kEpiWarps);
    tc::mbar_init(&ybar[0], 1);
    tc::mbar_init(&ybar[1], 1);
    tc::mbar_init(&dyrdy[0], kEpiWarps);
    tc::mbar_init(&dyrdy[1], kEpiWarps);
    tc::mbar_init(drain, 1);
    for (int i = 0; i < 12; i++) tc::mbar_init(&sh2[i], kEpiWarps);  // sh2 .. sd3
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t sbase = tc::smem_addr(sm);

  if (warp >= kEpiWarps + 1) {
    // ---------------------------------------------------------------- producers
    // The bulk copies one warp issues one after another do not overlap (a
    // ring fed by one warp moves about 25 B/cycle per SM on GB300, two warps
    // about 30, four about 55), so kProducers warps share the stream:
    // producer pp copies the units with u % kProducers == pp.  Two, because
    // the stream runs ahead of the MMA warp here, and four warps (21 in all)
    // would cap the epilogue at 80 registers a thread, which costs more.
    const uint32_t pp = (uint32_t)(warp - kEpiWarps - 1);
    if (lane == 0) {
      uint32_t u = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const bool first = t == blockIdx.x, next = t + gridDim.x < ntiles;
        const int n = stream_count(first, next);
        for (int j = 0; j < n; j++, u++) {
          if (u % kProducers != pp) continue;
          const int i = stream_unit(first, next, j);
          const uint32_t s = u % kStages, round = u / kStages;
          if (round > 0 && !tc::mbar_wait(&empty[s], (round - 1) & 1, kLimit)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&full[s], a.bytes[i]);
          tc::bulk_g2s(sbase + SM_ST + s * kStageBytes, a.pack + a.off[i], a.bytes[i], &full[s]);
        }
      }
      if (!ok) atomicOr(&g_fused_error, 1u);
      // before the CTA leaves, this producer's copies among the last kStages
      // units have landed (no stage was refilled after them; the MMA warp has
      // waited for them already unless it gave up)
      for (uint32_t v = u > kStages ? u - kStages : 0; v < u; v++)
        if (v % kProducers == pp) tc::mbar_wait(&full[v % kStages], (v / kStages) & 1, kLimit);
    }
  } else if (warp == kEpiWarps) {
    // ---------------------------------------------------------------- MMA issuer
    // The whole warp walks the schedule (so descriptors and loop state stay
    // warp-uniform) and votes on every wait; one elected lane issues the MMAs
    // and commits.  Descriptors are a base plus compile-time offsets.
    uint32_t u = 0, nopH = 0, nopT = 0;
    bool ok = true;
    const uint64_t dbase = tc::sdesc_base(sbase);
    auto wait_on = [&](uint64_t* bar, uint32_t& n) {
      ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(bar, n & 1, kLimit));
      n++;
      tc::fence_after();
    };
    auto commit = [&](uint64_t* bar) {
      if (ok && tc::elect_one()) tc::commit(bar);
      __syncwarp();
    };
    // a slice barrier completes once per tile: parity = the tile's parity
    auto wait_slice = [&](uint64_t* bar, uint32_t parity) {
      ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(bar, parity, kLimit));
      tc::fence_after();
    };
    // one weight unit: B = ring stage, A = activation tile at a_off (width
    // a_kw) from column k0, D = TMEM column dcol, N = n, K = kc; the stage is
    // released after its MMAs unless `hold` (an output unit, read again by
    // its chunk's B1); returns the stage.  With a_tcol >= 0, A is in TMEM from
    // that column instead
    auto unit = [&](uint32_t a_off, int a_kw, int k0, int kc, int n, uint32_t dcol, bool fresh,
                    bool hold = false, int a_tcol = -1) -> uint32_t {
      const uint32_t s = u % kStages, round = u / kStages;
      if (!ok) return s;
      ok = __all_sync(0xffffffffu, tc::mbar_wait(&full[s], round & 1, kLimit));
      if (!ok) return s;
      tc::fence_after();
      const uint64_t ad = dbase + tc::sdesc_off(a_off + (uint32_t)k0 * 16, (uint32_t)a_kw * 16);
      const uint64_t bd = dbase + tc::sdesc_off(SM_ST + s * kStageBytes, (uint32_t)kc * 16);
      const uint32_t idesc = tc::idesc_bf16(128, n);
      if (tc::elect_one()) {
        for (int j = 0; j < kc / 16; j++) {
          if (a_tcol >= 0)
            tc::mma_bf16_ts(tmem + dcol, tmem + (uint32_t)a_tcol + 8 * j, bd + 16 * j, idesc,
                            (fresh && j == 0) ? 0u : 1u);
          else
            tc::mma_bf16(tmem + dcol, ad + 16 * j, bd + 16 * j, idesc,
                         (fresh && j == 0) ? 0u : 1u);
        }
        if (!hold) tc::commit(&empty[s]);
      }
      __syncwarp();
      u++;
      return s;
    };
    // forward hidden layers into TMEM columns 256-511 (z in buffer zb)
    auto f1 = [&](uint32_t zb) { unit(zb, 16, 0, 16, 64, 256, true); commit(accH); };
    auto f2 = [&]() { unit(SM_H1, 64, 0, 64, 128, 256, true); commit(accH); };
    // F3 overwrites TMEM columns 256-511, where E2 reads F2's accumulator
    // until its last slice: it waits for both slices of h2
    auto f3 = [&](uint32_t parity) {
      wait_slice(&sh2[1], parity);                                   // h2 staged
      for (int k = 0; k < 4; k++) unit(SM_H2, 128, 32 * k, 32, 256, 256, k == 0);
      commit(accH);
    };
    if (blockIdx.x < ntiles) {
      wait_on(opH, nopH);                                            // z staged
      f1(SM_Z);
      wait_on(opH, nopH);                                            // h1 staged
      f2();
      f3(0);
    }
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, k++) {
      const bool next = t + gridDim.x < ntiles;
      const uint32_t zc = SM_Z + (uint32_t)(k & 1) * 4096, zn = SM_Z + (uint32_t)((k + 1) & 1) * 4096;
      const uint32_t par = (uint32_t)(k & 1);
      if (k > 0) wait_on(opT, nopT);                                 // dz of the last tile read
      // output chunk c (64 columns) -> TMEM buffer c & 1 (columns 256 + 64 (c &
      // 1)), announced on ybar[c & 1]; its two units stay in their stages
      // (held[c & 1]) until B1 c has read them.  Chunk 0's K-halves start as
      // the slices of h3 land; its buffer holds F3's columns 0-63 until E3
      // has read slice 0, which slice 1's arrival implies
      uint32_t held[2][2];
      auto f4 = [&](int c) {
        for (int h = 0; h < 2; h++) {
          if (c == 0) wait_slice(&sh3[2 * h + 1], par);             // h3 slices staged
          held[c & 1][h] = unit(SM_H3, 256, 128 * h, 128, 64, 256 + 64 * (c & 1), h == 0, true);
        }
        commit(&ybar[c & 1]);
      };
      // B1 c: dh3[:, 128 h ..] += dy_c W7[64 c .., 128 h ..]^T, A = dy_c in
      // TMEM buffer c & 1, B = the held unit h as an MN-major operand (K = the
      // chunk's 64 outputs, core matrices 2 KB apart; N = 128 of h3's columns,
      // 128 B apart); then both stages are released.  The epilogue refills
      // buffer c & 1 with chunk c + 2 only after ybar announces F4 c + 2,
      // which this thread issues after B1 c, so the commit covers B1 c too
      const uint32_t idesc_b1 = tc::idesc_bf16(128, 128) | (1u << 16);
      auto b1 = [&](int c) {
        if (!ok) return;
        if (tc::elect_one()) {
          for (int h = 0; h < 2; h++) {
            const uint32_t st = sbase + SM_ST + held[c & 1][h] * kStageBytes;
            for (int j = 0; j < 4; j++)
              tc::mma_bf16_ts(tmem + 128 * h, tmem + TM_DY + 32 * (c & 1) + 8 * j,
                              tc::sdesc(st + (uint32_t)j * 4096, 2048, 128), idesc_b1,
                              (c == 0 && j == 0) ? 0u : 1u);
          }
          tc::commit(&empty[held[c & 1][0]]);
          tc::commit(&empty[held[c & 1][1]]);
        }
        __syncwarp();
      };
      f4(0);
      f4(1);
#pragma unroll
      for (int c = 0; c < 8; c++) {
        wait_slice(&dyrdy[c & 1], (uint32_t)(c >> 1) & 1u);          // dy chunk c written
        b1(c);
        if (c < 6) f4(c + 2);
      }
      for (int kk = 0; kk < 4; kk++) unit(SM_H2, 128, 32 * kk, 32, 256, 256, kk == 0);  // R3
      commit(accT);
      // B2 writes TMEM columns 0-127, E5's dh3 input of slices 0 and 1: it
      // starts after slice 1, its later K-slices as theirs land; R2 (columns
      // 128-255) after the last
      for (int kk = 0; kk < 4; kk++) {                                                   // B2
        if (kk != 1) wait_slice(&sd3[kk == 0 ? 1 : kk], par);        // d3 slices written
        unit(SM_H3, 256, 64 * kk, 64, 128, 0, kk == 0);
      }
      unit(SM_H1, 64, 0, 64, 128, 128, true);                        // R2
      commit(accT);
      if (next) {
        wait_on(opH, nopH);                                          // next z staged
        f1(zn);
      }
      // B3 writes TMEM columns 0-63 (E6's slice 0 input); R1 (64-127) after
      // slice 1
      for (int kk = 0; kk < 2; kk++) {                                                   // B3
        wait_slice(&sd2[kk], par);                                   // d2 slice written
        unit(SM_H2, 128, 64 * kk, 64, 64, 0, kk == 0);
      }
      unit(zc, 16, 0, 16, 64, 64, true);                             // R1
      commit(accT);
      if (next) {
        wait_on(opH, nopH);                                          // next h1 staged
        f2();
      }
      wait_on(opT, nopT);                                            // d1 written
      unit(0, 64, 0, 64, 16, 0, true, false, (int)TM_D1);            // B4 (A = d1 in TMEM)
      commit(accT);
      if (next) f3(par ^ 1u);
    }
    if (!ok) {  // the MMAs issued so far finish before TMEM is released
      if (lane == 0) atomicOr(&g_fused_error, 2u);
      if (tc::elect_one()) tc::commit(drain);
      __syncwarp();
      tc::mbar_wait(drain, 0, kLimit);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // warp w reads TMEM lane quadrant w % 4 (rows 32 (w % 4) ..) and the
    // column quarter w / 4 of every accumulator
    const int q = warp & 3, qq = warp >> 2;
    const int r = 32 * q + lane;
    const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16);
    uint32_t nH = 0, nT = 0;
    bool ok = true;
    float lsum = 0.f;
    const uint32_t sbf = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a.scale));
    const uint32_t s2bf = sbf | (sbf << 16);  // BF16 scale in both halves
    auto wait_acc = [&](uint64_t* bar, uint32_t& n) {
      ok = ok && tc::mbar_wait(bar, n & 1, kLimit);
      n++;
      tc::fence_after();
    };
    // every thread publishes its shared-memory writes to the async proxy and
    // orders its TMEM loads; one lane per warp then arrives for the warp
    auto arrive = [&](uint64_t* bar) {
      tc::fence_async_smem();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(bar);
    };
    // the same after TMEM accesses only (no shared-memory writes to publish)
    auto arrive_tmem = [&](uint64_t* bar) {
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(bar);
    };
    // E0: z (f32) of tile t -> bf16 A operand in buffer zb, columns [8 qq, 8 qq + 8)
    auto stage_z = [&](int64_t t, uint32_t zb) {
      if (qq < 2) {
        const int64_t p = t * 128 + r;
        float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0;
        if (p < a.P) {
          const float4* src = reinterpret_cast<const float4*>(a.z + p * 16 + 8 * qq);
          f0 = src[0];
          f1 = src[1];
        }
        uint4 u;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
        h[0] = __floats2bfloat162_rn(f0.x, f0.y);
        h[1] = __floats2bfloat162_rn(f0.z, f0.w);
        h[2] = __floats2bfloat162_rn(f1.x, f1.y);
        h[3] = __floats2bfloat162_rn(f1.z, f1.w);
        *reinterpret_cast<uint4*>(sm + zb + tc::core_offset(r, qq, 16)) = u;
      }
      arrive(opH);
    };
    float v[32], pre[32];
    // E1..E3: forward hidden layers from TMEM columns 256-511 (this warp's
    // column quarter), GELU, BF16 activations into shared memory
    auto e1 = [&]() {
      wait_acc(accH, nH);
      const int c0 = 16 * qq;
      tc::tmem_ld16(tb + 256 + c0, v);
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const float2 g = gelu_tanh2(__fadd2_rn(f2(v[i], v[i + 1]),
                                               *reinterpret_cast<const float2*>(sb4 + c0 + i)));
        v[i] = g.x;
        v[i + 1] = g.y;
      }
      put_row<16>(sm + SM_H1, r, c0, 64, v);
      arrive(opH);
    };
    // GELU of NS consecutive 16-column slices from column c0 of the forward
    // accumulator into the BF16 tile (width kw); the next slice's TMEM load
    // is in flight while a slice is computed
    // slice s of NS: columns c0 + 64 s .. + 15 of this warp (the four column
    // quarters together write 64-column slice s, announced on bars[s])
    auto gelu_slices = [&](auto ns, int c0, const float* bias, uint8_t* tile, int kw,
                           uint64_t* bars) {
      constexpr int NS = decltype(ns)::value;
      uint32_t ra[16], rb[16];
      tc::tmem_ld16_issue(tb + 256 + c0, ra);
      tc::tmem_wait16(ra);
#pragma unroll
      for (int s2 = 0; s2 < NS; s2++) {
        const int cc = c0 + 64 * s2;
        uint32_t* cur = (s2 & 1) ? rb : ra;
        uint32_t* nxt = (s2 & 1) ? ra : rb;
        if (s2 + 1 < NS) tc::tmem_ld16_issue(tb + 256 + cc + 64, nxt);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const float2 g = gelu_tanh2(
              __fadd2_rn(f2(__uint_as_float(cur[i]), __uint_as_float(cur[i + 1])),
                         *reinterpret_cast<const float2*>(bias + cc + i)));
          v[i] = g.x;
          v[i + 1] = g.y;
        }
        put_row<16>(tile, r, cc, kw, v);
        arrive(&bars[s2]);
        if (s2 + 1 < NS) tc::tmem_wait16(nxt);
      }
    };
    auto e2 = [&]() {
      wait_acc(accH, nH);
      gelu_slices(std::integral_constant<int, 2>(), 16 * qq, sb5, sm + SM_H2, 128, sh2);
    };
    auto e3 = [&]() {
      wait_acc(accH, nH);
      gelu_slices(std::integral_constant<int, 4>(), 16 * qq, sb6, sm + SM_H3, 256, sh3);
    };
    // F_gt of output chunk c of tile t: this lane's row, this warp's 16
    // columns, one 32-byte load (a whole sector; F_gt is 32-byte aligned, so
    // the warp's load touches 32 sectors and uses every byte of them).  (The
    // same bytes as two 16-byte loads per lane cost twice the sector requests
    // and were slower; 16 rows x 32 bytes per instruction then a transpose
    // through shared memory, 0.302 ms against 0.297.)
    uint4 ld[2];
    auto load_fgt = [&](int64_t t, int c) {
      const int64_t pr = t * 128 + r;
      ld[0] = ld[1] = make_uint4(0u, 0u, 0u, 0u);
      if (pr < a.P) {
        const __nv_bfloat16* ptr = a.target + pr * 512 + 64 * c + 16 * qq;
        asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(ld[0].x), "=r"(ld[0].y), "=r"(ld[0].z), "=r"(ld[0].w), "=r"(ld[1].x),
                       "=r"(ld[1].y), "=r"(ld[1].z), "=r"(ld[1].w)
                     : "l"(ptr));
      }
    };
    if (blockIdx.x < ntiles) {
      const int64_t t = blockIdx.x;
      stage_z(t, SM_Z);
      e1();
      e2();
      load_fgt(t, 0);
      e3();
    }
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, k++) {
      const bool next = t + gridDim.x < ntiles;
      const int64_t p = t * 128 + r;
      const bool valid = p < a.P;
      // E4: output chunks, L1 against F_gt, dy into the chunk buffer
#pragma unroll 1
      for (int c = 0; c < 8; c++) {
        const uint4 tg[2] = {ld[0], ld[1]};  // F_gt of this row's 16 columns
        if (c < 7) load_fgt(t, c + 1);
        const int n0 = 64 * c + 16 * qq;
        ok = ok && tc::mbar_wait(&ybar[c & 1], (c >> 1) & 1, kLimit);
        tc::fence_after();
        // 16 columns; dy = +-scale or 0, packed to BF16 at once
        uint4 dy[2];
        uint32_t ya[16];
        float lc = 0.f;  // this chunk's sum of |d|
        bool anyz = false;
        const uint32_t ycol = tb + 256 + 64 * (c & 1) + 16 * qq;
        tc::tmem_ld16_issue(ycol, ya);
        tc::tmem_wait16(ya);
        // the BF16 pair of sign(d) * scale: d's sign bits applied to the BF16
        // pattern of scale; a d that is exactly 0 (its gradient is 0) only
        // raises anyz here and is handled below
#pragma unroll
        for (int kk = 0; kk < 2; kk++) {
          const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&tg[kk]);
          __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(&dy[kk]);
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const float2 nt = neg_bf16x2(h2[e]);
            const int i = 8 * kk + 2 * e;
            const float2 dd = __fadd2_rn(
                __fadd2_rn(f2(__uint_as_float(ya[i]), __uint_as_float(ya[i + 1])),
                           *reinterpret_cast<const float2*>(sb7 + n0 + i)),
                nt);
            lc += fabsf(dd.x) + fabsf(dd.y);
            anyz |= (dd.x == 0.f) | (dd.y == 0.f);
            reinterpret_cast<uint32_t*>(o2)[e] =
                (__byte_perm(__float_as_uint(dd.x), __float_as_uint(dd.y), 0x7632) & 0x80008000u) ^
                s2bf;
          }
        }
        if (__any_sync(0xffffffffu, anyz)) {
          // rare: some d of the warp is exactly 0; the warp reloads the chunk
          // (the TMEM load is warp-collective) and zeroes those halves
          tc::tmem_ld16_issue(ycol, ya);
          tc::tmem_wait16(ya);
#pragma unroll
          for (int kk = 0; kk < 2; kk++) {
            const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&tg[kk]);
            uint32_t* o = reinterpret_cast<uint32_t*>(&dy[kk]);
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const float2 nt = neg_bf16x2(h2[e]);
              const int i = 8 * kk + 2 * e;
              const float2 dd = __fadd2_rn(
                  __fadd2_rn(f2(__uint_as_float(ya[i]), __uint_as_float(ya[i + 1])),
                             *reinterpret_cast<const float2*>(sb7 + n0 + i)),
                  nt);
              if (dd.x == 0.f) o[e] &= 0xffff0000u;
              if (dd.y == 0.f) o[e] &= 0x0000ffffu;
            }
          }
        }
        if (valid) {
          lsum += lc;
        } else {  // rows past the end carry no loss and no gradient
          dy[0] = make_uint4(0u, 0u, 0u, 0u);
          dy[1] = make_uint4(0u, 0u, 0u, 0u);
        }
        // dy into TMEM buffer c & 1 (this warp's 16 columns = 8 TMEM columns),
        // whose last reader B1 c - 2 finished before ybar announced chunk c
        tc::tmem_st8(tb + TM_DY + 32 * (c & 1) + 8 * qq, reinterpret_cast<const uint32_t*>(dy));
        tc::tmem_wait_st();
        arrive_tmem(&dyrdy[c & 1]);
      }
      // E5: d3 = dh3 * gelu'(pre3), 64-column slice s by all 16 warps in step
      // s (this warp: columns 16 qq + 64 s ..), each slice announced on sd3[s]
      wait_acc(accT, nT);
      {  // the next slice's loads are in flight while this one is computed
        uint32_t ra[32], rb[32];
        tc::tmem_ld16x2_issue(tb + 16 * qq, tb + 256 + 16 * qq, ra);
        tc::tmem_wait32(ra);
#pragma unroll
        for (int s2 = 0; s2 < 4; s2++) {
          const int c0 = 16 * qq + 64 * s2;
          uint32_t* cur = (s2 & 1) ? rb : ra;
          uint32_t* nxt = (s2 & 1) ? ra : rb;
          if (s2 < 3) tc::tmem_ld16x2_issue(tb + c0 + 64, tb + 256 + c0 + 64, nxt);
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const float2 g = gelu_tanh_grad2(__fadd2_rn(
                f2(__uint_as_float(cur[16 + i]), __uint_as_float(cur[17 + i])),
                *reinterpret_cast<const float2*>(sb6 + c0 + i)));
            const float2 d =
                __fmul2_rn(f2(__uint_as_float(cur[i]), __uint_as_float(cur[i + 1])), g);
            v[i] = d.x;
            v[i + 1] = d.y;
          }
          put_row<16>(sm + SM_H3, r, c0, 256, v);
          arrive(&sd3[s2]);
          if (s2 < 3) tc::tmem_wait32(nxt);
        }
      }
      if (next) stage_z(t + gridDim.x, SM_Z + (uint32_t)((k + 1) & 1) * 4096);
      // E6: d2 = dh2 * gelu'(pre2), 64-column slices as in E5, on sd2[s]
      wait_acc(accT, nT);
      {
        uint32_t ra[32], rb[32];
        tc::tmem_ld16x2_issue(tb + 16 * qq, tb + 128 + 16 * qq, ra);
        tc::tmem_wait32(ra);
#pragma unroll
        for (int s2 = 0; s2 < 2; s2++) {
          const int c0 = 16 * qq + 64 * s2;
          uint32_t* cur = (s2 & 1) ? rb : ra;
          uint32_t* nxt = (s2 & 1) ? ra : rb;
          if (s2 < 1) tc::tmem_ld16x2_issue(tb + c0 + 64, tb + 128 + c0 + 64, nxt);
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const float2 g = gelu_tanh_grad2(__fadd2_rn(
                f2(__uint_as_float(cur[16 + i]), __uint_as_float(cur[17 + i])),
                *reinterpret_cast<const float2*>(sb5 + c0 + i)));
            const float2 d =
                __fmul2_rn(f2(__uint_as_float(cur[i]), __uint_as_float(cur[i + 1])), g);
            v[i] = d.x;
            v[i + 1] = d.y;
          }
          put_row<16>(sm + SM_H2, r, c0, 128, v);
          arrive(&sd2[s2]);
          if (s2 < 1) tc::tmem_wait32(nxt);
        }
      }
      if (next) e1();
      // E7: d1 = dh1 * gelu'(pre1), into TMEM columns TM_D1.. (pre2's: every
      // warp has read them in E6, which R1's commit implies)
      wait_acc(accT, nT);
      {
        const int c0 = 16 * qq;
        tc::tmem_ld16x2(tb + c0, v, tb + 64 + c0, pre);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const float2 g = gelu_tanh_grad2(__fadd2_rn(
              f2(pre[i], pre[i + 1]), *reinterpret_cast<const float2*>(sb4 + c0 + i)));
          const float2 d = __fmul2_rn(f2(v[i], v[i + 1]), g);
          v[i] = d.x;
          v[i + 1] = d.y;
        }
        // BF16 pairs into TMEM columns TM_D1 + 8 qq .. (B4's A operand)
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
          pk[i] = *reinterpret_cast<const uint32_t*>(&h);
        }
        tc::tmem_st8(tb + TM_D1 + 8 * qq, pk);
        tc::tmem_wait_st();
      }
      arrive_tmem(opT);
      if (next) e2();
      // E8: dz
      wait_acc(accT, nT);
      if (qq == 0) {
        tc::tmem_ld16(tb, v);
        if (valid) {
          float4* dst = reinterpret_cast<float4*>(a.dz + p * 16);
#pragma unroll
          for (int kk = 0; kk < 4; kk++)
            dst[kk] = make_float4(v[4 * kk], v[4 * kk + 1], v[4 * kk + 2], v[4 * kk + 3]);
        }
      }
      arrive_tmem(opT);
      if (next) {
        load_fgt(t + gridDim.x, 0);
        e3();
      }
    }
    if (!ok) atomicOr(&g_fused_error, 4u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(a.loss, lsum * a.scale);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

struct Plan {
  std::vector<Unit> units;
  uint32_t off[kUnits], bytes[kUnits], piece0[kUnits + 1];
  size_t total;
};

const Plan& plan() {
  static Plan P;
  static std::once_flag once;
  std::call_once(once, [] {
    P.units = schedule();
    uint32_t o = 0, pc = 0;
    for (int i = 0; i < kUnits; i++) {
      const Unit& U = P.units[i];
      P.off[i] = o;
      P.bytes[i] = (uint32_t)(U.rows * U.kc * 2);
      P.piece0[i] = pc;
      o += P.bytes[i];
      pc += (uint32_t)(U.rows * (U.kc / 8));
    }
    P.piece0[kUnits] = pc;
    P.total = o;
  });
  return P;
}

}  // namespace

size_t decode_pack_bytes() { return (plan().total + 255) & ~(size_t)255; }

lgs_status launch_decode_pack(const lgs_ae_weights* w, void* pack, cudaStream_t s) {
  const Plan& pl = plan();
  if ((int)pl.units.size() != kUnits) {
    set_error("decoder schedule size mismatch");
    return LGS_ERR_INVALID;
  }
  PackArgs pa;
  for (int m = 0; m < 4; m++) {
    pa.mats[m] = reinterpret_cast<const __nv_bfloat16*>(w->W[4 + m]);
    pa.mats[4 + m] = reinterpret_cast<const __nv_bfloat16*>(w->Wt[4 + m]);
  }
  for (int m = 0; m < 8; m++) pa.ld[m] = kCols[m];
  for (int i = 0; i < kUnits; i++) {
    pa.units[i] = pl.units[i];
    pa.off[i] = pl.off[i];
    pa.piece0[i] = pl.piece0[i];
  }
  pa.piece0[kUnits] = pl.piece0[kUnits];
  pa.pack = static_cast<uint8_t*>(pack);
  pack_units_kernel<<<(pl.piece0[kUnits] + 255) / 256, 256, 0, s>>>(pa);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

lgs_status launch_decode_fused(const lgs_ae_weights* w, const float* z, int64_t P,
                               const uint16_t* target, float weight, float* loss, float* dz,
                               void* pack, bool packed, cudaStream_t s) {
  const Plan& pl = plan();
  if (!packed) {
    const lgs_status st = launch_decode_pack(w, pack, s);
    if (st != LGS_OK) return st;
  }
  FusedArgs fa;
  fa.pack = static_cast<const uint8_t*>(pack);
  for (int i = 0; i < kUnits; i++) {
    fa.off[i] = pl.off[i];
    fa.bytes[i] = pl.bytes[i];
  }
  fa.b4 = w->b[4];
  fa.b5 = w->b[5];
  fa.b6 = w->b[6];
  fa.b7 = w->b[7];
  fa.z = z;
  fa.target = reinterpret_cast<const __nv_bfloat16*>(target);
  fa.dz = dz;
  fa.P = P;
  fa.scale = weight / ((float)P * 512.f);
  fa.loss = loss;
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(decode_fused_kernel), (int)SM_ALL));
  const int64_t ntiles = (P + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntiles, sm_count());
  decode_fused_kernel<<<grid, kFusedThreads, SM_ALL, s>>>(fa);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

unsigned fused_error_word(bool clear) {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_fused_error, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) cudaMemcpyToSymbol(g_fused_error, &zero, sizeof(zero));
  return v;
}

}  // namespace lgs
