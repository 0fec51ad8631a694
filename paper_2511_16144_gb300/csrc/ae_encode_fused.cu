// Fused encoder E_phi (LEGO-SLAM Sec. IV-A.2; the encoder prior of
// Sec. III-B.2 and the adaptation target of Eq. 3): z = E(x) for 128-pixel
// tiles, 512 -> 256 -> 128 -> 64 -> 16 with GELU (tanh form) after the first
// three layers and a linear latent, in one persistent kernel.
//
// Per tile, on the tensor cores (BF16 operands, FP32 accumulators in TMEM):
//   L0  x [128 x 512] W0^T in 16 K-steps of 32 columns: each ring stage holds
//       the x chunk (one 2-D TMA load in the 64-byte swizzle layout: 128 rows
//       of 64 bytes, each byte fetched once) and the matching 256 x 32 slice
//       of W0 (a bulk copy of a pre-packed unit);
//   L1..L3  the hidden activations stay in shared memory (BF16) and only
//       the weight units stream through the ring.
// Consecutive tiles of a CTA alternate TMEM halves (columns 0-255 / 256-511),
// so the tensor core runs the next tile's L0 while the epilogue warps apply
// GELU to the current tile's L0 accumulator.
// Warps 0-15 are the epilogue (warps w, w + 4, w + 8, w + 12 share TMEM lane
// quadrant w % 4 and split the columns in quarters), warp 16 issues the MMAs
// (converged; one elected lane issues), warps 17 and 18 stream the units.
// Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc05.cuh"

namespace lgs {

namespace {

constexpr int kUnits = 22;  // 16 L0 slices, 4 L1, 1 L2, 1 L3
constexpr int kStages = 4;
constexpr uint32_t kXBytes = 8192;     // x chunk: 128 rows x 32 columns
constexpr uint32_t kWBytes = 16384;    // largest weight unit
constexpr uint32_t kStageBytes = kXBytes + kWBytes;
constexpr uint32_t kLimit = 1u << 22;
constexpr int kEpiWarps = 16;
constexpr int kThreads = (kEpiWarps + 3) * 32;

// shared-memory map (bytes)
constexpr uint32_t SM_ST = 0;                              // ring
constexpr uint32_t SM_H1 = SM_ST + kStages * kStageBytes;  // 128 x 256 bf16
constexpr uint32_t SM_H2 = SM_H1 + 65536;                  // 128 x 128
constexpr uint32_t SM_H3 = SM_H2 + 32768;                  // 128 x 64
constexpr uint32_t SM_BAR = SM_H3 + 16384;
constexpr uint32_t SM_BIAS = SM_BAR + 256;                 // b0 | b1 | b2 | b3 (464 floats)
constexpr uint32_t SM_ALL = SM_BIAS + 464 * 4;
static_assert(SM_ALL <= 232448, "shared-memory map exceeds 227 KB");

struct EncUnit {
  int mat, row0, rows, col0, kc;
};

EncUnit enc_unit(int i) {
  if (i < 16) return {0, 0, 256, 32 * i, 32};
  if (i < 20) return {1, 0, 128, 64 * (i - 16), 64};
  if (i == 20) return {2, 0, 64, 0, 128};
  return {3, 0, 16, 0, 64};
}

struct EncPackArgs {
  const __nv_bfloat16* mats[4];
  EncUnit units[kUnits];
  uint32_t off[kUnits];
  uint32_t piece0[kUnits + 1];
  uint8_t* pack;
};

// Every unit as [rows/8][kc/8][8][8] bf16 core matrices.
__global__ void enc_pack_kernel(EncPackArgs a) {
  const uint32_t total = a.piece0[kUnits];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int u = 0;
    while (a.piece0[u + 1] <= i) u++;
    const EncUnit U = a.units[u];
    const uint32_t j = i - a.piece0[u];
    const int per_row = U.kc / 8;
    const int r = (int)(j / per_row), c = (int)(j % per_row);
    const __nv_bfloat16* src = a.mats[U.mat] + (int64_t)(U.row0 + r) * (512 >> U.mat) + U.col0 + 8 * c;  // K of W_l: 512 >> l
    *reinterpret_cast<uint4*>(a.pack + a.off[u] + tc::core_offset(r, c, U.kc)) =
        *reinterpret_cast<const uint4*>(src);
  }
}

struct EncArgs {
  const uint8_t* pack;
  uint32_t off[kUnits];
  uint32_t bytes[kUnits];
  const float* b[4];
  float* z;
  int64_t P;
};

__device__ unsigned g_enc_error;

// The ring's unit order: L0 of local tiles 0 and 1, then per local tile k:
// L1, L2, L3 of tile k (6 units) and, while tile k + 2 exists, its L0 (16).
// Position j of that order as (unit, local tile whose x it needs, or -1).
__device__ __forceinline__ void ring_unit(int j, int nloc, int& unit, int& tile) {
  const int head = 16 * (nloc < 2 ? nloc : 2);
  if (j < head) {
    unit = j & 15;
    tile = j >> 4;
    return;
  }
  j -= head;
  const int kfull = nloc > 2 ? nloc - 2 : 0;  // tiles followed by an L0
  if (j < 22 * kfull) {
    const int k = j / 22, r = j % 22;
    if (r < 6) {
      unit = 16 + r;
      tile = -1;
    } else {
      unit = r - 6;
      tile = k + 2;
    }
    return;
  }
  unit = 16 + (j - 22 * kfull) % 6;
  tile = -1;
}
// 16 L0 units and 6 small ones per tile
__device__ __forceinline__ int ring_count(int nloc) { return 22 * (nloc > 0 ? nloc : 0); }

__global__ void __launch_bounds__(kThreads, 1)
encode_fused_kernel(const __grid_constant__ EncArgs a, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + SM_BAR);
  uint64_t* empty = full + kStages;
  uint64_t* accL0 = empty + kStages;  // [2] MMA -> epilogue: L0 of a tile in TMEM half p
  uint64_t* accS = accL0 + 2;         // MMA -> epilogue: L1 / L2 / L3 done
  uint64_t* opL0 = accS + 1;          // epilogue -> MMA: L0 read out, h1 staged
  uint64_t* opS = opL0 + 1;           // epilogue -> MMA: h2 / h3 staged, z written
  uint64_t* drain = opS + 1;          // a give-up waits here for the MMAs already issued
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  float* sb = reinterpret_cast<float*>(sm + SM_BIAS);
  const float* sb0 = sb;
  const float* sb1 = sb + 256;
  const float* sb2 = sb + 384;
  const float* sb3 = sb + 448;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (a.P + 127) / 128;
  const int nloc = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  if (tc::smem_addr(sm) & 1023u) {  // the swizzled x chunks need 1 KB-aligned stages
    if (tid == 0) atomicOr(&g_enc_error, 8u);
    return;
  }
  for (int i = tid; i < 464; i += kThreads)
    sb[i] = i < 256 ? a.b[0][i] : i < 384 ? a.b[1][i - 256] : i < 448 ? a.b[2][i - 384] : a.b[3][i - 448];
  if (warp == 0) tc::tmem_alloc(tslot, 512);
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&accL0[0], 1);
    tc::mbar_init(&accL0[1], 1);
    tc::mbar_init(accS, 1);
    tc::mbar_init(opL0, kEpiWarps);
    tc::mbar_init(opS, kEpiWarps);
    tc::mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t sbase = tc::smem_addr(sm);

  if (warp >= kEpiWarps + 1) {
    // ---------------------------------------------------------------- producers
    const int pp = warp - kEpiWarps - 1;
    if (lane == 0) {
      bool ok = true;
      const int n = ring_count(nloc);
      int j = pp;
      for (; j < n && ok; j += 2) {
        int unit, tl;
        ring_unit(j, nloc, unit, tl);
        const uint32_t s = (uint32_t)j % kStages, round = (uint32_t)j / kStages;
        if (round > 0 && !tc::mbar_wait(&empty[s], (round - 1) & 1, kLimit)) {
          ok = false;
          break;
        }
        const uint32_t st = sbase + SM_ST + s * kStageBytes;
        tc::mbar_expect_tx(&full[s], a.bytes[unit] + (tl >= 0 ? kXBytes : 0u));
        if (tl >= 0) {
          const int64_t t = blockIdx.x + (int64_t)tl * gridDim.x;
          tc::tma_load_2d(st, &xmap, 32 * unit, (int)(t * 128), &full[s]);
        }
        tc::bulk_g2s(st + kXBytes, a.pack + a.off[unit], a.bytes[unit], &full[s]);
      }
      if (!ok) atomicOr(&g_enc_error, 1u);
      // before the CTA leaves, this producer's last copies have landed (ring
      // positions j - 2, j - 4, ... down to j - kStages; a stage belongs to
      // one producer since kStages is even)
      static_assert(kStages % 2 == 0, "a ring stage must belong to one producer");
      for (int v = j - 2; v >= 0 && v >= j - kStages; v -= 2)
        tc::mbar_wait(&full[(uint32_t)v % kStages], ((uint32_t)v / kStages) & 1, kLimit);
    }
  } else if (warp == kEpiWarps) {
    // ---------------------------------------------------------------- MMA issuer
    uint32_t u = 0, nL0 = 0, nS = 0;
    bool ok = true;
    const uint64_t dbase = tc::sdesc_base(sbase);            // K-adjacent core matrices 128 B apart
    const uint64_t xbase = tc::sdesc_sw64(sbase);             // TMA-staged x: 64-byte swizzle
    auto wait_on = [&](uint64_t* bar, uint32_t& n) {
      ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(bar, n & 1, kLimit));
      n++;
      tc::fence_after();
    };
    auto commit = [&](uint64_t* bar) {
      if (ok && tc::elect_one()) tc::commit(bar);
      __syncwarp();
    };
    auto take = [&]() -> uint32_t {  // wait for the next ring stage
      const uint32_t s = u % kStages, round = u / kStages;
      ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(&full[s], round & 1, kLimit));
      tc::fence_after();
      return s;
    };
    auto give = [&](uint32_t s) {  // release it once its MMAs are done
      if (ok && tc::elect_one()) tc::commit(&empty[s]);
      __syncwarp();
      u++;
    };
    // L0 of the tile in TMEM half hb: 16 stages of x chunk + W0 slice, N = 256
    auto l0 = [&](uint32_t hb) {
      for (int ks = 0; ks < 16 && ok; ks++) {
        const uint32_t s = take();
        if (!ok) break;
        const uint32_t st = SM_ST + s * kStageBytes;
        const uint64_t ad = xbase + tc::sdesc_off(st, 0);
        const uint64_t bd = dbase + tc::sdesc_off(st + kXBytes, 32 * 16);
        if (tc::elect_one()) {
          // K-step of 16 columns: 32 bytes along the x rows, 2 core matrices of W0
#pragma unroll
          for (int j = 0; j < 2; j++)
            tc::mma_bf16(tmem + hb, ad + 2 * j, bd + 16 * j, tc::idesc_bf16(128, 256),
                         (ks | j) != 0);
        }
        __syncwarp();
        give(s);
      }
    };
    // a weight unit against an activation tile at a_off (width a_kw) from
    // column k0: N = n, K = kc
    auto unit = [&](uint32_t a_off, int a_kw, int k0, int kc, int n, uint32_t dcol, bool fresh) {
      const uint32_t s = take();
      if (!ok) return;
      const uint64_t ad = dbase + tc::sdesc_off(a_off + (uint32_t)k0 * 16, (uint32_t)a_kw * 16);
      const uint64_t bd = dbase + tc::sdesc_off(SM_ST + s * kStageBytes + kXBytes, (uint32_t)kc * 16);
      const uint32_t idesc = tc::idesc_bf16(128, n);
      if (tc::elect_one()) {
        for (int j = 0; j < kc / 16; j++)
          tc::mma_bf16(tmem + dcol, ad + 16 * j, bd + 16 * j, idesc, (fresh && j == 0) ? 0u : 1u);
      }
      __syncwarp();
      give(s);
    };
    if (nloc > 0) {
      l0(0);
      commit(&accL0[0]);
    }
    if (nloc > 1) {
      l0(256);
      commit(&accL0[1]);
    }
    for (int k = 0; k < nloc && ok; k++) {
      const uint32_t hb = 256u * (uint32_t)(k & 1);
      wait_on(opL0, nL0);                                          // h1 staged
      for (int kk = 0; kk < 4; kk++) unit(SM_H1, 256, 64 * kk, 64, 128, hb, kk == 0);   // L1
      commit(accS);
      wait_on(opS, nS);                                            // h2 staged
      unit(SM_H2, 128, 0, 128, 64, hb, true);                      // L2
      commit(accS);
      wait_on(opS, nS);                                            // h3 staged
      unit(SM_H3, 64, 0, 64, 16, hb, true);                        // L3
      commit(accS);
      wait_on(opS, nS);                                            // z read out
      if (k + 2 < nloc) {
        l0(hb);
        commit(&accL0[k & 1]);
      }
    }
    if (!ok) {  // the MMAs issued so far finish before TMEM is released
      if (lane == 0) atomicOr(&g_enc_error, 2u);
      if (tc::elect_one()) tc::commit(drain);
      __syncwarp();
      tc::mbar_wait(drain, 0, kLimit);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3, qq = warp >> 2;
    const int r = 32 * q + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    uint32_t nS = 0;
    bool ok = true;
    float v[16];
    auto wait_acc = [&](uint64_t* bar, uint32_t parity) {
      ok = ok && tc::mbar_wait(bar, parity, kLimit);
      tc::fence_after();
    };
    auto arrive = [&](uint64_t* bar) {
      tc::fence_async_smem();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(bar);
    };
    // GELU of NS 16-column slices of the accumulator at TMEM column tb + c0
    // into the BF16 tile of width kw (next slice's load in flight)
    auto gelu_slices = [&](auto ns, uint32_t tb, int c0, const float* bias, uint8_t* tile, int kw) {
      constexpr int NS = decltype(ns)::value;
      uint32_t ra[16], rb[16];
      tc::tmem_ld16_issue(tb + c0, ra);
      tc::tmem_wait16(ra);
#pragma unroll
      for (int s2 = 0; s2 < NS; s2++) {
        const int cc = c0 + 16 * s2;
        uint32_t* cur = (s2 & 1) ? rb : ra;
        uint32_t* nxt = (s2 & 1) ? ra : rb;
        if (s2 + 1 < NS) tc::tmem_ld16_issue(tb + cc + 16, nxt);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const float2 g = gelu_tanh2(
              __fadd2_rn(f2(__uint_as_float(cur[i]), __uint_as_float(cur[i + 1])),
                         *reinterpret_cast<const float2*>(bias + cc + i)));
          v[i] = g.x;
          v[i + 1] = g.y;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
          uint4 pk;
          __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
          for (int e = 0; e < 4; e++) h2[e] = __floats2bfloat162_rn(v[8 * h + 2 * e], v[8 * h + 2 * e + 1]);
          *reinterpret_cast<uint4*>(tile + tc::core_offset(r, cc / 8 + h, kw)) = pk;
        }
        if (s2 + 1 < NS) tc::tmem_wait16(nxt);
      }
    };
    for (int k = 0; k < nloc && ok; k++) {
      const int64_t t = blockIdx.x + (int64_t)k * gridDim.x;
      const int64_t p = t * 128 + r;
      const uint32_t tb = tq + 256u * (uint32_t)(k & 1);
      wait_acc(&accL0[k & 1], (uint32_t)(k >> 1) & 1);             // E0: L0 -> h1
      gelu_slices(std::integral_constant<int, 4>(), tb, 64 * qq, sb0, sm + SM_H1, 256);
      arrive(opL0);
      wait_acc(accS, nS++ & 1);                                    // E1: L1 -> h2
      gelu_slices(std::integral_constant<int, 2>(), tb, 32 * qq, sb1, sm + SM_H2, 128);
      arrive(opS);
      wait_acc(accS, nS++ & 1);                                    // E2: L2 -> h3
      gelu_slices(std::integral_constant<int, 1>(), tb, 16 * qq, sb2, sm + SM_H3, 64);
      arrive(opS);
      wait_acc(accS, nS++ & 1);                                    // E3: L3 -> z
      if (qq == 0) {
        tc::tmem_ld16(tb, v);
        if (p < a.P) {
          float4* dst = reinterpret_cast<float4*>(a.z + p * 16);
#pragma unroll
          for (int kk = 0; kk < 4; kk++)
            dst[kk] = make_float4(v[4 * kk] + sb3[4 * kk], v[4 * kk + 1] + sb3[4 * kk + 1],
                                  v[4 * kk + 2] + sb3[4 * kk + 2], v[4 * kk + 3] + sb3[4 * kk + 3]);
        }
      }
      arrive(opS);
    }
    if (!ok) atomicOr(&g_enc_error, 4u);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

struct EncPlan {
  uint32_t off[kUnits], bytes[kUnits], piece0[kUnits + 1];
  size_t total;
};

const EncPlan& enc_plan() {
  static EncPlan P;
  static std::once_flag once;
  std::call_once(once, [] {
    uint32_t o = 0, pc = 0;
    for (int i = 0; i < kUnits; i++) {
      const EncUnit U = enc_unit(i);
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

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

size_t encode_pack_bytes() { return (enc_plan().total + 255) & ~(size_t)255; }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 152;
  return n;
}

bool make_kmajor_map(CUtensorMap* map, const void* base, int64_t rows, int K, int box_rows,
                     int box_groups) {
  auto encode = tensor_map_encoder();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return false;
  }
  const cuuint64_t dims[3] = {8, (cuuint64_t)rows, (cuuint64_t)(K / 8)};
  const cuuint64_t strides[2] = {(cuuint64_t)K * 2, 16};
  const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, (cuuint32_t)box_groups}, es[3] = {1, 1, 1};
  const CUresult cr =
      encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled refused a K-major map");
    return false;
  }
  return true;
}

bool make_swizzled_map(CUtensorMap* map, const void* base, int64_t rows, int K, int box_cols,
                       int box_rows) {
  auto encode = tensor_map_encoder();
  if (!encode || (box_cols != 64 && box_cols != 32)) {
    set_error(encode ? "swizzled maps take 32- or 64-column boxes"
                     : "cuTensorMapEncodeTiled is unavailable");
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows}, es[2] = {1, 1};
  const CUresult cr = encode(
      map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
      CU_TENSOR_MAP_INTERLEAVE_NONE,
      box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled refused a swizzled map");
    return false;
  }
  return true;
}

lgs_status launch_encode_fused(const lgs_ae_weights* w, const uint16_t* x, int64_t P, float* z,
                               void* pack, cudaStream_t s) {
  const EncPlan& pl = enc_plan();
  // x [P, 512] bf16 in 32-column x 128-row boxes with the 64-byte swizzle:
  // one box is one K-chunk of a tile, rows of 64 bytes in 512-byte atoms
  CUtensorMap xmap;
  if (!make_swizzled_map(&xmap, x, P, 512, 32, 128)) return LGS_ERR_CUDA;
  EncPackArgs pa;
  for (int m = 0; m < 4; m++) pa.mats[m] = reinterpret_cast<const __nv_bfloat16*>(w->W[m]);
  for (int i = 0; i < kUnits; i++) {
    pa.units[i] = enc_unit(i);
    pa.off[i] = pl.off[i];
    pa.piece0[i] = pl.piece0[i];
  }
  pa.piece0[kUnits] = pl.piece0[kUnits];
  pa.pack = static_cast<uint8_t*>(pack);
  enc_pack_kernel<<<(pl.piece0[kUnits] + 255) / 256, 256, 0, s>>>(pa);
  LGS_CHECK_LAUNCH();
  EncArgs ea;
  ea.pack = static_cast<const uint8_t*>(pack);
  for (int i = 0; i < kUnits; i++) {
    ea.off[i] = pl.off[i];
    ea.bytes[i] = pl.bytes[i];
  }
  for (int l = 0; l < 4; l++) ea.b[l] = w->b[l];
  ea.z = z;
  ea.P = P;
  LGS_CHECK_CUDA(set_smem_limit(reinterpret_cast<const void*>(encode_fused_kernel), (int)SM_ALL));
  const int64_t ntiles = (P + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntiles, sm_count());
  encode_fused_kernel<<<grid, kThreads, SM_ALL, s>>>(ea, xmap);
  LGS_CHECK_LAUNCH();
  return LGS_OK;
}

unsigned encode_error_word(bool clear) {
  unsigned v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_enc_error, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) cudaMemcpyToSymbol(g_enc_error, &zero, sizeof(zero));
  return v;
}

}  // namespace lgs
