// Internal launchers shared between translation units of liblgs.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace lgs {

// Validates the cameras and copies them into a kernel-parameter block.
lgs_status fill_cams(const lgs_camera* cams_host, int n_cams, CamBlock& cb);

// Projection backward: one thread per Gaussian sums the chain rule of every
// camera's 2D gradient record (u, v, a, b, c, o, tz, 0) into the parameters.
lgs_status launch_project_bwd(const float* means, const float* quats, const float* log_scales,
                              const float* logits, int64_t n, int n_cams, const CamBlock& cams,
                              const float* grad2d, float* d_means, float* d_quats,
                              float* d_log_scales, float* d_logits, cudaStream_t s);

// Fused Eq. 2 distillation (decoder forward, L1 against F_gt, gradient to
// z); `pack` is decode_pack_bytes() of scratch for the packed weights, which
// launch_decode_pack fills (and launch_decode_fused first, unless `packed`).
size_t decode_pack_bytes();
lgs_status launch_decode_pack(const lgs_ae_weights* w, void* pack, cudaStream_t s);
lgs_status launch_decode_fused(const lgs_ae_weights* w, const float* z, int64_t P,
                               const uint16_t* target, float weight, float* loss, float* dz,
                               void* pack, bool packed, cudaStream_t s);
// Reads (and with clear, clears) the fused decoder's timeout word.
unsigned fused_error_word(bool clear = true);
// Fused encoder z = E(x) (x bf16 [P,512] -> z f32 [P,16]); `pack` is
// encode_pack_bytes() of scratch for the packed weights.
size_t encode_pack_bytes();
lgs_status launch_encode_fused(const lgs_ae_weights* w, const uint16_t* x, int64_t P, float* z,
                               void* pack, cudaStream_t s);
// Reads (and with clear, clears) the fused encoder's timeout word.
unsigned encode_error_word(bool clear = true);
// Streaming multiprocessors of the current device.
int sm_count();
// A 3-D TMA tensor map that views a row-major bf16 matrix [rows, K] as
// [K / 8 column groups][rows][8 columns]: a box of box_rows rows and
// box_groups groups lands in shared memory as box_groups blocks of
// box_rows x 16 bytes, the K-major core-matrix layout whose K-adjacent core
// matrices are box_rows * 16 bytes apart (rows past the end read as zero).
// Read with the pixel as K, the same blocks are the MN-major layout: core
// matrices adjacent in K 128 bytes apart, adjacent in MN box_rows * 16.
// False (with the error string set) when the driver refuses the map.
bool make_kmajor_map(CUtensorMap* map, const void* base, int64_t rows, int K, int box_rows,
                     int box_groups);
// A 2-D TMA tensor map of a row-major bf16 matrix [rows, K] with box_cols x
// box_rows boxes in a swizzled layout: box_cols = 64 lands box_rows rows of
// 128 bytes with the 128-byte swizzle (the layout sdesc_sw128 describes),
// box_cols = 32 rows of 64 bytes with the 64-byte swizzle (sdesc_sw64).
// Rows past the end read as zero; the shared destination must be 1 KB
// aligned.  False (with the error string set) when the driver refuses it.
bool make_swizzled_map(CUtensorMap* map, const void* base, int64_t rows, int K, int box_cols,
                       int box_rows);
// Stable LSD radix sort of n (key, value) pairs on key bits [0, nbits)
// (nbits <= 32), one onesweep kernel per 8 bits.  `scratch` holds
// sort_pairs_scratch(n) bytes (256-byte aligned) and is cleared here.
// Returns true when the result is in (k1, v1), false when in (k0, v0).
size_t sort_pairs_scratch(int64_t n);
bool sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int nbits,
                void* scratch, cudaStream_t s);
// Reads (and with clear, clears) the radix sort's look-back timeout word.
unsigned sort_error_word(bool clear = true);
// Reads (and with clear, clears) the smallest Gaussian index gs_project
// found with a non-finite parameter (UINT64_MAX = none).
unsigned long long nonfinite_word(bool clear);
// Reads (and with clear, clears) the largest instance count gs_bin_sort
// needed beyond its capacity (0 = none).
unsigned long long capacity_word(bool clear);

}  // namespace lgs
