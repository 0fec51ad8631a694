/*
 * lgs.h -- C ABI of the GB300 language-feature Gaussian-splatting library.
 *
 * The library implements the data-parallel hot path of the mapping loop of
 * LEGO-SLAM (arXiv 2511.16144): rendering a map of language-embedded 3D
 * Gaussians (Sec. III-B.1) into RGB, depth and a compact feature map, the
 * backward pass that the map optimisation of Sec. III-B.3 needs (Eq. 1-2),
 * and the encoder / decoder GEMMs of the scene-adaptive autoencoder
 * (Sec. III-B.3 Eq. 2, Sec. III-B.4 Eq. 3, Sec. IV-A.2).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named *_host are host memory; every other pointer is device
 *   memory owned by the caller.  The library allocates nothing and frees
 *   nothing; scratch space is passed in (see gs_bin_sort_workspace and the
 *   grad2d argument of gs_render_bwd).
 * - Every call only enqueues work on `stream` (a cudaStream_t; NULL = the
 *   legacy default stream) and returns without synchronising.  Argument
 *   errors that the host can see (null or misaligned pointers, bad sizes)
 *   return LGS_ERR_INVALID before anything is enqueued (LGS_ERR_NONFINITE
 *   for a non-finite camera value); launch failures return LGS_ERR_CUDA.
 *   lgs_last_error() gives the message (thread-local).
 * - Errors that only the device sees (an instance buffer that is too small,
 *   a non-finite Gaussian parameter, a bounded wait that gave up) are
 *   recorded on the device and reported by lgs_sync_status(), which
 *   synchronises the stream; the enqueueing call has already returned
 *   LGS_OK.
 * - Arrays are dense, row-major, structure-of-arrays; images are [C,H,W,ch]
 *   (camera, row, column, channel).  Pointers read or written with 16-byte
 *   vector accesses must be 16-byte aligned (stated per argument).
 * - Gradient outputs (d_*) are ACCUMULATED into (+=); zero them first for a
 *   plain gradient.
 * - bf16 arrays are passed as uint16_t (IEEE bfloat16 bit patterns).
 * - A stream may carry calls from one host thread at a time; different
 *   streams may be used concurrently.  No call keeps state between calls.
 */
#ifndef LGS_H
#define LGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LGS_OK = 0,
  LGS_ERR_INVALID = 1,    /* bad argument (host-detected) */
  LGS_ERR_CAPACITY = 2,   /* instance buffer too small (gs_bin_sort; device-detected) */
  LGS_ERR_NONFINITE = 3,  /* NaN / inf in a camera (host) or a Gaussian (device) */
  LGS_ERR_TIMEOUT = 4,    /* a bounded device wait gave up (device-detected) */
  LGS_ERR_CUDA = 5        /* a CUDA launch or runtime call failed */
} lgs_status;

typedef enum { LGS_F32 = 0, LGS_BF16 = 1 } lgs_dtype;

/* Upper bound on cameras rendered in one launch (a keyframe window). */
#define LGS_MAX_CAMS 16
/* Tile edge in pixels (16x16 tiles, one CTA each). */
#define LGS_TILE 16
/* Floats per projected record and per 2D-gradient record. */
#define LGS_PROJ_STRIDE 8

/* Pinhole camera.  viewmat = row-major 3x4 world-to-camera [R | t] in
 * OpenCV axes (x right, y down, z forward); a pixel (i, j) has its centre at
 * (i + 0.5, j + 0.5); u = fx x/z + cx, v = fy y/z + cy.  Gaussians with
 * camera depth z <= znear are culled. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
  float viewmat[12];
  float znear;
} lgs_camera;

/* Library version string. */
const char* lgs_version(void);

/* Message of the last failing call on this host thread ("" if none). */
const char* lgs_last_error(void);

/* Number of kernel nodes in a captured CUDA graph (a cudaGraph_t, e.g. one
 * mapping step captured from the calls below), or -1 on error.  Utility for
 * counting launches; the paper has no counterpart. */
int64_t lgs_graph_kernel_nodes(void* graph);

/* Enqueues a zero fill of `bytes` bytes of device memory (a memset, no
 * kernel), e.g. gradient accumulators before gs_render_bwd. */
lgs_status lgs_zero(void* dev, size_t bytes, void* stream);

/* ------------------------------------------------------------------------
 * lgs_sync_status -- the deferred status of the device-side work.
 *
 * The paper states the problem (Sec. III-B.1: project, bin and composite
 * the map; Sec. III-B.3: optimise it by gradients) but no error contract;
 * this is the library's.  Synchronises `stream` (NULL = the legacy default
 * stream), then reports one error that kernels on the current device
 * recorded since it was last reported, and clears it:
 *   LGS_ERR_NONFINITE  gs_project met a NaN or infinite mean, quaternion,
 *                      log-scale or opacity logit (those Gaussians are culled
 *                      in every camera); *detail = the smallest such index;
 *   LGS_ERR_CAPACITY   gs_bin_sort needed more instances than its capacity
 *                      (nothing was sorted, every range is (0, 0));
 *                      *detail = the largest K required;
 *   LGS_ERR_TIMEOUT    a bounded wait gave up and its kernel returned
 *                      (results of that call are undefined but every
 *                      access stayed in bounds); *detail = the wait-site bit
 *                      word that lgs_device_error describes;
 *   LGS_OK             nothing recorded; *detail = 0.
 * When several kinds are pending they come out in the order above, one per
 * call (call again until LGS_OK).  Recorded errors are per device and
 * process-wide (not per stream): a caller that shares the device with other
 * users of the library sees theirs too.  detail may be NULL.  Returns
 * LGS_ERR_CUDA if the synchronisation itself fails (e.g. a faulted context).
 * ---------------------------------------------------------------------- */
lgs_status lgs_sync_status(void* stream, int64_t* detail);

/* Sets the number of polling rounds after which the decoupled look-back of
 * the radix sort behind gs_prune gives up (LGS_ERR_TIMEOUT), for calls
 * enqueued afterwards; polls <= 0 restores the default (4,194,304, about a
 * second).  A test hook for the timeout path: a small limit makes a look-back
 * that has to wait for a slower block give up at once.  Process-wide; no
 * counterpart in the paper. */
void lgs_set_sort_wait_limit(int64_t polls);

/* ------------------------------------------------------------------------
 * gs_project -- EWA projection of every Gaussian into every camera.
 *
 * Sec. III-B.1: a Gaussian has position p, rotation q, scale s, opacity
 * alpha, colour c and feature f, rendered "following the standard 3DGS
 * pipeline".  Per (camera c, Gaussian i), in FP32:
 *   t = R_c p + t_c;   Sigma3 = R(q/|q|) diag(exp(2 log_s)) R^T;
 *   J = [[fx/tz, 0, -fx tx'/tz^2], [0, fy/tz, -fy ty'/tz^2]] with tx'/tz
 *   clamped to [(-0.15W - cx)/fx, (1.15W - cx)/fx] (same in y);
 *   Sigma2 = J R_c Sigma3 R_c^T J^T + 0.3 I;  conic = Sigma2^-1;
 *   opacity o = sigmoid(logit).
 * A Gaussian is culled (rect empty) if tz <= znear, det(Sigma2) <= 0,
 * o < 1/255, its quaternion is zero or its support misses the image.  A
 * Gaussian with a NaN or infinite parameter is culled too and recorded as
 * LGS_ERR_NONFINITE (see lgs_sync_status); a camera with a non-finite
 * value returns LGS_ERR_NONFINITE at once.  The support radius is
 * sqrt(2 ln(255 o) lambda_max(Sigma2)) (1 + 1e-5) + 1e-3 px: every pixel
 * outside it has o exp(power) < 1/255, so tiled rendering equals per-pixel
 * rendering over all Gaussians.
 *
 * means [n,3], quats [n,4] (w,x,y,z), log_scales [n,3], opacity_logits [n]:
 *   float32 device arrays.
 * cams_host [n_cams]: host array, 1 <= n_cams <= LGS_MAX_CAMS.
 * proj [n_cams*n, 8] (16-byte aligned): per (camera, Gaussian) record
 *   (u, v, conic a, conic b, conic c, opacity, depth tz, cut); zero when
 *   culled.  cut = 2 ln(255 o) 1.001 + 0.01 bounds q = a dx^2 + 2 b dx dy +
 *   c dy^2 (= -2 power) over every pixel with o e^power >= 1/255, with a
 *   margin for FP32 rounding; gs_bin_sort's tile test uses it.
 * rect [n_cams*n, 4] uint16 (8-byte aligned): covered tiles
 *   [x0, y0, x1, y1) on the 16x16 grid, x1 == x0 and y1 == y0 when culled.
 * ---------------------------------------------------------------------- */
lgs_status gs_project(const float* means, const float* quats, const float* log_scales,
                      const float* opacity_logits, int64_t n, const lgs_camera* cams_host,
                      int n_cams, float* proj, uint16_t* rect, void* stream);

/* ------------------------------------------------------------------------
 * gs_bin_sort -- 16x16 tile binning, instances ordered by depth within each tile.
 *
 * Each (camera c, Gaussian i) emits one instance per tile of its rect that
 * its ellipse reaches: the minimum of q(d) = a dx^2 + 2 b dx dy + c dy^2,
 * d = (u - x, v - y), over the tile's pixel-centre square [16 tx + 0.5,
 * 16 tx + 15.5] x [16 ty + 0.5, 16 ty + 15.5] is at most the record's cut
 * (0 when the mean is inside, else the least of the four edges' 1-D
 * minima, in FP32 with round-to-nearest operations in a fixed order).  No
 * pixel that passes the 1/255 skip test is in a tile left out, so the tiled
 * render equals the per-pixel one.  The instances are ordered by the 64-bit
 * key ((c * tiles + tile) << 32) | bits(float depth), ties by ascending
 * Gaussian index (a stable sort of the emission order).  This is the
 * front-to-back order of Sec. III-B.1's alpha compositing within every
 * tile.
 *
 * proj, rect: gs_project outputs for n Gaussians and n_cams cameras.
 * tiles_x, tiles_y: grid size (ceil(W/16), ceil(H/16)); n_cams * tiles_x *
 *   tiles_y at most 2^24 (LGS_ERR_INVALID above).
 * capacity: length of ids (and keys_opt), below 2^30.
 * ids [capacity] uint32 out: Gaussian index of each sorted instance.
 * ranges [n_cams*tiles_x*tiles_y, 2] uint32 out: [start, end) of each
 *   tile's instances in ids; (0, 0) for an empty tile.
 * keys_opt [capacity] uint64 out or NULL: the sort keys.
 * n_instances_dev: device int64 out, the instance count K.  If K >
 *   capacity nothing is sorted, every range is (0, 0), LGS_ERR_CAPACITY is
 *   recorded for lgs_sync_status (detail = K) and the caller must retry
 *   with capacity >= K.  The call never synchronises, so capacity is not
 *   checked on the host.
 * workspace: device scratch of at least gs_bin_sort_workspace(...) bytes,
 *   256-byte aligned.
 * ---------------------------------------------------------------------- */
size_t gs_bin_sort_workspace(int64_t n, int n_cams, int tiles_x, int tiles_y,
                             int64_t capacity);
lgs_status gs_bin_sort(const float* proj, const uint16_t* rect, int64_t n, int n_cams,
                       int tiles_x, int tiles_y, int64_t capacity, uint32_t* ids,
                       uint32_t* ranges, uint64_t* keys_opt, int64_t* n_instances_dev,
                       void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * gs_render_fwd -- front-to-back alpha compositing of RGB, depth and a
 * feat_dim-channel feature map (Sec. III-B.1; F_render of Eq. 2).
 *
 * Per pixel, over its tile's sorted instances: power = -(a dx^2 + c dy^2)/2
 * - b dx dy with d = (u - px, v - py); skip if power > 0; alpha =
 * min(0.99, o e^power); skip if alpha < 1/255; T' = T (1 - alpha); stop,
 * without blending, when T' < 1e-4; else w = alpha T accumulates w c,
 * w tz, w f and T = T'.  rgb gets + T_final bg; depth is the unnormalised
 * sum of w tz.  alpha / T are FP32; channels are read as float32 or bf16
 * (chan_dtype) and accumulated in FP32.
 *
 * All cameras must share width and height.  colors [n,3], feats [n,D]
 * (16-byte aligned, D = feat_dim, a multiple of 8 in [8, 4096]).
 * bg_host: float[3] background colour.
 * Outputs (float32 unless stated): rgb [C,H,W,3], depth [C,H,W],
 * feat [C,H,W,D], T_final [C,H,W], last [C,H,W] uint32 (position + 1, in
 * the tile's range, of the last blended instance; the backward's start),
 * n_contrib_opt [C,H,W] uint32 (number blended) or NULL.
 * ---------------------------------------------------------------------- */
lgs_status gs_render_fwd(const float* proj, const uint32_t* ids, const uint32_t* ranges,
                         int64_t n, const lgs_camera* cams_host, int n_cams, const void* colors,
                         const void* feats, int feat_dim, int chan_dtype, const float* bg_host,
                         float* rgb, float* depth, float* feat, float* T_final, uint32_t* last,
                         uint32_t* n_contrib_opt, void* stream);

/* ------------------------------------------------------------------------
 * gs_render_bwd -- gradient of the rendered maps w.r.t. every Gaussian
 * parameter (the map optimisation of Sec. III-B.3, Eq. 1).
 *
 * Walks each pixel's blended instances back to front from `last`,
 * recovering T_i = T_{i+1} / (1 - alpha_i) from T_final instead of storing
 * it, and scatters per-Gaussian partials: colour and feature gradients
 * sum_px w g, and the 2D-mean, conic and opacity gradients through
 * dL/dalpha_i = T_i (x_i . g) - S_i / (1 - alpha_i), with S_i the suffix
 * sum of w_k (x_k . g) behind i plus T_final (bg . g).  Partials are summed
 * over each tile's 256 pixels on chip and added to global memory once per
 * (tile, instance).  The chain rule through the projection then gives the
 * parameter gradients, summed over cameras.
 *
 * Inputs: the Gaussian parameters and every gs_project / gs_bin_sort /
 * gs_render_fwd input and output named here, plus the upstream gradients
 * d_rgb [C,H,W,3], d_depth [C,H,W], d_feat [C,H,W,D] (float32).
 * grad2d [n_cams*n, 8] (16-byte aligned): scratch, overwritten with the
 *   per-(camera, Gaussian) 2D gradients (u, v, a, b, c, opacity, depth, 0).
 * Outputs (accumulated): d_means [n,3], d_quats [n,4], d_log_scales [n,3],
 * d_opacity_logits [n], d_colors [n,3], d_feats [n,D] (16-byte aligned).
 * ---------------------------------------------------------------------- */
lgs_status gs_render_bwd(const float* means, const float* quats, const float* log_scales,
                         const float* opacity_logits, const float* proj, const uint32_t* ids,
                         const uint32_t* ranges, int64_t n, const lgs_camera* cams_host,
                         int n_cams, const void* colors, const void* feats, int feat_dim,
                         int chan_dtype, const float* bg_host, const float* T_final,
                         const uint32_t* last, const float* d_rgb, const float* d_depth,
                         const float* d_feat, float* grad2d, float* d_means, float* d_quats,
                         float* d_log_scales, float* d_opacity_logits, float* d_colors,
                         float* d_feats, void* stream);

/* ------------------------------------------------------------------------
 * gs_render_bwd_static -- gs_render_bwd without the caller-owned grad2d
 * scratch, for callers that cannot allocate device memory: for example a
 * mapping thread with a hard real-time budget that must never take the
 * device-wide synchronisation a cudaMalloc / cudaFree implies, or a host
 * application that forbids libraries and plug-ins from owning device
 * memory.  The paper has no counterpart; this is a deployment variant.
 *
 * Same arguments, meaning and results as gs_render_bwd except grad2d.  The
 * scratch is a fixed array inside the library's device image, 524,288
 * (camera, Gaussian) records (16 MiB, see gs_render_bwd_static_capacity),
 * held by every GPU that loads the library until the process exits.
 * n_cams * n above that limit returns LGS_ERR_INVALID before anything is
 * enqueued.  Nothing is allocated by the caller or the library.
 * The first call on a device looks the array's device address up (with that
 * device current) and caches it with the ID of the device's current
 * context: make that first call before any stream capture.  A call in a new
 * context of the device (after cudaDeviceReset) looks it up again, so the
 * first call after a reset should also come before any capture.  All calls share the array, zero the part they use and leave
 * their contents in it; calls that overlap on the GPU (unordered streams)
 * race on it, so order them on one stream.
 * ---------------------------------------------------------------------- */
int64_t gs_render_bwd_static_capacity(void);
lgs_status gs_render_bwd_static(const float* means, const float* quats, const float* log_scales,
                                const float* opacity_logits, const float* proj,
                                const uint32_t* ids, const uint32_t* ranges, int64_t n,
                                const lgs_camera* cams_host, int n_cams, const void* colors,
                                const void* feats, int feat_dim, int chan_dtype,
                                const float* bg_host, const float* T_final, const uint32_t* last,
                                const float* d_rgb, const float* d_depth, const float* d_feat,
                                float* d_means, float* d_quats, float* d_log_scales,
                                float* d_opacity_logits, float* d_colors, float* d_feats,
                                void* stream);

/* ------------------------------------------------------------------------
 * lgs_l1_loss -- one L1 term of Eq. 1 / Eq. 2: loss_dev += weight *
 * mean|pred - target| and grad = weight * sign(pred - target) / count
 * (overwritten; sign(0) = 0).  pred, grad: float32 [count]; target float32
 * or bf16 (target_dtype) [count]; loss_dev: one float32 on the device.
 * ---------------------------------------------------------------------- */
lgs_status lgs_l1_loss(const float* pred, const void* target, int target_dtype, int64_t count,
                       float weight, float* grad, float* loss_dev, void* stream);

/* ------------------------------------------------------------------------
 * Scene-adaptive autoencoder (Sec. IV-A.2: stacks of 1x1 convolutions, i.e.
 * one MLP applied per pixel, pretrained as an autoencoder; Sec. III-B.3
 * Eq. 2: distillation through the frozen decoder; Sec. III-B.4 Eq. 3:
 * encoder adaptation).  Layers 0-3 are the encoder 512-256-128-64-16, layers
 * 4-7 the decoder 16-64-128-256-512; layer l maps width w[l] to w[l+1] with
 * y = x W_l^T + b_l, GELU after every layer except 3 and 7, in its tanh form
 * 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (the paper names no
 * activation; the hardware tanh approximation evaluates it).
 * GEMMs run on the tensor cores with BF16 operands and FP32 accumulation;
 * activations between layers are BF16.  Pixels are rows: x [P, 512],
 * z [P, 16], all row-major.
 * ---------------------------------------------------------------------- */
#define LGS_AE_LAYERS 8
#define LGS_AE_ENCODE 0
#define LGS_AE_DECODE 1
#define LGS_AE_TRAIN 2
#define LGS_AE_RECON 0     /* pretraining: L = mean_k (y-x)^2 + 1 - cos(y, x) */
#define LGS_AE_ENC_ADAPT 1 /* Eq. 3: L = mean |E(x) - F_render|, decoder frozen */

/* Inference weights: W[l] bf16 [w[l+1], w[l]] row-major, Wt[l] its
 * transpose (bf16 [w[l], w[l+1]], used by the backward), b[l] fp32.  All
 * 16-byte aligned device memory (ae_pack writes both copies). */
typedef struct {
  const uint16_t* W[LGS_AE_LAYERS];
  const uint16_t* Wt[LGS_AE_LAYERS];
  const float* b[LGS_AE_LAYERS];
} lgs_ae_weights;

/* Training state: FP32 master weights and biases, Adam moments, the last
 * step's gradients, and the BF16 copies (Wbf = W, Wtbf = W^T) that the GEMMs
 * read.  step counts Adam steps and is incremented by ae_train_step (host
 * field).  Every pointer is 16-byte aligned.  Each step overwrites the
 * gradient buffers gW / gb of the layers it trains with that step's
 * gradients.  The weight gradients are summed in a fixed order (per-CTA
 * partial sums in the workspace, added slice by slice), so the same inputs
 * give bit-identical gradients and updates on every run. */
typedef struct {
  float* W[LGS_AE_LAYERS];
  float* b[LGS_AE_LAYERS];
  float* mW[LGS_AE_LAYERS];
  float* vW[LGS_AE_LAYERS];
  float* mb[LGS_AE_LAYERS];
  float* vb[LGS_AE_LAYERS];
  float* gW[LGS_AE_LAYERS];
  float* gb[LGS_AE_LAYERS];
  uint16_t* Wbf[LGS_AE_LAYERS];
  uint16_t* Wtbf[LGS_AE_LAYERS];
  int64_t step;
} lgs_ae_state;

/* Scratch bytes for P pixels of LGS_AE_ENCODE, LGS_AE_DECODE or
 * LGS_AE_TRAIN work (0 for a bad argument), for the current device (the
 * training scratch holds the per-CTA partial weight gradients, about one
 * [N, K] slice per SM and layer: 81 MB on a 152-SM GPU at P >= 9,728). */
size_t ae_workspace_bytes(int64_t P, int what);

/* z [P,16] fp32 = E_phi(x), x bf16 [P,512] (the encoder prior of new
 * Gaussians' features, Sec. III-B.2). */
lgs_status ae_encode(const lgs_ae_weights* w, const uint16_t* x, int64_t P, float* z,
                     void* workspace, size_t workspace_bytes, void* stream);

/* Decoder D_theta on z [P,16] fp32 (the rendered F_render).  With target
 * (F_gt, bf16 [P,512], 32-byte aligned; the other pointers 16-byte aligned,
 * the workspace 256-byte): loss_dev += weight * mean|D(z) - F_gt| (Eq. 2) and
 * dz [P,16] fp32 = its gradient w.r.t. z (overwritten; the decoder is
 * frozen).  With y_opt: y_opt [P,512] fp32 = D(z).  Either or both. */
lgs_status ae_decode(const lgs_ae_weights* w, const float* z, int64_t P, const uint16_t* target,
                     float weight, float* loss_dev, float* dz, float* y_opt, void* workspace,
                     size_t workspace_bytes, void* stream);

/* ae_decode with a target splits into two calls, so that the weight packing
 * can run on another stream beside earlier work: ae_decode_pack writes the
 * decoder weights (layers 4-7) in the layout the fused distillation streams
 * into the first bytes of an ae_decode workspace (any P; workspace_bytes at
 * least ae_workspace_bytes(0, LGS_AE_DECODE)); ae_decode_packed then computes
 * exactly what ae_decode computes with that target and no y_opt, reading the
 * packed weights from the same workspace.  The weights must not change
 * between the two calls (the caller orders them, e.g. by an event). */
lgs_status ae_decode_pack(const lgs_ae_weights* w, void* workspace, size_t workspace_bytes,
                          void* stream);
lgs_status ae_decode_packed(const lgs_ae_weights* w, const float* z, int64_t P,
                            const uint16_t* target, float weight, float* loss_dev, float* dz,
                            void* workspace, size_t workspace_bytes, void* stream);

/* One Adam step (lr; beta 0.9, 0.999; eps 1e-8) on a batch x bf16 [P,512].
 * mode LGS_AE_RECON trains both networks on the reconstruction loss;
 * LGS_AE_ENC_ADAPT trains layers 0-3 on Eq. 3 against target = F_render
 * fp32 [P,16].  loss_dev += the batch loss (before the update); st->gW/gb
 * hold the gradients; the BF16 copies are refreshed. */
lgs_status ae_train_step(lgs_ae_state* st, const uint16_t* x, const float* target, int64_t P,
                         int mode, float lr, float* loss_dev, void* workspace,
                         size_t workspace_bytes, void* stream);

/* Refreshes Wbf / Wtbf of layers first..last from the FP32 masters. */
lgs_status ae_pack(lgs_ae_state* st, int first, int last, void* stream);

/* ------------------------------------------------------------------------
 * gs_prune -- language-guided pruning (Sec. III-C, Eq. 4) unioned with the
 * geometric criteria (low opacity, large scale), run periodically over the
 * map (every 200 mapping iterations in Sec. IV-A).
 *
 * Eq. 4: each Gaussian G_i takes its K nearest neighbours G_j in 3D; G_j is
 * redundant when d(p_i, p_j) < tau_dist and cos(f_i, f_j) > tau_sim on the
 * compact language features.  Readings where the paper is silent: the
 * neighbours are the K nearest among those closer than tau_dist, ranked by
 * (squared distance, index); G_i marks G_j only if G_i is the one to keep
 * (higher opacity logit, or the same logit and the lower index), so mutual
 * neighbours lose one member, not both; the cosine of a zero feature is 0;
 * low opacity is logit < logit(min_opacity), large scale is
 * max_k log_s_k > log(max_scale) (thresholds rounded to float once).
 * Each decision is taken in FP32 with a fixed operation order:
 * d2 = (dx dx + dy dy) + dz dz with dx = x_j - x_i, d = sqrt(d2);
 * |f| = sqrt of the left-to-right sum of f_k f_k; sim = (left-to-right
 * sum of f_ik f_jk) / (|f_i| |f_j|); no fused multiply-add.
 *
 * means [n,3], opacity_logits [n], log_scales [n,3] fp32; feats [n,feat_dim]
 * fp32 or bf16 (feat_dtype), feat_dim in [1, 64].  params (host): k in
 * [1, 16]; tau_dist > 0 (metres); tau_sim; min_opacity in [0, 1) (0 turns the
 * opacity test off); max_scale > 0 (+inf turns it off); lo/hi: bounds of the
 * neighbour grid (cells 1.05 tau_dist wide, at most 2^16 per axis and 2^32
 * in all).  Gaussians outside the bounds are still handled exactly (they
 * fall into the border cells); the bounds only affect speed.
 * mask [n] uint8 out: bit 0 geometric, bit 1 redundant; 0 keeps G_i.
 * n_pruned_dev: device int64 out, the number of nonzero entries.
 * workspace: gs_prune_workspace(n) bytes, 256-byte aligned.
 * Errors: LGS_ERR_INVALID for a bad argument (nothing enqueued).
 * ---------------------------------------------------------------------- */
typedef struct {
  int k;
  float tau_dist;
  float tau_sim;
  float min_opacity;
  float max_scale;
  float lo[3];
  float hi[3];
} lgs_prune_params;

size_t gs_prune_workspace(int64_t n);
lgs_status gs_prune(const float* means, const float* opacity_logits, const float* log_scales,
                    const void* feats, int feat_dim, int feat_dtype, int64_t n,
                    const lgs_prune_params* params, uint8_t* mask, int64_t* n_pruned_dev,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Order-preserving compaction after pruning (no counterpart in the paper,
 * which only says the pruned Gaussians are removed).
 * gs_compact_index: new_index [n] uint32 out = the rank of G_i among the
 * kept Gaussians (mask == 0), 0xffffffff for a pruned one; n_kept_dev:
 * device int64 out.  workspace: gs_compact_workspace(n) bytes, 256-byte
 * aligned.
 * gs_gather_rows: dst[new_index[i]] = src[i] for every kept row of
 * row_bytes bytes (a positive even number; rows aligned to 4 bytes when
 * row_bytes is a multiple of 4, else to 2; LGS_ERR_INVALID otherwise); dst holds
 * at least n_kept rows and must not overlap src. */
size_t gs_compact_workspace(int64_t n);
lgs_status gs_compact_index(const uint8_t* mask, int64_t n, uint32_t* new_index,
                            int64_t* n_kept_dev, void* workspace, size_t workspace_bytes,
                            void* stream);
lgs_status gs_gather_rows(const void* src, int64_t n, int row_bytes, const uint32_t* new_index,
                          void* dst, void* stream);

/* ------------------------------------------------------------------------
 * lgs_dssim_loss -- the D-SSIM term of the photometric loss L_rgb
 * (Sec. III-B.3, Eq. 1: L_rgb combines an L1 and a D-SSIM term).  The paper
 * gives no SSIM parameters; these are the standard ones: per colour channel,
 * an 11 x 11 Gaussian window of sigma 1.5 (normalised), images zero outside
 * their borders, C1 = 0.01^2, C2 = 0.03^2.
 * loss_dev (device float) += weight * (1 - mean SSIM(pred, target)) over all
 * pixels and channels; grad += its gradient w.r.t. pred (accumulated, so an
 * L1 term can share the buffer).  pred, target, grad: [n_img, H, W, 3] fp32.
 * workspace: lgs_dssim_workspace(...) bytes of device scratch (4-byte
 * aligned).  The standard L_rgb = 0.8 L1 + 0.2 D-SSIM is lgs_l1_loss with
 * weight 0.8 and this call with weight 0.2 on the same grad.
 * ---------------------------------------------------------------------- */
size_t lgs_dssim_workspace(int n_img, int height, int width);
lgs_status lgs_dssim_loss(const float* pred, const float* target, int n_img, int height,
                          int width, float weight, float* grad, float* loss_dev, void* workspace,
                          size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * gs_pose_grad -- camera pose gradient for the keyframe pose refinement of
 * Sec. III-B.2 (the pose is refined by minimising the render loss).
 * d_pose [n_cams, 6] fp32 out (overwritten): the gradient w.r.t. a left
 * perturbation T <- exp(xi^) T of each camera's world->camera transform,
 * xi = (rho, phi): rho translates the camera frame, phi rotates it (so a
 * camera-space mean t moves to t + phi x t + rho).  grad2d: the
 * per-(camera, Gaussian) 2D gradient records that gs_render_bwd wrote
 * ([n_cams*n, 8] fp32, 16-byte aligned); the other inputs as for gs_project.
 * ---------------------------------------------------------------------- */
lgs_status gs_pose_grad(const float* means, const float* quats, const float* log_scales,
                        const float* opacity_logits, int64_t n, const lgs_camera* cams_host,
                        int n_cams, const float* grad2d, float* d_pose, void* stream);

/* ------------------------------------------------------------------------
 * Language loop signature (Sec. III-D) and compact-space queries (Sec. I).
 *
 * lgs_codebook_assign: every row of x (bf16 [P, D], the keyframe's language
 * features; D = 16 or a multiple of 64) goes to its closest codeword of
 * codebook (bf16 [K, D], K in {16, 64, 128, 256, 512}) in Euclidean distance,
 * decided as argmin_k (|c_k|^2 - 2 x.c_k) with FP32 accumulation of the BF16
 * products on the tensor cores (ties to the lower index; two codewords whose
 * scores differ by less than that arithmetic's rounding may swap).
 * assign_opt [P] uint32 out or NULL; hist [K] uint32 += the counts (the
 * keyframe signature before normalisation).  workspace:
 * lgs_codebook_workspace(K) bytes, 4-byte aligned.
 * lgs_hist_cosine: out[m] = cos(hist, hists[m]) for M stored histograms
 * ([M, K] uint32); 0 for an empty histogram.
 * lgs_loop_candidates: out[0..top) = the indices m of past keyframes with
 * sim[m] > tau_hist and |centres[m] - cur| < radius (centres [M, 3] fp32,
 * cur on the host), most similar first, ties to the lower index, -1 padding;
 * top in [1, 8] (the paper verifies the top two).
 * gs_query_relevance: out [M, Q] fp32 = cos(feats[m], queries[q]) for
 * features [M, D] (fp32 or bf16, D <= 64: a rendered compact feature map or
 * the Gaussians' features) and queries [Q, D] fp32 already projected into the
 * compact space (ae_encode of the text embedding), Q <= 64; 0 for a zero norm.
 * ---------------------------------------------------------------------- */
size_t lgs_codebook_workspace(int K);
lgs_status lgs_codebook_assign(const uint16_t* x, int64_t P, int D, const uint16_t* codebook,
                               int K, uint32_t* assign_opt, uint32_t* hist, void* workspace,
                               size_t workspace_bytes, void* stream);
lgs_status lgs_hist_cosine(const uint32_t* hist, const uint32_t* hists, int M, int K, float* out,
                           void* stream);
lgs_status lgs_loop_candidates(const float* sim, const float* centres, int M,
                               const float* cur_centre_host, float tau_hist, float radius, int top,
                               int* out, void* stream);
lgs_status gs_query_relevance(const void* feats, int feat_dtype, int64_t M, int D,
                              const float* queries, int Q, float* out, void* stream);

/* Reads and clears the device error word that kernels with bounded waits
 * set when a wait gives up (0 = none; bits 0-3 the autoencoder layer
 * kernels -- 1: a wait gave up, 4: shared memory not on the 1 KB boundary
 * the 128-byte swizzle needs, so the kernel returned without work -- bits
 * 4-7 the fused decoder, 8-11 the sort's look-back, 12-15 the fused
 * encoder, whose bit 15 again means misaligned shared memory).  The same
 * word is the detail of LGS_ERR_TIMEOUT in lgs_sync_status; this call clears
 * it for both.  Synchronises the device. */
lgs_status lgs_device_error(int* code);

#ifdef __cplusplus
}
#endif
#endif /* LGS_H */
