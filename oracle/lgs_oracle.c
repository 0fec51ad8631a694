/*
 * FP64 CPU oracle for differentiable language-feature Gaussian splatting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header or constant table with the
 * CUDA library.
 *
 * What it computes (LEGO-SLAM, Sec. III-B.1 "Language-Embedded 3D Gaussians":
 * each Gaussian carries position p, rotation q, scale s, opacity alpha, colour c
 * and a compact language feature f, rendered "following the standard 3DGS
 * pipeline" into an RGB image, a depth map and a feature map; Eq. 1 and Eq. 2
 * are the losses those maps enter).  The paper gives no formulas for the
 * rasteriser itself, so this file writes out the textbook EWA-splatting
 * definition, with the readings listed below:
 *
 *   activations   q_hat = q/|q| (w,x,y,z order); R(q_hat) the unit-quaternion
 *                 rotation; S = diag(exp(log_s)); opacity o = sigmoid(logit);
 *                 colours are direct RGB (SH degree 0).
 *   camera        t = Rc p + tc (OpenCV axes: x right, y down, z forward);
 *                 valid iff t_z > znear; u = fx t_x/t_z + cx, v = fy t_y/t_z + cy
 *                 in pixel units; pixel (i, j) has its centre at (i+.5, j+.5).
 *   EWA           Sigma3 = R S S^T R^T; J = [[fx/tz, 0, -fx tx~/tz^2],
 *                 [0, fy/tz, -fy ty~/tz^2]] with tx~/tz clamped to
 *                 [(-0.15W - cx)/fx, (1.15W - cx)/fx] (same in y);
 *                 Sigma2 = J Rc Sigma3 Rc^T J^T + 0.3 I; invalid if det <= 0;
 *                 conic (a, b, c) = (S11, -S01, S00)/det.
 *   support       invalid if o < 1/255; otherwise every pixel with
 *                 o exp(power) >= 1/255 lies within
 *                 e = sqrt(2 ln(255 o) lambda_max) of (u, v); the tile rect
 *                 covers the pixels whose centres are within
 *                 r = e (1 + 1e-5) + 1e-3 of (u, v).
 *   compositing   per pixel, all valid Gaussians in ascending (t_z, index):
 *                 power = -(a dx^2 + c dy^2)/2 - b dx dy, d = (u - px, v - py);
 *                 skip if power > 0; alpha = min(0.99, o e^power); skip if
 *                 alpha < 1/255; T' = T (1 - alpha); stop (without blending)
 *                 if T' < 1e-4; else w = alpha T, accumulate w c, w t_z, w f.
 *                 Outputs RGB + T bg, depth sum (unnormalised), features,
 *                 T_final and the number blended.
 *   backward      analytic chain rule of all of the above, FP64.
 *   binning       key = ((camera * tiles + tile) << 32) | bits(float depth),
 *                 emitted in (camera, Gaussian index, tile row-major) order,
 *                 stable-sorted by key; per-tile [start, end) ranges, (0, 0)
 *                 for an empty tile.
 *
 * Camera array (double[19]): fx, fy, cx, cy, width, height, znear,
 * R (row-major 3x3, world -> camera), t (3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1e-4
#define DILATION 0.3
#define TILE 16

typedef struct {
  double fx, fy, cx, cy, znear;
  int width, height;
  double R[9], t[3];
} ocam;

static ocam read_cam(const double* c) {
  ocam k;
  k.fx = c[0]; k.fy = c[1]; k.cx = c[2]; k.cy = c[3];
  k.width = (int)c[4]; k.height = (int)c[5]; k.znear = c[6];
  for (int i = 0; i < 9; i++) k.R[i] = c[7 + i];
  for (int i = 0; i < 3; i++) k.t[i] = c[16 + i];
  return k;
}

/* Everything the forward projection of one Gaussian produces, plus the
 * intermediates its backward needs. */
typedef struct {
  int valid;
  double qn[4], qnorm;    /* normalised quaternion and |q| */
  double Rq[9];           /* rotation of the Gaussian */
  double s[3];            /* scales */
  double M[9];            /* R S */
  double S3[9];           /* 3D covariance */
  double t[3];            /* camera-space mean */
  double txc, tyc;        /* clamped tx~, ty~ used inside J */
  int clamp_x, clamp_y;   /* 0: inside, else sign of the clamp side */
  double limx, limy;      /* the active limit when clamped */
  double J[6];            /* 2x3 */
  double T2[6];           /* J Rc, 2x3 */
  double S2[3];           /* Sigma2 (00, 01, 11) incl. dilation */
  double det;
  double conic[3];
  double u, v, o;
  double radius;
  int rect[4];            /* tiles [x0, y0, x1, y1), x1 == x0 when empty */
} oproj;

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static void quat_to_rot(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void project_one(const double* p, const double* q, const double* ls, double logit,
                        const ocam* cam, oproj* P) {
  memset(P, 0, sizeof(*P));
  double qq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  P->qnorm = qq;
  for (int i = 0; i < 4; i++) P->qn[i] = q[i] / qq;
  quat_to_rot(P->qn, P->Rq);
  for (int k = 0; k < 3; k++) P->s[k] = exp(ls[k]);
  for (int j = 0; j < 3; j++)
    for (int k = 0; k < 3; k++) P->M[3 * j + k] = P->Rq[3 * j + k] * P->s[k];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double acc = 0;
      for (int k = 0; k < 3; k++) acc += P->M[3 * i + k] * P->M[3 * j + k];
      P->S3[3 * i + j] = acc;
    }
  for (int i = 0; i < 3; i++)
    P->t[i] = cam->R[3 * i] * p[0] + cam->R[3 * i + 1] * p[1] + cam->R[3 * i + 2] * p[2] + cam->t[i];
  P->o = sigmoid(logit);
  double tz = P->t[2];
  if (!(tz > cam->znear)) return;

  double W = cam->width, H = cam->height;
  double lox = (-0.15 * W - cam->cx) / cam->fx, hix = (1.15 * W - cam->cx) / cam->fx;
  double loy = (-0.15 * H - cam->cy) / cam->fy, hiy = (1.15 * H - cam->cy) / cam->fy;
  double rx = P->t[0] / tz, ry = P->t[1] / tz;
  P->clamp_x = rx < lox ? -1 : (rx > hix ? 1 : 0);
  P->clamp_y = ry < loy ? -1 : (ry > hiy ? 1 : 0);
  P->limx = P->clamp_x < 0 ? lox : hix;
  P->limy = P->clamp_y < 0 ? loy : hiy;
  P->txc = (P->clamp_x ? P->limx : rx) * tz;
  P->tyc = (P->clamp_y ? P->limy : ry) * tz;

  double* J = P->J;
  J[0] = cam->fx / tz; J[1] = 0; J[2] = -cam->fx * P->txc / (tz * tz);
  J[3] = 0; J[4] = cam->fy / tz; J[5] = -cam->fy * P->tyc / (tz * tz);
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) {
      double acc = 0;
      for (int k = 0; k < 3; k++) acc += J[3 * i + k] * cam->R[3 * k + j];
      P->T2[3 * i + j] = acc;
    }
  double S2f[4];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      double acc = 0;
      for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++) acc += P->T2[3 * i + k] * P->S3[3 * k + l] * P->T2[3 * j + l];
      S2f[2 * i + j] = acc;
    }
  P->S2[0] = S2f[0] + DILATION;
  P->S2[1] = S2f[1];
  P->S2[2] = S2f[3] + DILATION;
  P->det = P->S2[0] * P->S2[2] - P->S2[1] * P->S2[1];
  if (!(P->det > 0)) return;
  P->conic[0] = P->S2[2] / P->det;
  P->conic[1] = -P->S2[1] / P->det;
  P->conic[2] = P->S2[0] / P->det;
  P->u = cam->fx * P->t[0] / tz + cam->cx;
  P->v = cam->fy * P->t[1] / tz + cam->cy;
  if (P->o < ALPHA_MIN) return;

  double m = 0.5 * (P->S2[0] + P->S2[2]);
  double hd = 0.5 * (P->S2[0] - P->S2[2]);
  double lam = m + sqrt(hd * hd + P->S2[1] * P->S2[1]);
  double e = sqrt(2.0 * log(255.0 * P->o) * lam);
  double r = e * (1.0 + 1e-5) + 1e-3;
  P->radius = r;
  double pxmin = ceil(P->u - r - 0.5), pxmax = floor(P->u + r - 0.5);
  double pymin = ceil(P->v - r - 0.5), pymax = floor(P->v + r - 0.5);
  if (pxmin < 0) pxmin = 0;
  if (pymin < 0) pymin = 0;
  if (pxmax > W - 1) pxmax = W - 1;
  if (pymax > H - 1) pymax = H - 1;
  if (pxmin > pxmax || pymin > pymax) return;
  P->rect[0] = (int)pxmin / TILE;
  P->rect[1] = (int)pymin / TILE;
  P->rect[2] = (int)pxmax / TILE + 1;
  P->rect[3] = (int)pymax / TILE + 1;
  P->valid = 1;
}

/* ---------------------------------------------------------------------- */
/* projection                                                              */

int lgso_project(int64_t n, const double* means, const double* quats, const double* log_scales,
                 const double* op_logits, const double* camv, double* mean2d, double* depth,
                 double* conic, double* opacity, double* cov2d, double* radius, int32_t* rect,
                 int32_t* valid) {
  ocam cam = read_cam(camv);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    oproj P;
    project_one(means + 3 * i, quats + 4 * i, log_scales + 3 * i, op_logits[i], &cam, &P);
    if (mean2d) { mean2d[2 * i] = P.u; mean2d[2 * i + 1] = P.v; }
    if (depth) depth[i] = P.t[2];
    if (conic) for (int k = 0; k < 3; k++) conic[3 * i + k] = P.conic[k];
    if (opacity) opacity[i] = P.o;
    if (cov2d) for (int k = 0; k < 3; k++) cov2d[3 * i + k] = P.S2[k];
    if (radius) radius[i] = P.radius;
    if (rect) for (int k = 0; k < 4; k++) rect[4 * i + k] = P.rect[k];
    if (valid) valid[i] = P.valid;
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* compositing                                                             */

typedef struct { double z; int64_t idx; } zkey;

static int cmp_zkey(const void* a, const void* b) {
  const zkey* x = (const zkey*)a; const zkey* y = (const zkey*)b;
  if (x->z < y->z) return -1;
  if (x->z > y->z) return 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Projects all Gaussians and returns the valid ones ordered by (t_z, index). */
static int64_t project_and_order(int64_t n, const double* means, const double* quats,
                                 const double* log_scales, const double* op_logits,
                                 const ocam* cam, oproj* P, int64_t* order) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++)
    project_one(means + 3 * i, quats + 4 * i, log_scales + 3 * i, op_logits[i], cam, &P[i]);
  int64_t m = 0;
  for (int64_t i = 0; i < n; i++) m += P[i].valid;
  zkey* zk = (zkey*)malloc(sizeof(zkey) * (m ? m : 1));
  m = 0;
  for (int64_t i = 0; i < n; i++)
    if (P[i].valid) { zk[m].z = P[i].t[2]; zk[m].idx = i; m++; }
  qsort(zk, m, sizeof(zkey), cmp_zkey);
  for (int64_t j = 0; j < m; j++) order[j] = zk[j].idx;
  free(zk);
  return m;
}

typedef struct { int64_t g; double alpha, T, power; int clamped; } blend_rec;

/* Composites one pixel.  When `list` is non-null the blended Gaussians are
 * recorded (front to back) for the backward pass.  Returns the count. */
static int composite_pixel(int x, int y, int d, const oproj* P, const int64_t* order, int64_t m,
                           const double* colors, const double* feats, const double* bg,
                           double* rgb, double* dep, double* feat, double* T_out,
                           double* margin_out, double* zgap_out, blend_rec* list) {
  double px = x + 0.5, py = y + 0.5;
  double T = 1.0, C[3] = {0, 0, 0}, D = 0, margin = INFINITY, zgap = INFINITY, zprev = -1;
  for (int k = 0; k < d; k++) feat[k] = 0;
  int count = 0;
  for (int64_t j = 0; j < m; j++) {
    const oproj* g = &P[order[j]];
    double dx = g->u - px, dy = g->v - py;
    double power = -0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) - g->conic[1] * dx * dy;
    if (power > 0) continue;
    double lg = log(255.0 * g->o) + power;            /* ln(255 o e^power) */
    double mg = fabs(lg);
    if (mg < margin) margin = mg;
    if (lg < 0) continue;                             /* alpha < 1/255 */
    double araw = g->o * exp(power);
    double mc = fabs(araw / ALPHA_MAX - 1.0);
    if (mc < margin) margin = mc;
    double alpha = araw < ALPHA_MAX ? araw : ALPHA_MAX;
    if (zprev > 0) {
      double mz = fabs(g->t[2] - zprev) / g->t[2];
      if (mz < zgap) zgap = mz;
    }
    zprev = g->t[2];
    double Tn = T * (1.0 - alpha);
    double ms = fabs(Tn / T_STOP - 1.0);
    if (ms < margin) margin = ms;
    if (Tn < T_STOP) break;
    double w = alpha * T;
    int64_t gi = order[j];
    for (int k = 0; k < 3; k++) C[k] += w * colors[3 * gi + k];
    D += w * g->t[2];
    for (int k = 0; k < d; k++) feat[k] += w * feats[(int64_t)d * gi + k];
    if (list) {
      list[count].g = gi; list[count].alpha = alpha; list[count].T = T;
      list[count].power = power; list[count].clamped = araw >= ALPHA_MAX;
    }
    T = Tn;
    count++;
  }
  for (int k = 0; k < 3; k++) rgb[k] = C[k] + T * bg[k];
  *dep = D;
  *T_out = T;
  if (margin_out) *margin_out = margin;
  if (zgap_out) *zgap_out = zgap;
  return count;
}

int lgso_render_fwd(int64_t n, int d, const double* means, const double* quats,
                    const double* log_scales, const double* op_logits, const double* colors,
                    const double* feats, const double* camv, const double* bg, int x0, int y0,
                    int w, int h, double* rgb, double* dep, double* feat, double* T_final,
                    int32_t* n_contrib, double* margin, double* zgap) {
  ocam cam = read_cam(camv);
  oproj* P = (oproj*)malloc(sizeof(oproj) * (n ? n : 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  int64_t m = project_and_order(n, means, quats, log_scales, op_logits, &cam, P, order);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t pix = 0; pix < (int64_t)w * h; pix++) {
    int x = x0 + (int)(pix % w), y = y0 + (int)(pix / w);
    n_contrib[pix] = composite_pixel(x, y, d, P, order, m, colors, feats, bg, rgb + 3 * pix,
                                     dep + pix, feat + (int64_t)d * pix, T_final + pix,
                                     margin ? margin + pix : NULL, zgap ? zgap + pix : NULL,
                                     NULL);
  }
  free(P);
  free(order);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* backward                                                                */

static void atomic_add(double* p, double v) {
#pragma omp atomic
  *p += v;
}

/* The camera-space part of the projection backward of one Gaussian:
 * dp7 = gradient w.r.t. (u, v, conic a, conic b, conic c, opacity, depth t_z)
 * gives dS3 (world 3D covariance), dJ (the 2x3 Jacobian J of the EWA
 * linearisation) and dt (the camera-space mean t). */
static void camera_backward(const oproj* P, const ocam* cam, const double* dp7, double* dS3,
                            double* dJ, double* dt) {
  double du = dp7[0], dv = dp7[1], da = dp7[2], db = dp7[3], dc = dp7[4], dz = dp7[6];
  double tx = P->t[0], ty = P->t[1], tz = P->t[2];
  double fx = cam->fx, fy = cam->fy;
  /* conic = Sigma2^-1: dSigma2 = -Q dQ Q with dQ symmetric (b shared by 01/10) */
  double Q[4] = {P->conic[0], P->conic[1], P->conic[1], P->conic[2]};
  double G[4] = {da, 0.5 * db, 0.5 * db, dc};
  double QG[4], dS2[4];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) QG[2 * i + j] = Q[2 * i] * G[j] + Q[2 * i + 1] * G[2 + j];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++)
      dS2[2 * i + j] = -(QG[2 * i] * Q[j] + QG[2 * i + 1] * Q[2 + j]);
  /* Sigma2 = T Sigma3 T^T (+ const): dSigma3 = T^T dS2 T, dT = 2 dS2 T Sigma3 */
  double dT[6], TS3[6];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double acc = 0;
      for (int k = 0; k < 2; k++)
        for (int l = 0; l < 2; l++) acc += P->T2[3 * k + i] * dS2[2 * k + l] * P->T2[3 * l + j];
      dS3[3 * i + j] = acc;
    }
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) {
      double acc = 0;
      for (int k = 0; k < 3; k++) acc += P->T2[3 * i + k] * P->S3[3 * k + j];
      TS3[3 * i + j] = acc;
    }
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) dT[3 * i + j] = 2.0 * (dS2[2 * i] * TS3[j] + dS2[2 * i + 1] * TS3[3 + j]);
  /* T = J Rc: dJ = dT Rc^T */
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) {
      double acc = 0;
      for (int k = 0; k < 3; k++) acc += dT[3 * i + k] * cam->R[3 * j + k];
      dJ[3 * i + j] = acc;
    }
  dt[0] = dt[1] = dt[2] = 0;
  /* J00 = fx/tz, J02 = -fx txc/tz^2 with txc = tx (inside) or lim*tz (clamped) */
  dt[2] += dJ[0] * (-fx / (tz * tz));
  dt[2] += dJ[2] * (2.0 * fx * P->txc / (tz * tz * tz));
  if (P->clamp_x) dt[2] += dJ[2] * (-fx * P->limx / (tz * tz));
  else dt[0] += dJ[2] * (-fx / (tz * tz));
  dt[2] += dJ[4] * (-fy / (tz * tz));
  dt[2] += dJ[5] * (2.0 * fy * P->tyc / (tz * tz * tz));
  if (P->clamp_y) dt[2] += dJ[5] * (-fy * P->limy / (tz * tz));
  else dt[1] += dJ[5] * (-fy / (tz * tz));
  /* u = fx tx/tz + cx, v = fy ty/tz + cy, depth = tz */
  dt[0] += du * fx / tz;
  dt[2] += -du * fx * tx / (tz * tz);
  dt[1] += dv * fy / tz;
  dt[2] += -dv * fy * ty / (tz * tz);
  dt[2] += dz;
}

/* Projection backward of one Gaussian for one camera.  dp7 = gradient w.r.t.
 * (u, v, conic a, conic b, conic c, opacity, depth t_z).  Accumulates into
 * the parameter gradients. */
static void project_backward(const oproj* P, const ocam* cam, const double* dp7,
                             double* dmean, double* dquat, double* dls, double* dlogit) {
  double dS3[9], dJ[6], dt[3];
  camera_backward(P, cam, dp7, dS3, dJ, dt);
  /* opacity = sigmoid(logit) */
  *dlogit += dp7[5] * P->o * (1.0 - P->o);
  /* t = Rc p + tc */
  for (int j = 0; j < 3; j++)
    dmean[j] += cam->R[j] * dt[0] + cam->R[3 + j] * dt[1] + cam->R[6 + j] * dt[2];
  /* Sigma3 = M M^T: dM = 2 dSigma3 M; M = R S */
  double dM[9], dR[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double acc = 0;
      for (int k = 0; k < 3; k++) acc += dS3[3 * i + k] * P->M[3 * k + j];
      dM[3 * i + j] = 2.0 * acc;
    }
  for (int k = 0; k < 3; k++) {
    double ds = 0;
    for (int j = 0; j < 3; j++) ds += dM[3 * j + k] * P->Rq[3 * j + k];
    dls[k] += ds * P->s[k];
  }
  for (int j = 0; j < 3; j++)
    for (int k = 0; k < 3; k++) dR[3 * j + k] = dM[3 * j + k] * P->s[k];
  double w = P->qn[0], x = P->qn[1], y = P->qn[2], z = P->qn[3];
  double dqn[4];
  dqn[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  dqn[1] = 2 * (y * dR[1] + z * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] + z * dR[6] +
                w * dR[7] - 2 * x * dR[8]);
  dqn[2] = 2 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                z * dR[7] - 2 * y * dR[8]);
  dqn[3] = 2 * (-2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * z * dR[4] + y * dR[5] +
                x * dR[6] + y * dR[7]);
  double dotq = 0;
  for (int i = 0; i < 4; i++) dotq += P->qn[i] * dqn[i];
  for (int i = 0; i < 4; i++) dquat[i] += (dqn[i] - P->qn[i] * dotq) / P->qnorm;
}

int lgso_render_bwd(int64_t n, int d, const double* means, const double* quats,
                    const double* log_scales, const double* op_logits, const double* colors,
                    const double* feats, const double* camv, const double* bg, int x0, int y0,
                    int w, int h, const double* g_rgb, const double* g_dep, const double* g_feat,
                    double* d_means, double* d_quats, double* d_log_scales, double* d_logits,
                    double* d_colors, double* d_feats, double* d_proj) {
  ocam cam = read_cam(camv);
  oproj* P = (oproj*)malloc(sizeof(oproj) * (n ? n : 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  int64_t m = project_and_order(n, means, quats, log_scales, op_logits, &cam, P, order);
  double* dp7 = (double*)calloc((size_t)(n ? n : 1) * 7, sizeof(double));
#pragma omp parallel
  {
    blend_rec* list = (blend_rec*)malloc(sizeof(blend_rec) * (m ? m : 1));
    double* fbuf = (double*)malloc(sizeof(double) * (d ? 2 * d : 2));
    double* AF = fbuf + d;
#pragma omp for schedule(dynamic, 4)
    for (int64_t pix = 0; pix < (int64_t)w * h; pix++) {
      int x = x0 + (int)(pix % w), y = y0 + (int)(pix / w);
      double rgb[3], dep, T;
      int cnt = composite_pixel(x, y, d, P, order, m, colors, feats, bg, rgb, &dep, fbuf, &T,
                                NULL, NULL, list);
      const double* gr = g_rgb + 3 * pix;
      double gd = g_dep[pix];
      const double* gf = g_feat + (int64_t)d * pix;
      double AR[3] = {bg[0], bg[1], bg[2]}, AD = 0;
      for (int k = 0; k < d; k++) AF[k] = 0;
      for (int i = cnt - 1; i >= 0; i--) {
        const blend_rec* b = &list[i];
        const oproj* g = &P[b->g];
        const double* c = colors + 3 * b->g;
        const double* f = feats + (int64_t)d * b->g;
        double wgt = b->alpha * b->T;
        for (int k = 0; k < 3; k++) atomic_add(&d_colors[3 * b->g + k], wgt * gr[k]);
        for (int k = 0; k < d; k++) atomic_add(&d_feats[(int64_t)d * b->g + k], wgt * gf[k]);
        atomic_add(&dp7[7 * b->g + 6], wgt * gd);
        double dal = 0;
        for (int k = 0; k < 3; k++) dal += (c[k] - AR[k]) * gr[k];
        dal += (g->t[2] - AD) * gd;
        for (int k = 0; k < d; k++) dal += (f[k] - AF[k]) * gf[k];
        dal *= b->T;
        for (int k = 0; k < 3; k++) AR[k] = b->alpha * c[k] + (1 - b->alpha) * AR[k];
        AD = b->alpha * g->t[2] + (1 - b->alpha) * AD;
        for (int k = 0; k < d; k++) AF[k] = b->alpha * f[k] + (1 - b->alpha) * AF[k];
        if (b->clamped) continue;
        double dx = g->u - (x + 0.5), dy = g->v - (y + 0.5);
        double dpow = dal * b->alpha;
        atomic_add(&dp7[7 * b->g + 5], dal * exp(b->power));
        atomic_add(&dp7[7 * b->g + 0], -dpow * (g->conic[0] * dx + g->conic[1] * dy));
        atomic_add(&dp7[7 * b->g + 1], -dpow * (g->conic[2] * dy + g->conic[1] * dx));
        atomic_add(&dp7[7 * b->g + 2], -0.5 * dpow * dx * dx);
        atomic_add(&dp7[7 * b->g + 3], -dpow * dx * dy);
        atomic_add(&dp7[7 * b->g + 4], -0.5 * dpow * dy * dy);
      }
    }
    free(list);
    free(fbuf);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    if (!P[i].valid) continue;
    project_backward(&P[i], &cam, dp7 + 7 * i, d_means + 3 * i, d_quats + 4 * i,
                     d_log_scales + 3 * i, d_logits + i);
  }
  if (d_proj)
    for (int64_t i = 0; i < 7 * n; i++) d_proj[i] += dp7[i];
  free(dp7);
  free(P);
  free(order);
  return 0;
}

/* Projection backward alone, for checking the chain rule from given 2D
 * gradients (7 per Gaussian, as in lgso_render_bwd's d_proj). */
int lgso_project_bwd(int64_t n, const double* means, const double* quats, const double* log_scales,
                     const double* op_logits, const double* camv, const double* dp7,
                     double* d_means, double* d_quats, double* d_log_scales, double* d_logits) {
  ocam cam = read_cam(camv);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    oproj P;
    project_one(means + 3 * i, quats + 4 * i, log_scales + 3 * i, op_logits[i], &cam, &P);
    if (!P.valid) continue;
    project_backward(&P, &cam, dp7 + 7 * i, d_means + 3 * i, d_quats + 4 * i,
                     d_log_scales + 3 * i, d_logits + i);
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* binning                                                                 */

/* Whether a projected record reaches tile (tx, ty): its ellipse
   q(d) = a dx^2 + 2 b dx dy + c dy^2 <= cut, d = (u - x, v - y), meets the
   tile's pixel-centre square [16 tx + 0.5, 16 tx + 15.5] x [16 ty + 0.5,
   16 ty + 15.5].  The minimum of the convex q over the square is 0 when the
   mean is inside; otherwise it lies on one of the four edges, where q is a
   1-D quadratic whose minimiser (-b X / c, or -b Y / a, formed with the
   reciprocal of c or a) is clamped to the edge.  The decision turns
   a float into a bit, so it is taken in FP32 in one fixed order of
   operations, each rounded (compiled without contraction), as the GPU takes
   it.  rec = (u, v, a, b, c, o, tz, cut) as gs_project writes it. */
static int tile_hit32(const float* rec, int tx, int ty) {
  const float u = rec[0], v = rec[1], a = rec[2], b = rec[3], c = rec[4], cut = rec[7];
  const float ia = 1.0f / a, ic = 1.0f / c;  /* the edge minimisers use reciprocals */
  const float xa = (float)(16 * tx) + 0.5f, xb = (float)(16 * tx) + 15.5f;
  const float ya = (float)(16 * ty) + 0.5f, yb = (float)(16 * ty) + 15.5f;
  const float dx0 = u - xb, dx1 = u - xa, dy0 = v - yb, dy1 = v - ya;
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return 1;
  const float b2 = 2.f * b;
  float best = INFINITY;
  for (int e = 0; e < 4; e++) {
    float X, Y;
    if (e < 2) {  /* the edges dx = dx0 and dx = dx1 */
      X = e ? dx1 : dx0;
      Y = fminf(fmaxf(-(b * X) * ic, dy0), dy1);
    } else {      /* the edges dy = dy0 and dy = dy1 */
      Y = e == 3 ? dy1 : dy0;
      X = fminf(fmaxf(-(b * Y) * ia, dx0), dx1);
    }
    const float t1 = (a * X) * X, t2 = (b2 * X) * Y, t3 = (c * Y) * Y;
    const float q = (t1 + t2) + t3;
    best = fminf(best, q);
  }
  return best <= cut;
}

/* Instances of record i: the tiles of its rect that its ellipse reaches
   (proj NULL: every tile of the rect). */
static int64_t record_instances(const int32_t* r, const float* rec) {
  int64_t k = 0;
  if (!(r[2] > r[0] && r[3] > r[1])) return 0;
  for (int ty = r[1]; ty < r[3]; ty++)
    for (int tx = r[0]; tx < r[2]; tx++) k += !rec || tile_hit32(rec, tx, ty);
  return k;
}

int64_t lgso_bin_count(int64_t n, int ncams, const int32_t* rect, const float* proj) {
  int64_t k = 0;
  for (int64_t i = 0; i < (int64_t)ncams * n; i++)
    k += record_instances(rect + 4 * i, proj ? proj + 8 * i : NULL);
  return k;
}

typedef struct { uint64_t key; uint32_t id; } kv;

/* Stable bottom-up merge sort by key. */
static void merge_sort_kv(kv* a, int64_t n) {
  kv* tmp = (kv*)malloc(sizeof(kv) * (n ? n : 1));
  for (int64_t width = 1; width < n; width *= 2) {
    for (int64_t lo = 0; lo < n; lo += 2 * width) {
      int64_t mid = lo + width < n ? lo + width : n;
      int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
      int64_t i = lo, j = mid, o = lo;
      while (i < mid && j < hi) tmp[o++] = (a[j].key < a[i].key) ? a[j++] : a[i++];
      while (i < mid) tmp[o++] = a[i++];
      while (j < hi) tmp[o++] = a[j++];
    }
    memcpy(a, tmp, sizeof(kv) * n);
  }
  free(tmp);
}

int lgso_bin_sort(int64_t n, int ncams, int tiles_x, int tiles_y, const int32_t* rect,
                  const float* depth, const float* proj, uint64_t* keys, uint32_t* ids,
                  uint32_t* ranges) {
  int64_t ntiles = (int64_t)tiles_x * tiles_y;
  int64_t k = lgso_bin_count(n, ncams, rect, proj);
  kv* a = (kv*)malloc(sizeof(kv) * (k ? k : 1));
  int64_t o = 0;
  for (int c = 0; c < ncams; c++)
    for (int64_t i = 0; i < n; i++) {
      const int32_t* r = rect + 4 * ((int64_t)c * n + i);
      const float* rec = proj ? proj + 8 * ((int64_t)c * n + i) : NULL;
      uint32_t bits;
      memcpy(&bits, &depth[(int64_t)c * n + i], 4);
      for (int ty = r[1]; ty < r[3]; ty++)
        for (int tx = r[0]; tx < r[2]; tx++) {
          if (rec && !tile_hit32(rec, tx, ty)) continue;
          uint64_t tile = (uint64_t)c * ntiles + (uint64_t)ty * tiles_x + tx;
          a[o].key = (tile << 32) | bits;
          a[o].id = (uint32_t)i;
          o++;
        }
    }
  merge_sort_kv(a, k);
  memset(ranges, 0, sizeof(uint32_t) * 2 * ncams * ntiles);
  for (int64_t j = 0; j < k; j++) {
    keys[j] = a[j].key;
    ids[j] = a[j].id;
    uint64_t tile = a[j].key >> 32;
    if (j == 0 || (a[j - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)j;
    if (j == k - 1 || (a[j + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(j + 1);
  }
  free(a);
  return 0;
}

int lgso_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* camera pose gradient                                                     */

/* Gradient of the loss with respect to a left perturbation of the camera's
 * world->camera transform, T <- exp(xi^) T with xi = (rho, phi): the camera
 * frame moves by rho and rotates by phi (the keyframe pose refinement of
 * Sec. III-B.2 optimises this).  Under it t' = t + phi x t + rho and the
 * rotation in T = J Rc becomes (I + phi^) Rc, so per Gaussian
 *   dL/drho += dL/dt,   dL/dphi += t x dL/dt + vee(A^T - A),
 * A = J^T dJ... written out: with dT the gradient of T = J Rc,
 * dL = tr(dT^T J phi^ Rc) gives dL/dphi_k = -sum_ab A_ab eps_abk for
 * A = J^T dT Rc^T (= J^T dJ).  dproj [n,7] holds each Gaussian's gradient
 * w.r.t. (u, v, a, b, c, opacity, t_z) for this camera (as returned by
 * lgso_render_bwd).  out[6] = (dL/drho, dL/dphi). */
int lgso_pose_grad(int64_t n, const double* means, const double* quats, const double* log_scales,
                   const double* op_logits, const double* camv, const double* dproj,
                   double* out) {
  ocam cam = read_cam(camv);
  for (int k = 0; k < 6; k++) out[k] = 0;
  for (int64_t i = 0; i < n; i++) {
    oproj P;
    project_one(means + 3 * i, quats + 4 * i, log_scales + 3 * i, op_logits[i], &cam, &P);
    if (!P.valid) continue;
    const double* g = dproj + 7 * i;
    int nz = 0;
    for (int k = 0; k < 7; k++) nz |= g[k] != 0.0;
    if (!nz) continue;
    double dS3[9], dJ[6], dt[3];
    camera_backward(&P, &cam, g, dS3, dJ, dt);
    double A[9];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) A[3 * a + b] = P.J[a] * dJ[b] + P.J[3 + a] * dJ[3 + b];
    const double* t = P.t;
    out[0] += dt[0];
    out[1] += dt[1];
    out[2] += dt[2];
    out[3] += t[1] * dt[2] - t[2] * dt[1] + A[7] - A[5];
    out[4] += t[2] * dt[0] - t[0] * dt[2] + A[2] - A[6];
    out[5] += t[0] * dt[1] - t[1] * dt[0] + A[3] - A[1];
  }
  return 0;
}
