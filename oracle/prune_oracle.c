/*
 * CPU oracle of language-guided Gaussian pruning (LEGO-SLAM Sec. III-C,
 * Eq. 4) and the geometric criteria it is unioned with.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: only the tests,
 * the package's smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code with the CUDA library.
 *
 * The paper's rule: each Gaussian G_i looks at its K nearest neighbours in
 * 3D; a neighbour G_j is redundant when d(p_i, p_j) < tau_dist and
 * sim(f_i, f_j) > tau_sim (cosine of the compact language features); the
 * Gaussians pruned are the union of the redundant ones and those failing
 * the geometric criteria (low opacity, large scale).  Readings where the
 * paper is silent:
 *
 *   neighbours   the K nearest other Gaussians among those with
 *                d(p_i, p_j) < tau_dist, ranked by (squared distance, index);
 *   mutual case  G_i marks G_j only when G_i is the one to keep: higher
 *                opacity logit, or the same logit and the lower index (so a
 *                pair of mutual neighbours loses one member, not both);
 *   cosine       dot(f_i, f_j) / (|f_i| |f_j|), 0 when a norm is 0;
 *   geometric    opacity below min_opacity, taken as logit < logit(min_opacity),
 *                or largest scale above max_scale, taken as
 *                max_k log_s_k > log(max_scale) (the thresholds are rounded
 *                to float once, by the caller);
 *   output       mask[i] = geometric | redundant << 1 (0 keeps G_i).
 *
 * Precision: every decision here turns a float comparison into a bit of the
 * mask, so it is taken in FP32 with a fixed order of operations (products and
 * sums rounded one by one, left to right, no fused multiply-add; correctly
 * rounded sqrt and division), the precision the kernel uses:
 *   dx = x_j - x_i (same for y, z);  d2 = (dx dx + dy dy) + dz dz;
 *   d = sqrt(d2);  |f| = sqrt(sum_k f_k f_k);  dot = sum_k f_ik f_jk;
 *   sim = dot / (|f_i| |f_j|).
 * The search itself is brute force over all Gaussians (O(N^2)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PRUNE_KMAX 16

static float dist2f(const float* p, int64_t i, int64_t j) {
  const float dx = p[3 * j] - p[3 * i];
  const float dy = p[3 * j + 1] - p[3 * i + 1];
  const float dz = p[3 * j + 2] - p[3 * i + 2];
  const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
  const float s = xx + yy;
  return s + zz;
}

static float normf(const float* f, int d, int64_t i) {
  float s = 0.f;
  for (int k = 0; k < d; k++) {
    const float q = f[(int64_t)d * i + k] * f[(int64_t)d * i + k];
    s = s + q;
  }
  return sqrtf(s);
}

static float cosinef(const float* f, int d, const float* nrm, int64_t i, int64_t j) {
  float dot = 0.f;
  for (int k = 0; k < d; k++) {
    const float q = f[(int64_t)d * i + k] * f[(int64_t)d * j + k];
    dot = dot + q;
  }
  const float nn = nrm[i] * nrm[j];
  return nn > 0.f ? dot / nn : 0.f;
}

/* The K nearest neighbours of i within tau_dist, nearest first; returns the
 * count and writes their indices to nb. */
static int knn_within(int64_t n, const float* p, int64_t i, int k, float tau, int64_t* nb) {
  float bd[PRUNE_KMAX];
  int c = 0;
  for (int64_t j = 0; j < n; j++) {
    if (j == i) continue;
    const float d2 = dist2f(p, i, j);
    if (!(sqrtf(d2) < tau)) continue;
    /* rank by (d2, j); j ascends, so a tie never displaces an earlier j */
    if (c == k && !(d2 < bd[k - 1])) continue;
    int pos = c < k ? c : k - 1;
    while (pos > 0 && d2 < bd[pos - 1]) {
      bd[pos] = bd[pos - 1];
      nb[pos] = nb[pos - 1];
      pos--;
    }
    bd[pos] = d2;
    nb[pos] = j;
    if (c < k) c++;
  }
  return c;
}

static int keeps_over(const float* logit, int64_t i, int64_t j) {
  return logit[i] > logit[j] || (logit[i] == logit[j] && i < j);
}

static uint8_t geometric(const float* logit, const float* ls, int64_t i, float thr_logit,
                         float thr_logscale) {
  float m = ls[3 * i];
  if (ls[3 * i + 1] > m) m = ls[3 * i + 1];
  if (ls[3 * i + 2] > m) m = ls[3 * i + 2];
  return (uint8_t)((logit[i] < thr_logit || m > thr_logscale) ? 1 : 0);
}

/* Full mask.  means [n,3], logits [n], log_scales [n,3], feats [n,d], all
 * float32.  Returns 0, or -1 on bad arguments. */
int lgso_prune(int64_t n, int d, const float* means, const float* logits,
               const float* log_scales, const float* feats, int k, float tau_dist,
               float tau_sim, float thr_logit, float thr_logscale, uint8_t* mask) {
  if (n < 0 || d < 1 || k < 1 || k > PRUNE_KMAX) return -1;
  float* nrm = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  int64_t* nb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1) * PRUNE_KMAX);
  int* cnt = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  uint8_t* red = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!nrm || !nb || !cnt || !red) {
    free(nrm); free(nb); free(cnt); free(red);
    return -1;
  }
  for (int64_t i = 0; i < n; i++) nrm[i] = normf(feats, d, i);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; i++) cnt[i] = knn_within(n, means, i, k, tau_dist, nb + PRUNE_KMAX * i);
  for (int64_t i = 0; i < n; i++)
    for (int r = 0; r < cnt[i]; r++) {
      const int64_t j = nb[PRUNE_KMAX * i + r];
      if (cosinef(feats, d, nrm, i, j) > tau_sim && keeps_over(logits, i, j)) red[j] = 1;
    }
  for (int64_t i = 0; i < n; i++)
    mask[i] = (uint8_t)(geometric(logits, log_scales, i, thr_logit, thr_logscale) | (red[i] << 1));
  free(nrm); free(nb); free(cnt); free(red);
  return 0;
}

/* The mask of the m Gaussians idx[0..m) only, each decided from scratch: G_j
 * is redundant if some G_i within tau_dist has G_j among its K nearest, is
 * similar enough, and is the one to keep.  Same readings as lgso_prune. */
int lgso_prune_sample(int64_t n, int d, const float* means, const float* logits,
                      const float* log_scales, const float* feats, int k, float tau_dist,
                      float tau_sim, float thr_logit, float thr_logscale, const int64_t* idx,
                      int64_t m, uint8_t* out) {
  if (n < 0 || d < 1 || k < 1 || k > PRUNE_KMAX) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < m; s++) {
    const int64_t j = idx[s];
    if (j < 0 || j >= n) {
      bad = 1;
      continue;
    }
    uint8_t r = 0;
    const float nj = normf(feats, d, j);
    for (int64_t i = 0; i < n && !r; i++) {
      if (i == j || !(sqrtf(dist2f(means, i, j)) < tau_dist)) continue;
      if (!keeps_over(logits, i, j)) continue;
      /* cosine with the same operation order as cosinef */
      float dot = 0.f;
      for (int c = 0; c < d; c++) {
        const float q = feats[(int64_t)d * i + c] * feats[(int64_t)d * j + c];
        dot = dot + q;
      }
      const float nn = normf(feats, d, i) * nj;
      const float sim = nn > 0.f ? dot / nn : 0.f;
      if (!(sim > tau_sim)) continue;
      int64_t nb[PRUNE_KMAX];
      const int c = knn_within(n, means, i, k, tau_dist, nb);
      for (int q = 0; q < c; q++)
        if (nb[q] == j) r = 1;
    }
    out[s] = (uint8_t)(geometric(logits, log_scales, j, thr_logit, thr_logscale) | (r << 1));
  }
  return bad ? -1 : 0;
}
