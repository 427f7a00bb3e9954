/*
 * scsc_oracle.c -- FP64 CPU oracle for stochastic convolutional sparse coding.
 *
 * TEST INFRASTRUCTURE ONLY (see scsc_oracle.h).  Plain loops written from the
 * definitions in the paper; no blocking, fusion or reordering.  OpenMP, where
 * present, only splits independent output elements between threads and never
 * changes the order of any sum.
 */
#include "scsc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Counter-based hash and the subsampling matrix M^t (Sec. 3.1)              */
/* ------------------------------------------------------------------------ */

/* SplitMix64 output function, as published by Steele, Lea & Flood (2014):
 * add the golden-ratio increment, then two xor-shift-multiply rounds and a
 * final xor-shift, all modulo 2^64. */
uint64_t orc_splitmix64(uint64_t v) {
  uint64_t z = v + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Coordinate (k, y, x) of image n is kept at outer iteration t when the top
 * 32 bits of its hash fall below T = floor(p * 2^32), p = p_num / p_den.
 * p = 1 gives T = 2^32, so every coordinate is kept and M^t = I (Sec. 3.1). */
int orc_is_sampled(uint64_t seed, uint64_t t, uint64_t n, int H, int W,
                   int k, int y, int x, uint32_t p_num, uint32_t p_den) {
  uint64_t T = ((uint64_t)p_num << 32) / (uint64_t)p_den;
  uint64_t idx = ((uint64_t)k * (uint64_t)H + (uint64_t)y) * (uint64_t)W +
                 (uint64_t)x;
  uint64_t h = orc_splitmix64(seed);
  h = orc_splitmix64(h ^ t);
  h = orc_splitmix64(h ^ n);
  h = orc_splitmix64(h ^ idx);
  return (h >> 32) < T;
}

void orc_mask_image(uint64_t seed, uint64_t t, uint64_t n, int K, int H, int W,
                    uint32_t p_num, uint32_t p_den, uint8_t *mask) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x)
      for (int k = 0; k < K; ++k)
        mask[((size_t)y * W + x) * K + k] =
            (uint8_t)orc_is_sampled(seed, t, n, H, W, k, y, x, p_num, p_den);
}

/* ------------------------------------------------------------------------ */
/* The convolution operator D and its adjoints (Sec. 3.1)                    */
/* ------------------------------------------------------------------------ */

static double code_at(const double *z, int K, int H, int W, int k, int y,
                      int x) {
  if (y < 0 || y >= H || x < 0 || x >= W) return 0.0;
  return z[((size_t)y * W + x) * K + k];
}

static double pix_at(const double *r, int H, int W, int y, int x) {
  if (y < 0 || y >= H || x < 0 || x >= W) return 0.0;
  return r[(size_t)y * W + x];
}

/* xhat(i,j) = sum_k sum_{u,v} d_k(u,v) z_k(i+c-u, j+c-v): a true (flipped)
 * convolution with the filter centred at (c, c). */
void orc_synthesis(int K, int s, int H, int W, const double *d, const double *z,
                   double *xhat) {
  const int c = (s - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      double acc = 0.0;
      for (int k = 0; k < K; ++k)
        for (int u = 0; u < s; ++u)
          for (int v = 0; v < s; ++v)
            acc += d[((size_t)k * s + u) * s + v] *
                   code_at(z, K, H, W, k, i + c - u, j + c - v);
      xhat[(size_t)i * W + j] = acc;
    }
}

/* (D^T r)_k(a,b) = sum_{u,v} d_k(u,v) r(a-c+u, b-c+v): correlation. */
void orc_adjoint(int K, int s, int H, int W, const double *d, const double *r,
                 double *g) {
  const int c = (s - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < W; ++b)
      for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int u = 0; u < s; ++u)
          for (int v = 0; v < s; ++v)
            acc += d[((size_t)k * s + u) * s + v] *
                   pix_at(r, H, W, a - c + u, b - c + v);
        g[((size_t)a * W + b) * K + k] = acc;
      }
}

/* The same correlation at the sampled coordinates only (mask[(a W + b) K + k]
 * set): the gradient of Eq. 3 with respect to its pDK sampled variables
 * (Sec. 3.1).  Each value is the same sum, in the same order, as orc_adjoint's;
 * entries off the sampled set are not written. */
void orc_adjoint_sampled(int K, int s, int H, int W, const double *d, const double *r,
                         const uint8_t *mask, double *g) {
  const int c = (s - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < W; ++b)
      for (int k = 0; k < K; ++k) {
        const size_t i = ((size_t)a * W + b) * K + k;
        if (!mask[i]) continue;
        double acc = 0.0;
        for (int u = 0; u < s; ++u)
          for (int v = 0; v < s; ++v)
            acc += d[((size_t)k * s + u) * s + v] *
                   pix_at(r, H, W, a - c + u, b - c + v);
        g[i] = acc;
      }
}

/* G_k(u,v) = sum_{i,j} r(i,j) z_k(i+c-u, j+c-v) = (Z^T r)_{k,u,v}. */
void orc_filter_gradient(int K, int s, int H, int W, const double *r,
                         const double *z, double *G) {
  const int c = (s - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < K; ++k)
    for (int u = 0; u < s; ++u)
      for (int v = 0; v < s; ++v) {
        double acc = 0.0;
        for (int i = 0; i < H; ++i)
          for (int j = 0; j < W; ++j)
            acc += r[(size_t)i * W + j] *
                   code_at(z, K, H, W, k, i + c - u, j + c - v);
        G[((size_t)k * s + u) * s + v] = acc;
      }
}

/* ------------------------------------------------------------------------ */
/* Prox, projection, objective                                               */
/* ------------------------------------------------------------------------ */

/* sign(v) * max(|v| - tau, 0); |v| <= tau (equality included) gives 0. */
double orc_soft_threshold(double v, double tau) {
  if (v > tau) return v - tau;
  if (v < -tau) return v + tau;
  return 0.0;
}

/* d_k <- d_k / max(1, ||d_k||_2): Euclidean projection onto the unit ball. */
void orc_project_filters(int K, int M, double *d) {
  for (int k = 0; k < K; ++k) {
    double ss = 0.0;
    for (int m = 0; m < M; ++m) ss += d[(size_t)k * M + m] * d[(size_t)k * M + m];
    double nrm = sqrt(ss);
    if (nrm > 1.0)
      for (int m = 0; m < M; ++m) d[(size_t)k * M + m] /= nrm;
  }
}

double orc_objective_image(int K, int s, int H, int W, const double *d,
                           const double *z, const double *x, double lambda) {
  size_t D = (size_t)H * W;
  double *xh = (double *)malloc(D * sizeof(double));
  orc_synthesis(K, s, H, W, d, z, xh);
  double data = 0.0, l1 = 0.0;
  for (size_t i = 0; i < D; ++i) data += (x[i] - xh[i]) * (x[i] - xh[i]);
  for (size_t i = 0; i < D * (size_t)K; ++i) l1 += fabs(z[i]);
  free(xh);
  return 0.5 * data + lambda * l1;
}

/* ------------------------------------------------------------------------ */
/* Proximal gradient on the subsampled code problem (Eq. 3, Eq. 4)           */
/* ------------------------------------------------------------------------ */

void orc_code_update_image(int K, int s, int H, int W, const double *d,
                           const double *x, double *z, const uint8_t *mask,
                           double alpha, double lambda, int n_iters) {
  size_t D = (size_t)H * W, DK = D * (size_t)K;
  double *r = (double *)malloc(D * sizeof(double));
  double *g = (double *)malloc(DK * sizeof(double));
  /* Eq. 4: codes outside the sampled set are zero; the sampled ones start
   * from the previous codes (warm start). */
  for (size_t i = 0; i < DK; ++i)
    if (!mask[i]) z[i] = 0.0;
  for (int it = 0; it < n_iters; ++it) {
    orc_synthesis(K, s, H, W, d, z, r);
    for (size_t i = 0; i < D; ++i) r[i] -= x[i];
    orc_adjoint_sampled(K, s, H, W, d, r, mask, g);
    for (size_t i = 0; i < DK; ++i)
      if (mask[i]) z[i] = orc_soft_threshold(z[i] - alpha * g[i], alpha * lambda);
  }
  free(r);
  free(g);
}

/* Variant of the code update for the other reading of Sec. 3.1 (each
 * iteration works on the pDK sampled variables while the rest remain
 * unchanged): codes off the sampled set keep their previous values instead of
 * Eq. 4's zeros, and the sampled ones take n_iters proximal-gradient steps on
 * 1/2 || x - D z ||^2 + lambda || z_S ||_1 with z off S held fixed, i.e. with
 * the residual of all the codes. */
void orc_code_update_image_keep(int K, int s, int H, int W, const double *d,
                                const double *x, double *z, const uint8_t *mask,
                                double alpha, double lambda, int n_iters) {
  size_t D = (size_t)H * W, DK = D * (size_t)K;
  double *r = (double *)malloc(D * sizeof(double));
  double *g = (double *)malloc(DK * sizeof(double));
  for (int it = 0; it < n_iters; ++it) {
    orc_synthesis(K, s, H, W, d, z, r);
    for (size_t i = 0; i < D; ++i) r[i] -= x[i];
    orc_adjoint_sampled(K, s, H, W, d, r, mask, g);
    for (size_t i = 0; i < DK; ++i)
      if (mask[i]) z[i] = orc_soft_threshold(z[i] - alpha * g[i], alpha * lambda);
  }
  free(r);
  free(g);
}

/* ------------------------------------------------------------------------ */
/* Inpainting: observed pixels only in the data term (Sec. 4.3)              */
/* ------------------------------------------------------------------------ */

double orc_objective_image_observed(int K, int s, int H, int W, const double *d,
                                    const double *z, const double *x, const uint8_t *obs,
                                    double lambda) {
  size_t D = (size_t)H * W;
  double *xh = (double *)malloc(D * sizeof(double));
  orc_synthesis(K, s, H, W, d, z, xh);
  double data = 0.0, l1 = 0.0;
  for (size_t i = 0; i < D; ++i)
    if (obs[i]) data += (x[i] - xh[i]) * (x[i] - xh[i]);
  for (size_t i = 0; i < D * (size_t)K; ++i) l1 += fabs(z[i]);
  free(xh);
  return 0.5 * data + lambda * l1;
}

void orc_code_update_image_observed(int K, int s, int H, int W, const double *d,
                                    const double *x, double *z, const uint8_t *mask,
                                    const uint8_t *obs, double alpha, double lambda,
                                    int n_iters) {
  size_t D = (size_t)H * W, DK = D * (size_t)K;
  double *r = (double *)malloc(D * sizeof(double));
  double *g = (double *)malloc(DK * sizeof(double));
  for (size_t i = 0; i < DK; ++i)
    if (!mask[i]) z[i] = 0.0;
  for (int it = 0; it < n_iters; ++it) {
    orc_synthesis(K, s, H, W, d, z, r);
    /* gradient of 0.5 || O (x - D z) ||^2 is D^T O (D z - x) */
    for (size_t i = 0; i < D; ++i) r[i] = obs[i] ? r[i] - x[i] : 0.0;
    orc_adjoint_sampled(K, s, H, W, d, r, mask, g);
    for (size_t i = 0; i < DK; ++i)
      if (mask[i]) z[i] = orc_soft_threshold(z[i] - alpha * g[i], alpha * lambda);
  }
  free(r);
  free(g);
}

/* ------------------------------------------------------------------------ */
/* Power iterations for the Lipschitz constants of the gradient steps        */
/* ------------------------------------------------------------------------ */

typedef void (*orc_linop)(const void *ctx, const double *in, double *out);

static double dot(size_t n, const double *a, const double *b) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* u0_i = +1 or -1 by the top bit of mix(mix(seed ^ tag) ^ i); then `iters`
 * times u <- A u / ||A u||; the estimate is the Rayleigh quotient <u, A u>.
 * An operator that maps the iterate to zero gives the estimate 0. */
static double power_iteration(size_t n, orc_linop A, const void *ctx,
                              uint64_t seed, uint64_t tag, int iters) {
  double *u = (double *)malloc(n * sizeof(double));
  double *w = (double *)malloc(n * sizeof(double));
  uint64_t base = orc_splitmix64(seed ^ tag);
  for (size_t i = 0; i < n; ++i)
    u[i] = (orc_splitmix64(base ^ (uint64_t)i) >> 63) ? -1.0 : 1.0;
  double un = sqrt(dot(n, u, u));
  for (size_t i = 0; i < n; ++i) u[i] /= un;
  double est = 0.0;
  int dead = 0;
  for (int it = 0; it < iters; ++it) {
    A(ctx, u, w);
    double nrm = sqrt(dot(n, w, w));
    if (!(nrm > 0.0)) { dead = 1; break; }
    for (size_t i = 0; i < n; ++i) u[i] = w[i] / nrm;
  }
  if (!dead) {
    A(ctx, u, w);
    est = dot(n, u, w);
  }
  free(u);
  free(w);
  return est;
}

typedef struct { int K, s, H, W; const double *d; double *tmp; } ddt_ctx;

static void apply_ddt(const void *vctx, const double *in, double *out) {
  const ddt_ctx *c = (const ddt_ctx *)vctx;
  orc_adjoint(c->K, c->s, c->H, c->W, c->d, in, c->tmp);
  orc_synthesis(c->K, c->s, c->H, c->W, c->d, c->tmp, out);
}

double orc_power_ddt(int K, int s, int H, int W, const double *d, uint64_t seed,
                     uint64_t tag, int iters) {
  ddt_ctx c = {K, s, H, W, d, NULL};
  c.tmp = (double *)malloc((size_t)H * W * K * sizeof(double));
  double est = power_iteration((size_t)H * W, apply_ddt, &c, seed, tag, iters);
  free(c.tmp);
  return est;
}

typedef struct {
  int n_img; const int64_t *off; const int *H; const int *W; int K, s;
  const double *z_all; double *pix; double *gk;
} ztz_ctx;

/* (sum_n Z_n^T Z_n) v: synthesise every image's codes with filters v, then
 * take the filter gradient of that synthesis and sum over images. */
static void apply_ztz(const void *vctx, const double *in, double *out) {
  const ztz_ctx *c = (const ztz_ctx *)vctx;
  size_t KM = (size_t)c->K * c->s * c->s;
  memset(out, 0, KM * sizeof(double));
  for (int n = 0; n < c->n_img; ++n) {
    const double *z = c->z_all + (size_t)c->off[n] * c->K;
    orc_synthesis(c->K, c->s, c->H[n], c->W[n], in, z, c->pix);
    orc_filter_gradient(c->K, c->s, c->H[n], c->W[n], c->pix, z, c->gk);
    for (size_t i = 0; i < KM; ++i) out[i] += c->gk[i];
  }
}

double orc_power_ztz(int n_img, const int64_t *off, const int *H, const int *W,
                     int K, int s, const double *z_all, uint64_t seed,
                     uint64_t tag, int iters) {
  size_t maxD = 0, KM = (size_t)K * s * s;
  for (int n = 0; n < n_img; ++n)
    if ((size_t)H[n] * W[n] > maxD) maxD = (size_t)H[n] * W[n];
  ztz_ctx c = {n_img, off, H, W, K, s, z_all, NULL, NULL};
  c.pix = (double *)malloc((maxD ? maxD : 1) * sizeof(double));
  c.gk = (double *)malloc(KM * sizeof(double));
  double est = power_iteration(KM, apply_ztz, &c, seed, tag, iters);
  free(c.pix);
  free(c.gk);
  return est;
}

typedef struct { int n; const double *C; } dense_ctx;

static void apply_dense(const void *vctx, const double *in, double *out) {
  const dense_ctx *c = (const dense_ctx *)vctx;
  for (int i = 0; i < c->n; ++i) out[i] = dot((size_t)c->n, c->C + (size_t)i * c->n, in);
}

double orc_power_dense(int n, const double *C, uint64_t seed, uint64_t tag,
                       int iters) {
  dense_ctx c = {n, C};
  return power_iteration((size_t)n, apply_dense, &c, seed, tag, iters);
}

/* ------------------------------------------------------------------------ */
/* Online surrogates (Eq. 7)                                                 */
/* ------------------------------------------------------------------------ */

/* Row (i,j) of the code Toeplitz matrix Z is z_k(i+c-u, j+c-v) over the
 * column index (k,u,v).  Z^T Z is the sum of the outer products of its rows
 * and Z^T x the x-weighted sum of its rows. */
void orc_surrogate_accumulate(int K, int s, int H, int W, const double *z,
                              const double *x, double scale, double *C,
                              double *B) {
  const int c = (s - 1) / 2;
  const int M = s * s, KM = K * M;
  double *row = (double *)malloc((size_t)KM * sizeof(double));
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      for (int k = 0; k < K; ++k)
        for (int u = 0; u < s; ++u)
          for (int v = 0; v < s; ++v)
            row[k * M + u * s + v] = code_at(z, K, H, W, k, i + c - u, j + c - v);
      double xv = x[(size_t)i * W + j];
      for (int a = 0; a < KM; ++a) {
        if (row[a] == 0.0) continue; /* exact: the whole row a term is zero */
        double ra = scale * row[a];
        for (int b = 0; b < KM; ++b) C[(size_t)a * KM + b] += ra * row[b];
        B[a] += ra * xv;
      }
    }
  free(row);
}

/* ------------------------------------------------------------------------ */
/* ADMM on Eq. 3 (cross-check of the PG solution, Sec. 3.2)                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int K, s, H, W; const double *d; const uint8_t *mask; double rho;
  double *pix; double *tmp;
} qp_ctx;

/* v -> 1_S (D^T D (1_S v)) + rho v over the full code vector. */
static void apply_qp(const qp_ctx *c, const double *in, double *out) {
  size_t DK = (size_t)c->H * c->W * c->K;
  for (size_t i = 0; i < DK; ++i) c->tmp[i] = c->mask[i] ? in[i] : 0.0;
  orc_synthesis(c->K, c->s, c->H, c->W, c->d, c->tmp, c->pix);
  orc_adjoint(c->K, c->s, c->H, c->W, c->d, c->pix, out);
  for (size_t i = 0; i < DK; ++i)
    out[i] = c->mask[i] ? out[i] + c->rho * in[i] : 0.0;
}

void orc_admm_image(int K, int s, int H, int W, const double *d,
                    const double *x, double *z, const uint8_t *mask,
                    double lambda, double rho, double alpha_r, int n_iters,
                    int cg_iters) {
  size_t D = (size_t)H * W, DK = D * (size_t)K;
  double *y = (double *)calloc(DK, sizeof(double));
  double *u = (double *)calloc(DK, sizeof(double));
  double *b = (double *)malloc(DK * sizeof(double));
  double *atx = (double *)malloc(DK * sizeof(double));
  double *res = (double *)malloc(DK * sizeof(double));
  double *p = (double *)malloc(DK * sizeof(double));
  double *Ap = (double *)malloc(DK * sizeof(double));
  qp_ctx q = {K, s, H, W, d, mask, rho, NULL, NULL};
  q.pix = (double *)malloc(D * sizeof(double));
  q.tmp = (double *)malloc(DK * sizeof(double));

  orc_adjoint(K, s, H, W, d, x, atx);
  for (size_t i = 0; i < DK; ++i) {
    if (!mask[i]) z[i] = 0.0;
    y[i] = z[i];
  }
  for (int it = 0; it < n_iters; ++it) {
    /* QP substep: (A^T A + rho I) z = A^T x + rho (y - u), A = D (M^t)^T,
     * solved by conjugate gradient from the current z. */
    for (size_t i = 0; i < DK; ++i)
      b[i] = mask[i] ? atx[i] + rho * (y[i] - u[i]) : 0.0;
    apply_qp(&q, z, Ap);
    for (size_t i = 0; i < DK; ++i) { res[i] = b[i] - Ap[i]; p[i] = res[i]; }
    double rr = dot(DK, res, res);
    double bb = dot(DK, b, b);
    for (int k = 0; k < cg_iters && rr > 1e-30 * (bb > 0 ? bb : 1.0); ++k) {
      apply_qp(&q, p, Ap);
      double a = rr / dot(DK, p, Ap);
      for (size_t i = 0; i < DK; ++i) { z[i] += a * p[i]; res[i] -= a * Ap[i]; }
      double rr2 = dot(DK, res, res);
      for (size_t i = 0; i < DK; ++i) p[i] = res[i] + (rr2 / rr) * p[i];
      rr = rr2;
    }
    /* Over-relaxation, shrinkage substep, scaled dual update. */
    for (size_t i = 0; i < DK; ++i) {
      if (!mask[i]) continue;
      double zh = alpha_r * z[i] + (1.0 - alpha_r) * y[i];
      double yn = orc_soft_threshold(zh + u[i], lambda / rho);
      u[i] += zh - yn;
      y[i] = yn;
    }
  }
  /* The sparse split variable is the returned solution. */
  for (size_t i = 0; i < DK; ++i) z[i] = mask[i] ? y[i] : 0.0;
  free(y); free(u); free(b); free(atx); free(res); free(p); free(Ap);
  free(q.pix); free(q.tmp);
}

/* ------------------------------------------------------------------------ */
/* Safe screening of the code problem (Sec. 5)                               */
/* ------------------------------------------------------------------------ */

/* Margins of the sphere test (see scsc_oracle.h). */
#define SCREEN_ETA 1e-6
#define SCREEN_TAU 1e-4

/* ||a_j||^2 for column j = (k, a, b) of D: code z_k(a, b) reaches pixel
 * (a - c + u, b - c + v) with weight d_k(u, v); taps off the image drop. */
static double column_norm2(int s, int H, int W, const double *d, int k, int a,
                           int b) {
  const int c = (s - 1) / 2;
  double acc = 0.0;
  for (int u = 0; u < s; ++u)
    for (int v = 0; v < s; ++v) {
      int i = a - c + u, j = b - c + v;
      if (i < 0 || i >= H || j < 0 || j >= W) continue;
      double w = d[((size_t)k * s + u) * s + v];
      acc += w * w;
    }
  return acc;
}

int64_t orc_screen_image(int K, int s, int H, int W, const double *d,
                         const double *x, double *z, uint8_t *mask,
                         double lambda, double *gap_out, double *stat) {
  size_t D = (size_t)H * W, DK = D * (size_t)K;
  double *rho = (double *)malloc(D * sizeof(double));
  double *corr = (double *)malloc(DK * sizeof(double));
  for (size_t i = 0; i < DK; ++i)
    if (!mask[i]) z[i] = 0.0;
  /* residual rho = x - D z and correlations a_j . rho = (D^T rho)_j */
  orc_synthesis(K, s, H, W, d, z, rho);
  for (size_t i = 0; i < D; ++i) rho[i] = x[i] - rho[i];
  orc_adjoint(K, s, H, W, d, rho, corr);
  double scale = lambda, l1 = 0.0;
  for (size_t i = 0; i < DK; ++i)
    if (mask[i]) {
      if (fabs(corr[i]) > scale) scale = fabs(corr[i]);
      l1 += fabs(z[i]);
    }
  /* primal value, dual value at theta = rho / scale, their gap */
  double data = 0.0, dist = 0.0, xx = 0.0;
  for (size_t i = 0; i < D; ++i) {
    double theta = rho[i] / scale, e = theta - x[i] / lambda;
    data += rho[i] * rho[i];
    dist += e * e;
    xx += x[i] * x[i];
  }
  double primal = 0.5 * data + lambda * l1;
  double dual = 0.5 * xx - 0.5 * lambda * lambda * dist;
  double gap = primal - dual;
  if (gap < 0.0) gap = 0.0;
  /* the sphere uses the gap plus SCREEN_ETA (P + ||x||^2 / 2): a bound on the
   * rounding of P and the dual value in FP32 sums of that magnitude */
  double radius = sqrt(2.0 * (gap + SCREEN_ETA * (primal + 0.5 * xx))) / lambda;
  int64_t kept = 0;
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < W; ++b)
      for (int k = 0; k < K; ++k) {
        size_t i = ((size_t)a * W + b) * K + k;
        if (!mask[i]) {
          if (stat) stat[i] = NAN;
          continue;
        }
        double t = fabs(corr[i]) / scale +
                   radius * sqrt(column_norm2(s, H, W, d, k, a, b));
        if (stat) stat[i] = t;
        if (t < 1.0 - SCREEN_TAU) {
          mask[i] = 0;
          z[i] = 0.0;
        } else {
          ++kept;
        }
      }
  if (gap_out) *gap_out = gap;
  free(rho);
  free(corr);
  return kept;
}

int64_t orc_code_update_image_screened(int K, int s, int H, int W,
                                       const double *d, const double *x,
                                       double *z, uint8_t *mask, double alpha,
                                       double lambda, int n_iters,
                                       int screen_every, double *gap_out) {
  size_t DK = (size_t)H * W * K;
  int64_t kept = 0;
  for (size_t i = 0; i < DK; ++i) {
    if (!mask[i]) z[i] = 0.0;
    kept += mask[i] != 0;
  }
  for (int it = 0; it < n_iters; ++it) {
    if (screen_every > 0 && it % screen_every == 0)
      kept = orc_screen_image(K, s, H, W, d, x, z, mask, lambda, gap_out, NULL);
    orc_code_update_image(K, s, H, W, d, x, z, mask, alpha, lambda, 1);
  }
  return kept;
}
