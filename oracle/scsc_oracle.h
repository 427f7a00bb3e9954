/*
 * scsc_oracle.h -- FP64 CPU oracle for stochastic convolutional sparse coding
 * (Xiong, Richtarik, Heidrich, "Stochastic Convolutional Sparse Coding", 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Conventions (one image of H x W pixels, K filters of s x s taps, s odd,
 * c = (s-1)/2 is the filter centre, M = s*s):
 *   x    : image,  row-major [H][W]
 *   z    : codes,  [H][W][K]   (z_k(y,x) = z[(y*W + x)*K + k])
 *   d    : filters, [K][s][s]  (d_k(u,v) = d[(k*s + u)*s + v])
 *   mask : [H][W][K] bytes, 1 = coordinate sampled
 * Codes have the size of the image (Sec. 2, z_k in R^D) and both codes and
 * residuals are zero outside the image (spatial domain, zero padding).
 *
 * Parity status: every function below is pinned by a CPU test against a
 * closed form, an invariant, a library routine or brute force.
 */
#ifndef SCSC_ORACLE_H
#define SCSC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SplitMix64 output mix (Steele, Lea & Flood, OOPSLA 2014). */
uint64_t orc_splitmix64(uint64_t v);

/* Bernoulli(p_num/p_den) draw for code coordinate (k, y, x) of global image
 * index n at outer iteration t (subsampling matrix M^t, Sec. 3.1). */
int orc_is_sampled(uint64_t seed, uint64_t t, uint64_t n, int H, int W,
                   int k, int y, int x, uint32_t p_num, uint32_t p_den);

/* Whole mask of one image, [H][W][K] bytes. */
void orc_mask_image(uint64_t seed, uint64_t t, uint64_t n, int K, int H, int W,
                    uint32_t p_num, uint32_t p_den, uint8_t *mask);

/* Synthesis D z = sum_k d_k * z_k (Sec. 3.1, Eq. 1 data term). */
void orc_synthesis(int K, int s, int H, int W, const double *d, const double *z,
                   double *xhat);

/* Adjoint D^T r: (D^T r)_k(a,b) = sum_{u,v} d_k(u,v) r(a-c+u, b-c+v). */
void orc_adjoint(int K, int s, int H, int W, const double *d, const double *r,
                 double *g);
/* The adjoint at the sampled coordinates only (mask[(a W + b) K + k] set), the
 * gradient of Eq. 3 in its pDK variables; other entries of g are not written. */
void orc_adjoint_sampled(int K, int s, int H, int W, const double *d, const double *r,
                         const uint8_t *mask, double *g);

/* Filter gradient Z^T r: G_k(u,v) = sum_{i,j} r(i,j) z_k(i+c-u, j+c-v)
 * (gradient of Eq. 5's data term).  Writes G [K][s][s]. */
void orc_filter_gradient(int K, int s, int H, int W, const double *r,
                         const double *z, double *G);

/* Point-wise shrinkage: argmin_w 0.5 (w - v)^2 + tau |w|. */
double orc_soft_threshold(double v, double tau);

/* Projection of each filter onto the unit ball ||d_k||_2 <= 1 (Eq. 1, 5). */
void orc_project_filters(int K, int M, double *d);

/* 0.5 ||x - D z||^2 + lambda ||z||_1 for one image (Eq. 1). */
double orc_objective_image(int K, int s, int H, int W, const double *d,
                           const double *z, const double *x, double lambda);

/* Proximal-gradient solve of Eq. 3 for one image and one outer iteration:
 * unsampled codes are set to zero (Eq. 4), then n_iters times
 *   r = D z - x;  z_S <- soft(z_S - alpha (D^T r)_S, alpha lambda).
 * z is in/out: in = warm start (previous codes), out = Eq. 4 codes. */
void orc_code_update_image(int K, int s, int H, int W, const double *d,
                           const double *x, double *z, const uint8_t *mask,
                           double alpha, double lambda, int n_iters);
/* orc_code_update_image with the codes off the sampled set kept (not zeroed):
 * the sampled codes are updated against the residual of all the codes. */
void orc_code_update_image_keep(int K, int s, int H, int W, const double *d,
                                const double *x, double *z, const uint8_t *mask,
                                double alpha, double lambda, int n_iters);

/* Inpainting (Sec. 4.3, reconstruction from partially observed pixels): the
 * data term only counts observed pixels, 0.5 || O (x - D z) ||^2 with
 * O = diag(obs), obs[i] != 0 = observed.
 *   objective: 0.5 sum_i obs_i (x_i - (D z)_i)^2 + lambda ||z||_1;
 *   code update: as orc_code_update_image with r = O (D z - x). */
double orc_objective_image_observed(int K, int s, int H, int W, const double *d,
                                    const double *z, const double *x, const uint8_t *obs,
                                    double lambda);
void orc_code_update_image_observed(int K, int s, int H, int W, const double *d,
                                    const double *x, double *z, const uint8_t *mask,
                                    const uint8_t *obs, double alpha, double lambda,
                                    int n_iters);

/* Power iteration estimate of lambda_max(D D^T) on an H x W pixel domain.
 * Start u_i = +-1 from the top bit of mix(mix(seed ^ tag) ^ i); `iters`
 * normalised applications, then the Rayleigh quotient. */
double orc_power_ddt(int K, int s, int H, int W, const double *d, uint64_t seed,
                     uint64_t tag, int iters);

/* Power iteration estimate of lambda_max(sum_n Z_n^T Z_n) in filter space
 * (K*s*s), codes of a batch packed at off[n]*K. */
double orc_power_ztz(int n_img, const int64_t *off, const int *H, const int *W,
                     int K, int s, const double *z_all, uint64_t seed,
                     uint64_t tag, int iters);

/* Power iteration estimate of lambda_max of a dense symmetric n x n matrix. */
double orc_power_dense(int n, const double *C, uint64_t seed, uint64_t tag,
                       int iters);

/* C += scale * Z^T Z and B += scale * Z^T x for one image (Eq. 7 terms).
 * C is [K*M][K*M] row-major, B is [K*M]. */
void orc_surrogate_accumulate(int K, int s, int H, int W, const double *z,
                              const double *x, double scale, double *C,
                              double *B);

/* ADMM for the LASSO of Eq. 3 restricted to the sampled coordinates
 * (Sec. 3.2: split data term / L1 term, over-relaxation alpha_r, penalty rho,
 * QP substep by conjugate gradient).  z is in/out (warm start). */
void orc_admm_image(int K, int s, int H, int W, const double *d,
                    const double *x, double *z, const uint8_t *mask,
                    double lambda, double rho, double alpha_r, int n_iters,
                    int cg_iters);

/* Safe screening of the code problem (Sec. 5 names safe screening of this
 * sparse LASSO as a way to skip updates; the rule below is the duality-gap
 * sphere test).  Problem: Eq. 3 for one image restricted to the active set
 * S = {mask != 0}: P(z) = 0.5 ||x - D z||^2 + lambda ||z_S||_1.  Its dual is
 *   Dual(theta) = 0.5 ||x||^2 - 0.5 lambda^2 || theta - x / lambda ||^2
 *   over |a_j . theta| <= 1 for j in S  (a_j = column j of D).
 * At the current z (set to zero off S first): rho = x - D z, the dual point
 * theta = rho / max(lambda, max_{j in S} |a_j . rho|), gap = P(z) - Dual(theta)
 * (clamped at 0).  The optimal dual point lies within sqrt(2 gap) / lambda of
 * theta, so a coordinate j in S with |a_j . theta| + that radius x ||a_j|| < 1
 * is zero in every solution.  Two margins keep the test safe when P, the
 * dual value and the correlations carry FP32 rounding: the radius is
 *   R = sqrt(2 (gap + eta (P + ||x||^2 / 2))) / lambda,  eta = 1e-6,
 * and j is removed from S (mask = 0, z_j = 0) when
 *   stat_j = |a_j . theta| + R ||a_j||  <  1 - tau,  tau = 1e-4.
 * ||a_j|| is the norm of filter k restricted to the taps that land on the
 * image.  stat: [H][W][K] (NAN off the incoming S; may be NULL); *gap_out
 * (may be NULL).  Returns the number of coordinates left in S. */
int64_t orc_screen_image(int K, int s, int H, int W, const double *d,
                         const double *x, double *z, uint8_t *mask,
                         double lambda, double *gap_out, double *stat);

/* Proximal gradient on Eq. 3 as orc_code_update_image, with the screening test
 * above run on the active set before iterations 0, e, 2e, ... (e =
 * screen_every > 0; 0 = never).  mask is in/out (the active set left at the
 * end); *gap_out is the gap of the last test.  Returns the active count. */
int64_t orc_code_update_image_screened(int K, int s, int H, int W,
                                       const double *d, const double *x,
                                       double *z, uint8_t *mask, double alpha,
                                       double lambda, int n_iters,
                                       int screen_every, double *gap_out);

#ifdef __cplusplus
}
#endif
#endif
