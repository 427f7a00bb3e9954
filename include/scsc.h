/*
 * scsc.h -- C ABI of the GB300 library for stochastic convolutional sparse
 * coding (Xiong, Richtarik & Heidrich, "Stochastic Convolutional Sparse
 * Coding", 2019).
 *
 * Problem (Eq. 1): for every image x_n of H_n x W_n pixels,
 *     min_{d,z} 1/2 ||x_n - sum_k d_k * z_{n,k}||^2 + lambda sum_k ||z_{n,k}||_1
 *     s.t. ||d_k||_2 <= 1,
 * with K filters d_k of s x s taps (s odd, centre c = (s-1)/2) and codes z_k
 * of the image's size.  Convolution is the true (flipped) convolution with
 * zero padding:  (d_k * z_k)(i,j) = sum_{u,v} d_k(u,v) z_k(i+c-u, j+c-v).
 *
 * Memory conventions (all device pointers unless stated otherwise):
 *   x : float32 images packed back to back; image n starts at pixel
 *       offsets[n], row-major H[n] x W[n].
 *   z : float32 codes, image n starts at offsets[n] * K, layout [H][W][K]
 *       (filter index innermost).
 *   d : float32 filters [K][s][s].
 * The caller owns x, z and d; the library owns every workspace it needs and
 * grows it on demand.  Calls are asynchronous on the context's stream except
 * where a host-side result is returned (scsc_objective, scsc_lipschitz_codes,
 * scsc_online_save); those synchronise the stream.  A context is not
 * thread-safe.  Errors are returned as scsc_status codes; argument errors are
 * found on the host before anything is launched, and scsc_last_error() holds
 * a one-line description.  Device code never traps.
 *
 * Inputs are checked for NaN and infinities on the device, without a trap:
 * every call that reads x, z or d (or a gradient) enqueues a check that sets a
 * flag word of the context, and the next synchronising call (scsc_sync,
 * scsc_objective, scsc_objective_observed, scsc_lipschitz_codes,
 * scsc_code_step_host) returns SCSC_ENONFINITE and clears the word when it
 * was set.  The outputs of the calls since the previous report are then
 * undefined; the context stays usable.
 */
#ifndef SCSC_H
#define SCSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SCSC_OK = 0,
  SCSC_EINVAL = 1,       /* bad argument (detected on the host)            */
  SCSC_ENOMEM = 2,       /* device or pinned-host allocation failed        */
  SCSC_ECUDA = 3,        /* a CUDA runtime call or a kernel launch failed  */
  SCSC_ETIMEOUT = 4,     /* a bounded device-side wait ran out             */
  SCSC_ENONFINITE = 5,   /* NaN/Inf found in an input                      */
  SCSC_EUNSUPPORTED = 6  /* valid request that the library does not support */
} scsc_status;

typedef enum {
  SCSC_FP32 = 0, /* plain path: FP32 SIMT kernels on dense FP32 codes          */
  SCSC_BF16 = 1, /* tensor path: BF16 operands on tcgen05, FP32 accumulation,
                    FP32 residual / prox / projection, every K <= 512; the
                    sampled codes are stored in BF16 between iterations by
                    the fused kernel (K <= 112 at s = 11), in FP32 by the
                    two-kernel and single-stage kernels                       */
  SCSC_TF32 = 2  /* TF32 operands: not built; scsc_create returns
                    SCSC_EUNSUPPORTED (the BF16 path meets the objective bound
                    and SCSC_FP32 is the full-precision path)                  */
} scsc_precision;

typedef enum {
  SCSC_DICT_BATCH = 0,   /* Eq. 5, one projected-gradient step (Alg. 1 line 8) */
  SCSC_DICT_ONLINE = 1,  /* Eq. 7 surrogate update + one projected-gradient step
                            on Eq. 8 (Alg. 2 lines 8-9)                        */
  SCSC_DICT_BATCH_GS = 2 /* Eq. 5, one Gauss-Seidel pass of projected block
                            coordinate descent over the filters (Sec. 3.2)     */
} scsc_dict_mode;

typedef struct {
  int K;             /* number of filters, 1 <= K <= 512                        */
  int s;             /* filter side, odd, 1 <= s <= 11                          */
  double lambda;     /* L1 weight of Eq. 1 (> 0)                               */
  uint32_t p_num;    /* subsampling rate p = p_num / p_den, 0 <= p <= 1         */
  uint32_t p_den;    /* (Sec. 3.1: Bernoulli(p) per code coordinate)           */
  uint64_t seed;     /* seed of the counter-based subsampling hash             */
  scsc_precision prec;
  double step;       /* > 0: fixed code step alpha; 0: alpha = 1 / L_z          */
  uint32_t flags;    /* OR of SCSC_FLAG_* below; 0 = defaults                   */
} scsc_config;

/* SCSC_FLAG_PER_IMAGE: plain path launches its kernels once per image
 *   instead of once over the whole batch (the baseline of batched launches).
 * SCSC_FLAG_NO_GRAPH: tensor path launches every iteration directly instead
 *   of replaying a captured CUDA graph of the iteration loop.
 * SCSC_FLAG_NO_AUTOTUNE: tensor path skips the variant timing on the first
 *   call for a shape and uses the pipelined kernels when they apply.
 * SCSC_FLAG_UNSAMPLED_KEEP: the other reading of Sec. 3.1 (each iteration
 *   updates the pDK sampled variables "while the rest remain unchanged"):
 *   scsc_code_step, scsc_code_step_host and scsc_code_step_observed leave the
 *   codes off the sampled set as they were instead of zeroing them (Eq. 4),
 *   and the sampled codes take their proximal-gradient steps on
 *   1/2 || x - D z ||^2 + lambda || z_S ||_1 with those codes held fixed:
 *   x' = x - D z_off is formed once per call (FP32), then the same hot loop
 *   runs on x'.  The ADMM and screened steps return SCSC_EUNSUPPORTED. */
#define SCSC_FLAG_PER_IMAGE 1u
#define SCSC_FLAG_NO_GRAPH 2u
#define SCSC_FLAG_NO_AUTOTUNE 4u
#define SCSC_FLAG_UNSAMPLED_KEEP 8u
/* SCSC_FLAG_TWO_KERNEL: tensor path runs its two-kernel pipeline (adjoint +
 *   prox, then synthesis; FP32 packed codes) even where the fused
 *   one-launch-per-iteration kernel (BF16 packed codes) applies. */
#define SCSC_FLAG_TWO_KERNEL 16u

typedef struct {   /* host arrays, n_images entries each */
  int n_images;
  const int64_t *offsets;   /* pixel offset of each image in x            */
  const int *H;             /* rows    (>= 1)                             */
  const int *W;             /* columns (>= 1)                             */
  const int64_t *image_ids; /* global image index n used by the hash      */
} scsc_batch;

typedef struct scsc_ctx scsc_ctx;

/* Create a context bound to the current CUDA device and `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Validates cfg. */
scsc_status scsc_create(const scsc_config *cfg, void *cuda_stream, scsc_ctx **out);

/* Free the context and every workspace it owns.  NULL is accepted. */
scsc_status scsc_destroy(scsc_ctx *ctx);

/* One-line description of the last error on this context ("" if none). */
const char *scsc_last_error(const scsc_ctx *ctx);

/* Subsampling matrix M^t of outer iteration t (Sec. 3.1) as a bitmask:
 * bits_dev is uint32 [total_pixels][ceil(K/32)], bit (k % 32) of word k / 32
 * of pixel q is set when code coordinate (q, k) is sampled.  Coordinate
 * (k, y, x) of image n is sampled iff hi32(h) < floor(p * 2^32) with
 * h = mix(mix(mix(mix(seed) ^ t) ^ n) ^ ((k*H + y)*W + x)) and mix the
 * SplitMix64 output function. */
scsc_status scsc_mask(scsc_ctx *ctx, const scsc_batch *batch, uint64_t t, uint32_t *bits_dev);

/* One outer iteration of the code update (Alg. 1 lines 4-7, Alg. 2 lines
 * 5-7): draw M^t, take the previous codes on the sampled coordinates as the
 * warm start, run n_iters proximal-gradient steps on Eq. 3
 *     r = D z - x;   z_S <- soft(z_S - alpha (D^T r)_S, alpha lambda),
 * and write the Eq. 4 codes (zero off the sampled set) back to z_dev.
 * alpha = cfg.step if > 0, else 1 / L_z with L_z = 1.01 x the 50-step power
 * iteration estimate of lambda_max(D D^T) on the batch's max(H) x max(W)
 * domain.  n_iters >= 0; n_iters = 0 only applies Eq. 4 to the warm start. */
scsc_status scsc_code_step(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *d_dev, float *z_dev, uint64_t t, int n_iters);

/* scsc_code_step on HOST buffers: x_host (packed images), d_host (K x s x s)
 * and z_host (warm start in, Eq. 4 codes out), all float32 in scsc_code_step's
 * layouts.  The step size is taken once for the whole batch; the images are
 * then processed in up to 3 contiguous chunks (at least 2^20 pixels each), and
 * chunk c + 1's host-to-device copy and chunk c - 1's device-to-host copy run
 * on their own streams while chunk c computes.  Results equal scsc_code_step's
 * (every image's update is independent of the others).  Page-locked host
 * memory is needed for the copies to overlap (pageable memory is correct but
 * serialises them).  Returns once z_host holds the result.  Errors as
 * scsc_code_step. */
scsc_status scsc_code_step_host(scsc_ctx *ctx, const scsc_batch *batch, const float *x_host,
                                const float *d_host, float *z_host, uint64_t t, int n_iters);

/* Inpainting (Sec. 4.3: reconstruction from partially observed pixels): the
 * code update of scsc_code_step with the data term counted on observed pixels
 * only, 1/2 || O (x - D (M^t)^T z~) ||^2, O = diag(observed), so the residual
 * is r = O (D z - x).  observed_dev: device, one byte per pixel of the batch
 * (x's layout), nonzero = observed; the caller keeps it alive until the call's
 * work on the stream has run.  NULL observed_dev = every pixel observed
 * (exactly scsc_code_step).  The step size is scsc_code_step's 1 / L_z, a
 * valid step because ||O D|| <= ||D||.  Errors as scsc_code_step. */
scsc_status scsc_code_step_observed(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                    const float *d_dev, float *z_dev,
                                    const uint8_t *observed_dev, uint64_t t, int n_iters);

/* The paper's own solver for Eq. 3 (Sec. 3.2): ADMM on
 *   min 1/2 || x - D (M^t)^T z~ ||^2 + lambda || y ||_1  s.t.  z~ = y,
 * each image with its own CG scalars (the whole batch per launch), n_iters
 * times:
 *   z~ <- solution of (A^T A + rho I) z~ = A^T x + rho (y - u), A = D (M^t)^T,
 *         by cg_iters conjugate-gradient steps from the current z~ (stopped
 *         early once the squared residual is below 1e-30 max(||b||^2, 1));
 *   zh = alpha z~ + (1 - alpha) y  (over-relaxation);
 *   y <- soft(zh + u, lambda / rho);  u <- u + zh - y.
 * z_dev in: warm start (its sampled coordinates start z~ and y; u = 0);
 * out: y on the sampled set, zero elsewhere (Eq. 4).  rho <= 0 selects the
 * paper's 10 lambda, alpha <= 0 its 1.8 (alpha must be < 2).  Plain FP32
 * operators, FP64 CG reductions, for every precision setting.  Errors as
 * scsc_code_step; SCSC_EINVAL for n_iters or cg_iters < 0 and for batches of more
 * than 65535 images. */
scsc_status scsc_code_step_admm(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                const float *d_dev, float *z_dev, uint64_t t, int n_iters,
                                int cg_iters, double rho, double alpha);

/* Safe screening of the code problem (Sec. 5: the code subproblem is a sparse
 * LASSO, and safe screening proves coordinates zero so that their updates can
 * be skipped).  For each image, on its active set S = the set bits of bits_dev
 * ([total_pixels][ceil(K/32)] words, the layout scsc_mask writes; in/out):
 * codes off S are set to zero, then the duality-gap sphere test removes from S
 * every coordinate it proves zero in every solution of Eq. 3 restricted to S,
 * clearing its bit and its code.  With r = D z - x and g = D^T r:
 *   scale = max(lambda, max_S |g|),
 *   gap   = P(z) - Dual(-r / scale) >= 0  (P = 0.5 ||r||^2 + lambda ||z||_1,
 *           Dual(theta) = 0.5 ||x||^2 - 0.5 lambda^2 ||theta - x / lambda||^2),
 *   R     = sqrt(2 (gap + 1e-6 (P + 0.5 ||x||^2))) / lambda,
 *   j leaves S when |g_j| / scale + R ||a_j|| < 1 - 1e-4,
 * ||a_j|| the norm of filter k over the taps that land on the image; the two
 * margins cover FP32 rounding.  The data term is the plain one of Eq. 3
 * (every pixel observed).  Plain FP32 operators and FP64 reductions in
 * either precision.  gap_host (n_images doubles, may be NULL): each image's
 * duality gap at the input codes; n_active_host (n_images int64, may be NULL):
 * the coordinates left in each image's set.  Synchronises the stream when an
 * output is requested.  Errors as scsc_code_step; SCSC_EINVAL for batches of
 * more than 65535 images. */
scsc_status scsc_screen(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                        const float *d_dev, float *z_dev, uint32_t *bits_dev, double *gap_host,
                        int64_t *n_active_host);

/* scsc_code_step (step t, M^t, n_iters proximal-gradient iterations, Eq. 4
 * codes out) with the test of scsc_screen run on the active set, initially
 * M^t, before iterations 0, e, 2e, ... (e = screen_every >= 1); the iterations
 * update the active coordinates only, and the removed ones stay zero.  The
 * outputs are those of the last test (SCSC_EINVAL if one is requested with
 * n_iters = 0).  SCSC_EINVAL for n_iters < 0, screen_every < 1 or more than
 * 65535 images. */
scsc_status scsc_code_step_screened(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                    const float *d_dev, float *z_dev, uint64_t t, int n_iters,
                                    int screen_every, double *gap_host, int64_t *n_active_host);

/* Dictionary update.  SCSC_DICT_BATCH (Eq. 5): r = D z - x,
 * G_k(u,v) = sum_n sum_{i,j} r(i,j) z_k(i+c-u, j+c-v),
 * d_k <- P(d_k - G_k / L_d) with L_d from the power-iteration rule on
 * sum_n Z_n^T Z_n and P the projection onto ||d_k|| <= 1.
 * SCSC_DICT_BATCH_GS (Eq. 5, Sec. 3.2): the same L_d, then for k = 0..K-1 in
 * order: G_k from the current residual, d_k <- P(d_k - G_k / L_d), and the
 * residual r <- r + Z_k (d_k^new - d_k^old) before the next filter.
 * SCSC_DICT_ONLINE (Eq. 7-8, t >= 1 counts mini-batches): C, B <- (t-1)/t
 * C, B + (1/t) mean_n Z_n^T Z_n, Z_n^T x_n; d <- P(d - (C d - B) / L_C). */
scsc_status scsc_dict_step(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *z_dev, float *d_dev, scsc_dict_mode mode, uint64_t t);

/* Eq. 1 summed over the batch, accumulated in FP64; synchronises. */
scsc_status scsc_objective(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *z_dev, const float *d_dev, double *out_host);

/* Objective of the inpainting problem: 1/2 sum over observed pixels of
 * (x - D z)^2 + lambda ||z||_1, summed over the batch in FP64; observed_dev
 * as in scsc_code_step_observed (NULL = scsc_objective); synchronises. */
scsc_status scsc_objective_observed(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                    const float *z_dev, const float *d_dev,
                                    const uint8_t *observed_dev, double *out_host);

/* L_z = 1.01 x power-iteration estimate of lambda_max(D D^T) on the batch's
 * max(H) x max(W) domain (the step-size rule of scsc_code_step); synchronises. */
scsc_status scsc_lipschitz_codes(scsc_ctx *ctx, const scsc_batch *batch, const float *d_dev,
                                 double *out_host);

/* Synthesis xhat = sum_k d_k * (m_k . z_k) (Sec. 3.1, D (M^t)^T z~): masked
 * = 1 applies M^t of iteration t, masked = 0 uses every coordinate.
 * xhat_dev is float32 packed like x. */
scsc_status scsc_synth(scsc_ctx *ctx, const scsc_batch *batch, const float *z_dev,
                       const float *d_dev, uint64_t t, int masked, float *xhat_dev);

/* Backward of scsc_synth for an upstream gradient g (packed like x):
 * grad_z = m . (D^T g)  (layout of z), grad_d_k(u,v) = sum g(i,j) (m.z)_k(i+c-u, j+c-v).
 * Either output may be NULL.  Outputs are overwritten, not accumulated. */
scsc_status scsc_synth_backward(scsc_ctx *ctx, const scsc_batch *batch, const float *grad_dev,
                                const float *z_dev, const float *d_dev, uint64_t t, int masked,
                                float *grad_z_dev, float *grad_d_dev);

/* Wait for all work queued on the context, then report a device-side error
 * recorded by the tensor-core kernels: SCSC_ETIMEOUT when one of their
 * bounded waits on an mbarrier ran out (the kernel then skipped its
 * remaining work and released its tensor memory); else SCSC_ENONFINITE when
 * an input check found a NaN or an infinity since the last report. */
scsc_status scsc_sync(scsc_ctx *ctx);

/* Objective of Eq. 1 for n_images images that all have H x W pixels (packed
 * back to back; codes [H][W][K] per image), written to *out_dev (one device
 * double), enqueued on cuda_stream (NULL = legacy default stream).  It
 * allocates no device memory, so callers that cannot call cudaMalloc can use
 * it: code inside stream capture, services whose memory pool already holds
 * the whole device, loops that cannot take an allocation's implicit
 * synchronisation.  The paper has no counterpart; this is a service of this
 * library.  Needs no context: cfg supplies K, s and lambda (p, seed, prec and
 * step are ignored).
 * Scratch: a fixed array of 65,536 + 1,024 doubles (520 KiB) compiled into
 * the library, which every GPU that loads the library holds until the
 * process exits.  The batch may therefore span at most 65,536 tiles of
 * 32 x 32 pixels (n_images * ceil(H/32) * ceil(W/32) <= 65,536); larger
 * batches are rejected with SCSC_EINVAL before anything is launched.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call outside any stream capture.  The
 * address is cached with the id of the device's current CUDA context and
 * looked up again when that context changes (after cudaDeviceReset), so a
 * call after a reset is again a first call.  All
 * calls share the array and each call overwrites what it reads, so calls
 * that overlap on the GPU (on different streams or devices sharing nothing
 * else) race and must be serialised by the caller. */
scsc_status scsc_objective_noalloc(const scsc_config *cfg, int n_images, int H, int W,
                                   const float *x_dev, const float *z_dev, const float *d_dev,
                                   double *out_dev, void *cuda_stream);

/* Online surrogates (Eq. 7): reset to C = 0, B = 0, t = 0; query the byte
 * size of the serialised state; save to / load from a host buffer
 * (format: magic, K, s, t, then C [KM][KM] float32 and B [KM] float64). */
scsc_status scsc_online_reset(scsc_ctx *ctx);
scsc_status scsc_online_state_size(scsc_ctx *ctx, size_t *bytes);
scsc_status scsc_online_save(scsc_ctx *ctx, void *host_buf, size_t bytes);
scsc_status scsc_online_load(scsc_ctx *ctx, const void *host_buf, size_t bytes);

#ifdef __cplusplus
}
#endif
#endif /* SCSC_H */
