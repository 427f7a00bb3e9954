// scsc_internal.cuh -- declarations shared by the CUDA translation units of
// the SCSC library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace scsc {

constexpr int kMaxK = 512;
constexpr int kMaxS = 11;

// Device-side view of a batch of images packed back to back.
struct BatchDev {
  int n;                // number of images
  const int64_t *off;   // [n + 1] pixel offsets; off[n] = total pixels
  const int *H;         // [n]
  const int *W;         // [n]
  const int64_t *ids;   // [n] global image index (subsampling hash key)
  const int *tile0;     // [n + 1] first 32x32 tile of each image
  int64_t total_px;
  int n_tiles;          // tile0[n]
  int tile_base;        // global index of this view's first tile (sub-batches)
};

// Parameters of the proximal step, read by the kernels from device memory so
// that the step size computed on the device never round-trips to the host.
struct StepParams {
  float alpha;      // step 1/L
  float thresh;     // alpha * lambda
};

// ---------------------------------------------------------------- hashing

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t v) {
  uint64_t z = v + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Hash prefix shared by every coordinate of image `n` at outer iteration t.
__host__ __device__ __forceinline__ uint64_t mask_prefix(uint64_t seed, uint64_t t, uint64_t n) {
  return splitmix64(splitmix64(splitmix64(seed) ^ t) ^ n);
}

// Largest i in [0, n) with start[i] <= g (start ascending, start[0] = 0).
template <typename T>
__device__ __forceinline__ int upper_index(const T *start, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if ((int64_t)start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float soft_threshold(float v, float tau) {
  // sign(v) max(|v| - tau, 0); |v| <= tau gives exactly 0
  return v > tau ? v - tau : (v < -tau ? v + tau : 0.0f);
}

}  // namespace scsc

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns the launch status.
namespace scsc {

cudaError_t launch_mask_bits(const BatchDev &b, int K, uint64_t seed, uint64_t t, uint64_t T,
                             uint32_t *bits, cudaStream_t st);
cudaError_t launch_apply_mask_dense(const BatchDev &b, int K, const uint32_t *bits, float *z,
                                    cudaStream_t st);
// ksplit > 1 splits the filters over ksplit blocks per tile (small domains);
// the synthesis then needs `partial` of ksplit * total_px floats.
cudaError_t launch_synth_fp32(const BatchDev &b, int K, int s, const float *d, const float *z,
                              const uint32_t *bits, const float *x, float *out, cudaStream_t st,
                              int ksplit = 1, float *partial = nullptr);
cudaError_t launch_adjoint_fp32(const BatchDev &b, int K, int s, const float *d, const float *r,
                                const uint32_t *bits, int mode, const StepParams *prm,
                                float *z_or_g, cudaStream_t st, int ksplit = 1);
cudaError_t launch_filter_grad_fp32(const BatchDev &b, int K, int s, const float *r,
                                    const float *z, const uint32_t *bits, float *partial,
                                    int n_groups, cudaStream_t st);
cudaError_t launch_reduce_partials(const float *partial, int n_groups, int len, double *out,
                                   cudaStream_t st);
// The dictionary step's code operators on the nonzero codes (kernels_sparse.cu):
// count per pixel and per (filter, 128-pixel tile), exclusive scans into int64
// offsets (scratch: sparse_scan_scratch(n) int64), the pixel-major and
// filter-major entries, the gathered synthesis (minus x when given) and the
// filter gradient as `groups` partials [groups][K][s*s].
int sparse_tiles(int64_t total_px);
size_t sparse_scan_scratch(int64_t n);
cudaError_t launch_sparse_count(const BatchDev &b, int K, const float *z, int *cnt_px,
                                int *cnt_kt, cudaStream_t st);
cudaError_t launch_scan_counts(const int *in, int64_t n, int64_t *out, int64_t *scratch,
                               cudaStream_t st);
cudaError_t launch_sparse_fill(const BatchDev &b, int K, const float *z, const int64_t *row_ptr,
                               const int64_t *kt_off, int *pk, float *pv, int *kpix, int *kimg,
                               float *kv, cudaStream_t st);
cudaError_t launch_sparse_synth(const BatchDev &b, int K, int s, const float *d,
                                const int64_t *row_ptr, const int *pk, const float *pv,
                                const float *x, float *out, cudaStream_t st);
cudaError_t launch_sparse_grad(const BatchDev &b, int K, int s, const float *r,
                               const int64_t *kt_off, const int *kpix, const int *kimg,
                               const float *kv, float *partial, int groups, cudaStream_t st);
cudaError_t launch_sum_sq_abs(const float *a, int64_t n_sq, const float *b, int64_t n_abs,
                              double *partials, int n_blocks, cudaStream_t st);
cudaError_t launch_finish_sum(const double *partials, int n_blocks, double scale_sq,
                              double scale_abs, double *out, cudaStream_t st);
// ADMM vector steps over a batch (kernels_admm.cu): 2D grids, y = image, x =
// kAdmmBlocks blocks; codes in the batch's dense layout, bits = the batch's
// M^t; dot products as kAdmmBlocks FP64 partials per image.
constexpr int kAdmmBlocks = 64;
cudaError_t launch_seg_dot(const BatchDev &b, int K, const float *a, const float *c,
                           double *partials, cudaStream_t st);
cudaError_t launch_admm_init(const BatchDev &b, int K, float *z, float *y, float *u,
                             const uint32_t *bits, cudaStream_t st);
cudaError_t launch_admm_rhs(const BatchDev &b, int K, const float *atx, const float *y,
                            const float *u, float *bv, const uint32_t *bits, float rho,
                            cudaStream_t st);
cudaError_t launch_admm_qp_finish(const BatchDev &b, int K, const float *in, float *out,
                                  const uint32_t *bits, float rho, cudaStream_t st);
cudaError_t launch_cg_init(const BatchDev &b, int K, const float *bv, const float *Ap, float *res,
                           float *p, cudaStream_t st);
cudaError_t launch_cg_step(const BatchDev &b, int K, float *z, float *res, const float *p,
                           const float *Ap, const double *rr, const double *pap, const double *bb,
                           cudaStream_t st);
cudaError_t launch_cg_direction(const BatchDev &b, int K, float *p, const float *res,
                                const double *rr_new, const double *rr, const double *bb,
                                cudaStream_t st);
cudaError_t launch_admm_shrink(const BatchDev &b, int K, const float *z, float *y, float *u,
                               const uint32_t *bits, float ar, float tau, cudaStream_t st);
cudaError_t launch_admm_final(const BatchDev &b, int K, float *z, const float *y,
                              const uint32_t *bits, cudaStream_t st);
// One Gauss-Seidel block (filter k) of the dictionary pass (kernels_gs.cu):
// gradient of block k from residual r, d_k <- P(d_k - G_k / *L), r += Z_k delta.
// partial: n_groups * s * s floats; delta: s * s floats.
cudaError_t launch_gs_block(const BatchDev &b, int K, int s, int k, float *d, const float *z,
                            float *r, const double *L, float *partial, int n_groups, float *delta,
                            cudaStream_t st);
// r[i] = 0 where obs[i] == 0 (observed-pixel data term).
cudaError_t launch_mask_residual(float *r, const uint8_t *obs, int64_t n, cudaStream_t st);
// D D^T of the step-size domain as per-class stencils (kernels_ddt.cu):
// prepare builds the tap Gram matrix G (FP64, (s*s)^2) and the stencils A
// (ddt_stencil_floats(s, H, W) floats) from d; apply computes w = D D^T u.
size_t ddt_stencil_floats(int s, int H, int W);
cudaError_t launch_ddt_prepare(const float *d, int K, int s, int H, int W, double *G, float *A,
                               cudaStream_t st);
cudaError_t launch_ddt_apply(const float *A, int s, int H, int W, const float *u, float *w,
                             cudaStream_t st);
cudaError_t launch_power_init(float *u, int64_t n, uint64_t seed, uint64_t tag, cudaStream_t st);
cudaError_t launch_dot_partials(const float *a, const float *b, int64_t n, double *partials,
                                int n_blocks, cudaStream_t st);
cudaError_t launch_power_normalize(const float *w, float *u, int64_t n, const double *partials,
                                   int n_blocks, cudaStream_t st);
cudaError_t launch_power_finish(const double *partials, int n_blocks, double safety,
                                double *L_out, double lambda, double fixed_step,
                                StepParams *prm, cudaStream_t st);
cudaError_t launch_project_step(float *d, const float *G_or_null, const double *Gd_or_null,
                                const double *L, int K, int M, cudaStream_t st);
// *flag |= 1 when a[0, n) holds a NaN or an infinity.
cudaError_t launch_check_finite(const float *a, int64_t n, int *flag, cudaStream_t st);
// out = complement of in over the K filter bits of each of n_px pixels.
cudaError_t launch_complement_bits(const uint32_t *in, uint32_t *out, int64_t n_px, int K,
                                   cudaStream_t st);
cudaError_t launch_negate(float *a, int64_t n, cudaStream_t st);
// z <- zs on the coordinates whose bit is set, z unchanged elsewhere.
cudaError_t launch_merge_sampled(const BatchDev &b, int K, const uint32_t *bits, const float *zs,
                                 float *z, cudaStream_t st);
// Safe screening of the code problem (kernels_screen.cu): duality-gap sphere
// test per image on its active set.  prepare: per-filter prefix sums of the
// squared taps (pref, K (s+1)^2 doubles) and norms (nrm, K floats); stats:
// kScreenBlocks * 5 FP64 partials per image from r = D z - x, x, and z, g
// on the set; finish: one ScreenImage per image; test:
// clears the bits (and codes) of the coordinates the test removes and adds
// the survivors of image n to kept[n].
constexpr int kScreenBlocks = 64;
struct ScreenImage {
  double gap;        // duality gap at the tested codes (>= 0)
  double primal;     // the code problem's objective at the tested codes
  double inv_scale;  // 1 / max(lambda, max |g| on the set)
  double radius;     // sphere radius with the rounding margin
};
cudaError_t launch_screen_prepare(const float *d, int K, int s, double *pref, float *nrm,
                                  cudaStream_t st);
cudaError_t launch_screen_stats(const BatchDev &b, int K, const float *x, const float *r,
                                const float *z, const float *g, const uint32_t *bits,
                                double *part, cudaStream_t st);
cudaError_t launch_screen_finish(int n_img, const double *part, double lambda, ScreenImage *img,
                                 cudaStream_t st);
cudaError_t launch_screen_test(const BatchDev &b, int K, int s, const float *g, uint32_t *bits,
                               float *z, const ScreenImage *img, const double *pref,
                               const float *nrm, unsigned long long *kept, cudaStream_t st);

}  // namespace scsc
