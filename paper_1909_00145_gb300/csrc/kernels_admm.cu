// kernels_admm.cu -- element-wise steps of the paper's ADMM solver for the
// code subproblem (Eq. 3, Sec. 3.2: rho = 10 lambda, over-relaxation 1.8)
// with the QP substep (A^T A + rho I) z = A^T x + rho (y - u), A = D (M^t)^T,
// solved by conjugate gradient.  The operators A and A^T are the plain FP32
// synthesis and adjoint kernels over the whole batch; these kernels do the
// vector updates.  Vectors are dense codes [pixel][K] in the batch's layout;
// every image runs its own CG (its own scalars): a launch is a 2D grid, y =
// image, x = kAdmmBlocks blocks over that image's codes.  The CG scalars come
// from per-image FP64 block partials that every block sums in the same fixed
// order, so no value round-trips to the host.
#include <algorithm>

#include "scsc_internal.cuh"

namespace scsc {
namespace {

constexpr int kBlock = 256;

struct Range {
  int64_t lo, hi;  // the image's code indices [lo, hi)
};

__device__ __forceinline__ Range image_codes(const BatchDev &b, int K) {
  const int n = blockIdx.y;
  return {b.off[n] * K, b.off[n + 1] * K};
}

#define FOR_IMAGE_CODES(i, r)                                                                 \
  for (int64_t i = (r).lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (r).hi;      \
       i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ bool sampled(const uint32_t *bits, int KW, int K, int64_t i) {
  const int64_t pix = i / K;
  const int k = (int)(i - pix * K);
  return (bits[pix * KW + (k >> 5)] >> (k & 31)) & 1u;
}

// Sum of an image's nb FP64 partials, the same fixed order in every block.
__device__ double block_total(const double *partials, int nb) {
  __shared__ double sh[kBlock / 32];
  __shared__ double total;
  const double *pp = partials + (int64_t)blockIdx.y * nb;
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += kBlock) v += pp[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sh[w];
    total = t;
  }
  __syncthreads();
  return total;
}

// partials[n][blockIdx.x] = this block's part of <a, c> over image n's codes.
__global__ void __launch_bounds__(kBlock) seg_dot_kernel(BatchDev b, int K, const float *a,
                                                         const float *c, double *partials) {
  __shared__ double sh[kBlock / 32];
  const Range r = image_codes(b, K);
  double s = 0.0;
  FOR_IMAGE_CODES(i, r) s += (double)a[i] * (double)c[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sh[w];
    partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// z <- m z (Eq. 4 warm start); y <- z; u <- 0.
__global__ void admm_init_kernel(BatchDev b, int K, float *z, float *y, float *u,
                                 const uint32_t *bits, int KW) {
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) {
    const float v = sampled(bits, KW, K, i) ? z[i] : 0.0f;
    z[i] = v;
    y[i] = v;
    u[i] = 0.0f;
  }
}

// b <- m (A^T x + rho (y - u)).
__global__ void admm_rhs_kernel(BatchDev b, int K, const float *atx, const float *y,
                                const float *u, float *bv, const uint32_t *bits, int KW,
                                float rho) {
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) bv[i] = sampled(bits, KW, K, i) ? atx[i] + rho * (y[i] - u[i]) : 0.0f;
}

// out <- m (out + rho in): completes the QP operator after out = m D^T D (m in).
__global__ void admm_qp_finish_kernel(BatchDev b, int K, const float *in, float *out,
                                      const uint32_t *bits, int KW, float rho) {
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) out[i] = sampled(bits, KW, K, i) ? out[i] + rho * in[i] : 0.0f;
}

// res <- b - Ap; p <- res.
__global__ void cg_init_kernel(BatchDev b, int K, const float *bv, const float *Ap, float *res,
                               float *p) {
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) {
    const float v = bv[i] - Ap[i];
    res[i] = v;
    p[i] = v;
  }
}

// Per image: a = rr / <p, Ap> while rr > 1e-30 max(bb, 1) (else that image's
// iteration is finished and a = 0); z += a p; res -= a Ap.
__global__ void __launch_bounds__(kBlock) cg_step_kernel(BatchDev b, int K, float *z, float *res,
                                                         const float *p, const float *Ap,
                                                         const double *rr_p, const double *pap_p,
                                                         const double *bb_p, int nb) {
  const double rr = block_total(rr_p, nb), pap = block_total(pap_p, nb);
  const double bb = block_total(bb_p, nb);
  const bool live = rr > 1e-30 * (bb > 0.0 ? bb : 1.0) && pap != 0.0;
  const float a = live ? (float)(rr / pap) : 0.0f;
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) {
    z[i] += a * p[i];
    res[i] -= a * Ap[i];
  }
}

// Per image: p <- res + (rr_new / rr) p while the iteration is live.
__global__ void __launch_bounds__(kBlock) cg_direction_kernel(BatchDev b, int K, float *p,
                                                              const float *res,
                                                              const double *rr_new_p,
                                                              const double *rr_p,
                                                              const double *bb_p, int nb) {
  const double rr2 = block_total(rr_new_p, nb), rr = block_total(rr_p, nb);
  const double bb = block_total(bb_p, nb);
  if (!(rr > 1e-30 * (bb > 0.0 ? bb : 1.0))) return;
  const float beta = (float)(rr2 / rr);
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) p[i] = res[i] + beta * p[i];
}

// Over-relaxation, shrinkage, scaled dual update on the sampled set:
// zh = ar z + (1 - ar) y; y <- soft(zh + u, lambda / rho); u += zh - y.
__global__ void admm_shrink_kernel(BatchDev b, int K, const float *z, float *y, float *u,
                                   const uint32_t *bits, int KW, float ar, float tau) {
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) {
    if (!sampled(bits, KW, K, i)) continue;
    const float zh = ar * z[i] + (1.0f - ar) * y[i];
    const float yn = soft_threshold(zh + u[i], tau);
    u[i] += zh - yn;
    y[i] = yn;
  }
}

// z <- m y (the sparse split variable is the solution; Eq. 4 off the set).
__global__ void admm_final_kernel(BatchDev b, int K, float *z, const float *y,
                                  const uint32_t *bits, int KW) {
  const Range r = image_codes(b, K);
  FOR_IMAGE_CODES(i, r) z[i] = sampled(bits, KW, K, i) ? y[i] : 0.0f;
}

dim3 grid_of(const BatchDev &b) { return dim3(kAdmmBlocks, b.n); }

}  // namespace

cudaError_t launch_seg_dot(const BatchDev &b, int K, const float *a, const float *c,
                           double *partials, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  seg_dot_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, a, c, partials);
  return cudaGetLastError();
}

cudaError_t launch_admm_init(const BatchDev &b, int K, float *z, float *y, float *u,
                             const uint32_t *bits, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  admm_init_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, z, y, u, bits, (K + 31) / 32);
  return cudaGetLastError();
}

cudaError_t launch_admm_rhs(const BatchDev &b, int K, const float *atx, const float *y,
                            const float *u, float *bv, const uint32_t *bits, float rho,
                            cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  admm_rhs_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, atx, y, u, bv, bits, (K + 31) / 32, rho);
  return cudaGetLastError();
}

cudaError_t launch_admm_qp_finish(const BatchDev &b, int K, const float *in, float *out,
                                  const uint32_t *bits, float rho, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  admm_qp_finish_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, in, out, bits, (K + 31) / 32, rho);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const BatchDev &b, int K, const float *bv, const float *Ap, float *res,
                           float *p, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  cg_init_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, bv, Ap, res, p);
  return cudaGetLastError();
}

cudaError_t launch_cg_step(const BatchDev &b, int K, float *z, float *res, const float *p,
                           const float *Ap, const double *rr, const double *pap, const double *bb,
                           cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  cg_step_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, z, res, p, Ap, rr, pap, bb, kAdmmBlocks);
  return cudaGetLastError();
}

cudaError_t launch_cg_direction(const BatchDev &b, int K, float *p, const float *res,
                                const double *rr_new, const double *rr, const double *bb,
                                cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  cg_direction_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, p, res, rr_new, rr, bb, kAdmmBlocks);
  return cudaGetLastError();
}

cudaError_t launch_admm_shrink(const BatchDev &b, int K, const float *z, float *y, float *u,
                               const uint32_t *bits, float ar, float tau, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  admm_shrink_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, z, y, u, bits, (K + 31) / 32, ar, tau);
  return cudaGetLastError();
}

cudaError_t launch_admm_final(const BatchDev &b, int K, float *z, const float *y,
                              const uint32_t *bits, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  admm_final_kernel<<<grid_of(b), kBlock, 0, st>>>(b, K, z, y, bits, (K + 31) / 32);
  return cudaGetLastError();
}

}  // namespace scsc
