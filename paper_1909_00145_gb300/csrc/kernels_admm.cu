// kernels_admm.cu -- element-wise steps of the paper's ADMM solver for the
// code subproblem (Eq. 3, Sec. 3.2: rho = 10 lambda, over-relaxation 1.8)
// with the QP substep (A^T A + rho I) z = A^T x + rho (y - u), A = D (M^t)^T,
// solved by conjugate gradient.  The operators A and A^T are the plain FP32
// synthesis and adjoint kernels; these kernels do the vector updates.  All
// vectors are dense codes [pixel][K] of one image; m = the image's M^t bits.
// CG scalars come from FP64 block partials that every block sums in the same
// fixed order, so no value round-trips to the host.
#include <algorithm>

#include "scsc_internal.cuh"

namespace scsc {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool sampled(const uint32_t *bits, int KW, int K, int64_t i) {
  const int64_t pix = i / K;
  const int k = (int)(i - pix * K);
  return (bits[pix * KW + (k >> 5)] >> (k & 31)) & 1u;
}

// Sum of nb FP64 partials, the same fixed order in every block.
__device__ double block_total(const double *partials, int nb) {
  __shared__ double sh[kBlock / 32];
  __shared__ double total;
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += kBlock) v += partials[i];
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

// z <- m z (Eq. 4 warm start); y <- z; u <- 0.
__global__ void admm_init_kernel(float *z, float *y, float *u, const uint32_t *bits, int KW,
                                 int K, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = sampled(bits, KW, K, i) ? z[i] : 0.0f;
    z[i] = v;
    y[i] = v;
    u[i] = 0.0f;
  }
}

// b <- m (A^T x + rho (y - u)).
__global__ void admm_rhs_kernel(const float *atx, const float *y, const float *u, float *b,
                                const uint32_t *bits, int KW, int K, float rho, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = sampled(bits, KW, K, i) ? atx[i] + rho * (y[i] - u[i]) : 0.0f;
}

// out <- m (out + rho in): completes the QP operator after out = m D^T D (m in).
__global__ void admm_qp_finish_kernel(const float *in, float *out, const uint32_t *bits, int KW,
                                      int K, float rho, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = sampled(bits, KW, K, i) ? out[i] + rho * in[i] : 0.0f;
}

// res <- b - Ap; p <- res.
__global__ void cg_init_kernel(const float *b, const float *Ap, float *res, float *p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float r = b[i] - Ap[i];
    res[i] = r;
    p[i] = r;
  }
}

// a = rr / <p, Ap> while rr > 1e-30 max(bb, 1) (else the iteration is
// finished and a = 0); z += a p; res -= a Ap.
__global__ void __launch_bounds__(kBlock) cg_step_kernel(float *z, float *res, const float *p,
                                                         const float *Ap, const double *rr_p,
                                                         const double *pap_p, const double *bb_p,
                                                         int nb, int64_t n) {
  const double rr = block_total(rr_p, nb), pap = block_total(pap_p, nb);
  const double bb = block_total(bb_p, nb);
  const bool live = rr > 1e-30 * (bb > 0.0 ? bb : 1.0) && pap != 0.0;
  const float a = live ? (float)(rr / pap) : 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    z[i] += a * p[i];
    res[i] -= a * Ap[i];
  }
}

// p <- res + (rr_new / rr) p while the iteration is live.
__global__ void __launch_bounds__(kBlock) cg_direction_kernel(float *p, const float *res,
                                                              const double *rr_new_p,
                                                              const double *rr_p,
                                                              const double *bb_p, int nb,
                                                              int64_t n) {
  const double rr2 = block_total(rr_new_p, nb), rr = block_total(rr_p, nb);
  const double bb = block_total(bb_p, nb);
  const bool live = rr > 1e-30 * (bb > 0.0 ? bb : 1.0);
  if (!live) return;
  const float beta = (float)(rr2 / rr);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = res[i] + beta * p[i];
}

// Over-relaxation, shrinkage, scaled dual update on the sampled set:
// zh = ar z + (1 - ar) y; y <- soft(zh + u, lambda / rho); u += zh - y.
__global__ void admm_shrink_kernel(const float *z, float *y, float *u, const uint32_t *bits,
                                   int KW, int K, float ar, float tau, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!sampled(bits, KW, K, i)) continue;
    const float zh = ar * z[i] + (1.0f - ar) * y[i];
    const float yn = soft_threshold(zh + u[i], tau);
    u[i] += zh - yn;
    y[i] = yn;
  }
}

// z <- m y (the sparse split variable is the solution; Eq. 4 off the set).
__global__ void admm_final_kernel(float *z, const float *y, const uint32_t *bits, int KW, int K,
                                  int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = sampled(bits, KW, K, i) ? y[i] : 0.0f;
}

int grid_of(int64_t n) { return (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 152 * 8); }

}  // namespace

cudaError_t launch_admm_init(float *z, float *y, float *u, const uint32_t *bits, int K, int64_t n,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  admm_init_kernel<<<grid_of(n), kBlock, 0, st>>>(z, y, u, bits, (K + 31) / 32, K, n);
  return cudaGetLastError();
}

cudaError_t launch_admm_rhs(const float *atx, const float *y, const float *u, float *b,
                            const uint32_t *bits, int K, float rho, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  admm_rhs_kernel<<<grid_of(n), kBlock, 0, st>>>(atx, y, u, b, bits, (K + 31) / 32, K, rho, n);
  return cudaGetLastError();
}

cudaError_t launch_admm_qp_finish(const float *in, float *out, const uint32_t *bits, int K,
                                  float rho, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  admm_qp_finish_kernel<<<grid_of(n), kBlock, 0, st>>>(in, out, bits, (K + 31) / 32, K, rho, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const float *b, const float *Ap, float *res, float *p, int64_t n,
                           cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cg_init_kernel<<<grid_of(n), kBlock, 0, st>>>(b, Ap, res, p, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_step(float *z, float *res, const float *p, const float *Ap,
                           const double *rr, const double *pap, const double *bb, int nb,
                           int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cg_step_kernel<<<grid_of(n), kBlock, 0, st>>>(z, res, p, Ap, rr, pap, bb, nb, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_direction(float *p, const float *res, const double *rr_new,
                                const double *rr, const double *bb, int nb, int64_t n,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cg_direction_kernel<<<grid_of(n), kBlock, 0, st>>>(p, res, rr_new, rr, bb, nb, n);
  return cudaGetLastError();
}

cudaError_t launch_admm_shrink(const float *z, float *y, float *u, const uint32_t *bits, int K,
                               float ar, float tau, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  admm_shrink_kernel<<<grid_of(n), kBlock, 0, st>>>(z, y, u, bits, (K + 31) / 32, K, ar, tau, n);
  return cudaGetLastError();
}

cudaError_t launch_admm_final(float *z, const float *y, const uint32_t *bits, int K, int64_t n,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  admm_final_kernel<<<grid_of(n), kBlock, 0, st>>>(z, y, bits, (K + 31) / 32, K, n);
  return cudaGetLastError();
}

}  // namespace scsc
