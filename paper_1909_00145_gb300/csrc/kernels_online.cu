// kernels_online.cu -- online surrogates of Eq. 7 and the matrix-vector
// products of Eq. 8, plus small helpers.
//
// Z_n is the code Toeplitz matrix of image n: row (i,j), column (k,u,v),
// entry z_k(i+c-u, j+c-v).  The surrogate update
//     C <- a C + b sum_n Z_n^T Z_n,     B <- a B + b sum_n Z_n^T x_n
// is an implicit GEMM over all pixels of the batch: Z is never materialised,
// its entries are gathered from the codes while staging tiles in shared memory.
#include "scsc_internal.cuh"

namespace scsc {

namespace {

constexpr int kTB = 64;   // C tile edge
constexpr int kPB = 16;   // pixels per staged chunk

// Entry (row = pixel q of the batch, column col = (k,u,v)) of Z.
__device__ __forceinline__ float z_entry(const BatchDev &b, int K, int S, const float *z, int n,
                                         int y, int x, int col) {
  const int M = S * S, C = (S - 1) / 2;
  int k = col / M, m = col - k * M, u = m / S, v = m - u * S;
  int yy = y + C - u, xx = x + C - v;
  int H = b.H[n], W = b.W[n];
  if (yy < 0 || yy >= H || xx < 0 || xx >= W) return 0.0f;
  return z[(b.off[n] + (int64_t)yy * W + xx) * K + k];
}

// C[a][b] = alpha C[a][b] + beta sum_q Z[q][a] Z[q][b] for a 64x64 tile;
// 256 threads, 4x4 outputs each, FP32 accumulation per tile pass.
__global__ void __launch_bounds__(256) surrogate_gemm_kernel(BatchDev b, int K, int S,
                                                             const float *__restrict__ z,
                                                             int KM, float alpha, float beta,
                                                             float *__restrict__ Cm) {
  __shared__ float As[kPB][kTB + 4];
  __shared__ float Bs[kPB][kTB + 4];
  const int a0 = blockIdx.y * kTB, b0 = blockIdx.x * kTB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int64_t q0 = 0; q0 < b.total_px; q0 += kPB) {
    __syncthreads();
    for (int i = threadIdx.x; i < kPB * kTB; i += blockDim.x) {
      int p = i / kTB, c = i - p * kTB;
      int64_t q = q0 + p;
      float va = 0.0f, vb = 0.0f;
      if (q < b.total_px) {
        int n = upper_index(b.off, b.n, q);
        int64_t local = q - b.off[n];
        int W = b.W[n];
        int y = (int)(local / W), x = (int)(local - (int64_t)y * W);
        if (a0 + c < KM) va = z_entry(b, K, S, z, n, y, x, a0 + c);
        if (b0 + c < KM) vb = z_entry(b, K, S, z, n, y, x, b0 + c);
      }
      As[p][c] = va;
      Bs[p][c] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kPB; ++p) {
      float ra[4], rb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ra[i] = As[p][ty * 4 + i];
        rb[i] = Bs[p][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ra[i], rb[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int a = a0 + ty * 4 + i, c = b0 + tx * 4 + j;
      if (a < KM && c < KM) {
        float *p = Cm + (int64_t)a * KM + c;
        *p = alpha * *p + beta * acc[i][j];
      }
    }
}

// B[col] = alpha B[col] + beta sum_q Z[q][col] x[q]  (FP64 accumulation)
__global__ void surrogate_b_kernel(BatchDev b, int K, int S, const float *__restrict__ z,
                                   const float *__restrict__ x, int KM, double alpha, double beta,
                                   double *__restrict__ Bv) {
  const int col = blockIdx.x;
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < b.total_px; q += blockDim.x) {
    int n = upper_index(b.off, b.n, q);
    int64_t local = q - b.off[n];
    int W = b.W[n];
    int y = (int)(local / W), xcol = (int)(local - (int64_t)y * W);
    float e = z_entry(b, K, S, z, n, y, xcol, col);
    if (e != 0.0f) s += (double)e * (double)x[q];
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) Bv[col] = alpha * Bv[col] + beta * red[0];
}

// out[a] = sum_b C[a][b] v[b] (- Bv[a]), one warp per row.  Each lane keeps
// four FP32 partial sums over runs of 128 products (FP32 FMAs: this GPU's FP64
// rate would make the product FMA-bound instead of bandwidth-bound) and folds
// each run into an FP64 total, which the warp reduces in FP64.
template <bool kGrad>
__global__ void symv_kernel(const float *__restrict__ Cm, int64_t n, const float *__restrict__ v,
                            const double *__restrict__ Bv, float *__restrict__ outf,
                            double *__restrict__ outd) {
  int64_t row = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float *cr = Cm + row * n;
  double s = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += 32 * 128) {
    float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int64_t j1 = j0 + 32 * 128 < n ? j0 + 32 * 128 : n;
#pragma unroll 4
    for (int64_t j = j0 + lane; j < j1; j += 32) p[(j >> 5) & 3] = fmaf(cr[j], v[j], p[(j >> 5) & 3]);
    s += ((double)p[0] + (double)p[1]) + ((double)p[2] + (double)p[3]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    if (kGrad) outd[row] = s - Bv[row];
    else outf[row] = (float)s;
  }
}

// The same update from the index of the nonzero codes (kernels_sparse.cu):
// one warp per row a = (k, u, v) of C, over the columns of filters k2 >= k
// only (C is symmetric; mirror_lower_kernel copies the rest).  Row a of Z^T Z collects, for every
// nonzero z_k(q1), the pixel q = q1 - c + (u, v) whose patch holds it in
// column a, times every nonzero of q's patch: z_k2(q2) with q2 in the s x s
// window of q lands in column (k2, u2, v2), (u2, v2) = q + c - q2.  The row
// is decayed first; the lanes then split each patch's window, whose nonzeros
// fall in distinct columns, and a warp barrier orders one patch's updates
// before the next's, so the sums are deterministic.  B[a] accumulates
// z_k(q1) x(q) in FP64 on lane 0.
__global__ void __launch_bounds__(256) surrogate_sparse_kernel(
    BatchDev b, int K, int S, const float *__restrict__ x, const int64_t *__restrict__ row_ptr,
    const int *__restrict__ pk, const float *__restrict__ pv, const int64_t *__restrict__ kt_off,
    int ntiles, const int *__restrict__ kpix, const int *__restrict__ kimg,
    const float *__restrict__ kv, int KM, float alpha, float beta, float *__restrict__ Cm,
    double *__restrict__ Bv) {
  const int64_t a = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (a >= KM) return;
  const int M = S * S, C = (S - 1) / 2;
  const int k = (int)(a / M), m = (int)(a - (int64_t)k * M), u = m / S, v = m - (m / S) * S;
  float *const crow = Cm + a * KM;
  if (alpha != 1.0f)
    for (int64_t j = (int64_t)k * M + lane; j < KM; j += 32) crow[j] *= alpha;
  __syncwarp();
  double bsum = 0.0;
  const int64_t kb = kt_off[(int64_t)k * ntiles], ke = kt_off[(int64_t)(k + 1) * ntiles];
  for (int64_t e = kb; e < ke; ++e) {
    const int n = kimg[e];
    const int H = b.H[n], W = b.W[n];
    const int64_t base = b.off[n];
    const int local = (int)(kpix[e] - base);
    const int y = local / W - C + u, xx = local - (local / W) * W - C + v;
    if (y < 0 || y >= H || xx < 0 || xx >= W) continue;  // the same on every lane
    const float z1 = kv[e];
    if (lane == 0) bsum += (double)z1 * (double)x[base + (int64_t)y * W + xx];
    // the window's offsets first (up to 4 pixels per lane, s <= 11), so that
    // their loads are in flight together
    int64_t rb[4], re[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int wi = lane + 32 * r;
      rb[r] = re[r] = 0;
      if (wi < M) {
        const int u2 = wi / S, v2 = wi - (wi / S) * S;
        const int y2 = y + C - u2, x2 = xx + C - v2;
        if (y2 >= 0 && y2 < H && x2 >= 0 && x2 < W) {
          const int64_t g2 = base + (int64_t)y2 * W + x2;
          rb[r] = row_ptr[g2];
          re[r] = row_ptr[g2 + 1];
        }
      }
    }
    const float bz = beta * z1;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      for (int64_t e2 = rb[r]; e2 < re[r]; ++e2) {
        const int k2 = pk[e2];
        if (k2 >= k) crow[(int64_t)k2 * M + lane + 32 * r] += bz * pv[e2];
      }
    __syncwarp();
  }
  if (lane == 0) Bv[a] = (double)alpha * Bv[a] + (double)beta * bsum;
}

// Cross-correlations of the code maps for the surrogate update:
//   T[k][k2][dy][dx] = sum over nonzeros z_k(r1) with r1 + (dy, dx) in the
//   same image of z_k(r1) z_k2(r1 + (dy, dx)),  k2 >= k, |dy|, |dx| <= s - 1.
// Entry ((k,u,v),(k2,u2,v2)) of sum_q Z[q]^T Z[q] is T[k][k2][u-u2][v-v2]
// minus the products whose patch centre q = r1 - c + (u,v) lies outside the
// image (only codes within c of the border have such q; surrogate_border_
// kernel subtracts them).  Block k, thread = lag: each thread owns its lag's
// entries of row block k and walks filter k's nonzeros in order, so the sums
// are deterministic without barriers or atomics.
__global__ void __launch_bounds__(512) surrogate_corr_kernel(
    BatchDev b, int K, int S, const int64_t *__restrict__ row_ptr, const int *__restrict__ pk,
    const float *__restrict__ pv, const int64_t *__restrict__ kt_off, int ntiles,
    const int *__restrict__ kpix, const int *__restrict__ kimg, const float *__restrict__ kv,
    float *__restrict__ T) {
  const int k = blockIdx.x, D = 2 * S - 1, DD = D * D, t = threadIdx.x;
  if (t >= DD) return;
  const int dy = t / D - (S - 1), dx = t - (t / D) * D - (S - 1);
  float *const Tk = T + (int64_t)k * K * DD;
  for (int k2 = k; k2 < K; ++k2) Tk[(int64_t)k2 * DD + t] = 0.0f;
  const int64_t kb = kt_off[(int64_t)k * ntiles], ke = kt_off[(int64_t)(k + 1) * ntiles];
  for (int64_t e = kb; e < ke; ++e) {
    const int n = kimg[e];
    const int H = b.H[n], W = b.W[n];
    const int64_t base = b.off[n];
    const int local = (int)(kpix[e] - base);
    const int y2 = local / W + dy, x2 = local - (local / W) * W + dx;
    if (y2 < 0 || y2 >= H || x2 < 0 || x2 >= W) continue;
    const float z1 = kv[e];
    const int64_t g2 = base + (int64_t)y2 * W + x2;
    for (int64_t e2 = row_ptr[g2]; e2 < row_ptr[g2 + 1]; ++e2) {
      const int k2 = pk[e2];
      if (k2 >= k) Tk[(int64_t)k2 * DD + t] += z1 * pv[e2];
    }
  }
}

// C[a][b] <- alpha C[a][b] + beta T[k][k2][u-u2][v-v2] over the columns b of
// filters k2 >= k of row a = (k,u,v); one block per row.
__global__ void __launch_bounds__(256) surrogate_expand_kernel(float *__restrict__ Cm,
                                                               const float *__restrict__ T, int K,
                                                               int S, float alpha, float beta) {
  const int M = S * S, KM = K * M, D = 2 * S - 1, DD = D * D;
  const int a = blockIdx.x;
  const int k = a / M, m = a - k * M, u = m / S, v = m - (m / S) * S;
  float *const crow = Cm + (int64_t)a * KM;
  const float *const Tk = T + (int64_t)k * K * DD;
  for (int bcol = k * M + threadIdx.x; bcol < KM; bcol += blockDim.x) {
    const int k2 = bcol / M, m2 = bcol - k2 * M, u2 = m2 / S, v2 = m2 - (m2 / S) * S;
    const int lag = (u - u2 + S - 1) * D + (v - v2 + S - 1);
    crow[bcol] = alpha * crow[bcol] + beta * Tk[(int64_t)k2 * DD + lag];
  }
}

// The rest of the update, one warp per row a = (k,u,v).  The lanes take
// filter k's nonzeros z_k(r1) 32 at a time: for those whose patch centre
// q = r1 - c + (u,v) lies inside the image, B[a] accumulates z_k(r1) x(q)
// (FP64, per lane, then a fixed butterfly); those whose centre lies outside
// are then taken in order by the whole warp, which subtracts the products
// the correlation counted but no patch of the image holds (columns of
// filters k2 >= k, lanes over the window).
__global__ void __launch_bounds__(256) surrogate_border_kernel(
    BatchDev b, int K, int S, const float *__restrict__ x, const int64_t *__restrict__ row_ptr,
    const int *__restrict__ pk, const float *__restrict__ pv, const int64_t *__restrict__ kt_off,
    int ntiles, const int *__restrict__ kpix, const int *__restrict__ kimg,
    const float *__restrict__ kv, int KM, float alpha, float beta, float *__restrict__ Cm,
    double *__restrict__ Bv) {
  const int64_t a = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (a >= KM) return;  // whole warps
  const int M = S * S, C = (S - 1) / 2;
  const int k = (int)(a / M), m = (int)(a - (int64_t)k * M), u = m / S, v = m - (m / S) * S;
  float *const crow = Cm + a * KM;
  double bsum = 0.0;
  const int64_t kb = kt_off[(int64_t)k * ntiles], ke = kt_off[(int64_t)(k + 1) * ntiles];
  for (int64_t e0 = kb; e0 < ke; e0 += 32) {
    const int64_t e = e0 + lane;
    int n = 0, y = 0, xx = 0;
    float z1 = 0.0f;
    bool out = false;
    if (e < ke) {
      n = kimg[e];
      const int H = b.H[n], W = b.W[n];
      const int64_t base = b.off[n];
      const int local = (int)(kpix[e] - base);
      y = local / W - C + u;
      xx = local - (local / W) * W - C + v;
      z1 = kv[e];
      if (y >= 0 && y < H && xx >= 0 && xx < W)
        bsum += (double)z1 * (double)x[base + (int64_t)y * W + xx];
      else
        out = true;
    }
    unsigned todo = __ballot_sync(0xffffffffu, out);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const int nj = __shfl_sync(0xffffffffu, n, j);
      const int yj = __shfl_sync(0xffffffffu, y, j), xj = __shfl_sync(0xffffffffu, xx, j);
      const float bz = beta * __shfl_sync(0xffffffffu, z1, j);
      const int H = b.H[nj], W = b.W[nj];
      const int64_t base = b.off[nj];
      // the window's offsets first (up to 4 pixels per lane, s <= 11)
      int64_t rb[4], re[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int wi = lane + 32 * r;
        rb[r] = re[r] = 0;
        if (wi < M) {
          const int u2 = wi / S, v2 = wi - (wi / S) * S;
          const int y2 = yj + C - u2, x2 = xj + C - v2;
          if (y2 >= 0 && y2 < H && x2 >= 0 && x2 < W) {
            const int64_t g2 = base + (int64_t)y2 * W + x2;
            rb[r] = row_ptr[g2];
            re[r] = row_ptr[g2 + 1];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        for (int64_t e2 = rb[r]; e2 < re[r]; ++e2) {
          const int k2 = pk[e2];
          if (k2 >= k) crow[(int64_t)k2 * M + lane + 32 * r] -= bz * pv[e2];
        }
      __syncwarp();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
  if (lane == 0) Bv[a] = (double)alpha * Bv[a] + (double)beta * bsum;
}

// C[j][i] = C[i][j] for the columns j of filters below row i's filter: the
// lower block triangle from the upper one, by 32 x 32 tiles through shared
// memory (tile (bi, bj) with bj < bi reads the transposed tile (bj, bi)).
__global__ void __launch_bounds__(256) mirror_lower_kernel(float *__restrict__ Cm, int KM, int M) {
  __shared__ float t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // source: rows bj*32.., columns bi*32.. (upper), destination: rows bi*32.., columns bj*32..
  for (int r = ty; r < 32; r += 8) {
    const int64_t row = (int64_t)bj * 32 + r, col = (int64_t)bi * 32 + tx;
    t[r][tx] = (row < KM && col < KM) ? Cm[row * KM + col] : 0.0f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t row = (int64_t)bi * 32 + r, col = (int64_t)bj * 32 + tx;
    // only entries whose column's filter is below the row's filter
    if (row < KM && col < KM && col / M < row / M) Cm[row * KM + col] = t[tx][r];
  }
}

__global__ void double_to_float_kernel(const double *in, float *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

__global__ void set_step_kernel(StepParams *prm, double step, double lambda) {
  prm->alpha = (float)step;
  prm->thresh = (float)(step * lambda);
}

}  // namespace

cudaError_t launch_surrogate_update(const BatchDev &b, int K, int s, const float *z, const float *x,
                                    double alpha, double beta, float *Cm, double *Bv,
                                    cudaStream_t st) {
  const int KM = K * s * s;
  dim3 grid((KM + kTB - 1) / kTB, (KM + kTB - 1) / kTB);
  surrogate_gemm_kernel<<<grid, 256, 0, st>>>(b, K, s, z, KM, (float)alpha, (float)beta, Cm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  surrogate_b_kernel<<<KM, 256, 0, st>>>(b, K, s, z, x, KM, alpha, beta, Bv);
  return cudaGetLastError();
}

size_t surrogate_corr_floats(int K, int s) {
  const size_t D = (size_t)(2 * s - 1);
  return (size_t)K * K * D * D;
}

cudaError_t launch_surrogate_update_sparse(const BatchDev &b, int K, int s, const float *x,
                                           const int64_t *row_ptr, const int *pk, const float *pv,
                                           const int64_t *kt_off, const int *kpix,
                                           const int *kimg, const float *kv, double alpha,
                                           double beta, float *Cm, double *Bv, float *T,
                                           cudaStream_t st) {
  const int KM = K * s * s;
  const int nt_px = sparse_tiles(b.total_px);
  cudaError_t e;
  if (T != nullptr) {
    // correlations, then C = alpha C + beta T (upper blocks), then the
    // border corrections and B
    surrogate_corr_kernel<<<K, 512, 0, st>>>(b, K, s, row_ptr, pk, pv, kt_off, nt_px, kpix, kimg,
                                             kv, T);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    surrogate_expand_kernel<<<KM, 256, 0, st>>>(Cm, T, K, s, (float)alpha, (float)beta);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t blocks = ((int64_t)KM + 7) / 8;
    surrogate_border_kernel<<<(unsigned)blocks, 256, 0, st>>>(
        b, K, s, x, row_ptr, pk, pv, kt_off, nt_px, kpix, kimg, kv, KM, (float)alpha,
        (float)beta, Cm, Bv);
  } else {
    const int64_t blocks = ((int64_t)KM + 7) / 8;
    surrogate_sparse_kernel<<<(unsigned)blocks, 256, 0, st>>>(
        b, K, s, x, row_ptr, pk, pv, kt_off, nt_px, kpix, kimg, kv, KM, (float)alpha,
        (float)beta, Cm, Bv);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = (KM + 31) / 32;
  mirror_lower_kernel<<<dim3(nt, nt), 256, 0, st>>>(Cm, KM, s * s);
  return cudaGetLastError();
}

cudaError_t launch_symv(const float *Cm, int64_t n, const float *v, const double *unused, float *out,
                        cudaStream_t st) {
  (void)unused;
  int64_t blocks = (n + 7) / 8;
  symv_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(Cm, n, v, nullptr, out, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_symv_grad(const float *Cm, int64_t n, const float *d, const double *Bv,
                             double *out, cudaStream_t st) {
  int64_t blocks = (n + 7) / 8;
  symv_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(Cm, n, d, Bv, nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_double_to_float(const double *in, float *out, int n, cudaStream_t st) {
  double_to_float_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_set_step(StepParams *prm, double step, double lambda, cudaStream_t st) {
  set_step_kernel<<<1, 1, 0, st>>>(prm, step, lambda);
  return cudaGetLastError();
}

}  // namespace scsc
