// kernels_online.cu -- online surrogates of Eq. 7 and the matrix-vector
// products of Eq. 8, plus small helpers.
//
// Z_n is the code Toeplitz matrix of image n: row (i,j), column (k,u,v),
// entry z_k(i+c-u, j+c-v).  The surrogate update
//     C <- a C + b sum_n Z_n^T Z_n,     B <- a B + b sum_n Z_n^T x_n
// has two forms.  For dense codes it is an implicit GEMM over all pixels of
// the batch: Z is never materialised, its entries are gathered from the codes
// while staging tiles in shared memory.  For codes sparser than 1/16 it is
// built from the nonzero codes: cross-correlations of the code maps at the
// lag between two columns, expanded into C's upper block triangle, minus the
// products of patches centred outside the image, then mirrored.  The
// products with C read its upper block triangle only.
#include <algorithm>

#include "scsc_internal.cuh"
#include "scsc_tc.cuh"

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

// out = C v (- Bv) for the symmetric C, reading its upper block triangle
// only.  C is cut into panels of kSymB rows and columns; CTA b takes block
// (I, J), J >= I, of the upper triangle (row by row).  It writes the block's
// row products C_IJ v_J (rows of panel I) into slot J of panel I and, off the
// diagonal, its column products C_IJ^T v_I (rows of panel J) into slot I of
// panel J, so every (slot, row) of the partial buffer part[NP][n] is written
// exactly once.  The partials are FP32 sums of at most kSymB products; the
// reduction sums a row's NP slots in FP64 in a fixed order.
constexpr int kSymB = 128;

__device__ __forceinline__ int64_t upper_offset(int64_t I, int64_t NP) {
  return I * NP - I * (I - 1) / 2;  // blocks in the triangle's rows 0 .. I-1
}

template <bool kVec>
__global__ void __launch_bounds__(256) symv_upper_kernel(const float *__restrict__ Cm, int64_t n,
                                                         int NP, const float *__restrict__ v,
                                                         float *__restrict__ part) {
  __shared__ float s_col[8][kSymB];
  const int64_t b = blockIdx.x;
  // row I of the triangle holding block b: the root of offset(I) = b, then
  // corrected against the exact integer offsets
  const double tn = 2.0 * NP + 1.0;
  int64_t I = (int64_t)((tn - sqrt(tn * tn - 8.0 * (double)b)) * 0.5);
  if (I < 0) I = 0;
  if (I > NP - 1) I = NP - 1;
  while (I > 0 && upper_offset(I, NP) > b) --I;
  while (I + 1 < NP && upper_offset(I + 1, NP) <= b) ++I;
  const int64_t J = I + (b - upper_offset(I, NP));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r0 = I * kSymB, c0 = J * kSymB + 4 * lane;
  float vj[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) vj[q] = c0 + q < n ? v[c0 + q] : 0.0f;
  // rows r0 + w + 8 k, k < 16; this lane's 4 columns c0 .. c0 + 3
  float4 c[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t r = r0 + w + 8 * k;
    c[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (r < n) {
      const float *src = Cm + r * n + c0;
      if (kVec) {
        if (c0 < n) c[k] = *reinterpret_cast<const float4 *>(src);
      } else {
        if (c0 < n) c[k].x = src[0];
        if (c0 + 1 < n) c[k].y = src[1];
        if (c0 + 2 < n) c[k].z = src[2];
        if (c0 + 3 < n) c[k].w = src[3];
      }
    }
  }
  float col[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t r = r0 + w + 8 * k;
    const float vi = r < n ? v[r] : 0.0f;
    float rp = c[k].x * vj[0];
    rp = fmaf(c[k].y, vj[1], rp);
    rp = fmaf(c[k].z, vj[2], rp);
    rp = fmaf(c[k].w, vj[3], rp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rp += __shfl_xor_sync(0xffffffffu, rp, o);
    if (lane == k && r < n) part[J * n + r] = rp;
    col[0] = fmaf(c[k].x, vi, col[0]);
    col[1] = fmaf(c[k].y, vi, col[1]);
    col[2] = fmaf(c[k].z, vi, col[2]);
    col[3] = fmaf(c[k].w, vi, col[3]);
  }
  if (I == J) return;  // whole CTA: the diagonal block's rows cover it
#pragma unroll
  for (int q = 0; q < 4; ++q) s_col[w][4 * lane + q] = col[q];
  __syncthreads();
  if (threadIdx.x < kSymB) {
    float sum = 0.0f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) sum += s_col[ww][threadIdx.x];
    const int64_t cc = J * kSymB + threadIdx.x;
    if (cc < n) part[I * n + cc] = sum;
  }
}

// out[i] = sum over the NP slots of part[.][i] in FP64 (- Bv[i]).  Block
// (32, 8): x over 32 consecutive rows, y over the slots y, y + 8, ...; the 8
// partial sums are added in a fixed order.
template <bool kGrad>
__global__ void __launch_bounds__(256) symv_reduce_kernel(const float *__restrict__ part,
                                                          int64_t n, int NP,
                                                          const double *__restrict__ Bv,
                                                          float *__restrict__ outf,
                                                          double *__restrict__ outd) {
  __shared__ double s_sum[8][33];
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
#pragma unroll 4
    for (int sl = threadIdx.y; sl < NP; sl += 8) acc += (double)part[(int64_t)sl * n + i];
  }
  s_sum[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < n) {
    double t = 0.0;
#pragma unroll
    for (int y = 0; y < 8; ++y) t += s_sum[y][threadIdx.x];
    if (kGrad) outd[i] = t - Bv[i];
    else outf[i] = (float)t;
  }
}

// Cross-correlations of the code maps for the surrogate update:
//   T[k][k2][dy][dx] = sum over nonzeros z_k(r1) with r1 + (dy, dx) in the
//   same image of z_k(r1) z_k2(r1 + (dy, dx)),  k2 >= k, |dy|, |dx| <= s - 1.
// Entry ((k,u,v),(k2,u2,v2)) of sum_q Z[q]^T Z[q] is T[k][k2][u-u2][v-v2]
// minus the products whose patch centre q = r1 - c + (u,v) lies outside the
// image (only codes within c of the border have such q; surrogate_border_
// kernel subtracts them).
// The nonzeros of a filter are cut into segments of seg_len (how many codes
// each filter holds varies widely, and a filter's walk is sequential); block
// = segment, thread = lag.  Each thread walks its segment in order into the
// segment's own slice (T itself for a filter of one segment), and
// corr_reduce_kernel adds a filter's slices in segment order, so the sums
// are deterministic without atomics.

// seg_off[k] = first segment of filter k, seg_off[K] = segment count.
__global__ void corr_segments_kernel(const int64_t *__restrict__ kt_off, int ntiles, int K,
                                     int seg_len, int *__restrict__ seg_off) {
  if (threadIdx.x != 0) return;
  int run = 0;
  for (int k = 0; k < K; ++k) {
    const int64_t cnt = kt_off[(int64_t)(k + 1) * ntiles] - kt_off[(int64_t)k * ntiles];
    seg_off[k] = run;
    run += (int)((cnt + seg_len - 1) / seg_len);
  }
  seg_off[K] = run;
}

__global__ void __launch_bounds__(512) surrogate_corr_kernel(
    BatchDev b, int K, int S, const int64_t *__restrict__ row_ptr, const int *__restrict__ pk,
    const float *__restrict__ pv, const int64_t *__restrict__ kt_off, int ntiles,
    const int *__restrict__ kpix, const int *__restrict__ kimg, const float *__restrict__ kv,
    const int *__restrict__ seg_off, int seg_len, float *__restrict__ P, float *__restrict__ T) {
  const int seg = blockIdx.x, D = 2 * S - 1, DD = D * D, t = threadIdx.x;
  if (seg >= seg_off[K] || t >= DD) return;
  // the filter of this segment: the last k with seg_off[k] <= seg (filters
  // without segments share their offset with the next one)
  int lo = 0, hi = K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= seg) lo = mid;
    else hi = mid - 1;
  }
  const int k = lo;
  const int dy = t / D - (S - 1), dx = t - (t / D) * D - (S - 1);
  const int64_t kb = kt_off[(int64_t)k * ntiles], ke = kt_off[(int64_t)(k + 1) * ntiles];
  const int64_t e0 = kb + (int64_t)(seg - seg_off[k]) * seg_len;
  const int64_t e1 = e0 + seg_len < ke ? e0 + seg_len : ke;
  float *const Tk = (seg_off[k + 1] - seg_off[k] == 1 ? T + (int64_t)k * K * DD
                                                      : P + (int64_t)seg * K * DD);
  for (int k2 = k; k2 < K; ++k2) Tk[(int64_t)k2 * DD + t] = 0.0f;
  for (int64_t e = e0; e < e1; ++e) {
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

// T[k][k2 >= k][.] of the filters without a single segment: the sum of their
// segments' slices in segment order, or zero for a filter without nonzeros.
__global__ void __launch_bounds__(256) corr_reduce_kernel(const float *__restrict__ P,
                                                          const int *__restrict__ seg_off, int K,
                                                          int DD, float *__restrict__ T) {
  const int k = blockIdx.y;
  const int s0 = seg_off[k], s1 = seg_off[k + 1];
  if (s1 - s0 == 1) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)(K - k) * DD) return;
  const int64_t off = (int64_t)k * DD + i;  // k2 * DD + lag, k2 >= k
  float acc = 0.0f;
  for (int sg = s0; sg < s1; ++sg) acc += P[(int64_t)sg * K * DD + off];
  T[(int64_t)k * K * DD + off] = acc;
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

// Segment length and slice count of the correlation walk for nnz nonzero
// codes: segments of 256 nonzeros, longer where the slices would pass 4 GB.
void surrogate_corr_segments(int K, int s, int64_t nnz, int *seg_len, int64_t *max_segments) {
  const int64_t D = 2 * s - 1, slice = (int64_t)K * D * D * 4;
  const int64_t budget = std::max<int64_t>(K + 1, ((int64_t)4 << 30) / slice);
  int64_t len = 256;
  if (nnz / len + K > budget) len = (nnz + (budget - K) - 1) / (budget - K);
  *seg_len = (int)std::min<int64_t>(len, 0x7fffffff);
  *max_segments = nnz / *seg_len + K;
}

cudaError_t launch_surrogate_update_sparse(const BatchDev &b, int K, int s, const float *x,
                                           const int64_t *row_ptr, const int *pk, const float *pv,
                                           const int64_t *kt_off, const int *kpix,
                                           const int *kimg, const float *kv, double alpha,
                                           double beta, float *Cm, double *Bv, float *T,
                                           const CorrSegments *segs, cudaStream_t st) {
  const int KM = K * s * s;
  const int nt_px = sparse_tiles(b.total_px);
  cudaError_t e;
  if (T == nullptr || segs == nullptr || segs->max_segments > 0x7fffffff)
    return cudaErrorInvalidValue;
  // correlations, then C = alpha C + beta T (upper blocks), then the border
  // corrections and B, then the lower blocks
  corr_segments_kernel<<<1, 32, 0, st>>>(kt_off, nt_px, K, segs->seg_len, segs->seg_off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  surrogate_corr_kernel<<<(unsigned)segs->max_segments, 512, 0, st>>>(
      b, K, s, row_ptr, pk, pv, kt_off, nt_px, kpix, kimg, kv, segs->seg_off, segs->seg_len,
      segs->P, T);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int DD = (2 * s - 1) * (2 * s - 1);
  corr_reduce_kernel<<<dim3((unsigned)(((int64_t)K * DD + 255) / 256), K), 256, 0, st>>>(
      segs->P, segs->seg_off, K, DD, T);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  surrogate_expand_kernel<<<KM, 256, 0, st>>>(Cm, T, K, s, (float)alpha, (float)beta);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t blocks = ((int64_t)KM + 7) / 8;
  surrogate_border_kernel<<<(unsigned)blocks, 256, 0, st>>>(
      b, K, s, x, row_ptr, pk, pv, kt_off, nt_px, kpix, kimg, kv, KM, (float)alpha,
      (float)beta, Cm, Bv);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = (KM + 31) / 32;
  mirror_lower_kernel<<<dim3(nt, nt), 256, 0, st>>>(Cm, KM, s * s);
  return cudaGetLastError();
}

int symv_panels(int64_t n) { return (int)((n + kSymB - 1) / kSymB); }

template <bool kGrad>
static cudaError_t symv_both(const float *Cm, int64_t n, const float *v, const double *Bv,
                             float *outf, double *outd, float *part, cudaStream_t st) {
  const int NP = symv_panels(n);
  const int64_t nblocks = (int64_t)NP * (NP + 1) / 2;
  if (nblocks > 0x7fffffff) return cudaErrorInvalidValue;
  if (n % 4 == 0)
    symv_upper_kernel<true><<<(unsigned)nblocks, 256, 0, st>>>(Cm, n, NP, v, part);
  else
    symv_upper_kernel<false><<<(unsigned)nblocks, 256, 0, st>>>(Cm, n, NP, v, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  symv_reduce_kernel<kGrad><<<(unsigned)((n + 31) / 32), dim3(32, 8), 0, st>>>(part, n, NP, Bv,
                                                                               outf, outd);
  return cudaGetLastError();
}

cudaError_t launch_symv(const float *Cm, int64_t n, const float *v, float *out, float *part,
                        cudaStream_t st) {
  return symv_both<false>(Cm, n, v, nullptr, out, nullptr, part, st);
}

cudaError_t launch_symv_grad(const float *Cm, int64_t n, const float *d, const double *Bv,
                             double *out, float *part, cudaStream_t st) {
  return symv_both<true>(Cm, n, d, Bv, nullptr, out, part, st);
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
