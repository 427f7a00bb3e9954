// kernels_ddt.cu -- the pixel-space operator D D^T of the code step size
// (power iteration for L_z) as one 21x21 stencil per pixel class.
//
// With zero padding and same-size codes, D^T u keeps the code maps only on
// the image grid, and D then sums them back:
//   (D D^T u)(i, j) = sum_{u,v,u',v'} G[(u,v),(u',v')] u(i + u' - u, j + v' - v)
//                     over taps (u, v) whose code position (i + c - u,
//                     j + c - v) lies on the grid,
//   G[(u,v),(u',v')] = sum_k d_k(u, v) d_k(u', v')        (tap Gram matrix).
// The grid condition only restricts u to [max(0, i + c - H + 1), min(s-1, i + c)]
// and v likewise, so every row i falls into one of at most s classes (c rows
// at each edge, one interior class) and every column too.  Per class pair the
// operator is a stencil A[dy][dx], dy, dx in [-(s-1), s-1]; the result equals
// the composition of the adjoint and the synthesis exactly, summed in another
// order.  Cost per application: (2s-1)^2 multiply-adds per pixel instead of
// 2 K s^2.
#include "scsc_internal.cuh"

namespace scsc {
namespace {

constexpr int kTile = 16;  // output tile side of the apply kernel

// Row class of row i of an n-row grid (see above) and its representative row.
__host__ __device__ inline int row_class(int i, int n, int c) {
  if (n <= 2 * c + 1) return i;
  if (i < c) return i;
  if (i >= n - c) return i - (n - 2 * c - 1);
  return c;
}
__host__ __device__ inline int class_row(int k, int n, int c) {
  if (n <= 2 * c + 1) return k;
  if (k < c) return k;
  if (k > c) return k + (n - 2 * c - 1);
  return c;
}
inline int n_classes(int n, int c) { return n < 2 * c + 1 ? n : 2 * c + 1; }

// G[t][t'] = sum_k d_k[t] d_k[t'] in FP64; one thread per (t, t').
__global__ void tap_gram_kernel(const float *d, int K, int M, double *G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * M) return;
  const int t = idx / M, t2 = idx - t * M;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) acc += (double)d[(int64_t)k * M + t] * (double)d[(int64_t)k * M + t2];
  G[idx] = acc;
}

// A[cy][cx][dy + s - 1][dx + s - 1] for every class pair; one thread per entry.
__global__ void stencil_kernel(const double *G, int s, int H, int W, int ncy, int ncx, float *A) {
  const int n_a = 2 * s - 1, per = n_a * n_a;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncy * ncx * per) return;
  const int cls = idx / per, e = idx - cls * per;
  const int cy = cls / ncx, cx = cls - cy * ncx;
  const int dy = e / n_a - (s - 1), dx = e % n_a - (s - 1);
  const int c = (s - 1) / 2, M = s * s;
  const int iy = class_row(cy, H, c), ix = class_row(cx, W, c);
  const int u_lo = max(max(0, iy + c - H + 1), -dy), u_hi = min(min(s - 1, iy + c), s - 1 - dy);
  const int v_lo = max(max(0, ix + c - W + 1), -dx), v_hi = min(min(s - 1, ix + c), s - 1 - dx);
  double acc = 0.0;
  for (int u = u_lo; u <= u_hi; ++u)
    for (int v = v_lo; v <= v_hi; ++v) acc += G[(u * s + v) * M + (u + dy) * s + (v + dx)];
  A[idx] = (float)acc;
}

// w = (D D^T) u on an H x W grid: 16x16 output tiles, the input tile with its
// (s-1)-pixel halo (zero outside the grid) in shared memory, one output per
// thread, the pixel's class stencil read through the L1 (a warp mostly shares
// one class, so the reads broadcast).
template <int S>
__global__ void __launch_bounds__(kTile *kTile) ddt_apply_kernel(const float *__restrict__ u,
                                                                  const float *__restrict__ A,
                                                                  int H, int W, int ncx,
                                                                  float *__restrict__ w) {
  constexpr int R = S - 1, C = (S - 1) / 2, NA = 2 * S - 1, T = kTile + 2 * R;
  __shared__ float tile[T][T + 1];
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  for (int k = threadIdx.x; k < T * T; k += kTile * kTile) {
    const int ty = k / T, tx = k - ty * T;
    const int gy = y0 - R + ty, gx = x0 - R + tx;
    tile[ty][tx] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? u[(int64_t)gy * W + gx] : 0.0f;
  }
  __syncthreads();
  const int ty = threadIdx.x / kTile, tx = threadIdx.x % kTile;
  const int i = y0 + ty, j = x0 + tx;
  if (i >= H || j >= W) return;
  const float *a = A + (int64_t)(row_class(i, H, C) * ncx + row_class(j, W, C)) * NA * NA;
  float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll
  for (int dy = 0; dy < NA; ++dy) {
#pragma unroll
    for (int dx = 0; dx < NA; ++dx) {
      const float t = __ldg(a + dy * NA + dx) * tile[ty + dy][tx + dx];
      if (dx & 1) acc1 += t;
      else acc0 += t;
    }
  }
  w[(int64_t)i * W + j] = acc0 + acc1;
}

}  // namespace

size_t ddt_stencil_floats(int s, int H, int W) {
  const int c = (s - 1) / 2;
  return (size_t)n_classes(H, c) * n_classes(W, c) * (2 * s - 1) * (2 * s - 1);
}

cudaError_t launch_ddt_prepare(const float *d, int K, int s, int H, int W, double *G, float *A,
                               cudaStream_t st) {
  if (s < 1 || s > kMaxS || H < 1 || W < 1) return cudaErrorInvalidValue;
  const int M = s * s, c = (s - 1) / 2;
  tap_gram_kernel<<<(M * M + 255) / 256, 256, 0, st>>>(d, K, M, G);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ncy = n_classes(H, c), ncx = n_classes(W, c);
  const int n = ncy * ncx * (2 * s - 1) * (2 * s - 1);
  stencil_kernel<<<(n + 255) / 256, 256, 0, st>>>(G, s, H, W, ncy, ncx, A);
  return cudaGetLastError();
}

cudaError_t launch_ddt_apply(const float *A, int s, int H, int W, const float *u, float *w,
                             cudaStream_t st) {
  const int c = (s - 1) / 2, ncx = n_classes(W, c);
  const dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  switch (s) {
#define SCSC_DDT_CASE(SV)                                                              \
  case SV:                                                                             \
    ddt_apply_kernel<SV><<<grid, kTile * kTile, 0, st>>>(u, A, H, W, ncx, w);          \
    break;
    SCSC_DDT_CASE(1)
    SCSC_DDT_CASE(3)
    SCSC_DDT_CASE(5)
    SCSC_DDT_CASE(7)
    SCSC_DDT_CASE(9)
    SCSC_DDT_CASE(11)
#undef SCSC_DDT_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace scsc
