// kernels_screen.cu -- safe screening of the code problem (Eq. 3 restricted to
// each image's active set S; Sec. 5 names safe screening of this sparse LASSO
// as a way to skip coordinate updates).  The test is the duality-gap sphere
// test.  With r = D z - x (codes zero off S) and g = D^T r on S, from the
// plain FP32 synthesis and adjoint, per image:
//   rr = ||r||^2, xr = <x, r>, xx = ||x||^2, l1 = ||z_S||_1, gm = max_S |g|
//   (FP64 block partials, summed in a fixed order);
//   scale = max(lambda, gm), beta = lambda / scale;
//   P = rr / 2 + lambda l1; the dual value at theta = -r / scale is
//   -(beta xr + beta^2 rr / 2); gap = max(P - dual, 0);
//   R = sqrt(2 (gap + eta (P + xx / 2))) / lambda,  eta = 1e-6;
//   j in S leaves S (bit cleared, z_j = 0) when
//     |g_j| / scale + R ||a_j|| < 1 - tau,  tau = 1e-4,
// ||a_j|| the norm of filter k over the taps that land on the image.  The
// optimal dual point lies within sqrt(2 gap) / lambda of theta, so such a
// coordinate is zero in every solution; eta and tau cover the FP32 rounding of
// P, the dual value and g.
#include <math.h>

#include "scsc_internal.cuh"

namespace scsc {
namespace {

constexpr int kBlock = 256;
constexpr double kEta = 1e-6;
constexpr float kTau = 1e-4f;
constexpr int kStats = 5;  // rr, xr, xx, l1, gm
constexpr int kU = 4;      // codes per thread and round in the stats and test loops

// pref[k][a][b] = sum_{u < a, v < b} d_k(u, v)^2 (FP64, (s+1)^2 per filter);
// nrm[k] = ||d_k||.  One thread per filter.
__global__ void screen_norms_kernel(const float *d, int K, int s, double *pref, float *nrm) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int n1 = s + 1;
  double *p = pref + (int64_t)k * n1 * n1;
  for (int b = 0; b < n1; ++b) p[b] = 0.0;
  for (int a = 1; a < n1; ++a) {
    double row = 0.0;
    p[a * n1] = 0.0;
    for (int b = 1; b < n1; ++b) {
      const double w = d[((int64_t)k * s + (a - 1)) * s + (b - 1)];
      row += w * w;
      p[a * n1 + b] = p[(a - 1) * n1 + b] + row;
    }
  }
  nrm[k] = (float)sqrt(p[s * n1 + s]);
}

// Walks the codes [0, npx K) of one image in a grid-stride loop, keeping the
// pixel p and filter k of the current code without a division per step.
struct CodeWalk {
  int64_t e, p;  // code index within the image, its pixel
  int k;         // its filter
  int64_t dp;    // pixels per stride
  int dk;        // filters per stride (remainder)
  int K;
  __device__ CodeWalk(int64_t start, int64_t stride, int K_) : e(start), K(K_) {
    p = start / K_;
    k = (int)(start - p * K_);
    dp = stride / K_;
    dk = (int)(stride - dp * K_);
  }
  // advance by one stride; returns the pixel increment (dp or dp + 1)
  __device__ __forceinline__ int64_t step(int64_t stride) {
    e += stride;
    k += dk;
    int64_t inc = dp;
    if (k >= K) {
      k -= K;
      ++inc;
    }
    p += inc;
    return inc;
  }
};

// part[(n * gridDim.x + block) * 5 + q]: this block's share of image n's
// rr, xr, xx (pixels) and l1, gm (codes of the set); consecutive threads take
// consecutive codes (coalesced), each checks its own mask bit.
__global__ void __launch_bounds__(kBlock) screen_stats_kernel(BatchDev b, int K, const float *x,
                                                              const float *r, const float *z,
                                                              const float *g,
                                                              const uint32_t *bits,
                                                              double *part) {
  __shared__ double sh[kBlock / 32][kStats];
  const int n = blockIdx.y, KW = (K + 31) >> 5, lane = threadIdx.x & 31;
  const int64_t p0 = b.off[n], npx = b.off[n + 1] - p0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0, xr = 0.0, xx = 0.0, l1 = 0.0;
  for (int64_t p = t0; p < npx; p += stride) {
    const double rv = r[p0 + p], xv = x[p0 + p];
    rr += rv * rv;
    xr += xv * rv;
    xx += xv * xv;
  }
  // codes, kU strides per round with every load issued before any use (the
  // loop is bound by memory latency otherwise); FP32 within a round, FP64
  // across rounds
  const float *zi = z + p0 * K, *gi = g + p0 * K;
  const uint32_t *bi = bits + p0 * KW;
  const int64_t total = npx * K;
  float gm = 0.0f;
  for (CodeWalk c(t0, stride, K); c.e < total;) {
    float zv[kU], gv[kU];
    uint32_t on[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      on[u] = 0u;
      zv[u] = gv[u] = 0.0f;
      if (c.e < total) {
        on[u] = bi[c.p * KW + (c.k >> 5)] >> (c.k & 31);
        zv[u] = zi[c.e];
        gv[u] = gi[c.e];
        c.step(stride);
      }
    }
    float l1p = 0.0f;
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (on[u] & 1u) {
        l1p += fabsf(zv[u]);
        gm = fmaxf(gm, fabsf(gv[u]));
      }
    l1 += l1p;
  }
  double gmd = gm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    xr += __shfl_down_sync(0xffffffffu, xr, o);
    xx += __shfl_down_sync(0xffffffffu, xx, o);
    l1 += __shfl_down_sync(0xffffffffu, l1, o);
    gmd = fmax(gmd, __shfl_down_sync(0xffffffffu, gmd, o));
  }
  const int wi = threadIdx.x >> 5;
  if (lane == 0) {
    sh[wi][0] = rr;
    sh[wi][1] = xr;
    sh[wi][2] = xx;
    sh[wi][3] = l1;
    sh[wi][4] = gmd;
  }
  __syncthreads();
  if (threadIdx.x < kStats) {
    const int q = threadIdx.x;
    double t = sh[0][q];
    for (int i = 1; i < kBlock / 32; ++i) t = q == 4 ? fmax(t, sh[i][q]) : t + sh[i][q];
    part[((int64_t)n * gridDim.x + blockIdx.x) * kStats + q] = t;
  }
}

// One thread per image: the gap, 1 / scale and the sphere radius.
__global__ void screen_finish_kernel(int n_img, const double *part, int nb, double lambda,
                                     ScreenImage *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_img) return;
  double v[kStats] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < nb; ++i)
    for (int q = 0; q < kStats; ++q) {
      const double t = part[((int64_t)n * nb + i) * kStats + q];
      v[q] = q == 4 ? fmax(v[q], t) : v[q] + t;
    }
  const double rr = v[0], xr = v[1], xx = v[2], l1 = v[3], gm = v[4];
  const double scale = fmax(lambda, gm), beta = lambda / scale;
  const double primal = 0.5 * rr + lambda * l1;
  const double dual = -(beta * xr + 0.5 * beta * beta * rr);
  const double gap = fmax(primal - dual, 0.0);
  ScreenImage o;
  o.gap = gap;
  o.primal = primal;
  o.inv_scale = 1.0 / scale;
  o.radius = sqrt(2.0 * (gap + kEta * (primal + 0.5 * xx))) / lambda;
  out[n] = o;
}

// ||a_j|| for filter k at code position (a, c2) of an H x W image: the full
// norm inside, the rectangle of taps that land on the image near the edges.
__device__ __forceinline__ float column_norm(const double *pref, const float *nrm, int k, int s,
                                             int H, int W, int a, int c2) {
  const int c = (s - 1) / 2;
  if (a >= c && a < H - c && c2 >= c && c2 < W - c) return nrm[k];
  // pixel a - c + u on the image: u in [c - a, H - 1 - a + c]
  const int u0 = max(0, c - a), u1 = min(s - 1, H - 1 - a + c);
  const int v0 = max(0, c - c2), v1 = min(s - 1, W - 1 - c2 + c);
  const int n1 = s + 1;
  const double *p = pref + (int64_t)k * n1 * n1;
  const double sum = p[(u1 + 1) * n1 + v1 + 1] - p[u0 * n1 + v1 + 1] - p[(u1 + 1) * n1 + v0] +
                     p[u0 * n1 + v0];
  return (float)sqrt(fmax(sum, 0.0));
}

// Consecutive threads test consecutive codes of image n (coalesced); a
// removed coordinate clears its bit with an atomic AND (words are shared
// between threads) and its code.  kept[n] += the block's survivors.
__global__ void __launch_bounds__(kBlock) screen_test_kernel(BatchDev b, int K, int s,
                                                             const float *g, uint32_t *bits,
                                                             float *z, const ScreenImage *img,
                                                             const double *pref, const float *nrm,
                                                             unsigned long long *kept) {
  __shared__ unsigned long long sh[kBlock / 32];
  const int n = blockIdx.y, KW = (K + 31) >> 5;
  const int H = b.H[n], W = b.W[n];
  const int64_t p0 = b.off[n], npx = b.off[n + 1] - p0;
  const ScreenImage im = img[n];
  const float inv_scale = (float)im.inv_scale, radius = (float)im.radius;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float *zi = z + p0 * K;
  const float *gi = g + p0 * K;
  uint32_t *bi = bits + p0 * KW;
  CodeWalk c(t0, stride, K);
  // row a and column c2 of pixel c.p, advanced with it
  int a = (int)(c.p / W), c2 = (int)(c.p - (int64_t)a * W);
  const int64_t da = c.dp / W;
  const int dc = (int)(c.dp - da * W);
  const int64_t total = npx * K;
  unsigned long long cnt = 0;
  while (c.e < total) {
    // kU codes per round: every load issued before any use
    int64_t ev[kU], wv[kU];
    int kv[kU], av[kU], cv[kU];
    uint32_t word[kU];
    float gv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      ev[u] = -1;
      word[u] = 0u;
      gv[u] = 0.0f;
      kv[u] = av[u] = cv[u] = 0;
      wv[u] = 0;
      if (c.e < total) {
        ev[u] = c.e;
        kv[u] = c.k;
        av[u] = a;
        cv[u] = c2;
        wv[u] = c.p * KW + (c.k >> 5);
        word[u] = bi[wv[u]];
        gv[u] = gi[c.e];
        const int64_t inc = c.step(stride);
        a += (int)da;
        c2 += dc + (int)(inc - c.dp);
        if (c2 >= W) {
          c2 -= W;
          ++a;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t bit = 1u << (kv[u] & 31);
      if (ev[u] < 0 || !(word[u] & bit)) continue;
      const float stat = fabsf(gv[u]) * inv_scale +
                         radius * column_norm(pref, nrm, kv[u], s, H, W, av[u], cv[u]);
      if (stat < 1.0f - kTau) {
        zi[ev[u]] = 0.0f;
        atomicAnd(bi + wv[u], ~bit);
      } else {
        ++cnt;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < kBlock / 32; ++i) t += sh[i];
    if (t) atomicAdd(kept + n, t);
  }
}

}  // namespace

cudaError_t launch_screen_prepare(const float *d, int K, int s, double *pref, float *nrm,
                                  cudaStream_t st) {
  screen_norms_kernel<<<(K + 127) / 128, 128, 0, st>>>(d, K, s, pref, nrm);
  return cudaGetLastError();
}

cudaError_t launch_screen_stats(const BatchDev &b, int K, const float *x, const float *r,
                                const float *z, const float *g, const uint32_t *bits,
                                double *part, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  screen_stats_kernel<<<dim3(kScreenBlocks, b.n), kBlock, 0, st>>>(b, K, x, r, z, g, bits, part);
  return cudaGetLastError();
}

cudaError_t launch_screen_finish(int n_img, const double *part, double lambda, ScreenImage *img,
                                 cudaStream_t st) {
  if (n_img == 0) return cudaSuccess;
  screen_finish_kernel<<<(n_img + 127) / 128, 128, 0, st>>>(n_img, part, kScreenBlocks, lambda,
                                                           img);
  return cudaGetLastError();
}

cudaError_t launch_screen_test(const BatchDev &b, int K, int s, const float *g, uint32_t *bits,
                               float *z, const ScreenImage *img, const double *pref,
                               const float *nrm, unsigned long long *kept, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  screen_test_kernel<<<dim3(kScreenBlocks, b.n), kBlock, 0, st>>>(b, K, s, g, bits, z, img, pref,
                                                                  nrm, kept);
  return cudaGetLastError();
}

}  // namespace scsc
