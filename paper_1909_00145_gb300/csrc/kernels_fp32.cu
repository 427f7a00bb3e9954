// kernels_fp32.cu -- FP32 SIMT kernels: subsampling mask (Sec. 3.1), masked
// synthesis with fused residual, adjoint correlation with fused proximal step
// (Eq. 3), filter gradient (Eq. 5), FP64 reductions for the objective (Eq. 1)
// and the power iterations that set the step sizes, filter projection.
//
// Spatial tiles are 32 x 32 pixels.  Codes are float32 [pixel][K]; images are
// packed back to back (see scsc.h).
#include <algorithm>

#include "scsc_internal.cuh"

namespace scsc {

namespace {

constexpr int kTile = 32;

struct TileCoord {
  int n, y0, x0, H, W;
  int64_t base;
};

__device__ __forceinline__ TileCoord tile_coord(const BatchDev &b, int tile) {
  tile += b.tile_base;
  TileCoord c;
  c.n = upper_index(b.tile0, b.n, tile);
  c.H = b.H[c.n];
  c.W = b.W[c.n];
  int tiles_x = (c.W + kTile - 1) / kTile;
  int lt = tile - b.tile0[c.n];
  c.y0 = (lt / tiles_x) * kTile;
  c.x0 = (lt % tiles_x) * kTile;
  c.base = b.off[c.n];
  return c;
}

__device__ __forceinline__ bool bit_of(const uint32_t *bits, int64_t pix, int KW, int k) {
  return (bits[pix * KW + (k >> 5)] >> (k & 31)) & 1u;
}

// ------------------------------------------------------------------ mask

// One block per 32x32 tile (image and position found once per block), one
// thread per pixel column and every eighth row; the coordinate index
// (k H + y) W + x advances by H W per filter.
__global__ void __launch_bounds__(256) mask_bits_kernel(BatchDev b, int K, int KW, uint64_t seed,
                                                        uint64_t t, uint64_t T, uint32_t *bits) {
  const TileCoord tc = tile_coord(b, blockIdx.x);
  const uint64_t pre = mask_prefix(seed, t, (uint64_t)b.ids[tc.n]);
  const uint64_t HW = (uint64_t)tc.H * (uint64_t)tc.W;
  const int x = tc.x0 + (threadIdx.x & 31);
  if (x >= tc.W) return;
  for (int yy = threadIdx.x >> 5; yy < kTile; yy += 8) {
    const int y = tc.y0 + yy;
    if (y >= tc.H) break;
    const int64_t pix = tc.base + (int64_t)y * tc.W + x;
    uint64_t idx = (uint64_t)y * (uint64_t)tc.W + (uint64_t)x;
    for (int w = 0; w < KW; ++w) {
      uint32_t word = 0;
      const int kn = min(32, K - 32 * w);
      for (int j = 0; j < kn; ++j, idx += HW)
        if ((splitmix64(pre ^ idx) >> 32) < T) word |= 1u << j;
      bits[pix * KW + w] = word;
    }
  }
}

// r <- O r: zero the residual at unobserved pixels (inpainting data term).
__global__ void mask_residual_kernel(float *r, const uint8_t *obs, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (obs[i] == 0) r[i] = 0.0f;
}

__global__ void apply_mask_dense_kernel(int64_t total, int K, int KW, const uint32_t *bits,
                                        float *z) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t pix = g / K;
    int k = (int)(g - pix * K);
    if (!bit_of(bits, pix, KW, k)) z[g] = 0.0f;
  }
}

// ------------------------------------------------------------------ synthesis
// out(i,j) = sum_k sum_{u,v} d_k(u,v) z_k(i+c-u, j+c-v)  [- x(i,j)]
// 128 threads; thread (tx, ty) owns column tx and rows 8 ty .. 8 ty + 7.

// gridDim.y > 1 splits the filters into gridDim.y ranges of `kspan`; each
// range writes its partial sum to out + blockIdx.y * total_px (no residual).
template <int S, int KC>
__global__ void __launch_bounds__(128) synth_fp32_kernel(BatchDev b, int K, int kspan,
                                                         const float *__restrict__ d,
                                                         const float *__restrict__ z,
                                                         const uint32_t *__restrict__ bits,
                                                         const float *__restrict__ x,
                                                         float *__restrict__ out) {
  constexpr int C = (S - 1) / 2;
  constexpr int HS = kTile + S - 1;
  constexpr int R = 8;
  __shared__ float zs[KC][HS][HS + 1];
  __shared__ float ds[KC][S * S];
  const TileCoord tc = tile_coord(b, blockIdx.x);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int KW = (K + 31) >> 5;
  float acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0f;

  const int kbeg = blockIdx.y * kspan, kend = min(K, kbeg + kspan);
  for (int k0 = kbeg; k0 < kend; k0 += KC) {
    __syncthreads();
    for (int i = threadIdx.x; i < HS * HS; i += blockDim.x) {
      int hy = i / HS, hx = i - hy * HS;
      int yy = tc.y0 - C + hy, xx = tc.x0 - C + hx;
      bool in = yy >= 0 && yy < tc.H && xx >= 0 && xx < tc.W;
      int64_t pix = tc.base + (int64_t)yy * tc.W + xx;
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        int k = k0 + kk;
        float v = 0.0f;
        if (in && k < kend) {
          v = z[pix * K + k];
          if (bits != nullptr && !bit_of(bits, pix, KW, k)) v = 0.0f;
        }
        zs[kk][hy][hx] = v;
      }
    }
    for (int i = threadIdx.x; i < KC * S * S; i += blockDim.x) {
      int kk = i / (S * S), m = i - kk * S * S;
      ds[kk][m] = (k0 + kk < kend) ? d[(int64_t)(k0 + kk) * S * S + m] : 0.0f;
    }
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < KC; ++kk) {
#pragma unroll 1
      for (int v = 0; v < S; ++v) {
        float col[R + S - 1];
#pragma unroll
        for (int q = 0; q < R + S - 1; ++q) col[q] = zs[kk][ty * R + q][tx + 2 * C - v];
#pragma unroll
        for (int u = 0; u < S; ++u) {
          float dv = ds[kk][u * S + v];
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] = fmaf(dv, col[r + 2 * C - u], acc[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int i = tc.y0 + ty * R + r, j = tc.x0 + tx;
    if (i < tc.H && j < tc.W) {
      int64_t p = tc.base + (int64_t)i * tc.W + j;
      if (gridDim.y > 1) out[blockIdx.y * b.total_px + p] = acc[r];
      else out[p] = x != nullptr ? acc[r] - x[p] : acc[r];
    }
  }
}

// out[p] = sum_s part[s][p] (- x[p]), fixed order over s.
__global__ void sum_split_kernel(const float *__restrict__ part, int nsplit, int64_t n,
                                 const float *__restrict__ x, float *__restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.0f;
    for (int s2 = 0; s2 < nsplit; ++s2) v += part[s2 * n + p];
    out[p] = x != nullptr ? v - x[p] : v;
  }
}

// ------------------------------------------------------------------ adjoint
// g_k(a,b) = sum_{u,v} d_k(u,v) r(a-c+u, b-c+v).
// mode 0: store g (zero at unsampled coordinates when bits != null)
// mode 1: proximal step at sampled coordinates,
//         z <- soft(z - alpha g, alpha lambda); other coordinates untouched.

template <int S>
__global__ void __launch_bounds__(128) adjoint_fp32_kernel(BatchDev b, int K,
                                                           const float *__restrict__ d,
                                                           const float *__restrict__ r,
                                                           const uint32_t *__restrict__ bits,
                                                           int mode,
                                                           const StepParams *__restrict__ prm,
                                                           float *__restrict__ zg) {
  constexpr int C = (S - 1) / 2;
  constexpr int HS = kTile + S - 1;
  constexpr int R = 8;
  constexpr int KCH = 32;  // filters staged per pass
  constexpr int KC = 4;    // filters per register block
  __shared__ float rs[HS][HS + 1];
  __shared__ __align__(16) float ds[S][S][KCH];  // [v][u][k]
  const TileCoord tc = tile_coord(b, blockIdx.x);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int KW = (K + 31) >> 5;
  float alpha = 0.0f, thr = 0.0f;
  if (mode == 1) {
    alpha = prm->alpha;
    thr = prm->thresh;
  }
  for (int i = threadIdx.x; i < HS * HS; i += blockDim.x) {
    int hy = i / HS, hx = i - hy * HS;
    int yy = tc.y0 - C + hy, xx = tc.x0 - C + hx;
    bool in = yy >= 0 && yy < tc.H && xx >= 0 && xx < tc.W;
    rs[hy][hx] = in ? r[tc.base + (int64_t)yy * tc.W + xx] : 0.0f;
  }
  const int kspan = (K + gridDim.y - 1) / gridDim.y;
  const int kbeg = blockIdx.y * ((kspan + KCH - 1) / KCH) * KCH;
  for (int kc0 = kbeg; kc0 < K && kc0 < kbeg + ((kspan + KCH - 1) / KCH) * KCH; kc0 += KCH) {
    __syncthreads();
    for (int i = threadIdx.x; i < KCH * S * S; i += blockDim.x) {
      int kk = i / (S * S), m = i - kk * S * S;
      int u = m / S, v = m - u * S;
      ds[v][u][kk] = (kc0 + kk < K) ? d[(int64_t)(kc0 + kk) * S * S + m] : 0.0f;
    }
    __syncthreads();
    const int kend = min(KCH, K - kc0);
#pragma unroll 1
    for (int kb = 0; kb < kend; kb += KC) {
      float acc[KC][R];
#pragma unroll
      for (int q = 0; q < KC; ++q)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) acc[q][rr] = 0.0f;
#pragma unroll 1
      for (int v = 0; v < S; ++v) {
        float col[R + S - 1];
#pragma unroll
        for (int q = 0; q < R + S - 1; ++q) col[q] = rs[ty * R + q][tx + v];
#pragma unroll
        for (int u = 0; u < S; ++u) {
          float4 dv = *reinterpret_cast<const float4 *>(&ds[v][u][kb]);
#pragma unroll
          for (int rr = 0; rr < R; ++rr) {
            acc[0][rr] = fmaf(dv.x, col[rr + u], acc[0][rr]);
            acc[1][rr] = fmaf(dv.y, col[rr + u], acc[1][rr]);
            acc[2][rr] = fmaf(dv.z, col[rr + u], acc[2][rr]);
            acc[3][rr] = fmaf(dv.w, col[rr + u], acc[3][rr]);
          }
        }
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        int a = tc.y0 + ty * R + rr, bb = tc.x0 + tx;
        if (a >= tc.H || bb >= tc.W) continue;
        int64_t pix = tc.base + (int64_t)a * tc.W + bb;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          int k = kc0 + kb + q;
          if (kb + q >= kend) break;
          bool on = bits == nullptr || bit_of(bits, pix, KW, k);
          float *p = zg + pix * K + k;
          if (mode == 0) {
            *p = on ? acc[q][rr] : 0.0f;
          } else if (on) {
            *p = soft_threshold(*p - alpha * acc[q][rr], thr);
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ filter gradient
// G_k(u,v) = sum_a z_k(a) r(a_y-c+u, a_x-c+v), summed over the pixels of the
// tiles this block visits; one partial per (block row, k, u, v).
// Thread = (filter kk in a chunk of 32, tap row u); 11 v accumulators.

template <int S>
__global__ void __launch_bounds__(32 * S) filter_grad_fp32_kernel(BatchDev b, int K,
                                                                  const float *__restrict__ r,
                                                                  const float *__restrict__ z,
                                                                  const uint32_t *__restrict__ bits,
                                                                  float *__restrict__ partial) {
  constexpr int C = (S - 1) / 2;
  constexpr int HR = 16;               // code rows per pass
  constexpr int HS_Y = HR + S - 1, HS_X = kTile + S - 1;
  constexpr int KCH = 32;
  extern __shared__ float smem[];
  float *zs = smem;                              // [HR][kTile][KCH]
  float *rs = smem + HR * kTile * KCH;           // [HS_Y][HS_X + 1]
  const int kk = threadIdx.x % KCH, u = threadIdx.x / KCH;  // u < S
  const int k0 = blockIdx.y * KCH;
  const int KW = (K + 31) >> 5;
  float acc[S];
#pragma unroll
  for (int v = 0; v < S; ++v) acc[v] = 0.0f;

  for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
    const TileCoord tc = tile_coord(b, tile);
    for (int half = 0; half < kTile / HR; ++half) {
      const int ya = tc.y0 + half * HR;
      if (ya >= tc.H) break;
      __syncthreads();
      for (int i = threadIdx.x; i < HR * kTile * KCH; i += blockDim.x) {
        int q = i % KCH, px = (i / KCH) % kTile, py = i / (KCH * kTile);
        int yy = ya + py, xx = tc.x0 + px, k = k0 + q;
        float v = 0.0f;
        if (yy < tc.H && xx < tc.W && k < K) {
          int64_t pix = tc.base + (int64_t)yy * tc.W + xx;
          v = z[pix * K + k];
          if (bits != nullptr && !bit_of(bits, pix, KW, k)) v = 0.0f;
        }
        zs[i] = v;
      }
      for (int i = threadIdx.x; i < HS_Y * HS_X; i += blockDim.x) {
        int hy = i / HS_X, hx = i - hy * HS_X;
        int yy = ya - C + hy, xx = tc.x0 - C + hx;
        bool in = yy >= 0 && yy < tc.H && xx >= 0 && xx < tc.W;
        rs[hy * (HS_X + 1) + hx] = in ? r[tc.base + (int64_t)yy * tc.W + xx] : 0.0f;
      }
      __syncthreads();
      if (u < S) {
#pragma unroll 1
        for (int py = 0; py < HR; ++py) {
          const float *rrow = rs + (py + u) * (HS_X + 1);
          float win[S];
#pragma unroll
          for (int v = 0; v < S; ++v) win[v] = rrow[v];
#pragma unroll 4
          for (int px = 0; px < kTile; ++px) {
            float zv = zs[(py * kTile + px) * KCH + kk];
#pragma unroll
            for (int v = 0; v < S; ++v) acc[v] = fmaf(zv, win[v], acc[v]);
#pragma unroll
            for (int v = 0; v < S - 1; ++v) win[v] = win[v + 1];
            win[S - 1] = (px + S < HS_X) ? rrow[px + S] : 0.0f;
          }
        }
      }
    }
  }
  const int k = k0 + kk;
  if (u < S && k < K) {
    float *dst = partial + ((int64_t)blockIdx.x * K + k) * S * S + u * S;
#pragma unroll
    for (int v = 0; v < S; ++v) dst[v] = acc[v];
  }
}

// out[i] = sum_g partial[g][i] in FP64, fixed order over g.
__global__ void reduce_partials_kernel(const float *partial, int n_groups, int len, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double s = 0.0;
  for (int g = 0; g < n_groups; ++g) s += (double)partial[(int64_t)g * len + i];
  out[i] = s;
}

// ------------------------------------------------------------------ FP64 reductions

template <int BS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[BS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < BS / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// partials[blk] = sum a_i^2 (i < n_sq) and partials[NB + blk] = sum |b_i| (i < n_abs)
__global__ void __launch_bounds__(256) sum_sq_abs_kernel(const float *a, int64_t n_sq,
                                                         const float *bv, int64_t n_abs,
                                                         double *partials) {
  double s = 0.0, t = 0.0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_sq; i += stride) {
    double v = a[i];
    s += v * v;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_abs; i += stride)
    t += fabs((double)bv[i]);
  s = block_sum<256>(s);
  t = block_sum<256>(t);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    partials[gridDim.x + blockIdx.x] = t;
  }
}

// out = scale_sq * sum partials[0..nb) + scale_abs * sum partials[nb..2nb)
__global__ void finish_sum_kernel(const double *partials, int nb, double scale_sq,
                                  double scale_abs, double *out) {
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s += partials[i];
    t += partials[nb + i];
  }
  s = block_sum<256>(s);
  t = block_sum<256>(t);
  if (threadIdx.x == 0) *out = scale_sq * s + scale_abs * t;
}

__global__ void __launch_bounds__(256) dot_partials_kernel(const float *a, const float *bv,
                                                           int64_t n, double *partials) {
  double s = 0.0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    s += (double)a[i] * (double)bv[i];
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// u0_i = +1 / -1 by the top bit of mix(mix(seed ^ tag) ^ i)
__global__ void power_init_kernel(float *u, int64_t n, uint64_t seed, uint64_t tag) {
  uint64_t base = splitmix64(seed ^ tag);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] = (splitmix64(base ^ (uint64_t)i) >> 63) ? -1.0f : 1.0f;
}

// u = w / ||w|| with ||w||^2 = sum of partials (fixed order: strided per
// thread, then the block tree); u = 0 if ||w|| = 0.
__global__ void __launch_bounds__(256) power_normalize_kernel(const float *w, float *u, int64_t n,
                                                              const double *partials, int nb) {
  __shared__ double inv;
  double p = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) p += partials[i];
  p = block_sum<256>(p);
  if (threadIdx.x == 0) inv = p > 0.0 ? 1.0 / sqrt(p) : 0.0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] = (float)((double)w[i] * inv);
}

// lambda_hat = <u, A u> (sum of partials); L = safety * lambda_hat;
// step = fixed_step if > 0 else 1 / L (0 when L = 0).
__global__ void power_finish_kernel(const double *partials, int nb, double safety, double *L_out,
                                    double lambda, double fixed_step, StepParams *prm) {
  if (blockIdx.x != 0) return;
  double s = 0.0;  // one warp, fixed order
  for (int i = threadIdx.x; i < nb; i += 32) s += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x != 0) return;
  double L = safety * s;
  if (L_out != nullptr) *L_out = L;
  if (prm != nullptr) {
    double a = fixed_step > 0.0 ? fixed_step : (L > 0.0 ? 1.0 / L : 0.0);
    prm->alpha = (float)a;
    prm->thresh = (float)(a * lambda);
  }
}

// d_k <- P(d_k - G_k / L): one block per filter, FP32 arithmetic.
// G may be float or double (exactly one non-null); L <= 0 skips the step.
__global__ void project_step_kernel(float *d, const float *G, const double *Gd, const double *Lp,
                                    int M) {
  __shared__ float red[32];
  const int k = blockIdx.x;
  const double L = *Lp;
  float *dk = d + (int64_t)k * M;
  float v[4];
  float ss = 0.0f;
  for (int j = 0; j < 4; ++j) {
    int m = threadIdx.x + j * blockDim.x;
    float val = 0.0f;
    if (m < M) {
      val = dk[m];
      if (L > 0.0) {
        float g = G != nullptr ? G[(int64_t)k * M + m] : (float)Gd[(int64_t)k * M + m];
        val = val - g * (float)(1.0 / L);
      }
    }
    v[j] = val;
    ss = fmaf(val, val, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) t += red[i];
    red[0] = t;
  }
  __syncthreads();
  float nrm = sqrtf(red[0]);
  float scale = nrm > 1.0f ? 1.0f / nrm : 1.0f;
  for (int j = 0; j < 4; ++j) {
    int m = threadIdx.x + j * blockDim.x;
    if (m < M) dk[m] = v[j] * scale;
  }
}

// *flag = 1 if any of a[0, n) is NaN or +-Inf.  The aligned body is read as
// float4 (coalesced 16-byte loads), the unaligned head and the tail as floats;
// the bits are tested (exponent all ones) so that fast-math cannot drop it.
__device__ __forceinline__ bool nonfinite_bits(float v) {
  return (__float_as_uint(v) & 0x7F800000u) == 0x7F800000u;
}
__global__ void check_finite_kernel(const float *a, int64_t head, int64_t n4, int64_t n,
                                    int *flag) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  const float4 *a4 = reinterpret_cast<const float4 *>(a + head);
  for (int64_t i = tid; i < n4; i += stride) {
    const float4 v = a4[i];
    bad |= nonfinite_bits(v.x) | nonfinite_bits(v.y) | nonfinite_bits(v.z) | nonfinite_bits(v.w);
  }
  for (int64_t i = tid; i < head; i += stride) bad |= nonfinite_bits(a[i]);
  for (int64_t i = head + 4 * n4 + tid; i < n; i += stride) bad |= nonfinite_bits(a[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// bits_out = the complement of bits_in on the K filters of every pixel
// (unused high bits of each pixel's last word stay zero).
__global__ void complement_bits_kernel(const uint32_t *in, uint32_t *out, int64_t n_words, int KW,
                                       int K) {
  const uint32_t last = (K & 31) ? ((1u << (K & 31)) - 1u) : 0xFFFFFFFFu;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_words;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(i % KW);
    out[i] = ~in[i] & (w == KW - 1 ? last : 0xFFFFFFFFu);
  }
}

__global__ void negate_kernel(float *a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = -a[i];
}

// z <- zs on the sampled set, z unchanged elsewhere.
__global__ void merge_sampled_kernel(int64_t total, int K, int KW, const uint32_t *bits,
                                     const float *zs, float *z) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pix = g / K;
    const int k = (int)(g - pix * K);
    if (bit_of(bits, pix, KW, k)) z[g] = zs[g];
  }
}

template <typename F>
cudaError_t dispatch_s(int s, F &&f) {
  switch (s) {
    case 1: return f(std::integral_constant<int, 1>());
    case 3: return f(std::integral_constant<int, 3>());
    case 5: return f(std::integral_constant<int, 5>());
    case 7: return f(std::integral_constant<int, 7>());
    case 9: return f(std::integral_constant<int, 9>());
    case 11: return f(std::integral_constant<int, 11>());
    default: return cudaErrorInvalidValue;
  }
}

inline int grid_for(int64_t n, int bs, int cap = 1 << 20) {
  int64_t g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  return (int)(g > cap ? cap : g);
}

}  // namespace

// ------------------------------------------------------------------ launchers

cudaError_t launch_mask_bits(const BatchDev &b, int K, uint64_t seed, uint64_t t, uint64_t T,
                             uint32_t *bits, cudaStream_t st) {
  int KW = (K + 31) / 32;
  if (b.total_px == 0 || b.n_tiles == 0) return cudaSuccess;
  mask_bits_kernel<<<b.n_tiles, 256, 0, st>>>(b, K, KW, seed, t, T, bits);
  return cudaGetLastError();
}

cudaError_t launch_mask_residual(float *r, const uint8_t *obs, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  mask_residual_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(r, obs, n);
  return cudaGetLastError();
}

cudaError_t launch_apply_mask_dense(const BatchDev &b, int K, const uint32_t *bits, float *z,
                                    cudaStream_t st) {
  int64_t n = b.total_px * K;
  if (n == 0) return cudaSuccess;
  apply_mask_dense_kernel<<<grid_for(n, 256, 152 * 64), 256, 0, st>>>(n, K, (K + 31) / 32, bits, z);
  return cudaGetLastError();
}

cudaError_t launch_synth_fp32(const BatchDev &b, int K, int s, const float *d, const float *z,
                              const uint32_t *bits, const float *x, float *out, cudaStream_t st,
                              int ksplit, float *partial) {
  if (b.n_tiles == 0) return cudaSuccess;
  if (ksplit < 1 || partial == nullptr) ksplit = 1;
  const int kspan = ((K + ksplit - 1) / ksplit + 3) / 4 * 4;
  ksplit = (K + kspan - 1) / kspan;
  cudaError_t e = dispatch_s(s, [&](auto SC) {
    constexpr int S = decltype(SC)::value;
    dim3 grid(b.n_tiles, ksplit);
    synth_fp32_kernel<S, 4><<<grid, 128, 0, st>>>(b, K, kspan, d, z, bits, x,
                                                   ksplit > 1 ? partial : out);
    return cudaGetLastError();
  });
  if (e != cudaSuccess || ksplit == 1) return e;
  sum_split_kernel<<<grid_for(b.total_px, 256, 152 * 8), 256, 0, st>>>(partial, ksplit, b.total_px,
                                                                         x, out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_fp32(const BatchDev &b, int K, int s, const float *d, const float *r,
                                const uint32_t *bits, int mode, const StepParams *prm,
                                float *zg, cudaStream_t st, int ksplit) {
  if (b.n_tiles == 0) return cudaSuccess;
  ksplit = std::max(1, std::min(ksplit, (K + 31) / 32));
  return dispatch_s(s, [&](auto SC) {
    constexpr int S = decltype(SC)::value;
    dim3 grid(b.n_tiles, ksplit);
    adjoint_fp32_kernel<S><<<grid, 128, 0, st>>>(b, K, d, r, bits, mode, prm, zg);
    return cudaGetLastError();
  });
}

cudaError_t launch_filter_grad_fp32(const BatchDev &b, int K, int s, const float *r,
                                    const float *z, const uint32_t *bits, float *partial,
                                    int n_groups, cudaStream_t st) {
  return dispatch_s(s, [&](auto SC) {
    constexpr int S = decltype(SC)::value;
    constexpr int HR = 16, KCH = 32;
    size_t smem = (size_t)(HR * kTile * KCH + (HR + S - 1) * (kTile + S)) * sizeof(float);
    auto kern = filter_grad_fp32_kernel<S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n_groups, (K + KCH - 1) / KCH);
    kern<<<grid, 32 * S, smem, st>>>(b, K, r, z, bits, partial);
    return cudaGetLastError();
  });
}

cudaError_t launch_reduce_partials(const float *partial, int n_groups, int len, double *out,
                                   cudaStream_t st) {
  reduce_partials_kernel<<<(len + 255) / 256, 256, 0, st>>>(partial, n_groups, len, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_sq_abs(const float *a, int64_t n_sq, const float *bv, int64_t n_abs,
                              double *partials, int n_blocks, cudaStream_t st) {
  sum_sq_abs_kernel<<<n_blocks, 256, 0, st>>>(a, n_sq, bv, n_abs, partials);
  return cudaGetLastError();
}

cudaError_t launch_finish_sum(const double *partials, int n_blocks, double scale_sq,
                              double scale_abs, double *out, cudaStream_t st) {
  finish_sum_kernel<<<1, 256, 0, st>>>(partials, n_blocks, scale_sq, scale_abs, out);
  return cudaGetLastError();
}

cudaError_t launch_power_init(float *u, int64_t n, uint64_t seed, uint64_t tag, cudaStream_t st) {
  power_init_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(u, n, seed, tag);
  return cudaGetLastError();
}

cudaError_t launch_dot_partials(const float *a, const float *bv, int64_t n, double *partials,
                                int n_blocks, cudaStream_t st) {
  dot_partials_kernel<<<n_blocks, 256, 0, st>>>(a, bv, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_power_normalize(const float *w, float *u, int64_t n, const double *partials,
                                   int n_blocks, cudaStream_t st) {
  power_normalize_kernel<<<grid_for(n, 256, 2048), 256, 0, st>>>(w, u, n, partials, n_blocks);
  return cudaGetLastError();
}

cudaError_t launch_power_finish(const double *partials, int n_blocks, double safety,
                                double *L_out, double lambda, double fixed_step,
                                StepParams *prm, cudaStream_t st) {
  power_finish_kernel<<<1, 32, 0, st>>>(partials, n_blocks, safety, L_out, lambda, fixed_step, prm);
  return cudaGetLastError();
}

cudaError_t launch_project_step(float *d, const float *G, const double *Gd, const double *L, int K,
                                int M, cudaStream_t st) {
  project_step_kernel<<<K, 128, 0, st>>>(d, G, Gd, L, M);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *a, int64_t n, int *flag, cudaStream_t st) {
  if (n == 0 || a == nullptr) return cudaSuccess;
  int64_t head = (int64_t)(((16u - ((uintptr_t)a & 15u)) & 15u) / 4u);
  if ((uintptr_t)a & 3u) head = n;  // not even float-aligned: scalar loads only
  if (head > n) head = n;
  const int64_t n4 = (n - head) / 4;
  check_finite_kernel<<<grid_for(n4 > 0 ? n4 : n, 256, 152 * 16), 256, 0, st>>>(a, head, n4, n,
                                                                                   flag);
  return cudaGetLastError();
}

cudaError_t launch_complement_bits(const uint32_t *in, uint32_t *out, int64_t n_px, int K,
                                   cudaStream_t st) {
  const int KW = (K + 31) / 32;
  const int64_t n = n_px * KW;
  if (n == 0) return cudaSuccess;
  complement_bits_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n, KW, K);
  return cudaGetLastError();
}

cudaError_t launch_negate(float *a, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  negate_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(a, n);
  return cudaGetLastError();
}

cudaError_t launch_merge_sampled(const BatchDev &b, int K, const uint32_t *bits, const float *zs,
                                 float *z, cudaStream_t st) {
  const int64_t n = b.total_px * K;
  if (n == 0) return cudaSuccess;
  merge_sampled_kernel<<<grid_for(n, 256, 152 * 64), 256, 0, st>>>(n, K, (K + 31) / 32, bits, zs,
                                                                    z);
  return cudaGetLastError();
}

}  // namespace scsc
