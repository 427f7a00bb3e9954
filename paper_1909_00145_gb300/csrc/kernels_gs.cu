// kernels_gs.cu -- one pass of projected block coordinate descent on Eq. 5
// (Sec. 3.2), the blocks being the filters, in order k = 0..K-1:
//   G_k(u,v) = sum_n sum_{i,j} r_n(i,j) z_{n,k}(i+c-u, j+c-v)   (gs_grad)
//   d_k <- P(d_k - G_k / L_d), delta = d_k^new - d_k^old         (gs_update)
//   r_n(i,j) += sum_{u,v} delta(u,v) z_{n,k}(i+c-u, j+c-v)       (gs_synth)
// over 32x32 tiles of the batch; block partials of G_k are summed in FP64
// in a fixed order (deterministic).
#include "scsc_internal.cuh"

namespace scsc {
namespace {

constexpr int kTile = 32;

struct TileCoordGs {
  int n, y0, x0, H, W;
  int64_t base;
};

__device__ __forceinline__ TileCoordGs tile_of(const BatchDev &b, int tile) {
  tile += b.tile_base;
  TileCoordGs c;
  c.n = upper_index(b.tile0, b.n, tile);
  c.H = b.H[c.n];
  c.W = b.W[c.n];
  const int tiles_x = (c.W + kTile - 1) / kTile;
  const int lt = tile - b.tile0[c.n];
  c.y0 = (lt / tiles_x) * kTile;
  c.x0 = (lt % tiles_x) * kTile;
  c.base = b.off[c.n];
  return c;
}

// partial[g][t] = sum over the tiles of group g of r(i,j) z_k(i+c-u, j+c-v),
// t = u s + v; thread t of the block owns tap t.
template <int S>
__global__ void __launch_bounds__(128) gs_grad_kernel(BatchDev b, int K, int k,
                                                      const float *__restrict__ r,
                                                      const float *__restrict__ z,
                                                      float *__restrict__ partial) {
  constexpr int C = (S - 1) / 2, HS = kTile + S - 1, M = S * S;
  __shared__ float zs[HS][HS + 1];
  __shared__ float rs[kTile][kTile + 1];
  const int t = threadIdx.x, u = t / S, v = t - u * S;
  float acc = 0.0f;
  for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
    const TileCoordGs tc = tile_of(b, tile);
    __syncthreads();
    for (int i = threadIdx.x; i < HS * HS; i += blockDim.x) {
      const int hy = i / HS, hx = i - hy * HS;
      const int yy = tc.y0 - C + hy, xx = tc.x0 - C + hx;
      const bool in = yy >= 0 && yy < tc.H && xx >= 0 && xx < tc.W;
      zs[hy][hx] = in ? z[(tc.base + (int64_t)yy * tc.W + xx) * K + k] : 0.0f;
    }
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
      const int ry = i / kTile, rx = i - ry * kTile;
      const int yy = tc.y0 + ry, xx = tc.x0 + rx;
      rs[ry][rx] = (yy < tc.H && xx < tc.W) ? r[tc.base + (int64_t)yy * tc.W + xx] : 0.0f;
    }
    __syncthreads();
    if (t < M) {
      // z index (i + c - u, j + c - v) - (y0 - c, x0 - c) = (ry + 2c - u, rx + 2c - v)
      for (int ry = 0; ry < kTile; ++ry)
#pragma unroll 8
        for (int rx = 0; rx < kTile; ++rx)
          acc = fmaf(rs[ry][rx], zs[ry + 2 * C - u][rx + 2 * C - v], acc);
    }
  }
  if (t < M) partial[(int64_t)blockIdx.x * M + t] = acc;
}

// d_k <- P(d_k - G_k / L) with G_k the FP64 sum of the groups' partials in
// group order; delta = new - old.  One block of 128 threads.
__global__ void __launch_bounds__(128) gs_update_kernel(float *d, const float *partial,
                                                        int n_groups, const double *Lp, int k,
                                                        int M, float *delta) {
  __shared__ float red[4];
  const double L = *Lp;
  float *dk = d + (int64_t)k * M;
  float v[2], old[2];
  float ss = 0.0f;
  for (int j = 0; j < 2; ++j) {
    const int m = threadIdx.x + j * 128;
    float val = 0.0f;
    if (m < M) {
      val = dk[m];
      if (L > 0.0) {
        double g = 0.0;
        for (int q = 0; q < n_groups; ++q) g += (double)partial[(int64_t)q * M + m];
        val = val - (float)g * (float)(1.0 / L);
      }
    }
    old[j] = m < M ? dk[m] : 0.0f;
    v[j] = val;
    ss = fmaf(val, val, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  const float nrm = sqrtf(red[0] + red[1] + red[2] + red[3]);
  const float scale = nrm > 1.0f ? 1.0f / nrm : 1.0f;
  for (int j = 0; j < 2; ++j) {
    const int m = threadIdx.x + j * 128;
    if (m < M) {
      const float nv = v[j] * scale;
      dk[m] = nv;
      delta[m] = nv - old[j];
    }
  }
}

// r(i,j) += sum_{u,v} delta(u,v) z_k(i+c-u, j+c-v): thread (tx, ty) owns
// column tx and rows 8 ty .. 8 ty + 7 of the tile.
template <int S>
__global__ void __launch_bounds__(128) gs_synth_kernel(BatchDev b, int K, int k,
                                                       const float *__restrict__ delta,
                                                       const float *__restrict__ z,
                                                       float *__restrict__ r) {
  constexpr int C = (S - 1) / 2, HS = kTile + S - 1, R = 8;
  __shared__ float zs[HS][HS + 1];
  __shared__ float ds[S * S];
  const TileCoordGs tc = tile_of(b, blockIdx.x);
  for (int i = threadIdx.x; i < HS * HS; i += blockDim.x) {
    const int hy = i / HS, hx = i - hy * HS;
    const int yy = tc.y0 - C + hy, xx = tc.x0 - C + hx;
    const bool in = yy >= 0 && yy < tc.H && xx >= 0 && xx < tc.W;
    zs[hy][hx] = in ? z[(tc.base + (int64_t)yy * tc.W + xx) * K + k] : 0.0f;
  }
  for (int i = threadIdx.x; i < S * S; i += blockDim.x) ds[i] = delta[i];
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = 0.0f;
  // z row (i + c - u) - (y0 - c) = ry + 2c - u
  for (int u = 0; u < S; ++u)
    for (int v = 0; v < S; ++v) {
      const float dv = ds[u * S + v];
#pragma unroll
      for (int q = 0; q < R; ++q) acc[q] = fmaf(dv, zs[ty * R + q + 2 * C - u][tx + 2 * C - v], acc[q]);
    }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = tc.y0 + ty * R + q, j = tc.x0 + tx;
    if (i < tc.H && j < tc.W) r[tc.base + (int64_t)i * tc.W + j] += acc[q];
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

}  // namespace

cudaError_t launch_gs_block(const BatchDev &b, int K, int s, int k, float *d, const float *z,
                            float *r, const double *L, float *partial, int n_groups, float *delta,
                            cudaStream_t st) {
  if (b.n_tiles == 0) return cudaSuccess;
  return dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    gs_grad_kernel<S><<<n_groups, 128, 0, st>>>(b, K, k, r, z, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gs_update_kernel<<<1, 128, 0, st>>>(d, partial, n_groups, L, k, S * S, delta);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gs_synth_kernel<S><<<b.n_tiles, 128, 0, st>>>(b, K, k, delta, z, r);
    return cudaGetLastError();
  });
}

}  // namespace scsc
