// kernels_sparse.cu -- the code operators of the dictionary step (Eq. 5) on
// the nonzero codes only.  After a code step the codes are sparse (the l1
// term of Eq. 1; a fraction of a percent of the coordinates on the benchmark
// batch), so the synthesis D z and the filter gradient Z^T r, and with them
// every application of Z^T Z in the power iteration for L_d, cost
// O(nnz s^2) instead of the dense O(D K s^2) -- the sparsity the paper's
// complexity analysis counts on.
//
// Index, built once per dictionary step from the dense codes z [pixel][K]:
// - pixel-major: row_ptr[p] .. row_ptr[p + 1] are pixel p's nonzero codes,
//   filter index pk and value pv, in filter order;
// - filter-major: kt_off[k * ntiles + t] is the first entry of filter k's
//   nonzeros in 128-pixel tile t; the entries (global pixel kpix, image kimg,
//   value kv) are in (filter, pixel) order, and kt_off[K * ntiles] = nnz.
// Both orders come from per-tile counts and exclusive scans, so the index,
// and every sum below (fixed order, no atomics), is deterministic.
#include "scsc_internal.cuh"

namespace scsc {
namespace {

constexpr int kSpTile = 128;   // pixels per block of the index build
constexpr int kScanBlock = 1024;
constexpr int kSynTile = 32;   // output tile of the synthesis (32 x 32 pixels)
constexpr int kMaxHalo = kSynTile + 10;  // s <= 11

// Counts: nonzeros per pixel, and per (filter, 128-pixel tile).
__global__ void __launch_bounds__(kSpTile) sparse_count_kernel(int64_t total_px, int K,
                                                               const float *__restrict__ z,
                                                               int *cnt_px, int *cnt_kt,
                                                               int ntiles) {
  __shared__ float zs[kSpTile][33];
  __shared__ int wcnt[kSpTile / 32][32];
  const int tile = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t p0 = (int64_t)tile * kSpTile, p = p0 + t;
  int mine = 0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int kn = min(32, K - k0);
    __syncthreads();
    for (int i = t; i < kSpTile * 32; i += kSpTile) {
      const int pp = i >> 5, kk = i & 31;
      zs[pp][kk] = (kk < kn && p0 + pp < total_px) ? z[(p0 + pp) * K + k0 + kk] : 0.0f;
    }
    __syncthreads();
    for (int kk = 0; kk < kn; ++kk) {
      const bool nz = zs[t][kk] != 0.0f;
      mine += nz ? 1 : 0;
      const unsigned bal = __ballot_sync(0xffffffffu, nz);
      if (lane == 0) wcnt[w][kk] = __popc(bal);
    }
    __syncthreads();
    if (t < kn) {
      int c = 0;
#pragma unroll
      for (int q = 0; q < kSpTile / 32; ++q) c += wcnt[q][t];
      cnt_kt[(int64_t)(k0 + t) * ntiles + tile] = c;
    }
  }
  if (p < total_px) cnt_px[p] = mine;
}

// Entries at the positions the scans of the counts give.
__global__ void __launch_bounds__(kSpTile) sparse_fill_kernel(BatchDev b, int K,
                                                              const float *__restrict__ z,
                                                              const int64_t *__restrict__ row_ptr,
                                                              const int64_t *__restrict__ kt_off,
                                                              int ntiles, int *pk, float *pv,
                                                              int *kpix, int *kimg, float *kv) {
  __shared__ float zs[kSpTile][33];
  __shared__ int wcnt[kSpTile / 32][32];
  const int tile = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t p0 = (int64_t)tile * kSpTile, p = p0 + t;
  const bool live = p < b.total_px;
  int64_t pos = live ? row_ptr[p] : 0;
  const int img = live ? upper_index(b.off, b.n, p) : 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int kn = min(32, K - k0);
    __syncthreads();
    for (int i = t; i < kSpTile * 32; i += kSpTile) {
      const int pp = i >> 5, kk = i & 31;
      zs[pp][kk] = (kk < kn && p0 + pp < b.total_px) ? z[(p0 + pp) * K + k0 + kk] : 0.0f;
    }
    __syncthreads();
    for (int kk = 0; kk < kn; ++kk) {
      const unsigned bal = __ballot_sync(0xffffffffu, zs[t][kk] != 0.0f);
      if (lane == 0) wcnt[w][kk] = __popc(bal);
    }
    __syncthreads();
    for (int kk = 0; kk < kn; ++kk) {
      const float v = zs[t][kk];
      const unsigned bal = __ballot_sync(0xffffffffu, v != 0.0f);
      if (v != 0.0f) {
        int before = __popc(bal & lt);
        for (int q = 0; q < w; ++q) before += wcnt[q][kk];
        const int64_t e = kt_off[(int64_t)(k0 + kk) * ntiles + tile] + before;
        kpix[e] = (int)p;
        kimg[e] = img;
        kv[e] = v;
        pk[pos] = k0 + kk;
        pv[pos] = v;
        ++pos;
      }
    }
  }
}

// Exclusive scan of int counts into int64 offsets, out[n] = total: block
// sums, a one-block scan of the sums, then each block's own scan.
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *warp_tot, int64_t &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  if (lane == 31) warp_tot[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t x = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t o = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += o;
    }
    if (lane < nw) warp_tot[lane] = x;
  }
  __syncthreads();
  if (w > 0) v += warp_tot[w - 1];
  total = warp_tot[nw - 1];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const int *in, int64_t n,
                                                                 int64_t *bsum) {
  __shared__ int64_t wt[32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int64_t total;
  block_incl_scan(i < n ? in[i] : 0, wt, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block: bsum[0..nb) -> exclusive offsets, bsum[nb] = total.
__global__ void __launch_bounds__(kScanBlock) scan_bsum_kernel(int64_t *bsum, int nb) {
  __shared__ int64_t wt[32];
  int64_t carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int i = b0 + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    int64_t total;
    const int64_t incl = block_incl_scan(v, wt, total);
    if (i < nb) bsum[i] = carry + incl - v;
    carry += total;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanBlock) scan_apply_kernel(const int *in, int64_t n,
                                                                const int64_t *bsum, int nb,
                                                                int64_t *out) {
  __shared__ int64_t wt[32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int64_t v = i < n ? in[i] : 0;
  int64_t total;
  const int64_t incl = block_incl_scan(v, wt, total);
  if (i < n) out[i] = bsum[blockIdx.x] + incl - v;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

// out = sum_k d_k * z_k (minus x when given), gathered per output pixel from
// the nonzero codes of the s x s pixels that reach it; one 32 x 32 tile per
// block, the tile's halo offsets staged in shared memory.
__global__ void __launch_bounds__(256) sparse_synth_kernel(BatchDev b, int K, int s,
                                                           const float *__restrict__ d,
                                                           const int64_t *__restrict__ row_ptr,
                                                           const int *__restrict__ pk,
                                                           const float *__restrict__ pv,
                                                           const float *__restrict__ x,
                                                           float *__restrict__ out) {
  __shared__ int64_t hb[kMaxHalo * kMaxHalo];
  __shared__ int hc[kMaxHalo * kMaxHalo];
  const int c = (s - 1) / 2, M = s * s, hw = kSynTile + 2 * c;
  const int tile = blockIdx.x + b.tile_base;
  const int n = upper_index(b.tile0, b.n, tile);
  const int H = b.H[n], W = b.W[n];
  const int tiles_x = (W + kSynTile - 1) / kSynTile, lt = tile - b.tile0[n];
  const int y0 = (lt / tiles_x) * kSynTile, x0 = (lt % tiles_x) * kSynTile;
  const int64_t base = b.off[n];
  for (int i = threadIdx.x; i < hw * hw; i += blockDim.x) {
    const int yy = y0 - c + i / hw, xx = x0 - c + i % hw;
    int cnt = 0;
    int64_t beg = 0;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      const int64_t g = base + (int64_t)yy * W + xx;
      beg = row_ptr[g];
      cnt = (int)(row_ptr[g + 1] - beg);
    }
    hb[i] = beg;
    hc[i] = cnt;
  }
  __syncthreads();
  const int px = threadIdx.x & 31;
  for (int py = threadIdx.x >> 5; py < kSynTile; py += 8) {
    const int yy = y0 + py, xx = x0 + px;
    if (yy >= H || xx >= W) continue;
    float acc = 0.0f;
    for (int u = 0; u < s; ++u) {
      const int hrow = (py + 2 * c - u) * hw + px + 2 * c;
      for (int v = 0; v < s; ++v) {
        const int h = hrow - v;
        const int cnt = hc[h];
        if (cnt != 0) {
          const int64_t beg = hb[h];
          for (int e = 0; e < cnt; ++e) acc = fmaf(d[pk[beg + e] * M + u * s + v], pv[beg + e], acc);
        }
      }
    }
    const int64_t g = base + (int64_t)yy * W + xx;
    out[g] = x != nullptr ? acc - x[g] : acc;
  }
}

// partial[g][k][u][v] = sum over group g of filter k's nonzeros (q, z) of
// z * r(q_y - c + u, q_x - c + v): thread = tap, the group's entries in order.
__global__ void __launch_bounds__(128) sparse_grad_kernel(BatchDev b, int K, int s,
                                                          const float *__restrict__ r,
                                                          const int64_t *__restrict__ kt_off,
                                                          int ntiles, const int *__restrict__ kpix,
                                                          const int *__restrict__ kimg,
                                                          const float *__restrict__ kv,
                                                          float *__restrict__ partial) {
  const int k = blockIdx.x, g = blockIdx.y, G = gridDim.y;
  const int c = (s - 1) / 2, M = s * s, t = threadIdx.x;
  const int u = t / s, v = t - (t / s) * s;
  const int64_t kb = kt_off[(int64_t)k * ntiles], ke = kt_off[(int64_t)(k + 1) * ntiles];
  const int64_t len = ke - kb;
  const int64_t e0 = kb + len * g / G, e1 = kb + len * (g + 1) / G;
  float acc = 0.0f;
  if (t < M) {
#pragma unroll 4
    for (int64_t e = e0; e < e1; ++e) {
      const int n = kimg[e];
      const int W = b.W[n], H = b.H[n];
      const int64_t base = b.off[n];
      const int local = (int)(kpix[e] - base);
      const int qi = local / W, qj = local - (local / W) * W;
      const int i = qi - c + u, j = qj - c + v;
      if (i >= 0 && i < H && j >= 0 && j < W) acc = fmaf(kv[e], r[base + (int64_t)i * W + j], acc);
    }
    partial[(int64_t)g * K * M + (int64_t)k * M + t] = acc;
  }
}

}  // namespace

int sparse_tiles(int64_t total_px) { return (int)((total_px + kSpTile - 1) / kSpTile); }

size_t sparse_scan_scratch(int64_t n) { return (size_t)((n + kScanBlock - 1) / kScanBlock + 1); }

cudaError_t launch_sparse_count(const BatchDev &b, int K, const float *z, int *cnt_px,
                                int *cnt_kt, cudaStream_t st) {
  const int nt = sparse_tiles(b.total_px);
  if (nt == 0) return cudaSuccess;
  sparse_count_kernel<<<nt, kSpTile, 0, st>>>(b.total_px, K, z, cnt_px, cnt_kt, nt);
  return cudaGetLastError();
}

cudaError_t launch_scan_counts(const int *in, int64_t n, int64_t *out, int64_t *scratch,
                               cudaStream_t st) {
  const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  if (nb > 0) {
    scan_reduce_kernel<<<nb, kScanBlock, 0, st>>>(in, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  scan_bsum_kernel<<<1, kScanBlock, 0, st>>>(scratch, nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nb == 0) {
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    return e;
  }
  scan_apply_kernel<<<nb, kScanBlock, 0, st>>>(in, n, scratch, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_sparse_fill(const BatchDev &b, int K, const float *z, const int64_t *row_ptr,
                               const int64_t *kt_off, int *pk, float *pv, int *kpix, int *kimg,
                               float *kv, cudaStream_t st) {
  const int nt = sparse_tiles(b.total_px);
  if (nt == 0) return cudaSuccess;
  sparse_fill_kernel<<<nt, kSpTile, 0, st>>>(b, K, z, row_ptr, kt_off, nt, pk, pv, kpix, kimg, kv);
  return cudaGetLastError();
}

cudaError_t launch_sparse_synth(const BatchDev &b, int K, int s, const float *d,
                                const int64_t *row_ptr, const int *pk, const float *pv,
                                const float *x, float *out, cudaStream_t st) {
  if (s > 11 || s < 1) return cudaErrorInvalidValue;
  if (b.n_tiles == 0) return cudaSuccess;
  sparse_synth_kernel<<<b.n_tiles, 256, 0, st>>>(b, K, s, d, row_ptr, pk, pv, x, out);
  return cudaGetLastError();
}

cudaError_t launch_sparse_grad(const BatchDev &b, int K, int s, const float *r,
                               const int64_t *kt_off, const int *kpix, const int *kimg,
                               const float *kv, float *partial, int groups, cudaStream_t st) {
  if (s > 11 || s < 1 || K < 1) return cudaErrorInvalidValue;
  sparse_grad_kernel<<<dim3(K, groups), 128, 0, st>>>(b, K, s, r, kt_off,
                                                       sparse_tiles(b.total_px), kpix, kimg, kv,
                                                       partial);
  return cudaGetLastError();
}

}  // namespace scsc
