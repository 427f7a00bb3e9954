// tc_items.cuh -- row items and the packed sampled-code layout shared by the
// tensor-core kernels.
//
// Row item q: image row a of the 128-column strip js of image n; items are
// ordered (n, js, a), item0[n] is the first item of image n.  The sampled
// codes of item q are stored pixel-major from seg_base[q]: the values of
// pixel p, in filter order, start at seg_base[q] + pxoff[q * 128 + p].  Every
// item's storage is padded to a multiple of 4 floats (8 for the BF16 codes
// of the fused kernel) so that it starts 16-byte aligned.
#pragma once
#include "scsc_internal.cuh"

namespace scsc {
namespace tcitems {

constexpr int kStrip = 128;

struct ItemMap {
  int n;
  const int *item0;  // [n + 1]
  const int *H;
  const int *W;
  const int64_t *off;
  int total;
};

struct Item {
  int n, js, a, H, W, JS;
  int64_t base;
  int q_row0;  // item index of row 0 of this strip
};

__device__ __forceinline__ Item item_of(const ItemMap &m, int q) {
  Item it;
  it.n = upper_index(m.item0, m.n, q);
  it.H = m.H[it.n];
  it.W = m.W[it.n];
  it.JS = (it.W + kStrip - 1) / kStrip;
  int local = q - m.item0[it.n];
  it.js = local / it.H;
  it.a = local - it.js * it.H;
  it.base = m.off[it.n];
  it.q_row0 = q - it.a;
  return it;
}

// 16-bit sampled mask of chunk c (filters 16c..16c+15) of pixel (a, col).
__device__ __forceinline__ uint32_t chunk_mask(const uint32_t *bits, int KW, const Item &it, int a,
                                               int col, int c) {
  if (col >= it.W || a < 0 || a >= it.H) return 0u;
  int64_t pix = it.base + (int64_t)a * it.W + col;
  return (bits[pix * KW + (c >> 1)] >> ((c & 1) * 16)) & 0xFFFFu;
}

// Exclusive scan of one int per thread over a 128-thread block.
__device__ __forceinline__ int scan128(int v, int *sh, int &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  int pre = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) pre += (i < w) ? sh[i] : 0;
  total = sh[0] + sh[1] + sh[2] + sh[3];
  __syncthreads();
  return pre + x - v;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&h);
}

}  // namespace tcitems
}  // namespace scsc
