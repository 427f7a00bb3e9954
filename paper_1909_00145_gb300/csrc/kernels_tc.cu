// kernels_tc.cu -- tensor-core code update (Eq. 3 by proximal gradient) on
// sm_103a: BF16 operands in shared memory, FP32 accumulators in TMEM.
//
// Work unit ("row item"): one image row a of one 128-column strip js of
// image n, i.e. 128 code pixels = the M = 128 rows of one tcgen05 MMA.
// Items are ordered (n, js, a); a persistent CTA takes a contiguous range.
//
// Sampled codes (the pDK variables of Eq. 3) are stored packed in FP32,
// pixel-major per item: the sampled values of pixel p of item q, in filter
// order, start at seg_base[q] + pxoff[q * 128 + p].  Unsampled codes are not
// stored (Eq. 4).  Each item is padded to a multiple of 4 floats (16-byte
// aligned bulk copies).  seg_base and pxoff depend only on the mask M^t and
// are built once per outer iteration.
//
// Synthesis  P[p][(u,v)] = sum_k z_k(a, b0+p) d_k(u,v)  (MMA, N = 16 s taps)
//            xhat(a-c+u, b0+p-c+v) += P[p][(u,v)]       (col2im, registers)
// Adjoint    G[p][k] = sum_u sum_v r(a-c+u, b0+p-c+v) d_k(u,v)
//            one MMA per tap row u: the A operand is a Toeplitz view of the
//            residual row a-c+u (8 shifted copies, LBO = SBO = 128 bytes).
// Prox       z <- soft(z - alpha G, alpha lambda) on the packed values.
#include <algorithm>
#include <cstring>

#include "scsc_internal.cuh"
#include "scsc_tc.cuh"
#include "tc_items.cuh"
#include "tc_ptx.cuh"

namespace scsc {
namespace {

using namespace tcitems;
constexpr int kThreads = 128;
constexpr uint64_t kWaitNs = 1000000000ull;  // bounded waits: 1 s
constexpr int kPad = 10;                     // col2im padding (>= 2c)
constexpr int kPuRow = kStrip + 2 * kPad;    // 148

// ------------------------------------------------------------------ filter images
// B operand of the adjoint: per tap row u a [Kp filters x 16 taps] K-major
// tile; core (filter group g, tap half j) at u*Kp*32 + j*Kp*16 + g*128.
// B operand of the synthesis: [16 s taps x Kp filters] K-major; core (tap
// group T, filter chunk j) at j*(2 s*128) + T*128; tap n = 16 u + v.
__global__ void prep_filters_kernel(const float *d, int K, int S, int Kp, __nv_bfloat16 *badj,
                                    __nv_bfloat16 *bsyn) {
  const int M = S * S;
  const int n_adj = S * Kp * 16;
  const int n_syn = Kp * 16 * S;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_adj + n_syn;
       i += gridDim.x * blockDim.x) {
    if (i < n_adj) {
      int e = i & 7, r = (i >> 3) & 7, rest = i >> 6;  // rest = (u*2 + j)*(Kp/8) + g
      int g = rest % (Kp / 8), uj = rest / (Kp / 8);
      int j = uj & 1, u = uj >> 1;
      int k = 8 * g + r, v = 8 * j + e;
      float val = (k < K && v < S) ? d[(int64_t)k * M + u * S + v] : 0.0f;
      badj[i] = __float2bfloat16_rn(val);
    } else {
      int t = i - n_adj;
      int e = t & 7, r = (t >> 3) & 7, rest = t >> 6;  // rest = j*(2S) + T
      int T = rest % (2 * S), j = rest / (2 * S);
      int n = 8 * T + r, k = 8 * j + e;
      int u = n >> 4, v = n & 15;
      float val = (k < K && v < S) ? d[(int64_t)k * M + u * S + v] : 0.0f;
      bsyn[t] = __float2bfloat16_rn(val);
    }
  }
}

// ------------------------------------------------------------------ packed layout

// Per item: its sampled-value count (padded to a multiple of 4) and the
// exclusive offsets of its 128 pixels' values inside it.
__global__ void __launch_bounds__(kThreads) seg_count_kernel(ItemMap im, int KW,
                                                             const uint32_t *bits,
                                                             uint32_t *counts, uint16_t *pxoff,
                                                             int pad) {
  __shared__ int sh[4];
  const int q = blockIdx.x;
  const Item it = item_of(im, q);
  const int col = it.js * kStrip + threadIdx.x;
  int cnt = 0;
  if (col < it.W) {
    const uint32_t *w = bits + (it.base + (int64_t)it.a * it.W + col) * KW;
    for (int k = 0; k < KW; ++k) cnt += __popc(w[k]);
  }
  int total;
  const int off = scan128(cnt, sh, total);
  pxoff[(int64_t)q * kStrip + threadIdx.x] = (uint16_t)off;
  if (threadIdx.x == 0) counts[q] = (uint32_t)((total + pad - 1) / pad * pad);
}

// Exclusive scan u32 -> u64 in three passes over blocks of 1024 elements.
__global__ void scan_local_kernel(const uint32_t *in, uint64_t *out, int n, uint64_t *block_sums) {
  __shared__ uint64_t sh[32];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  uint64_t v = i < n ? in[i] : 0, x = v;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t s = sh[lane], t = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t - s;
    if (lane == 31) block_sums[blockIdx.x] = t;
  }
  __syncthreads();
  if (i < n) out[i] = sh[w] + x - v;
}

__global__ void scan_blocks_kernel(uint64_t *block_sums, int nb, uint64_t *total_out) {
  if (threadIdx.x != 0) return;
  uint64_t run = 0;
  for (int i = 0; i < nb; ++i) {
    uint64_t s = block_sums[i];
    block_sums[i] = run;
    run += s;
  }
  *total_out = run;
}

__global__ void scan_add_kernel(uint64_t *out, int n, const uint64_t *block_sums) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += block_sums[blockIdx.x];
}

// mode 0: packed <- z on the sampled set (warm start); *nonfinite |= 1 if
//         any code of the item is NaN or infinite
// mode 1: z <- packed on the sampled set, 0 elsewhere (Eq. 4)
// mode 2: z <- packed on the sampled set, unchanged elsewhere (the variant
//         that keeps the unsampled codes)
// One block per item.  The item's dense codes are one contiguous block of
// npx * K floats, walked linearly by the block (coalesced); each element
// finds its packed slot from per-pixel chunk offsets staged in shared memory.
constexpr int kMaxChunks = 32;  // K <= 512
__global__ void __launch_bounds__(kThreads) pack_kernel(ItemMap im, int K, int KW, int NC,
                                                        const uint32_t *bits,
                                                        const uint64_t *seg_base,
                                                        const uint16_t *pxoff, float *packed,
                                                        float *z, int mode, int *nonfinite) {
  __shared__ uint16_t s_m[kMaxChunks][kStrip];
  __shared__ uint32_t s_off[kMaxChunks][kStrip];
  const int q = blockIdx.x;
  const Item it = item_of(im, q);
  const int col = it.js * kStrip + threadIdx.x;
  const uint64_t item_base = seg_base[q];
  uint32_t run = pxoff[(int64_t)q * kStrip + threadIdx.x];
  for (int c = 0; c < NC; ++c) {
    const uint32_t m = chunk_mask(bits, KW, it, it.a, col, c);
    s_m[c][threadIdx.x] = (uint16_t)m;
    s_off[c][threadIdx.x] = run;
    run += __popc(m);
  }
  __syncthreads();
  const int npx = min(kStrip, it.W - it.js * kStrip);
  float *zb = z + (it.base + (int64_t)it.a * it.W + it.js * kStrip) * K;
  const int n = npx * K;
  // (pixel, filter) of element j, advanced by kThreads elements per step
  // without a division; kU elements per round, every load issued before any
  // store (the loop is bound by memory latency otherwise)
  constexpr int kU = 4;
  int pl = threadIdx.x / K, k = threadIdx.x - pl * K;
  const int dpl = kThreads / K, dk = kThreads - dpl * K;
  bool bad = false;
  for (int j0 = threadIdx.x; j0 < n; j0 += kU * kThreads) {
    float v[kU];
    uint64_t idx[kU];
    bool on[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u * kThreads;
      on[u] = false;
      idx[u] = 0;
      v[u] = 0.0f;
      if (j < n) {
        const int c = k >> 4, e = k & 15;
        const uint32_t m = s_m[c][pl];
        on[u] = (m >> e) & 1u;
        idx[u] = item_base + s_off[c][pl] + __popc(m & ((1u << e) - 1u));
        if (mode == 0) v[u] = zb[j];
        else if (on[u]) v[u] = packed[idx[u]];
        pl += dpl;
        k += dk;
        if (k >= K) {
          k -= K;
          ++pl;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u * kThreads;
      if (j >= n) break;
      if (mode == 0) {
        bad |= (__float_as_uint(v[u]) & 0x7F800000u) == 0x7F800000u;
        if (on[u]) packed[idx[u]] = v[u];
      } else if (mode == 1 || on[u]) {
        zb[j] = v[u];  // mode 1: 0 off the sampled set (Eq. 4)
      }
    }
  }
  if (mode == 0 && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

// Dense BF16 code tile of every row item in the synthesis A-operand layout
// (K-major cores of 8 pixels x 8 filters; chunk c of 16 filters at c * 4096
// bytes): the packed sampled codes, zero elsewhere.  One block per item,
// thread = pixel of the strip.
__global__ void __launch_bounds__(kThreads) abuf_kernel(ItemMap im, int Kp, int KW,
                                                        const uint32_t *bits,
                                                        const uint64_t *seg_base,
                                                        const uint16_t *pxoff, const float *packed,
                                                        uint8_t *abuf) {
  const int q = blockIdx.x, e = threadIdx.x;
  const Item it = item_of(im, q);
  const int NC = Kp / 16;
  const float *src = packed + seg_base[q] + pxoff[(int64_t)q * kStrip + e];
  uint8_t *tile = abuf + (size_t)q * kStrip * Kp * 2;
  for (int c = 0; c < NC; ++c) {
    const uint32_t m = chunk_mask(bits, KW, it, it.a, it.js * kStrip + e, c);
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      v[j] = ((m >> j) & 1u) ? *src : 0.0f;
      src += (m >> j) & 1u;
    }
    uint8_t *dst = tile + (size_t)(2 * c) * 2048 + (e >> 3) * 128 + (e & 7) * 16;
    *reinterpret_cast<uint4 *>(dst) = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                                 pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
    *reinterpret_cast<uint4 *>(dst + 2048) =
        make_uint4(pack_bf16x2(v[8], v[9]), pack_bf16x2(v[10], v[11]), pack_bf16x2(v[12], v[13]),
                   pack_bf16x2(v[14], v[15]));
  }
}

// BF16 packed codes of the fused path (a multiple of 8 values per item) and
// the A-tile element index of each value, e = (k / 8) * 1024 + (p / 8) * 64 +
// (p % 8) * 8 + k % 8 (0xFFFF for the padding).
// mode 0: vals <- BF16(z) on the sampled set and idx <- e (warm start), the
//         padding set to 0 / 0xFFFF; *nonfinite |= 1 if a code is NaN or Inf
// mode 1: z <- vals on the sampled set, 0 elsewhere (Eq. 4)
// mode 2: z <- vals on the sampled set, unchanged elsewhere
// One block per item, as pack_kernel.
__global__ void __launch_bounds__(kThreads) pack16_kernel(ItemMap im, int K, int KW, int NC,
                                                          const uint32_t *bits,
                                                          const uint64_t *seg_base,
                                                          const uint16_t *pxoff, uint16_t *vals,
                                                          uint16_t *idx, float *z, int mode,
                                                          int *nonfinite) {
  __shared__ uint16_t s_m[kMaxChunks][kStrip];
  __shared__ uint32_t s_off[kMaxChunks][kStrip];
  __shared__ uint32_t s_total;
  const int q = blockIdx.x;
  const Item it = item_of(im, q);
  const int col = it.js * kStrip + threadIdx.x;
  const uint64_t item_base = seg_base[q];
  uint32_t run = pxoff[(int64_t)q * kStrip + threadIdx.x];
  for (int c = 0; c < NC; ++c) {
    const uint32_t m = chunk_mask(bits, KW, it, it.a, col, c);
    s_m[c][threadIdx.x] = (uint16_t)m;
    s_off[c][threadIdx.x] = run;
    run += __popc(m);
  }
  if (threadIdx.x == kStrip - 1) s_total = run;
  __syncthreads();
  if (mode == 0) {
    // padding up to the next multiple of 8
    const uint64_t item_end = seg_base[q + 1];
    for (uint64_t j = item_base + s_total + threadIdx.x; j < item_end; j += kThreads) {
      vals[j] = 0;
      idx[j] = 0xFFFFu;
    }
  }
  const int npx = min(kStrip, it.W - it.js * kStrip);
  float *zb = z + (it.base + (int64_t)it.a * it.W + it.js * kStrip) * K;
  const int n = npx * K;
  constexpr int kU = 4;
  int pl = threadIdx.x / K, k = threadIdx.x - pl * K;
  const int dpl = kThreads / K, dk = kThreads - dpl * K;
  bool bad = false;
  for (int j0 = threadIdx.x; j0 < n; j0 += kU * kThreads) {
    float v[kU];
    uint64_t ix[kU];
    uint32_t e[kU];
    bool on[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u * kThreads;
      on[u] = false;
      ix[u] = 0;
      e[u] = 0;
      v[u] = 0.0f;
      if (j < n) {
        const int c = k >> 4, b = k & 15;
        const uint32_t m = s_m[c][pl];
        on[u] = (m >> b) & 1u;
        ix[u] = item_base + s_off[c][pl] + __popc(m & ((1u << b) - 1u));
        e[u] = (uint32_t)((k >> 3) * 1024 + (pl >> 3) * 64 + (pl & 7) * 8 + (k & 7));
        if (mode == 0) v[u] = zb[j];
        else if (on[u]) v[u] = __uint_as_float((uint32_t)vals[ix[u]] << 16);
        pl += dpl;
        k += dk;
        if (k >= K) {
          k -= K;
          ++pl;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u * kThreads;
      if (j >= n) break;
      if (mode == 0) {
        bad |= (__float_as_uint(v[u]) & 0x7F800000u) == 0x7F800000u;
        if (on[u]) {
          vals[ix[u]] = __bfloat16_as_ushort(__float2bfloat16_rn(v[u]));
          idx[ix[u]] = (uint16_t)e[u];
        }
      } else if (mode == 1 || on[u]) {
        zb[j] = v[u];
      }
    }
  }
  if (mode == 0 && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

// ------------------------------------------------------------------ row staging
// The single-stage kernels read, per code row, every pixel's mask words and
// the item's packed values.  Issued one by one these are dependent global
// loads (one round trip per 16-filter chunk); here they are asynchronous
// copies into shared memory, issued ahead of their use: the mask words of
// pixel i into s_mw[w * 128 + i], and the item's packed values (contiguous,
// 16-byte aligned, a multiple of 4 floats) into `stage` when they fit.
// Returns whether the values were staged (the same on every thread).
constexpr int kMaxKW = 16;  // mask words per pixel, K <= 512
__device__ __forceinline__ bool issue_row_copies(const Item &it, int a, int qa,
                                                 const uint32_t *__restrict__ bits, int KW,
                                                 const uint64_t *__restrict__ seg_base,
                                                 const float *packed, float *stage,
                                                 int stage_cap, uint32_t *s_mw) {
  const int i = threadIdx.x;
  const uint64_t sb = seg_base[qa];
  const int cnt = (int)(seg_base[qa + 1] - sb);
  const bool staged = cnt <= stage_cap;
  if (staged)
    for (int j = 4 * i; j < cnt; j += 4 * kThreads) tc::cp_async16(stage + j, packed + sb + j);
  const int col = it.js * kStrip + i;
  if (col < it.W) {
    const uint32_t *w = bits + (it.base + (int64_t)a * it.W + col) * KW;
    for (int k = 0; k < KW; ++k) tc::cp_async4(s_mw + k * kThreads + i, w + k, 4);
  } else {
    for (int k = 0; k < KW; ++k) s_mw[k * kThreads + i] = 0u;
  }
  tc::cp_async_commit();
  return staged;
}

// 16-bit sampled mask of chunk c of this thread's pixel, from the staged words.
__device__ __forceinline__ uint32_t staged_mask(const uint32_t *s_mw, int c) {
  return (s_mw[(c >> 1) * kThreads + threadIdx.x] >> ((c & 1) * 16)) & 0xFFFFu;
}

// ------------------------------------------------------------------ synthesis

template <int S>
struct SynthSmem {
  static constexpr int C = (S - 1) / 2;
  static constexpr int N = 16 * S;
  // A holds a_chunks filter chunks of 16 (4 KB each): all Kp / 16 where they
  // fit beside B, else the chunks are built and multiplied in groups
  // Then B, the col2im rows, the staged packed values of one code row
  // (stage_cap floats) and the staged mask words.
  __host__ __device__ static size_t a_bytes(int a_chunks) { return (size_t)a_chunks * 4096; }
  __host__ __device__ static size_t b_bytes(int Kp) { return (size_t)N * Kp * 2; }
  __host__ __device__ static size_t pu_bytes() { return (size_t)2 * S * kPuRow * 4; }
  __host__ __device__ static size_t total(int Kp, int a_chunks, int stage_cap) {
    return 1024 + a_bytes(a_chunks) + b_bytes(Kp) + pu_bytes() + (size_t)stage_cap * 4 +
           (size_t)kMaxKW * kThreads * 4;
  }
};

template <int S>
__global__ void __launch_bounds__(kThreads) synth_tc_kernel(ItemMap im, int K, int Kp, int KW,
                                                            const uint32_t *__restrict__ bits,
                                                            const uint64_t *__restrict__ seg_base,
                                                            const uint16_t *__restrict__ pxoff,
                                                            const float *__restrict__ packed,
                                                            const uint4 *__restrict__ bsyn,
                                                            float *__restrict__ xcore,
                                                            float *__restrict__ spill,
                                                            int a_chunks, int stage_cap,
                                                            int *err) {
  using L = SynthSmem<S>;
  constexpr int C = L::C, N = L::N;
  const int NC = Kp / 16;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *As = smem;
  uint8_t *Bs = As + L::a_bytes(a_chunks);
  float *Pu = reinterpret_cast<float *>(Bs + L::b_bytes(Kp));  // [2][S][kPuRow]
  float *stage = reinterpret_cast<float *>(Bs + L::b_bytes(Kp) + L::pu_bytes());
  uint32_t *s_mw = reinterpret_cast<uint32_t *>(stage + stage_cap);
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  {
    const int n16 = (int)(L::b_bytes(Kp) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(Bs);
    for (int i = tid; i < n16; i += kThreads) dst[i] = bsyn[i];
    for (int i = tid; i < 2 * S * kPuRow; i += kThreads) Pu[i] = 0.0f;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const uint32_t lane_addr = taddr + ((uint32_t)(32 * warp) << 16);
  const uint32_t idesc = tc::idesc_bf16_f32(128, N);
  const uint32_t a_base = tc::smem_u32(As), b_base = tc::smem_u32(Bs);
  const uint32_t b_lbo = 2 * S * 128;
  uint32_t phase = 0;
  bool failed = false;

  const int Q = im.total;
  int q = (int)((int64_t)Q * blockIdx.x / gridDim.x);
  const int q_end = (int)((int64_t)Q * (blockIdx.x + 1) / gridDim.x);
  const int i = tid;  // pixel lane
  while (q < q_end && !failed) {
    const Item it = item_of(im, q);
    const int seg_end = min(q_end, it.q_row0 + it.H);
    const int o0 = it.a, o1 = o0 + (seg_end - q);
    const int a_start = max(0, o0 - C), a_end = min(it.H, o1 + C);
    const int b0 = it.js * kStrip;
    float acc[S], acch[S];
#pragma unroll
    for (int u = 0; u < S; ++u) acc[u] = acch[u] = 0.0f;
    const bool halo = i < 2 * C;
    const int hcol = i < C ? i - C : kStrip + i - C;  // halo output column (strip-local)

    // row a's copies are issued while row a-1 is multiplied and folded
    bool staged = issue_row_copies(it, a_start, it.q_row0 + a_start, bits, KW, seg_base, packed,
                                   stage, stage_cap, s_mw);
    for (int a = a_start; a < a_end; ++a) {
      const int qa = it.q_row0 + a;
      const uint32_t po = pxoff[(int64_t)qa * kStrip + i];
      tc::cp_async_wait<0>();
      __syncthreads();
      const float *src = staged ? stage + po : packed + seg_base[qa] + po;
      for (int g0 = 0; g0 < NC; g0 += a_chunks) {
        const int g1 = min(NC, g0 + a_chunks);
        // 1. expand the packed codes of code row a (this thread: pixel i),
        // filter chunks g0 .. g1-1, into the A operand (BF16)
        for (int c = g0; c < g1; ++c) {
          const uint32_t m = staged_mask(s_mw, c);
          float v[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            v[e] = ((m >> e) & 1u) ? *src : 0.0f;
            src += (m >> e) & 1u;
          }
          uint4 lo = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
          uint4 hi = make_uint4(pack_bf16x2(v[8], v[9]), pack_bf16x2(v[10], v[11]),
                                pack_bf16x2(v[12], v[13]), pack_bf16x2(v[14], v[15]));
          uint8_t *dst = As + (size_t)(2 * (c - g0)) * 2048 + (i >> 3) * 128 + (i & 7) * 16;
          *reinterpret_cast<uint4 *>(dst) = lo;
          *reinterpret_cast<uint4 *>(dst + 2048) = hi;
        }
        tc::fence_proxy_async();
        __syncthreads();
        // 2. P += Z_row * D^T over these filter chunks; the wait also frees A
        // for the next group
        if (tid == 0) {
          tc::fence_after_sync();
          for (int kk = g0; kk < g1; ++kk) {
            uint64_t ad = tc::smem_desc(a_base + (kk - g0) * 2 * 2048, 2048, 128);
            uint64_t bd = tc::smem_desc(b_base + kk * 2 * b_lbo, b_lbo, 128);
            tc::mma_bf16(taddr, ad, bd, idesc, kk > 0 ? 1u : 0u);
          }
          tc::mma_commit(&mbar);
        }
        bool ok = tc::mbar_wait_bounded(&mbar, phase, kWaitNs);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
          if (tid == 0) atomicExch(err, 1);
          failed = true;
          break;
        }
        tc::fence_after_sync();
      }
      if (failed) break;
      // every thread is past its reads of the staged row: fetch the next one
      if (a + 1 < a_end)
        staged = issue_row_copies(it, a + 1, qa + 1, bits, KW, seg_base, packed, stage, stage_cap,
                                  s_mw);
      // 3. col2im: output row a-c+u gets sum_v P[b + c - v][(u, v)]
#pragma unroll
      for (int u = 0; u < S; ++u) {
        float p[16];
        tc::tmem_ld16(lane_addr + 16 * u, p);
        float *pu = Pu + (u & 1) * S * kPuRow;
#pragma unroll
        for (int v = 0; v < S; ++v) pu[v * kPuRow + i + kPad] = p[v];
        __syncthreads();
        float sum = 0.0f;
#pragma unroll
        for (int v = 0; v < S; ++v) sum += pu[v * kPuRow + i + C + kPad - v];
        acc[u] += sum;
        if (halo) {
          float hs = 0.0f;
#pragma unroll
          for (int v = 0; v < S; ++v) hs += pu[v * kPuRow + hcol + C + kPad - v];
          acch[u] += hs;
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      // 4. output row a - c is complete
      const int o = a - C;
      if (o >= o0 && o < o1) {
        if (b0 + i < it.W) xcore[it.base + (int64_t)o * it.W + b0 + i] = acc[0];
        if (halo) spill[(int64_t)(it.q_row0 + o) * (2 * C) + i] = acch[0];
      }
#pragma unroll
      for (int u = 0; u < S - 1; ++u) {
        acc[u] = acc[u + 1];
        acch[u] = acch[u + 1];
      }
      acc[S - 1] = acch[S - 1] = 0.0f;
    }
    if (failed) break;
    // rows whose remaining contributors lie below the image
#pragma unroll
    for (int j = 0; j < S - 1; ++j) {
      const int o = a_end - C + j;
      if (o >= o0 && o < o1 && o < it.H) {
        if (b0 + i < it.W) xcore[it.base + (int64_t)o * it.W + b0 + i] = acc[j];
        if (halo) spill[(int64_t)(it.q_row0 + o) * (2 * C) + i] = acch[j];
      }
    }
    q = seg_end;
  }
  if (failed) {
    // let any MMA still in flight finish before the TMEM is released
    tc::mbar_wait_bounded(&mbar, phase, kWaitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 256);
  }
}

// r = xcore + spills of the neighbouring strips - x
// Each block takes a contiguous range of row items (image n, strip js, row
// a); thread = column of the strip.  The first item is found by search, the
// next ones by stepping the row (and, at a strip's end, a search).
__global__ void __launch_bounds__(kThreads) finalize_r_kernel(ItemMap im, int C,
                                                              const float *__restrict__ xcore,
                                                              const float *__restrict__ spill,
                                                              const float *__restrict__ x,
                                                              const uint8_t *__restrict__ obs,
                                                              float *__restrict__ r) {
  const int q_begin = (int)((int64_t)im.total * blockIdx.x / gridDim.x);
  const int q_end = (int)((int64_t)im.total * (blockIdx.x + 1) / gridDim.x);
  if (q_begin >= q_end) return;
  Item it = item_of(im, q_begin);
  const int lc = threadIdx.x;
  for (int q = q_begin; q < q_end; ++q) {
    if (q > q_begin) {
      if (it.a + 1 < it.H) {
        ++it.a;
      } else {
        it = item_of(im, q);
      }
    }
    const int col = it.js * kStrip + lc;
    if (col >= it.W) continue;
    const int64_t p = it.base + (int64_t)it.a * it.W + col;
    float v = xcore[p];
    if (C > 0) {
      if (lc < C && it.js > 0) v += spill[(int64_t)(q - it.H) * (2 * C) + C + lc];
      if (lc >= kStrip - C && it.js + 1 < it.JS)
        v += spill[(int64_t)(q + it.H) * (2 * C) + lc - (kStrip - C)];
    }
    // inpainting: the data term counts observed pixels only
    r[p] = (obs != nullptr && obs[p] == 0) ? 0.0f : v - x[p];
  }
}

// ------------------------------------------------------------------ adjoint + prox

template <int S>
struct AdjSmem {
  static constexpr int C = (S - 1) / 2;
  static constexpr int kSRow = 17 * 128;  // one Toeplitz residual row (17 blocks)
  __host__ __device__ static size_t b_bytes(int Kp) { return (size_t)S * Kp * 32; }
  // B, the residual ring, its staging row, the staged packed values of one
  // code row (stage_cap floats), the staged mask words and the prox's
  // gradient scratch
  __host__ __device__ static size_t total(int Kp, int stage_cap) {
    return 1024 + b_bytes(Kp) + (size_t)S * kSRow + 144 * 4 + (size_t)stage_cap * 4 +
           (size_t)kMaxKW * kThreads * 4 + (size_t)16 * kThreads * 4;
  }
};

__host__ __device__ inline int tmem_cols_for(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

template <int S>
__global__ void __launch_bounds__(kThreads) adj_tc_kernel(ItemMap im, int K, int Kp, int KW,
                                                          const uint32_t *__restrict__ bits,
                                                          const uint64_t *__restrict__ seg_base,
                                                          const uint16_t *__restrict__ pxoff,
                                                          float *__restrict__ packed,
                                                          const uint4 *__restrict__ badj,
                                                          const float *__restrict__ r,
                                                          const StepParams *__restrict__ prm,
                                                          int stage_cap, int *err) {
  using L = AdjSmem<S>;
  constexpr int C = L::C;
  const int NC = Kp / 16;
  const int tcols = tmem_cols_for(Kp);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *Bs = smem;
  uint8_t *ring = Bs + L::b_bytes(Kp);
  float *rstage = reinterpret_cast<float *>(ring + (size_t)S * L::kSRow);
  float *stage = rstage + 144;
  uint32_t *s_mw = reinterpret_cast<uint32_t *>(stage + stage_cap);
  float *s_g = reinterpret_cast<float *>(s_mw + kMaxKW * kThreads);  // [16][kThreads]
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, tcols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  {
    const int n16 = (int)(L::b_bytes(Kp) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(Bs);
    for (int i = tid; i < n16; i += kThreads) dst[i] = badj[i];
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const uint32_t lane_addr = taddr + ((uint32_t)(32 * warp) << 16);
  // N <= 256 per MMA: above that the filters go in two column ranges of the
  // accumulator, [0, n1) and [n1, Kp)
  const int n1 = Kp <= 256 ? Kp : (Kp / 2 + 15) / 16 * 16;
  const uint32_t idesc = tc::idesc_bf16_f32(128, n1);
  const uint32_t idesc2 = tc::idesc_bf16_f32(128, Kp > n1 ? Kp - n1 : 16);
  const uint32_t ring_base = tc::smem_u32(ring), b_base = tc::smem_u32(Bs);
  const float alpha = prm->alpha, thr = prm->thresh;
  uint32_t phase = 0;
  bool failed = false;

  // Toeplitz row of residual row ar into its ring slot:
  // slot[g][i][e] = r(ar, b0 - c + 8 g + i + e), g < 17, i, e < 8.
  auto build_row = [&](const Item &it, int ar) {
    const int b0 = it.js * kStrip;
    for (int j = tid; j < 144; j += kThreads) {
      int col = b0 - C + j;
      float v = 0.0f;
      if (ar >= 0 && ar < it.H && col >= 0 && col < it.W)
        v = r[it.base + (int64_t)ar * it.W + col];
      rstage[j] = v;
    }
    __syncthreads();
    uint8_t *slot = ring + (size_t)(((ar % S) + S) % S) * L::kSRow;
    for (int t = tid; t < 17 * 8; t += kThreads) {
      int g = t >> 3, ii = t & 7;
      const float *src = rstage + 8 * g + ii;
      uint4 w = make_uint4(pack_bf16x2(src[0], src[1]), pack_bf16x2(src[2], src[3]),
                           pack_bf16x2(src[4], src[5]), pack_bf16x2(src[6], src[7]));
      *reinterpret_cast<uint4 *>(slot + g * 128 + ii * 16) = w;
    }
    __syncthreads();
  };

  const int Q = im.total;
  int q = (int)((int64_t)Q * blockIdx.x / gridDim.x);
  const int q_end = (int)((int64_t)Q * (blockIdx.x + 1) / gridDim.x);
  const int i = tid;
  while (q < q_end && !failed) {
    const Item it0 = item_of(im, q);
    const int seg_end = min(q_end, it0.q_row0 + it0.H);
    const int o0 = it0.a, o1 = o0 + (seg_end - q);
    for (int ar = o0 - C; ar < o0 + C; ++ar) build_row(it0, ar);
    for (int a = o0; a < o1; ++a) {
      const int qa = it0.q_row0 + a;
      build_row(it0, a + C);
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        for (int u = 0; u < S; ++u) {
          int ar = a - C + u;
          uint32_t slot = (uint32_t)(((ar % S) + S) % S) * L::kSRow;
          uint64_t ad = tc::smem_desc(ring_base + slot, 128, 128);
          uint64_t bd = tc::smem_desc(b_base + u * Kp * 32, Kp * 16, 128);
          tc::mma_bf16(taddr, ad, bd, idesc, u > 0 ? 1u : 0u);
          if (Kp > n1) {
            // filters n1 .. Kp-1 start n1 / 8 core groups (128 bytes each) in
            bd = tc::smem_desc(b_base + u * Kp * 32 + n1 * 16, Kp * 16, 128);
            tc::mma_bf16(taddr + (uint32_t)n1, ad, bd, idesc2, u > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&mbar);
      }
      // the row's packed values and mask words, copied while the MMAs run
      const bool staged = issue_row_copies(it0, a, qa, bits, KW, seg_base, packed, stage,
                                           stage_cap, s_mw);
      const uint32_t po = pxoff[(int64_t)qa * kStrip + i];
      tc::cp_async_wait<0>();
      bool ok = tc::mbar_wait_bounded(&mbar, phase, kWaitNs);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(err, 1);
        failed = true;
        break;
      }
      tc::fence_after_sync();
      // prox on the packed sampled codes of this item (this thread: pixel i),
      // in shared memory when staged
      // A chunk whose masks are sparse on every lane of the warp goes through
      // its set bits only, its gradients staged in s_g[e][thread]
      // (conflict-free); otherwise the unrolled form takes all 16 filters.
      float *dst = (staged ? stage : packed + seg_base[qa]) + po;
      float *const gs = s_g + tid;
      for (int c = 0; c < NC; ++c) {
        uint32_t m = staged_mask(s_mw, c);
        float g[16];
        tc::tmem_ld16(lane_addr + 16 * c, g);
        if (__any_sync(0xffffffffu, __popc(m) > 6)) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if ((m >> e) & 1u) {
              *dst = soft_threshold(*dst - alpha * g[e], thr);
              ++dst;
            }
          }
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) gs[e * kThreads] = g[e];
          while (m != 0u) {
            const int e = __ffs(m) - 1;
            m &= m - 1u;
            *dst = soft_threshold(*dst - alpha * gs[e * kThreads], thr);
            ++dst;
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      if (staged) {
        // the updated row back, coalesced
        const uint64_t sb = seg_base[qa];
        const int cnt = (int)(seg_base[qa + 1] - sb);
        for (int j = 4 * tid; j < cnt; j += 4 * kThreads)
          *reinterpret_cast<float4 *>(packed + sb + j) = *reinterpret_cast<const float4 *>(stage + j);
      }
    }
    q = seg_end;
  }
  if (failed) tc::mbar_wait_bounded(&mbar, phase, kWaitNs);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, tcols);
  }
}

// ------------------------------------------------------------------ self-test GEMM
// D[128 x N] = A[128 x 64] B[N x 64]^T; canonical K-major layouts with
// LBO = rows * 16 bytes (K-direction core stride) and SBO = 128 bytes.
__global__ void __launch_bounds__(kThreads) selftest_gemm_kernel(int N, const float *A,
                                                                 const float *B, float *D,
                                                                 int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *As = smem;                  // 128 x 64 bf16 = 16 KB
  uint8_t *Bs = smem + 128 * 64 * 2;   // N x 64 bf16
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  // element (row, k) -> (k/8)*(rows*16) + (row/8)*128 + (row%8)*16 + (k%8)*2
  for (int t = tid; t < 128 * 64; t += kThreads) {
    int row = t / 64, k = t % 64;
    size_t o = (size_t)(k / 8) * (128 * 16) + (row / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
    *reinterpret_cast<__nv_bfloat16 *>(As + o) = __float2bfloat16_rn(A[t]);
  }
  for (int t = tid; t < N * 64; t += kThreads) {
    int row = t / 64, k = t % 64;
    size_t o = (size_t)(k / 8) * (N * 16) + (row / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
    *reinterpret_cast<__nv_bfloat16 *>(Bs + o) = __float2bfloat16_rn(B[t]);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(128, N);
    for (int kk = 0; kk < 4; ++kk) {
      uint64_t ad = tc::smem_desc(tc::smem_u32(As) + kk * 2 * 128 * 16, 128 * 16, 128);
      uint64_t bd = tc::smem_desc(tc::smem_u32(Bs) + kk * 2 * N * 16, N * 16, 128);
      tc::mma_bf16(taddr, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&mbar);
  }
  bool ok = tc::mbar_wait_bounded(&mbar, 0, kWaitNs);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(err, 1);
    tc::mbar_wait_bounded(&mbar, 0, kWaitNs);
  } else {
    tc::fence_after_sync();
    const uint32_t lane_addr = taddr + ((uint32_t)(32 * warp) << 16);
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tc::tmem_ld16(lane_addr + c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) D[(size_t)tid * N + c + e] = v[e];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 256);
  }
}

// D[128 x N] = A[128 x 64] B[N x 64]^T with B stored MN-major: core matrix
// (n block nb, k block kb) at nb * 1024 + kb * 128 bytes, its row r holding
// B[8 nb .. 8 nb + 7][8 kb + r] (8 N values, 16 bytes).  `swap` selects which
// descriptor field carries the K-direction core stride (128 bytes): 0 = the
// leading-dimension offset, 1 = the stride-dimension offset.  Either way
// every address the MMA forms lies inside the 32 KB B buffer.
__global__ void __launch_bounds__(kThreads) selftest_gemm_mn_kernel(int N, const float *A,
                                                                    const float *B, float *D,
                                                                    int swap, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *As = smem;               // 128 x 64 bf16 = 16 KB, K-major
  uint8_t *Bs = smem + 128 * 64 * 2;  // 32 KB, MN-major
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  for (int t = tid; t < 128 * 64; t += kThreads) {
    int row = t / 64, k = t % 64;
    size_t o = (size_t)(k / 8) * (128 * 16) + (row / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
    *reinterpret_cast<__nv_bfloat16 *>(As + o) = __float2bfloat16_rn(A[t]);
  }
  for (int t = tid; t < 32 * 1024 / 2; t += kThreads)
    reinterpret_cast<__nv_bfloat16 *>(Bs)[t] = __float2bfloat16_rn(0.0f);
  __syncthreads();
  for (int t = tid; t < N * 64; t += kThreads) {
    int n = t / 64, k = t % 64;
    size_t o = (size_t)(n / 8) * 1024 + (k / 8) * 128 + (k % 8) * 16 + (n % 8) * 2;
    *reinterpret_cast<__nv_bfloat16 *>(Bs + o) = __float2bfloat16_rn(B[t]);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32_bmn(128, N);
    const uint32_t lbo = swap ? 1024 : 128, sbo = swap ? 128 : 1024;
    for (int kk = 0; kk < 4; ++kk) {
      uint64_t ad = tc::smem_desc(tc::smem_u32(As) + kk * 2 * 128 * 16, 128 * 16, 128);
      uint64_t bd = tc::smem_desc(tc::smem_u32(Bs) + kk * 2 * 128, lbo, sbo);
      tc::mma_bf16(taddr, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&mbar);
  }
  bool ok = tc::mbar_wait_bounded(&mbar, 0, kWaitNs);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(err, 1);
    tc::mbar_wait_bounded(&mbar, 0, kWaitNs);
  } else {
    tc::fence_after_sync();
    const uint32_t lane_addr = taddr + ((uint32_t)(32 * warp) << 16);
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tc::tmem_ld16(lane_addr + c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) D[(size_t)tid * N + c + e] = v[e];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 256);
  }
}

// ------------------------------------------------------------------ host helpers

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

cudaError_t ensure(TcWorkspace::Buf &b, size_t need) {
  if (need <= b.bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = need + need / 8 + 256;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e == cudaSuccess) b.bytes = want;
  return e;
}

template <typename T>
T *as(const TcWorkspace::Buf &b) {
  return reinterpret_cast<T *>(b.p);
}

#define TRY(expr)                            \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

}  // namespace

cudaError_t launch_syn2(const tcitems::ItemMap &im, int K, int s, const uint8_t *abuf,
                        const uint4 *bsyn, float *xcore, float *spill, int *err, int grid,
                        int max_smem, cudaStream_t st);
cudaError_t launch_adj2(const tcitems::ItemMap &im, int K, int s, const uint32_t *bits,
                        const uint64_t *seg_base, const uint16_t *pxoff, float *packed,
                        uint8_t *abuf, const uint4 *badj, const float *xcore, const float *spill,
                        const float *x, const uint8_t *obs, const StepParams *prm, int *err,
                        int grid, cudaStream_t st);
size_t tc_abuf_bytes(int K, int Q);
cudaError_t prepare_pipe(int K, int s, int max_smem);
int fused_chunk_buffers(int K, int s, int max_smem);
cudaError_t prepare_fused(int K, int s, int ncb);
cudaError_t launch_fused(const tcitems::ItemMap &im, int K, int s, int mode, int ncb,
                         const uint64_t *seg_base, const uint16_t *vin, uint16_t *vout,
                         const uint16_t *idx, const uint4 *bimg, const float *xin,
                         const float *sin, float *xout, float *sout, const float *x,
                         const uint8_t *obs, const StepParams *prm, int *err, int grid,
                         cudaStream_t st);

namespace {
// Launch `n` iterations (iteration(it), it = 0..n-1) as one CUDA graph: the
// graph captured for key gk is replayed if one of the slots holds it, else it
// is captured into the least recently used slot.
template <typename F>
cudaError_t replay_graph(TcWorkspace &ws, const GraphKey &gk, int n, F &&iteration,
                         cudaStream_t st) {
  GraphSlot *slot = nullptr;
  for (GraphSlot &g : ws.graphs_cached)
    if (g.exec && std::memcmp(&gk, &g.key, sizeof gk) == 0) slot = &g;
  if (!slot) {
    slot = &ws.graphs_cached[0];
    for (GraphSlot &g : ws.graphs_cached)
      if (!g.exec || g.used < slot->used) slot = &g;
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    slot->exec = nullptr;
    cudaGraph_t g = nullptr;
    TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int it = 0; it < n && err == cudaSuccess; ++it) err = iteration(it);
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&slot->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    TRY(err);
    slot->key = gk;
  }
  slot->used = ++ws.graph_clock;
  return cudaGraphLaunch(slot->exec, st);
}

// The fused path of tc_code_step (seg_base and pxoff already built with a
// multiple of 8 values per item): BF16 packed warm start and A-tile indices,
// the synthesis of the warm start, n_iters fused iterations alternating
// between two sets of buffers (replayed from a CUDA graph), unpack.
cudaError_t fused_code_step(TcWorkspace &ws, const ItemMap &im, int Q, const BatchDev &b, int K,
                            int s, const float *x, float *z, const uint32_t *bits,
                            const uint64_t *seg_base, const uint16_t *pxoff, const uint8_t *obs,
                            const StepParams *prm, int n_iters, bool keep_unsampled,
                            int *nonfinite, int ncb, cudaStream_t st) {
  const int Kp = (K + 15) / 16 * 16, NC = Kp / 16, KW = (K + 31) / 32, C = (s - 1) / 2;
  if (n_iters == 0) {
    // no step: only Eq. 4 (or nothing, for the keep variant) on the warm
    // start, which must not go through the BF16 packed storage
    if (!keep_unsampled) TRY(launch_apply_mask_dense(b, K, bits, z, st));
    return launch_check_finite(z, b.total_px * K, nonfinite, st);
  }
  // values: at most K per pixel plus 7 padding per item
  const size_t nval = (size_t)b.total_px * K + 8 * (size_t)Q + 16;
  TRY(ensure(ws.v16[0], nval * 2));
  TRY(ensure(ws.v16[1], nval * 2));
  TRY(ensure(ws.idx16, nval * 2));
  TRY(ensure(ws.xcore2, (size_t)b.total_px * 4));
  TRY(ensure(ws.spill2, (size_t)Q * (2 * C > 0 ? 2 * C : 1) * 4));
  uint16_t *v[2] = {as<uint16_t>(ws.v16[0]), as<uint16_t>(ws.v16[1])};
  float *xc[2] = {as<float>(ws.xcore), as<float>(ws.xcore2)};
  float *sp[2] = {as<float>(ws.spill), as<float>(ws.spill2)};
  uint16_t *idx = as<uint16_t>(ws.idx16);
  int pr = ws.prof ? ws.prof->begin(KID_PACK, st) : -1;
  pack16_kernel<<<Q, kThreads, 0, st>>>(im, K, KW, NC, bits, seg_base, pxoff, v[0], idx, z, 0,
                                        nonfinite);
  TRY(cudaGetLastError());
  if (ws.prof) ws.prof->end(pr, st);
  TRY(prepare_fused(K, s, ncb));
  const int grid = std::min(Q, ws.sm_count);
  const uint4 *bimg = as<uint4>(ws.badj);
  int *err = as<int>(ws.err);
  // the synthesis of the warm start: the first iteration's input
  int p0 = ws.prof ? ws.prof->begin(KID_FUSED, st) : -1;
  TRY(launch_fused(im, K, s, 0, ncb, seg_base, v[0], nullptr, idx, bimg, nullptr, nullptr, xc[0],
                   sp[0], x, obs, prm, err, grid, st));
  if (ws.prof) ws.prof->end(p0, st);
  auto iteration = [&](int it) -> cudaError_t {
    const int i = it & 1, o = i ^ 1;
    int p1 = ws.prof ? ws.prof->begin(KID_FUSED, st) : -1;
    TRY(launch_fused(im, K, s, 1, ncb, seg_base, v[i], v[o], idx, bimg, xc[i], sp[i], xc[o],
                     sp[o], x, obs, prm, err, grid, st));
    if (ws.prof) ws.prof->end(p1, st);
    return cudaSuccess;
  };
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TRY(cudaStreamIsCapturing(st, &cap));
  const bool use_graph = ws.graphs && n_iters > 0 && st != nullptr &&
                         cap == cudaStreamCaptureStatusNone && !(ws.prof && ws.prof->on);
  if (use_graph) {
    GraphKey gk{};  // zero-filled, so that memcmp sees no padding bytes
    gk.seg_base = seg_base;
    gk.v16a = ws.v16[0].p;
    gk.v16b = ws.v16[1].p;
    gk.idx16 = idx;
    gk.badj = ws.badj.p;
    gk.xcore = ws.xcore.p;
    gk.spill = ws.spill.p;
    gk.xcore2 = ws.xcore2.p;
    gk.spill2 = ws.spill2.p;
    gk.err = ws.err.p;
    gk.x = x;
    gk.prm = prm;
    gk.item0 = ws.item0.p;
    gk.off = b.off;
    gk.obs = obs;
    gk.total_px = b.total_px;
    gk.n_images = b.n;
    gk.K = K;
    gk.s = s;
    gk.Q = Q;
    gk.variant = 2 + 8 * ncb;
    gk.iters = n_iters;
    TRY(replay_graph(ws, gk, n_iters, iteration, st));
  } else {
    for (int it = 0; it < n_iters; ++it) TRY(iteration(it));
  }
  // Eq. 4 (or the keep variant): dense codes from the last iterate
  int pu = ws.prof ? ws.prof->begin(KID_UNPACK, st) : -1;
  pack16_kernel<<<Q, kThreads, 0, st>>>(im, K, KW, NC, bits, seg_base, pxoff, v[n_iters & 1],
                                        idx, z, keep_unsampled ? 2 : 1, nonfinite);
  TRY(cudaGetLastError());
  if (ws.prof) ws.prof->end(pu, st);
  return cudaSuccess;
}
}  // namespace

int *tc_error_word(TcWorkspace &ws) {
  if (ensure(ws.err, sizeof(int)) != cudaSuccess) return nullptr;
  return as<int>(ws.err);
}

const char *tc_last_error(const TcWorkspace &ws) { return ws.last_error.c_str(); }

void tc_release(TcWorkspace &ws) {
  for (GraphSlot &g : ws.graphs_cached) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  for (TcWorkspace::Buf *b : {&ws.item0, &ws.seg_count, &ws.seg_base, &ws.pxoff, &ws.scan_blocks,
                              &ws.packed, &ws.xcore, &ws.spill, &ws.r, &ws.badj, &ws.bsyn,
                              &ws.err, &ws.abuf, &ws.v16[0], &ws.v16[1], &ws.idx16, &ws.xcore2,
                              &ws.spill2}) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->bytes = 0;
  }
}

cudaError_t tc_code_step(TcWorkspace &ws, const BatchDev &b, const int *H_host, const int *W_host,
                         int K, int s, const float *x, const float *d, float *z,
                         const uint32_t *bits, const uint8_t *obs, const StepParams *prm,
                         int n_iters, bool keep_unsampled, int *nonfinite, cudaStream_t st) {
  if (K > kMaxChunks * 16) {
    ws.last_error = "the tensor path supports K <= 512";
    return cudaErrorNotSupported;
  }
  const int Kp = (K + 15) / 16 * 16, NC = Kp / 16, KW = (K + 31) / 32, C = (s - 1) / 2;
  if (ws.sm_count == 0) {
    int dev;
    TRY(cudaGetDevice(&dev));
    TRY(cudaDeviceGetAttribute(&ws.sm_count, cudaDevAttrMultiProcessorCount, dev));
  }
  // row-item map (host, cached per batch shape)
  const int n = b.n;
  std::vector<int> Hh(H_host, H_host + n), Wh(W_host, W_host + n);
  if (Hh != ws.host_H || Wh != ws.host_W) {
    std::vector<int> item0(n + 1);
    int64_t q = 0;
    for (int i = 0; i < n; ++i) {
      item0[i] = (int)q;
      q += (int64_t)Hh[i] * ((Wh[i] + kStrip - 1) / kStrip);
    }
    if (q > 0x7fffffff) {
      ws.last_error = "batch has too many row items";
      return cudaErrorNotSupported;
    }
    item0[n] = (int)q;
    TRY(ensure(ws.item0, (size_t)(n + 1) * 4));
    TRY(cudaMemcpyAsync(ws.item0.p, item0.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, st));
    TRY(cudaStreamSynchronize(st));  // the host vector is released after this call
    ws.host_item0.swap(item0);
    ws.host_H.swap(Hh);
    ws.host_W.swap(Wh);
    ws.n_items = (int)q;
  }
  const int Q = ws.n_items;
  ItemMap im{n, as<int>(ws.item0), b.H, b.W, b.off, Q};
  const int64_t nseg = Q;
  const int nblk = (int)((nseg + 1023) / 1024);
  TRY(ensure(ws.seg_count, (size_t)nseg * 4));
  TRY(ensure(ws.seg_base, (size_t)(nseg + 1) * 8));
  TRY(ensure(ws.pxoff, (size_t)nseg * kStrip * 2));
  TRY(ensure(ws.scan_blocks, (size_t)(nblk + 1) * 8));
  TRY(ensure(ws.packed, ((size_t)b.total_px * K + 4 * (size_t)Q + 16) * 4));
  TRY(ensure(ws.xcore, (size_t)b.total_px * 4));
  TRY(ensure(ws.r, (size_t)b.total_px * 4));
  TRY(ensure(ws.spill, (size_t)Q * (2 * C > 0 ? 2 * C : 1) * 4));
  TRY(ensure(ws.badj, (size_t)s * Kp * 32));
  TRY(ensure(ws.bsyn, (size_t)Kp * 16 * s * 2));
  TRY(ensure(ws.err, sizeof(int)));

  if (ws.max_smem == 0) {
    int dev;
    TRY(cudaGetDevice(&dev));
    TRY(cudaDeviceGetAttribute(&ws.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  }
  // the fused kernel (BF16 packed codes) where it fits, else the two-kernel
  // paths (FP32 packed codes).  It also needs at least two row items per SM:
  // each CTA recomputes the 2c rows around its range, so with fewer items the
  // recomputation outweighs the saved launch (100 items of 100^2 at K = 16:
  // 1.84 Gpix*filter/s fused, 2.07 on two kernels)
  const bool fused_fits_p = ws.sample_p * kStrip * K <= 4096.0;
  const bool fused_fits_q = Q >= 2 * ws.sm_count;
  const int fused_ncb =
      ws.fused && fused_fits_p && fused_fits_q ? fused_chunk_buffers(K, s, ws.max_smem) : 0;
  const bool use_fused = fused_ncb > 0;
  // filter operand images, sampled-code layout, warm start
  prep_filters_kernel<<<64, 256, 0, st>>>(d, K, s, Kp, as<__nv_bfloat16>(ws.badj),
                                          as<__nv_bfloat16>(ws.bsyn));
  TRY(cudaGetLastError());
  if (Q == 0) return cudaSuccess;
  uint16_t *pxoff = as<uint16_t>(ws.pxoff);
  seg_count_kernel<<<Q, kThreads, 0, st>>>(im, KW, bits, as<uint32_t>(ws.seg_count), pxoff,
                                           use_fused ? 8 : 4);
  TRY(cudaGetLastError());
  uint64_t *seg_base = as<uint64_t>(ws.seg_base);
  scan_local_kernel<<<nblk, 1024, 0, st>>>(as<uint32_t>(ws.seg_count), seg_base, (int)nseg,
                                           as<uint64_t>(ws.scan_blocks));
  TRY(cudaGetLastError());
  scan_blocks_kernel<<<1, 32, 0, st>>>(as<uint64_t>(ws.scan_blocks), nblk, seg_base + nseg);
  TRY(cudaGetLastError());
  scan_add_kernel<<<nblk, 1024, 0, st>>>(seg_base, (int)nseg, as<uint64_t>(ws.scan_blocks));
  TRY(cudaGetLastError());
  if (use_fused)
    return fused_code_step(ws, im, Q, b, K, s, x, z, bits, seg_base, pxoff, obs, prm, n_iters,
                           keep_unsampled, nonfinite, fused_ncb, st);
  int pr = ws.prof ? ws.prof->begin(KID_PACK, st) : -1;
  pack_kernel<<<Q, kThreads, 0, st>>>(im, K, KW, NC, bits, seg_base, pxoff, as<float>(ws.packed),
                                      z, 0, nonfinite);
  TRY(cudaGetLastError());
  if (ws.prof) ws.prof->end(pr, st);

  const bool pipe_ok = tc_pipe_supported(K, s, ws.max_smem);
  const int fin_grid = std::min(Q, ws.sm_count * 16);  // finalize: blocks over row items
  // launch geometry of the single-stage kernels (several CTAs per SM)
  int grid_s1 = 1, grid_a1 = 1, a_chunks = NC, stage_s = 0, stage_a = 0;
  size_t smem_s1 = 0, smem_a1 = 0;
  if (ws.smem_sm == 0) {
    int dev;
    TRY(cudaGetDevice(&dev));
    TRY(cudaDeviceGetAttribute(&ws.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  }
  TRY(dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    using SL = SynthSmem<S>;
    using AL = AdjSmem<S>;
    // 1 KB of each CTA's share is left for static shared memory and 1 KB is
    // reserved by the system
    const size_t smem_cap = (size_t)ws.max_smem - 1024;
    auto per_cta = [&](int occ) {
      return std::min(smem_cap, (size_t)ws.smem_sm / (size_t)occ - 2048);
    };
    // staged values of one code row: the expected count with a margin (rows
    // above it are read in place)
    const int want = (int)std::min(16384.0, ws.sample_p * K * kStrip * 1.25 + 512.0) & ~3;
    // synthesis: as many CTAs per SM as its 256 TMEM columns allow where the
    // filters and all chunks fit; the staging takes what is left, down to 8
    // chunks in shared memory (the rest are built and multiplied in groups)
    const size_t s_all = SL::total(Kp, NC, 0);
    const int occ_s_t = std::max(1, std::min(2, (int)(ws.smem_sm / (s_all + 2048))));
    const size_t cap_s = per_cta(occ_s_t);
    const size_t s_keep = SL::total(Kp, std::min(NC, 8), 0);
    stage_s = cap_s > s_keep ? (int)std::min<size_t>(want, (cap_s - s_keep) / 4) & ~3 : 0;
    const size_t s_fixed = SL::total(Kp, 0, stage_s);
    a_chunks = s_fixed < cap_s ? std::min(NC, (int)((cap_s - s_fixed) / 4096)) : 0;
    smem_s1 = SL::total(Kp, a_chunks, stage_s);
    // adjoint: the CTAs per SM its TMEM columns and unstaged layout allow
    const size_t a_min = AL::total(Kp, 0);
    const int occ_a_t = std::max(
        1, std::min(512 / tmem_cols_for(Kp), (int)(ws.smem_sm / (a_min + 2048))));
    const size_t cap_a = per_cta(occ_a_t);
    stage_a = cap_a > a_min ? (int)std::min<size_t>(want, (cap_a - a_min) / 4) & ~3 : 0;
    smem_a1 = AL::total(Kp, stage_a);
    if (a_chunks < 1 || smem_a1 > smem_cap) {
      ws.last_error = "the filters do not fit in shared memory";
      return cudaErrorNotSupported;
    }
    TRY(cudaFuncSetAttribute(synth_tc_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_s1));
    TRY(cudaFuncSetAttribute(adj_tc_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_a1));
    int occ_s = 0, occ_a = 0;
    TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, synth_tc_kernel<S>, kThreads,
                                                      smem_s1));
    TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, adj_tc_kernel<S>, kThreads,
                                                      smem_a1));
    occ_s = std::max(1, std::min(occ_s, 512 / 256));
    occ_a = std::max(1, std::min(occ_a, 512 / tmem_cols_for(Kp)));
    grid_s1 = std::min(Q, ws.sm_count * occ_s);
    grid_a1 = std::min(Q, ws.sm_count * occ_a);
    return cudaSuccess;
  }));
  if (pipe_ok) TRY(prepare_pipe(K, s, ws.max_smem));
  const int grid2 = std::min(Q, ws.sm_count);
  // the pipelined synthesis reads every code row as a dense BF16 A tile,
  // which the pipelined adjoint rewrites after each prox; built here from the
  // packed warm start (and again whenever the single-stage adjoint, which
  // does not write it, has run)
  auto build_abuf = [&]() -> cudaError_t {
    abuf_kernel<<<Q, kThreads, 0, st>>>(im, Kp, KW, bits, seg_base, pxoff, as<float>(ws.packed),
                                        as<uint8_t>(ws.abuf));
    return cudaGetLastError();
  };
  if (pipe_ok) {
    TRY(ensure(ws.abuf, tc_abuf_bytes(K, Q)));
    TRY(build_abuf());
  }

  // One proximal-gradient iteration with kernel variant v (0 single-stage,
  // 1 pipelined): synthesis, residual, adjoint + prox.
  auto iteration = [&](int v) -> cudaError_t {
    int p1 = ws.prof ? ws.prof->begin(KID_SYNTH_TC, st) : -1;
    if (v == 1) {
      TRY(launch_syn2(im, K, s, as<uint8_t>(ws.abuf), as<uint4>(ws.bsyn), as<float>(ws.xcore),
                      as<float>(ws.spill), as<int>(ws.err), grid2, ws.max_smem, st));
    } else {
      TRY(dispatch_s(s, [&](auto SC) -> cudaError_t {
        constexpr int S = decltype(SC)::value;
        synth_tc_kernel<S><<<grid_s1, kThreads, smem_s1, st>>>(
            im, K, Kp, KW, bits, seg_base, pxoff, as<float>(ws.packed), as<uint4>(ws.bsyn),
            as<float>(ws.xcore), as<float>(ws.spill), a_chunks, stage_s, as<int>(ws.err));
        return cudaGetLastError();
      }));
    }
    if (ws.prof) ws.prof->end(p1, st);
    // the pipelined adjoint forms the residual rows itself from xcore, the
    // spill columns and x; with an observation mask (inpainting), and for
    // the single-stage adjoint, r is formed here
    if (v != 1 || obs != nullptr) {
      int p2 = ws.prof ? ws.prof->begin(KID_FINALIZE, st) : -1;
      finalize_r_kernel<<<fin_grid, kThreads, 0, st>>>(im, C, as<float>(ws.xcore),
                                                        as<float>(ws.spill), x, obs, as<float>(ws.r));
      TRY(cudaGetLastError());
      if (ws.prof) ws.prof->end(p2, st);
    }
    int p3 = ws.prof ? ws.prof->begin(KID_ADJ_TC, st) : -1;
    if (v == 1) {
      if (obs == nullptr)
        TRY(launch_adj2(im, K, s, bits, seg_base, pxoff, as<float>(ws.packed),
                        as<uint8_t>(ws.abuf), as<uint4>(ws.badj), as<float>(ws.xcore),
                        as<float>(ws.spill), x, nullptr, prm, as<int>(ws.err), grid2, st));
      else
        TRY(launch_adj2(im, K, s, bits, seg_base, pxoff, as<float>(ws.packed),
                        as<uint8_t>(ws.abuf), as<uint4>(ws.badj), as<float>(ws.r), nullptr,
                        nullptr, nullptr, prm, as<int>(ws.err), grid2, st));
    } else {
      TRY(dispatch_s(s, [&](auto SC) -> cudaError_t {
        constexpr int S = decltype(SC)::value;
        adj_tc_kernel<S><<<grid_a1, kThreads, smem_a1, st>>>(
            im, K, Kp, KW, bits, seg_base, pxoff, as<float>(ws.packed), as<uint4>(ws.badj),
            as<float>(ws.r), prm, stage_a, as<int>(ws.err));
        return cudaGetLastError();
      }));
    }
    if (ws.prof) ws.prof->end(p3, st);
    return cudaSuccess;
  };

  // Autotuner: the first call for a (device, K, s, shape class) runs its
  // first two iterations once with each variant, times them with events and
  // keeps the faster one for every later call with the same key.
  int variant = pipe_ok ? 1 : 0;
  int done = 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TRY(cudaStreamIsCapturing(st, &cap));
  const bool user_capture = cap != cudaStreamCaptureStatusNone;
  if (pipe_ok && ws.autotune) {
    int dev = 0;
    TRY(cudaGetDevice(&dev));
    int qclass = 0;
    while ((1 << (qclass + 1)) <= Q) ++qclass;
    const TuneKey key{dev, K, s, qclass};
    auto hit = ws.tune.find(key);
    if (hit != ws.tune.end()) {
      variant = hit->second;
    } else if (n_iters >= 2 && !user_capture) {
      cudaEvent_t ev[4];
      for (auto &e : ev) TRY(cudaEventCreate(&e));
      float ms[2] = {0.f, 0.f};
      cudaError_t err = cudaSuccess;
      for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
        // the single-stage adjoint (v = 0) leaves the A tiles behind
        if (v == 1) err = build_abuf();
        if (err == cudaSuccess) err = cudaEventRecord(ev[2 * v], st);
        if (err == cudaSuccess) err = iteration(v);
        if (err == cudaSuccess) err = cudaEventRecord(ev[2 * v + 1], st);
      }
      if (err == cudaSuccess) err = cudaEventSynchronize(ev[3]);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[1], ev[2], ev[3]);
      for (auto &e : ev) cudaEventDestroy(e);
      TRY(err);
      variant = ms[1] <= ms[0] ? 1 : 0;
      ws.tune[key] = variant;
      ws.tune_ms[key] = std::make_pair(ms[0], ms[1]);
      done = 2;
    }
  }

  // Remaining iterations: replayed from a CUDA graph captured once per
  // (buffers, shape, variant, count), or launched directly when profiling,
  // when the caller is itself capturing, or on the legacy default stream.
  const int rem = n_iters - done;
  const bool use_graph = ws.graphs && rem > 0 && st != nullptr && !user_capture &&
                         !(ws.prof && ws.prof->on);
  if (use_graph) {
    GraphKey gk{};  // zero-filled, so that memcmp sees no padding bytes
    gk.bits = bits;
    gk.seg_base = seg_base;
    gk.pxoff = pxoff;
    gk.packed = ws.packed.p;
    gk.bsyn = ws.bsyn.p;
    gk.badj = ws.badj.p;
    gk.xcore = ws.xcore.p;
    gk.spill = ws.spill.p;
    gk.r = ws.r.p;
    gk.err = ws.err.p;
    gk.x = x;
    gk.prm = prm;
    gk.item0 = ws.item0.p;
    gk.off = b.off;
    gk.obs = obs;
    gk.abuf = ws.abuf.p;
    gk.total_px = b.total_px;
    gk.n_images = b.n;
    gk.K = K;
    gk.s = s;
    gk.Q = Q;
    gk.variant = variant;
    gk.iters = rem;
    gk.a_chunks = a_chunks;
    gk.stage_s = stage_s;
    gk.stage_a = stage_a;
    TRY(replay_graph(ws, gk, rem, [&](int) { return iteration(variant); }, st));
  } else {
    for (int it = 0; it < rem; ++it) TRY(iteration(variant));
  }
  // Eq. 4: dense codes, zero off the sampled set
  int pu = ws.prof ? ws.prof->begin(KID_UNPACK, st) : -1;
  pack_kernel<<<Q, kThreads, 0, st>>>(im, K, KW, NC, bits, seg_base, pxoff, as<float>(ws.packed),
                                      z, keep_unsampled ? 2 : 1, nonfinite);
  TRY(cudaGetLastError());
  if (ws.prof) ws.prof->end(pu, st);
  return cudaSuccess;
}

namespace {
// A bounded wait on an mbarrier that nothing arrives on: the wait gives up
// after limit_ns, as every wait of the tensor kernels does, and raises the
// error word (one thread, one block).
__global__ void selftest_wait_kernel(uint64_t limit_ns, int *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    if (!tc::mbar_wait_bounded(&bar, 0, limit_ns)) atomicExch(err, 1);
  }
}
// The issue and completion rate of back-to-back tcgen05 MMAs of M = 128,
// K = 16 and the given N from one thread, on zero operands (the rate does not
// depend on the values).  layout 0: A K-major (8 x 16-byte core matrices, 256
// bytes apart along M), B K-major; 1: A the overlapping Toeplitz view of the
// adjoint (core matrices 128 bytes apart in both directions), B K-major;
// 2: A K-major, B MN-major (the synthesis's filter operand).  Every operand
// lies inside the 24 KB zeroed here: A spans at most 4 KB, B at most 8 KB at
// N = 256.  out[0]: cycles to issue the timed MMAs, out[1]: cycles until
// their completion barrier.
__global__ void __launch_bounds__(kThreads) selftest_mma_rate_kernel(int N, int layout, int reps,
                                                                     long long *out, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::fence_mbar_init();
  }
  for (int t = tid; t < 24 * 1024 / 16; t += kThreads)
    reinterpret_cast<uint4 *>(smem)[t] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  bool ok = true;
  if (tid == 0) {
    const uint32_t a0 = tc::smem_u32(smem), b0 = a0 + 16 * 1024;
    const uint64_t ad = layout == 1 ? tc::smem_desc(a0, 128, 128) : tc::smem_desc(a0, 128, 256);
    const uint64_t bd = layout == 2 ? tc::smem_desc(b0, 128, 256) : tc::smem_desc(b0, N * 16, 128);
    const uint32_t idesc = layout == 2 ? tc::idesc_bf16_f32_bmn(128, N) : tc::idesc_bf16_f32(128, N);
    // one untimed round, then the timed one
    for (int round = 0; round < 2 && ok; ++round) {
      const long long t0 = clock64();
      for (int r = 0; r < reps; ++r) tc::mma_bf16(taddr, ad, bd, idesc, r > 0 ? 1u : 0u);
      const long long t1 = clock64();
      tc::mma_commit(&mbar);
      ok = tc::mbar_wait_bounded(&mbar, (uint32_t)round, kWaitNs);
      const long long t2 = clock64();
      out[0] = t1 - t0;
      out[1] = t2 - t0;
      if (!ok) {
        // the MMAs in flight finish (bounded) before the TMEM is released
        atomicExch(err, 1);
        tc::mbar_wait_bounded(&mbar, (uint32_t)round, kWaitNs);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 256);
  }
}

}  // namespace

cudaError_t tc_selftest_mma_rate(int N, int layout, int reps, long long *out, int *err,
                                 cudaStream_t st) {
  if (N < 16 || N > 256 || N % 16 != 0 || layout < 0 || layout > 2 || reps < 1 || reps > 4096)
    return cudaErrorInvalidValue;
  selftest_mma_rate_kernel<<<1, kThreads, 1024 + 24 * 1024, st>>>(N, layout, reps, out, err);
  return cudaGetLastError();
}

cudaError_t tc_selftest_wait(uint64_t limit_ns, int *err, cudaStream_t st) {
  selftest_wait_kernel<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}

cudaError_t tc_selftest_gemm_mn(int N, const float *A, const float *B, float *D, int swap,
                                int *err, cudaStream_t st) {
  if (N < 16 || N > 256 || N % 16 != 0) return cudaErrorInvalidValue;
  size_t smem = 1024 + 128 * 64 * 2 + 32 * 1024;
  TRY(cudaFuncSetAttribute(selftest_gemm_mn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem));
  selftest_gemm_mn_kernel<<<1, kThreads, smem, st>>>(N, A, B, D, swap, err);
  return cudaGetLastError();
}

cudaError_t tc_selftest_gemm(int N, const float *A, const float *B, float *D, int *err,
                             cudaStream_t st) {
  if (N < 16 || N > 256 || N % 16 != 0) return cudaErrorInvalidValue;
  size_t smem = 1024 + 128 * 64 * 2 + (size_t)N * 64 * 2;
  TRY(cudaFuncSetAttribute(selftest_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem));
  selftest_gemm_kernel<<<1, kThreads, smem, st>>>(N, A, B, D, err);
  return cudaGetLastError();
}

}  // namespace scsc
