// kernels_fused.cu -- one proximal-gradient iteration of the code update
// (Eq. 3) in a single persistent launch: residual, adjoint at the sampled
// coordinates, soft-threshold prox, and the synthesis of the updated codes,
// with the codes kept packed in BF16 between launches (one CTA per SM).
//
// Work unit: row item q = image row a of a 128-column strip (see
// tc_items.cuh).  A CTA owns a contiguous range of items; per strip segment
// [o0, o1) it also recomputes the c items on each side that belong to its
// neighbours ([e0, e1) = [o0 - c, o1 + c) clipped to the image), so that the
// synthesis of every owned output row o in [o0, o1) sees all its code rows
// [o - c, o + c] and is complete: no exchange between CTAs.  The input codes
// and the input synthesis are read from one set of buffers and the outputs
// written to another (they alternate between launches), so that a CTA never
// reads a value a neighbour rewrites in the same launch.
//
// Packed codes: per item, its sampled values (BF16) in pixel-major order, a
// multiple of 8 per item (16-byte aligned); beside each value, in a second
// array, its element index in the item's A tile (the synthesis A operand:
// 128 pixels x Kp filters, K-major core matrices of 8 pixels x 8 filters,
// e = (k / 8) * 1024 + (p / 8) * 64 + (p % 8) * 8 + k % 8); padding values
// carry the index 0xFFFF.  The index array depends only on the mask M^t and
// is built once per outer iteration.
//
// Warp roles (17 warps):
//   0       MMA issue (lane 0): per item, 11 adjoint MMAs (one per tap row,
//           A = Toeplitz view of a residual row, B = filter image) into one
//           of two TMEM accumulators; then the synthesis MMAs of the previous
//           item (A = its BF16 code tile, B = the same filter image read
//           MN-major) into a TMEM ring of 16 output-row blocks.
//   1-3     residual rows: r = xhat_in + neighbours' spill - x (0 off the
//           image or at unobserved pixels), as 8 shifted BF16 copies per row.
//   4-11    epilogue: drain the adjoint accumulator to shared memory (FP32),
//           zero the item's A tile, then over the staged packed values:
//           z <- soft(z - alpha g, alpha lambda) in FP32, the BF16 result to
//           the staging buffer and to the A tile at its index.
//   12-15   fold: an output row's ring block is complete once its last code
//           row has been multiplied; x_hat(o, j) = sum_v Q_o[j + c - v][v] by
//           warp shuffles (warp-edge halo through shared memory), written for
//           the owned rows; the block is zeroed for reuse.
//   16      copies (lane 0): packed values and indices of each item in
//           chunks of up to 4096 into a ring of staging buffers by bulk copy, and
//           the updated values of owned items back to the output array.
// Every wait is bounded; on timeout the CTA raises an abort flag, every role
// leaves its loop, the copies and MMAs in flight are waited for (bounded) and
// the tensor memory is released.
#include "scsc_tc.cuh"
#include "tc_items.cuh"
#include "tc_ptx.cuh"

namespace scsc {
namespace {

using namespace tcitems;

constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return p + ((1024u - (tc::smem_u32(p) & 1023u)) & 1023u);
}

template <int S>
struct Fus {
  static constexpr int C = (S - 1) / 2;
  static constexpr int RS = 16;          // residual ring slots (slot = row & 15)
  static_assert(S + 3 <= RS, "ring too small");
  static constexpr int kSRow = 17 * 128;  // one Toeplitz residual row
  static constexpr int kProd = 3;
  static constexpr int kEpiW = 8;
  static constexpr int kFoldW = 4;
  static constexpr int kRB = 16;          // synthesis ring blocks of 16 TMEM columns
  static_assert(S <= kRB, "synthesis ring too small");
  static constexpr int kCH = 4096;        // packed values per staging chunk (one item at p = 1/4, K <= 112)
  static constexpr int W_PROD0 = 1, W_EPI0 = 4, W_FOLD0 = 12, W_COPY = 16;
  static constexpr int kThreads = 32 * 17;
  __host__ __device__ static size_t b_bytes(int Kp) { return (size_t)S * Kp * 32; }
  __host__ __device__ static size_t ring_bytes() { return (size_t)RS * kSRow; }
  __host__ __device__ static size_t g_bytes(int Kp) { return (size_t)kStrip * Kp * 4; }
  __host__ __device__ static size_t a_bytes(int Kp) { return (size_t)kStrip * Kp * 2; }
  __host__ __device__ static size_t chunk_bytes() { return (size_t)kCH * 4; }  // values + indices
  __host__ __device__ static size_t prod_bytes() { return (size_t)kProd * 4 * 144 * 4; }
  __host__ __device__ static size_t xb_bytes() { return (size_t)2 * 4 * 2 * (C > 0 ? C : 1) * 4; }
  __host__ __device__ static size_t total(int Kp, int ncb) {
    return 1024 + b_bytes(Kp) + ring_bytes() + g_bytes(Kp) + 2 * a_bytes(Kp) +
           (size_t)ncb * chunk_bytes() + prod_bytes() + xb_bytes();
  }
};

struct FusedArgs {
  ItemMap im;
  int K, Kp, mode;            // mode 0: synthesis of the input codes only; 1: one iteration
  int ncb;                    // staging chunk buffers
  const uint64_t *seg_base;   // [Q + 1] element offset of each item's packed values
  const uint16_t *vin;        // packed BF16 codes of the input iterate
  uint16_t *vout;             // packed BF16 codes of the output iterate (owned items)
  const uint16_t *idx;        // per packed value: its A-tile element index (0xFFFF = padding)
  const uint4 *bimg;          // filter image (per tap row u: [Kp filters x 16 taps], K-major)
  const float *xin, *sin;     // synthesis of the input codes: core columns, strip spills
  float *xout, *sout;         // synthesis of the output codes
  const float *x;             // image
  const uint8_t *obs;         // observation mask (nullptr: every pixel observed)
  const StepParams *prm;
  int *err;
};

// Strip segments of a CTA's item range with their extended ranges.
struct ExtSeg {
  int q, q_end;
  Item it;
  int o0, o1, e0, e1;  // owned rows, extended rows
  int C;
  __device__ bool next(const ItemMap &im) {
    if (q >= q_end) return false;
    it = item_of(im, q);
    const int seg_end = min(q_end, it.q_row0 + it.H);
    o0 = it.a;
    o1 = o0 + (seg_end - q);
    e0 = max(0, o0 - C);
    e1 = min(it.H, o1 + C);
    q = seg_end;
    return true;
  }
};

// Residual rows in the order the MMA consumes them: per segment, rows
// e0 - c .. e1 - 1 + c; j counts them across segments.
struct ExtRowGen {
  ExtSeg sg;
  int j_seg, j, t, nrows;
  bool live;
  __device__ void init(int q0, int q1, int c) {
    sg.q = q0;
    sg.q_end = q1;
    sg.C = c;
    j_seg = j = t = nrows = 0;
    live = false;
  }
  __device__ bool next(const ItemMap &im) {
    while (!live || t >= nrows) {
      if (live) j_seg += nrows;
      if (!sg.next(im)) return false;
      live = true;
      t = 0;
      nrows = sg.e1 - sg.e0 + 2 * sg.C;
    }
    j = j_seg + t;
    ++t;
    return true;
  }
  __device__ int ar() const { return sg.e0 - sg.C + (t - 1); }
};

// Staging chunks of the packed values in CTA order: item by item (extended
// ranges), kCH values per chunk.
template <int CH>
struct ChunkIter {
  ExtSeg sg;
  bool live;
  int a;           // current row of the segment
  uint64_t beg, end, pos;  // current item's packed range and chunk start
  bool owned;
  __device__ void init(int q0, int q1, int c) {
    sg.q = q0;
    sg.q_end = q1;
    sg.C = c;
    live = false;
    a = 0;
    beg = end = pos = 0;
    owned = false;
  }
  // Advance to the next non-empty chunk; false when none is left.
  __device__ bool next(const ItemMap &im, const uint64_t *seg_base) {
    if (live && pos + CH < end) {
      pos += CH;
      return true;
    }
    while (true) {
      if (live) ++a;
      while (!live || a >= sg.e1) {
        if (!sg.next(im)) return false;
        live = true;
        a = sg.e0;
      }
      const int q = sg.it.q_row0 + a;
      beg = seg_base[q];
      end = seg_base[q + 1];
      owned = a >= sg.o0 && a < sg.o1;
      if (end > beg) {
        pos = beg;
        return true;
      }
    }
  }
  __device__ uint32_t count() const { return (uint32_t)(end - pos < (uint64_t)CH ? end - pos : (uint64_t)CH); }
};

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__device__ __forceinline__ void st_shared_u16(uint32_t saddr, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(saddr), "h"((unsigned short)v) : "memory");
}

// 16 TMEM columns of this warp's lanes set to zero.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int S>
__global__ void __launch_bounds__(Fus<S>::kThreads, 1) fused_kernel(const FusedArgs A) {
  using L = Fus<S>;
  constexpr int C = L::C, RS = L::RS, kRB = L::kRB, kCH = L::kCH;
  const ItemMap &im = A.im;
  const int Kp = A.Kp, NC = Kp / 16, ncb = A.ncb;
  const bool iterate = A.mode == 1;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *const Bs = smem;
  uint8_t *const ring = Bs + L::b_bytes(Kp);
  float *const Gs = reinterpret_cast<float *>(ring + L::ring_bytes());
  uint8_t *const As = reinterpret_cast<uint8_t *>(Gs) + L::g_bytes(Kp);  // 2 A tiles
  uint8_t *const stage = As + 2 * L::a_bytes(Kp);                        // ncb chunks
  float *const rst = reinterpret_cast<float *>(stage + (size_t)ncb * L::chunk_bytes());
  float *const xb = rst + L::prod_bytes() / 4;
  auto chunk_vals = [&](int b) { return reinterpret_cast<uint16_t *>(stage + (size_t)b * L::chunk_bytes()); };
  auto chunk_idx = [&](int b) { return chunk_vals(b) + kCH; };
  const uint32_t a_bytes = (uint32_t)L::a_bytes(Kp);

  __shared__ uint64_t ring_full[RS], ring_empty[RS], adj_full[2], adj_empty[2], a_full[2],
      a_free[2], s_full[kRB], r_free[kRB], cb_full[4], cb_done[4], ring_init, done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  // per A tile: the 16-filter chunks that hold a nonzero code; the synthesis
  // multiplies only those (the other chunks of the tile are zero: exact)
  __shared__ uint32_t s_chunks[2];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < RS; ++i) {
      tc::mbar_init(&ring_full[i], 1);
      tc::mbar_init(&ring_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&adj_full[i], 1);
      tc::mbar_init(&adj_empty[i], L::kEpiW);
      tc::mbar_init(&a_full[i], L::kEpiW);
      tc::mbar_init(&a_free[i], 1);
      s_chunks[i] = 0u;
    }
    // one phase per code row (s_full) and per folded output row (r_free); the
    // MMA issue runs at most kRB - 1 rows ahead of the fold, so kRB barriers
    // never alias a phase
    for (int i = 0; i < kRB; ++i) {
      tc::mbar_init(&s_full[i], 1);
      tc::mbar_init(&r_free[i], L::kFoldW);
    }
    for (int i = 0; i < 4; ++i) {
      tc::mbar_init(&cb_full[i], 1);
      tc::mbar_init(&cb_done[i], L::kEpiW);
    }
    tc::mbar_init(&ring_init, L::kFoldW);
    tc::mbar_init(&done_bar, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  {
    const int n16 = (int)(L::b_bytes(Kp) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(Bs);
    for (int i = tid; i < n16; i += blockDim.x) dst[i] = A.bimg[i];
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const uint32_t ring_col = 256;  // synthesis ring blocks at columns 256 + 16 r
  const int Q = im.total;
  const int q_begin = (int)((int64_t)Q * blockIdx.x / gridDim.x);
  const int q_end = (int)((int64_t)Q * (blockIdx.x + 1) / gridDim.x);
  volatile int *abort_v = &abort_flag;

  if (warp == 0) {
    // ================================================== MMA issue
    if (lane == 0) {
      bool ok = tc::mbar_wait_abortable(&ring_init, 0, abort_v, kWaitNs);
      const uint32_t idesc_adj = tc::idesc_bf16_f32(128, Kp);
      const uint32_t ring_base = tc::smem_u32(ring), b_base = tc::smem_u32(Bs);
      const uint32_t a_base = tc::smem_u32(As);
      // synthesis of item i (CTA order) whose first output row has ring
      // counter J0
      auto synth = [&](int i, int J0) -> bool {
        if (!tc::mbar_wait_abortable(&a_full[i & 1], (uint32_t)((i >> 1) & 1), abort_v, kWaitNs))
          return false;
        const int Jr = J0 + 2 * C - kRB;  // the rows up to Jr must have been folded
        if (Jr >= 0 &&
            !tc::mbar_wait_abortable(&r_free[Jr & (kRB - 1)], (uint32_t)((Jr / kRB) & 1), abort_v,
                                     kWaitNs))
          return false;
        tc::fence_after_sync();
        const int rb0 = J0 & (kRB - 1);
        const int n1 = min(S, kRB - rb0), n2 = S - n1;
        const uint32_t ab = a_base + (uint32_t)(i & 1) * a_bytes;
        const uint32_t chunks = *reinterpret_cast<volatile uint32_t *>(&s_chunks[i & 1]);
#pragma unroll 1
        for (uint32_t rest = chunks & ((NC < 32 ? (1u << NC) : 0u) - 1u); rest != 0u;
             rest &= rest - 1u) {
          const int kk = __ffs(rest) - 1;
          const uint64_t ad = tc::smem_desc(ab + kk * 2 * 2048, 2048, 128);
          const uint32_t bk = b_base + kk * 2 * 128;
          tc::mma_bf16(taddr + ring_col + 16 * rb0, ad, tc::smem_desc(bk, 128, Kp * 16),
                       tc::idesc_bf16_f32_bmn(128, 16 * n1), 1u);
          if (n2 > 0)
            tc::mma_bf16(taddr + ring_col, ad,
                         tc::smem_desc(bk + (uint32_t)n1 * 2 * Kp * 16, 128, Kp * 16),
                         tc::idesc_bf16_f32_bmn(128, 16 * n2), 1u);
        }
        tc::mma_commit(&s_full[i & (kRB - 1)]);
        tc::mma_commit(&a_free[i & 1]);
        return true;
      };
      ExtSeg sg;
      sg.q = q_begin;
      sg.q_end = q_end;
      sg.C = C;
      int i = 0, j_seg = 0, J_seg = 0;
      int pend_i = -1, pend_J = 0;  // synthesis not yet issued
      while (ok && sg.next(im)) {
        const int ne = sg.e1 - sg.e0;
        for (int t = 0; t < ne && ok; ++t, ++i) {
          if (iterate) {
            const int b = i & 1;
            ok = tc::mbar_wait_abortable(&adj_empty[b], (uint32_t)(((i >> 1) & 1) ^ 1), abort_v,
                                         kWaitNs);
            const int jr = j_seg + t;
            for (int u = (t == 0 ? 0 : S - 1); u < S && ok; ++u) {
              const int j = jr + u;
              ok = tc::mbar_wait_abortable(&ring_full[j & (RS - 1)], (uint32_t)((j / RS) & 1),
                                           abort_v, kWaitNs);
            }
            if (!ok) break;
            tc::fence_after_sync();
#pragma unroll 1
            for (int u = 0; u < S; ++u) {
              const uint32_t slot = (uint32_t)((jr + u) & (RS - 1));
              const uint64_t ad = tc::smem_desc(ring_base + slot * L::kSRow, 128, 128);
              const uint64_t bd = tc::smem_desc(b_base + u * Kp * 32, Kp * 16, 128);
              tc::mma_bf16(taddr + b * 128, ad, bd, idesc_adj, u > 0 ? 1u : 0u);
            }
            tc::mma_commit(&adj_full[b]);
            tc::mma_commit(&ring_empty[jr & (RS - 1)]);
            if (t == ne - 1)
              for (int e2 = 1; e2 <= 2 * C; ++e2) tc::mma_commit(&ring_empty[(jr + e2) & (RS - 1)]);
          }
          // the previous item's synthesis runs while this item's epilogue works
          if (pend_i >= 0) ok = synth(pend_i, pend_J);
          pend_i = i;
          pend_J = J_seg + t;
        }
        j_seg += ne + 2 * C;
        J_seg += ne + 2 * C;
      }
      if (ok && pend_i >= 0) synth(pend_i, pend_J);
      tc::mma_commit(&done_bar);
      tc::mbar_wait_bounded(&done_bar, 0, kWaitNs);
    }
  } else if (warp < L::W_EPI0) {
    // ================================================== residual rows
    if (iterate) {
      const int pw = warp - L::W_PROD0;
      const bool form_r = A.x != nullptr;
      float *const stg0 = rst + pw * 4 * 144, *const stg1 = stg0 + 144;
      float *const sx0 = stg0 + 2 * 144, *const sx1 = sx0 + 144;
      const float *const xcore = A.xin, *const spill = A.sin;
      const float *const x = A.x;
      const uint8_t *const obs = A.obs;
      ExtRowGen g;
      g.init(q_begin, q_end, C);
      auto next_mine = [&](ExtRowGen &gg) -> bool {
        while (gg.next(im))
          if ((int)(gg.j % L::kProd) == pw) return true;
        return false;
      };
      auto issue = [&](const ExtRowGen &gg, float *dst, float *dx) {
        const Item &it = gg.sg.it;
        const int ar = gg.ar(), b0 = it.js * kStrip;
        for (int k = lane; k < 144; k += 32) {
          const int col = b0 - C + k;
          const bool in = ar >= 0 && ar < it.H && col >= 0 && col < it.W;
          const int64_t p = in ? it.base + (int64_t)ar * it.W + col : 0;
          tc::cp_async4(dst + k, xcore + p, in ? 4u : 0u);
          if (form_r) tc::cp_async4(dx + k, x + p, in ? 4u : 0u);
        }
        tc::cp_async_commit();
      };
      ExtRowGen cur = g;
      bool have = next_mine(cur);
      if (have) issue(cur, stg0, sx0);
      int sbuf = 0;
      while (have) {
        ExtRowGen nxt = cur;
        const bool have_next = next_mine(nxt);
        if (have_next) issue(nxt, sbuf ? stg0 : stg1, sbuf ? sx0 : sx1);
        else tc::cp_async_commit();
        const int j = cur.j, slot = j & (RS - 1);
        bool w = true;
        if (lane == 0)
          w = tc::mbar_wait_abortable(&ring_empty[slot], (uint32_t)(((j / RS) & 1) ^ 1), abort_v,
                                      kWaitNs);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (!w) break;
        tc::cp_async_wait<1>();
        __syncwarp();
        float *const src0 = sbuf ? stg1 : stg0;
        if (form_r) {
          // r = the core columns plus the halo columns the neighbouring
          // strips spilled onto them, minus the image (0 off the image and at
          // unobserved pixels)
          const float *const srcx = sbuf ? sx1 : sx0;
          const Item &it = cur.sg.it;
          const int ar = cur.ar(), b0 = it.js * kStrip;
          const bool row_in = ar >= 0 && ar < it.H;
          const int64_t qr = (int64_t)it.q_row0 + ar;
          for (int k = lane; k < 144; k += 32) {
            const int col = b0 - C + k;
            float v = 0.0f;
            if (row_in && col >= 0 && col < it.W) {
              v = src0[k];
              if (C > 0) {
                if (k < C) v += spill[qr * (2 * C) + k];
                else if (k < 2 * C) {
                  if (it.js > 0) v += spill[(qr - it.H) * (2 * C) + k];
                } else if (k >= kStrip && k < kStrip + C) {
                  if (it.js + 1 < it.JS) v += spill[(qr + it.H) * (2 * C) + k - kStrip];
                } else if (k >= kStrip + C && k < kStrip + 2 * C) {
                  v += spill[qr * (2 * C) + k - kStrip];
                }
              }
              const int64_t p = it.base + (int64_t)ar * it.W + col;
              v = (obs != nullptr && obs[p] == 0) ? 0.0f : v - srcx[k];
            }
            src0[k] = v;
          }
          __syncwarp();
        }
        uint8_t *dst = ring + (size_t)slot * L::kSRow;
        for (int t2 = lane; t2 < 17 * 8; t2 += 32) {
          const int gq = t2 >> 3, ii = t2 & 7;
          const float *src = src0 + 8 * gq + ii;
          uint4 v = make_uint4(pack_bf16x2(src[0], src[1]), pack_bf16x2(src[2], src[3]),
                               pack_bf16x2(src[4], src[5]), pack_bf16x2(src[6], src[7]));
          *reinterpret_cast<uint4 *>(dst + gq * 128 + ii * 16) = v;
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&ring_full[slot]);
        cur = nxt;
        have = have_next;
        sbuf ^= 1;
      }
      tc::cp_async_wait<0>();
    }
  } else if (warp < L::W_FOLD0) {
    // ================================================== epilogue
    const int et = tid - 32 * L::W_EPI0, ew = et >> 5;
    const int quarter = ew & 3, half = ew >> 2;  // TMEM lane quarter, column half
    const int p = 32 * quarter + lane;           // pixel of this thread's TMEM lane
    const float alpha = iterate ? A.prm->alpha : 0.0f, thr = iterate ? A.prm->thresh : 0.0f;
    const uint32_t g_base = tc::smem_u32(Gs), a_base = tc::smem_u32(As);
    const uint32_t lane_base = taddr + ((uint32_t)(32 * quarter) << 16);
    // this thread's pixel row inside a core matrix (G in the A-tile layout,
    // FP32); the two 16-byte halves of the 32-byte row are swapped for pixels
    // with bit 2 set, so that the 16-byte stores of 8 consecutive pixels fall
    // in different bank groups (element e at byte 4e ^ ((e >> 1) & 16))
    const uint32_t g_row = 4u * (uint32_t)((p >> 3) * 64 + (p & 7) * 8);
    const uint32_t g_sw = (uint32_t)((p >> 2) & 1) << 4;
    const int cols = Kp / 2, c0 = half * cols;  // this warp's accumulator columns
    const uint32_t e_max = (uint32_t)(kStrip * Kp);  // elements of G and of an A tile
    ChunkIter<kCH> ci;
    ci.init(q_begin, q_end, C);
    ExtSeg sg;
    sg.q = q_begin;
    sg.q_end = q_end;
    sg.C = C;
    int i = 0, m = 0;  // item, chunk counters
    bool okw = true;     // this warp's waits so far
    bool have_chunk = ci.next(im, A.seg_base);
    // Every epilogue warp passes the same two block-wide barriers per item;
    // they OR the warps' wait results, so that all of them leave together
    // after a wait has run out.
    while (sg.next(im)) {
      bool stop = false;
      for (int a = sg.e0; a < sg.e1; ++a, ++i) {
        if (tc::named_sync_or(1, 32 * L::kEpiW, !okw)) {  // done with the last item's G
          stop = true;
          break;
        }
        const int q = sg.it.q_row0 + a;
        const uint64_t ibeg = A.seg_base[q], iend = A.seg_base[q + 1];
        const int b = i & 1;
        if (iterate) {
          bool w = true;
          if (lane == 0)
            w = tc::mbar_wait_abortable(&adj_full[b], (uint32_t)((i >> 1) & 1), abort_v, kWaitNs);
          okw = __shfl_sync(0xffffffffu, w, 0);
          if (okw) {
            tc::fence_after_sync();
            // accumulator columns [c0, c0 + cols) of pixel p into G, 8 at a time
#pragma unroll 1
            for (int k0 = 0; k0 < cols; k0 += 32) {
              uint32_t r[32];
              const int n8 = min(4, (cols - k0) / 8);
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (j < n8)
                  tc::tmem_ld8_nowait(lane_base + b * 128 + c0 + k0 + 8 * j,
                                      *reinterpret_cast<uint32_t(*)[8]>(&r[8 * j]));
              tc::tmem_ld_wait();
              tc::reg_fence(r);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (j < n8) {
                  const int k = c0 + k0 + 8 * j;
                  const uint32_t so = g_row + 4u * (uint32_t)((k >> 3) * 1024);
                  const uint32_t sa = g_base + (so ^ g_sw), sb = g_base + ((so + 16) ^ g_sw);
                  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(sa), "r"(r[8 * j]),
                               "r"(r[8 * j + 1]), "r"(r[8 * j + 2]), "r"(r[8 * j + 3])
                               : "memory");
                  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(sb),
                               "r"(r[8 * j + 4]), "r"(r[8 * j + 5]), "r"(r[8 * j + 6]),
                               "r"(r[8 * j + 7])
                               : "memory");
                }
              }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&adj_empty[b]);
          }
        }
        // the A tile of item i - 2 has been multiplied: zero it for item i
        if (okw && i >= 2) {
          bool w = true;
          if (lane == 0)
            w = tc::mbar_wait_abortable(&a_free[b], (uint32_t)(((i >> 1) & 1) ^ 1), abort_v,
                                        kWaitNs);
          okw = __shfl_sync(0xffffffffu, w, 0);
        }
        if (okw) {
          uint4 *at = reinterpret_cast<uint4 *>(As + (size_t)b * a_bytes);
          const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
          for (int k = et; k < (int)(a_bytes / 16); k += 32 * L::kEpiW) at[k] = zero;
          if (et == 0) s_chunks[b] = 0u;
        }
        if (tc::named_sync_or(1, 32 * L::kEpiW, !okw)) {  // G written, A tile zeroed
          stop = true;
          break;
        }
        const uint32_t at_base = a_base + (uint32_t)b * a_bytes;
        uint32_t cmask = 0u;  // 16-filter chunks this thread wrote a nonzero code to
        // the item's staged chunks: prox (or, for the input synthesis, the
        // codes as they are) into the staging buffer and the A tile
        while (okw && have_chunk && ci.pos >= ibeg && ci.pos < iend) {
          const int cb = m % ncb;
          bool w2 = true;
          if (lane == 0)
            w2 = tc::mbar_wait_abortable(&cb_full[cb], (uint32_t)((m / ncb) & 1), abort_v,
                                         kWaitNs);
          okw = __shfl_sync(0xffffffffu, w2, 0);
          if (!okw) break;
          const uint32_t n = ci.count();  // a multiple of 8
          uint16_t *const vals = chunk_vals(cb);
          const uint16_t *const ids = chunk_idx(cb);
          for (uint32_t g0 = 8u * et; g0 < n; g0 += 8u * 32 * L::kEpiW) {
            const uint4 vv = *reinterpret_cast<const uint4 *>(vals + g0);
            const uint4 ii = *reinterpret_cast<const uint4 *>(ids + g0);
            uint32_t vw[4] = {vv.x, vv.y, vv.z, vv.w};
            const uint32_t iw[4] = {ii.x, ii.y, ii.z, ii.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              // padding (0xFFFF) and any index past the tile are skipped, so
              // that every shared-memory access stays inside G and the A tile
              const uint32_t e_lo = iw[h] & 0xFFFFu, e_hi = iw[h] >> 16;
              const bool in_lo = e_lo < e_max, in_hi = e_hi < e_max;
              if (iterate) {
                const float g_lo =
                    in_lo ? tc::ld_shared(g_base + ((4u * e_lo) ^ ((e_lo >> 1) & 16u))) : 0.0f;
                const float g_hi =
                    in_hi ? tc::ld_shared(g_base + ((4u * e_hi) ^ ((e_hi >> 1) & 16u))) : 0.0f;
                const float v0 = bf16_lo(vw[h]) - alpha * g_lo;
                const float v1 = bf16_hi(vw[h]) - alpha * g_hi;
                vw[h] = pack_bf16x2(v0 - fminf(fmaxf(v0, -thr), thr),
                                    v1 - fminf(fmaxf(v1, -thr), thr));
              }
              if (in_lo) st_shared_u16(at_base + 2u * e_lo, vw[h] & 0xFFFFu);
              if (in_hi) st_shared_u16(at_base + 2u * e_hi, vw[h] >> 16);
              if (in_lo && (vw[h] & 0x7FFFu)) cmask |= 1u << (e_lo >> 11);
              if (in_hi && (vw[h] & 0x7FFF0000u)) cmask |= 1u << (e_hi >> 11);
            }
            if (iterate)
              *reinterpret_cast<uint4 *>(vals + g0) = make_uint4(vw[0], vw[1], vw[2], vw[3]);
          }
          tc::fence_proxy_async();  // staging (bulk write-back) and A tile (MMA)
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&cb_done[cb]);
          ++m;
          have_chunk = ci.next(im, A.seg_base);
        }
        if (okw) {
          cmask = __reduce_or_sync(0xffffffffu, cmask);
          if (lane == 0 && cmask != 0u) atomicOr(&s_chunks[b], cmask);
          tc::fence_proxy_async();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&a_full[b]);
        }
      }
      if (stop) break;
    }
  } else if (warp < L::W_COPY) {
    // ================================================== fold
    const int ft = tid - 32 * L::W_FOLD0, fw = ft >> 5;  // fw = TMEM lane quarter
    const uint32_t lane_base = taddr + ((uint32_t)(32 * fw) << 16);
    // start: every ring block zero
#pragma unroll 1
    for (int r = 0; r < kRB; ++r) tmem_zero16(lane_base + ring_col + 16 * r);
    tmem_st_wait();
    tc::fence_before_sync();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&ring_init);
    const bool left_edge = lane < C, right_edge = lane >= 32 - C;
    uint32_t own_taps = 0u;
#pragma unroll
    for (int v = 0; v < S; ++v)
      if ((unsigned)(lane + C - v) < 32u) own_taps |= 1u << v;
    const bool spill_lane = (fw == 0 && right_edge) || (fw == 3 && left_edge);
    const int spill_slot = fw == 0 ? lane - (32 - C) : C + lane;
    ExtSeg sg;
    sg.q = q_begin;
    sg.q_end = q_end;
    sg.C = C;
    int i = 0, Jg = 0;  // code row (item) counter, output row counter
    bool ok = true;
    while (ok && sg.next(im)) {
      const Item &it = sg.it;
      const int ne = sg.e1 - sg.e0, b0 = it.js * kStrip, col = b0 + 32 * fw + lane;
      for (int J = 0; J < ne + 2 * C && ok; ++J, ++Jg) {
        if (J < ne) {
          // output row J of the segment is complete once code row J is in;
          // one thread waits, the barrier shares the outcome with the others
          bool w = true;
          if (ft == 0)
            w = tc::mbar_wait_abortable(&s_full[(i + J) & (kRB - 1)],
                                        (uint32_t)(((i + J) / kRB) & 1), abort_v, kWaitNs);
          if (tc::named_sync_or(2, 32 * L::kFoldW, !w)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
        }
        const uint32_t blk = lane_base + ring_col + 16 * (uint32_t)(Jg & (kRB - 1));
        uint32_t qv[16];
        tc::tmem_ld16_nowait(blk, qv);
        tc::tmem_ld_wait();
        tc::reg_fence(qv);
        float own0 = 0.0f, own1 = 0.0f, hal = 0.0f;
#pragma unroll
        for (int v = 0; v < S; ++v) {
          const float t = __shfl_sync(0xffffffffu, __uint_as_float(qv[v]), (lane + C - v) & 31);
          if ((own_taps >> v) & 1u) {
            if (v & 1) own1 += t;
            else own0 += t;
          } else {
            hal += t;
          }
        }
        // the block is read: zero it for output row Jg + kRB
        tmem_zero16(blk);
        tmem_st_wait();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&r_free[Jg & (kRB - 1)]);
        float acc = own0 + own1, acch = 0.0f;
        if (C > 0) {
          float *x2 = xb + (Jg & 1) * (4 * 2 * C);
          if (left_edge || right_edge) x2[fw * 2 * C + (right_edge ? lane - (32 - C) : C + lane)] = hal;
          tc::named_sync(2, 32 * L::kFoldW);
          if (left_edge && fw > 0) acc += x2[(fw - 1) * 2 * C + C + lane];
          if (right_edge && fw < 3) acc += x2[(fw + 1) * 2 * C + lane - (32 - C)];
          if (spill_lane) acch = hal;
        }
        const int o = sg.e0 - C + J;
        if (o >= sg.o0 && o < sg.o1) {
          if (col < it.W) A.xout[it.base + (int64_t)o * it.W + col] = acc;
          if (spill_lane) A.sout[(int64_t)(it.q_row0 + o) * (2 * C) + spill_slot] = acch;
        }
      }
      i += ne;
    }
  } else if (lane == 0) {
    // ================================================== copies
    ChunkIter<kCH> fill, drain;
    fill.init(q_begin, q_end, C);
    drain.init(q_begin, q_end, C);
    auto stage_chunk = [&](const ChunkIter<kCH> &c, int buf) {
      const uint32_t n = c.count();
      tc::fence_proxy_async();
      tc::mbar_arrive_expect_tx(&cb_full[buf], 4u * n);
      tc::bulk_g2s(chunk_vals(buf), A.vin + c.pos, 2u * n, &cb_full[buf]);
      tc::bulk_g2s(chunk_idx(buf), A.idx + c.pos, 2u * n, &cb_full[buf]);
    };
    int staged = 0;  // chunks whose staging copy was issued
    bool more = fill.next(im, A.seg_base);
    for (; more && staged < ncb; ++staged) {
      stage_chunk(fill, staged);
      more = fill.next(im, A.seg_base);
    }
    int m = 0;
    for (; m < staged; ++m) {
      drain.next(im, A.seg_base);
      const int cb = m % ncb;
      if (!tc::mbar_wait_abortable(&cb_done[cb], (uint32_t)((m / ncb) & 1), abort_v, kWaitNs))
        break;
      if (iterate && drain.owned) {
        tc::bulk_s2g(A.vout + drain.pos, chunk_vals(cb), 2u * drain.count());
        tc::bulk_commit();
      }
      if (more) {
        tc::bulk_wait_read0();  // the write-back has read the buffer
        stage_chunk(fill, cb);
        ++staged;
        more = fill.next(im, A.seg_base);
      }
    }
    // staging copies issued but not consumed (after an abort) land, and the
    // write-backs complete, before the CTA exits
    for (int j = m; j < staged; ++j)
      tc::mbar_wait_bounded(&cb_full[j % ncb], (uint32_t)((j / ncb) & 1), kWaitNs);
    tc::bulk_wait0();
  }

  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 512);
  }
  if (tid == 0 && abort_flag) atomicExch(A.err, 1);
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

// Largest number of staging chunk buffers (2..4) that fits, 0 if none does.
int fused_chunk_buffers(int K, int s, int max_smem) {
  const int Kp = (K + 15) / 16 * 16;
  if (Kp > 128) return 0;
  int ncb = 0;
  dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    // 2 KB are left for the kernel's static shared memory (barriers)
    for (int n = 4; n >= 2; --n)
      if (Fus<S>::total(Kp, n) + 2048 <= (size_t)max_smem) {
        ncb = n;
        break;
      }
    return cudaSuccess;
  });
  return ncb;
}

// The kernel's shared-memory size for (K, s, ncb); called before any launch
// (and outside stream capture).
cudaError_t prepare_fused(int K, int s, int ncb) {
  const int Kp = (K + 15) / 16 * 16;
  return dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    return cudaFuncSetAttribute(fused_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Fus<S>::total(Kp, ncb));
  });
}

cudaError_t launch_fused(const tcitems::ItemMap &im, int K, int s, int mode, int ncb,
                         const uint64_t *seg_base, const uint16_t *vin, uint16_t *vout,
                         const uint16_t *idx, const uint4 *bimg, const float *xin,
                         const float *sin, float *xout, float *sout, const float *x,
                         const uint8_t *obs, const StepParams *prm, int *err, int grid,
                         cudaStream_t st) {
  FusedArgs a;
  a.im = im;
  a.K = K;
  a.Kp = (K + 15) / 16 * 16;
  a.mode = mode;
  a.ncb = ncb;
  a.seg_base = seg_base;
  a.vin = vin;
  a.vout = vout;
  a.idx = idx;
  a.bimg = bimg;
  a.xin = xin;
  a.sin = sin;
  a.xout = xout;
  a.sout = sout;
  a.x = x;
  a.obs = obs;
  a.prm = prm;
  a.err = err;
  return dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    const size_t smem = Fus<S>::total(a.Kp, ncb);
    fused_kernel<S><<<grid, Fus<S>::kThreads, smem, st>>>(a);
    return cudaGetLastError();
  });
}

}  // namespace scsc
