// kernels_tc_pipe.cu -- warp-specialised, pipelined tcgen05 kernels of the
// code update for K <= 128 (one persistent CTA per SM).
//
// Adjoint + prox (Eq. 3), 13 warps: warps 1-3 form residual rows (the
// synthesis output staged by cp.async, plus the neighbours' spill columns,
// minus the image; or r itself when an observation mask applies) and write
// each as 8 shifted BF16 copies (a Toeplitz view) into a 16-slot
// shared-memory ring; warp 0 (lane 0) issues, per row item, one MMA per tap
// row into one of two TMEM accumulators; warps 4-11 are two epilogue groups of
// four warps (each covers all 128 pixels of the item and half of its units of
// 8 filters), which run without block barriers: they apply the soft-threshold
// step to the sampled coordinates of the staged packed codes and write the
// item's dense BF16 codes (zero off the sample) in the synthesis's A-operand
// layout; warp 12 (lane 0) stages each item's packed codes by one bulk copy
// and writes them back by another once every epilogue warp is done.
//
// Synthesis, 5 warps: warp 4 (lane 0) fetches each code row's dense BF16 A
// tile by one bulk copy (up to 4 rows ahead) and issues the MMAs P = Z D^T
// into one of two TMEM accumulators; warps 0-3 fold P into output rows
// (col2im by warp shuffles, the warp-edge halo exchanged through shared
// memory) and write the strip's core columns and its 2c spill columns.
//
// Every wait is bounded; on timeout the CTA raises an abort flag, all roles
// leave their loops, the MMAs already issued are waited for (bounded) and the
// tensor memory is released.
#include "scsc_tc.cuh"
#include "tc_items.cuh"
#include "tc_ptx.cuh"

namespace scsc {
namespace {

using namespace tcitems;

constexpr uint64_t kWaitNs = 1000000000ull;

// Offset the dynamic shared-memory base to a 1024-byte boundary by pointer
// arithmetic on the shared array itself, so that the compiler keeps treating
// every derived pointer as a shared-memory address (LDS/STS, not generic).
__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return p + ((1024u - (tc::smem_u32(p) & 1023u)) & 1023u);
}

// Output-row segments of a CTA's item range [q, q_end): maximal runs of items
// in one strip.  o0..o1 are the segment's rows.
struct SegIter {
  int q, q_end;
  Item it;
  int o0, o1;
  __device__ bool next(const ItemMap &im) {
    if (q >= q_end) return false;
    it = item_of(im, q);
    int seg_end = min(q_end, it.q_row0 + it.H);
    o0 = it.a;
    o1 = o0 + (seg_end - q);
    q = seg_end;
    return true;
  }
};

// Mask words of pixel e of row a of the item's strip (zero beyond the image)
// and the offset of the pixel's sampled values inside the item, into registers.
__device__ __forceinline__ void load_masks(const Item &it, int a, int KW, const uint32_t *bits,
                                           const uint16_t *pxoff, int e, uint32_t (&mw)[4],
                                           uint32_t &po) {
  const int col = it.js * kStrip + e;
#pragma unroll
  for (int w = 0; w < 4; ++w) mw[w] = 0u;
  if (col < it.W) {
    const uint32_t *src = bits + (it.base + (int64_t)a * it.W + col) * KW;
#pragma unroll
    for (int w = 0; w < 4; ++w)
      if (w < KW) mw[w] = src[w];
  }
  po = pxoff[(int64_t)(it.q_row0 + a) * kStrip + e];
}

// Mask word w of a pixel's four (0 past the end), by selects, so that a
// runtime index keeps the words in registers.
__device__ __forceinline__ uint32_t pick4(const uint32_t (&mw)[4], int w) {
  return w == 0 ? mw[0] : w == 1 ? mw[1] : w == 2 ? mw[2] : w == 3 ? mw[3] : 0u;
}

// One bulk copy of an item's packed codes [beg, end) (16-byte aligned, a
// multiple of 4 floats) into shared memory; `bar` completes when it lands.
// Issued by one thread once every reader of dv's previous contents is done.
__device__ __forceinline__ void stage_item(uint64_t beg, uint64_t end, const float *packed,
                                           float *dv, uint64_t *bar) {
  const uint32_t bytes = (uint32_t)(end - beg) * 4u;
  tc::fence_proxy_async();
  tc::mbar_arrive_expect_tx(bar, bytes);
  if (bytes) tc::bulk_g2s(dv, packed + beg, bytes, bar);
}

// Item following `it` (next row of the strip, or the first row of the next
// strip / image, found by search only at strip ends).
__device__ __forceinline__ Item next_item(const ItemMap &im, const Item &it) {
  if (it.a + 1 < it.H) {
    Item n = it;
    n.a += 1;
    return n;
  }
  return item_of(im, it.q_row0 + it.H);
}

// ================================================================== adjoint + prox

template <int S>
struct Adj2 {
  static constexpr int C = (S - 1) / 2;
  static constexpr int RS = 16;  // ring slots: a power of two >= S + 3 (slot = j & 15)
  static_assert(S + 3 <= RS, "ring too small");
  static constexpr int kSRow = 17 * 128;
  static constexpr int kProd = 3;
  // Epilogue: kEpi groups of four warps; each covers all 128 pixels (TMEM lane
  // quarters) and a share of the filter chunks.
  static constexpr int kEpi = 2;
  // warp 0: MMA; 1..kProd: residual rows; then 4 kEpi epilogue warps; last: copies
  static constexpr int kThreads = 32 * (1 + kProd + 4 * kEpi + 1);
  __host__ __device__ static size_t b_bytes(int Kp) { return (size_t)S * Kp * 32; }
  __host__ __device__ static size_t vals_bytes(int Kp) { return (size_t)kStrip * Kp * 4; }
  __host__ __device__ static size_t mask_bytes(int KW) { return (size_t)kStrip * KW * 4; }
  __host__ __device__ static size_t total(int Kp, int KW) {
    return 1024 + b_bytes(Kp) + (size_t)RS * kSRow + 2 * vals_bytes(Kp) +
           (size_t)kProd * 4 * 144 * 4;
  }
};

// Rows of the residual that the ring holds, in the order the MMA consumes
// them: per segment, rows o0 - c .. o1 - 1 + c; j counts them across segments.
struct RowGen {
  SegIter sg;
  int j_seg, j;  // 32-bit: a CTA's range holds far fewer than 2^31 rows
  int t, nrows;
  bool live;
  int C;
  __device__ void init(int q0, int q1, int c) {
    sg.q = q0;
    sg.q_end = q1;
    j_seg = 0;
    j = 0;
    t = 0;
    nrows = 0;
    live = false;
    C = c;
  }
  // Advance to the next row; false when exhausted.
  __device__ bool next(const ItemMap &im) {
    while (!live || t >= nrows) {
      if (live) j_seg += nrows;
      if (!sg.next(im)) return false;
      live = true;
      t = 0;
      nrows = sg.o1 - sg.o0 + 2 * C;
    }
    j = j_seg + t;
    ++t;
    return true;
  }
  __device__ int ar() const { return sg.o0 - C + (t - 1); }
};

template <int S>
__global__ void __launch_bounds__(Adj2<S>::kThreads, 1) adj2_kernel(ItemMap im, int K, int Kp, int KW,
                                                      const uint32_t *__restrict__ bits,
                                                      const uint64_t *__restrict__ seg_base,
                                                      const uint16_t *__restrict__ pxoff,
                                                      float *__restrict__ packed,
                                                      uint8_t *__restrict__ abuf,
                                                      const uint4 *__restrict__ badj,
                                                      const float *__restrict__ xcore,
                                                      const float *__restrict__ spill,
                                                      const float *__restrict__ x,
                                                      const uint8_t *__restrict__ obs,
                                                      const StepParams *__restrict__ prm,
                                                      int *err) {
  using L = Adj2<S>;
  constexpr int C = L::C, RS = L::RS;
  const int NC = Kp / 16;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *Bs = smem;
  uint8_t *ring = Bs + L::b_bytes(Kp);
  uint8_t *p = ring + (size_t)RS * L::kSRow;
  float *const vals0 = reinterpret_cast<float *>(p);
  p += L::vals_bytes(Kp);
  float *const vals1 = reinterpret_cast<float *>(p);
  p += L::vals_bytes(Kp);
  auto vals = [&](int k) { return (k & 1) ? vals1 : vals0; };
  float *rst = reinterpret_cast<float *>(p);

  __shared__ uint64_t ring_full[RS], ring_empty[RS], tfull[2], tempty[2], stg_full[2], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < RS; ++i) {
      tc::mbar_init(&ring_full[i], 1);
      tc::mbar_init(&ring_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], 4 * L::kEpi);
      tc::mbar_init(&stg_full[i], 1);
    }
    tc::mbar_init(&done_bar, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  {
    const int n16 = (int)(L::b_bytes(Kp) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(Bs);
    for (int i = tid; i < n16; i += blockDim.x) dst[i] = badj[i];
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const int Q = im.total;
  const int q_begin = (int)((int64_t)Q * blockIdx.x / gridDim.x);
  const int q_end = (int)((int64_t)Q * (blockIdx.x + 1) / gridDim.x);
  volatile int *abort_v = &abort_flag;

  if (warp == 0) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(128, Kp);
      const uint32_t ring_base = tc::smem_u32(ring), b_base = tc::smem_u32(Bs);
      SegIter sg{q_begin, q_end};
      int j_seg = 0;
      int i = 0;
      bool ok = true;
      while (ok && sg.next(im)) {
        const int nrows = sg.o1 - sg.o0 + 2 * C;
        for (int a = sg.o0; a < sg.o1; ++a, ++i) {
          const int b = i & 1;
          const uint32_t use = (uint32_t)(i >> 1);
          ok = tc::mbar_wait_abortable(&tempty[b], (use & 1u) ^ 1u, abort_v, kWaitNs);
          const int jr = j_seg + (a - sg.o0);
          // rows jr .. jr + S - 2 were waited for by the previous row of the
          // segment; only the first row of a segment waits for its whole window
          for (int u = (a == sg.o0 ? 0 : S - 1); u < S && ok; ++u) {
            const int j = jr + u;
            ok = tc::mbar_wait_abortable(&ring_full[j & (RS - 1)], (uint32_t)((j / RS) & 1), abort_v,
                                         kWaitNs);
          }
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll 1
          for (int u = 0; u < S; ++u) {
            const uint32_t slot = (uint32_t)((jr + u) & (RS - 1));
            uint64_t ad = tc::smem_desc(ring_base + slot * L::kSRow, 128, 128);
            uint64_t bd = tc::smem_desc(b_base + u * Kp * 32, Kp * 16, 128);
            tc::mma_bf16(taddr + b * 128, ad, bd, idesc, u > 0 ? 1u : 0u);
          }
          tc::mma_commit(&tfull[b]);
          tc::mma_commit(&ring_empty[jr & (RS - 1)]);
          if (a == sg.o1 - 1)
            for (int e2 = 1; e2 <= 2 * C; ++e2) tc::mma_commit(&ring_empty[(jr + e2) & (RS - 1)]);
        }
        j_seg += nrows;
      }
      tc::mma_commit(&done_bar);
      tc::mbar_wait_bounded(&done_bar, 0, kWaitNs);
    }
  } else if (warp <= L::kProd) {
    // ------------------------------------------------ residual row producers
    const int pw = warp - 1;
    // staged rows of the synthesis output (stg) and of the image (sx), two
    // each; with x == nullptr, xcore already holds the residual r and the rows
    // are used as they arrive
    const bool form_r = x != nullptr;
    float *const stg0 = rst + pw * 4 * 144, *const stg1 = stg0 + 144;
    float *const sx0 = stg0 + 2 * 144, *const sx1 = sx0 + 144;
    RowGen g;
    g.init(q_begin, q_end, C);
    // rows of this warp: sequence indices j = pw (mod kProd)
    auto next_mine = [&](RowGen &gg) -> bool {
      while (gg.next(im))
        if ((int)(gg.j % L::kProd) == pw) return true;
      return false;
    };
    auto issue = [&](const RowGen &gg, float *dst, float *dx) {
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
    RowGen cur = g;
    bool have = next_mine(cur);
    if (have) issue(cur, stg0, sx0);
    int sbuf = 0;
    bool ok = true;
    while (have && ok) {
      RowGen nxt = cur;
      bool have_next = next_mine(nxt);
      if (have_next) issue(nxt, sbuf ? stg0 : stg1, sbuf ? sx0 : sx1);
      else tc::cp_async_commit();
      const int j = cur.j;
      const int slot = j & (RS - 1);
      bool w = true;
      if (lane == 0)
        w = tc::mbar_wait_abortable(&ring_empty[slot], (uint32_t)(((j / RS) & 1) ^ 1), abort_v,
                                    kWaitNs);
      w = __shfl_sync(0xffffffffu, w, 0);
      if (!w) {
        ok = false;
        break;
      }
      tc::cp_async_wait<1>();
      __syncwarp();
      float *const src0 = sbuf ? stg1 : stg0;
      if (form_r) {
        // residual row ar: the synthesis's core columns plus the halo
        // columns its neighbours spilled onto them (the left outer spill of
        // this strip's item on k < c, the right outer spill of the left
        // neighbour's item on c <= k < 2c, the left outer spill of the right
        // neighbour's item on 128 <= k < 128 + c, this item's right outer
        // spill beyond), minus the image; 0 off the image and at unobserved
        // pixels
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
  } else if (warp <= L::kProd + 4 * L::kEpi) {
    // ------------------------------------------------ epilogue: prox on packed codes
    // thread e: pixel px = e & 127 (TMEM lane), group gi = units of 8 filters
    // [u_lo, u_hi): the groups split the 2 NC units evenly, at most 8 each.
    // The warps run unsynchronised with one another: lane 0 of each waits on
    // the item's staged codes and accumulator, and arrives on tempty when the
    // warp is done with the item (TMEM, the staged codes and the A tile).
    const int e = tid - 32 * (1 + L::kProd), px = e & 127, gi = e >> 7, ew = px >> 5;
    const int u_lo = gi * 2 * NC / L::kEpi, u_hi = (gi + 1) * 2 * NC / L::kEpi;
    const int nu = u_hi - u_lo;
    const int w0 = (8 * u_lo) >> 5, sh = (8 * u_lo) & 31;  // mask word and bit of unit u_lo
    const float alpha = prm->alpha, thr = prm->thresh;
    const int n_items = q_end - q_begin;
    const uint32_t lane_base = taddr + ((uint32_t)(32 * ew) << 16);
    // item bookkeeping one step ahead: cur = item i, nxt = item i + 1
    Item cur = item_of(im, q_begin), nxt = cur;
    uint32_t mw[4], mwn[4], po = 0, pon = 0;
    if (n_items > 0) {
      load_masks(cur, cur.a, KW, bits, pxoff, px, mw, po);
      if (n_items > 1) nxt = next_item(im, cur);
    }
    for (int i = 0; i < n_items; ++i) {
      const int q = q_begin + i;
      if (i + 1 < n_items) load_masks(nxt, nxt.a, KW, bits, pxoff, px, mwn, pon);
      // this group's mask bits (8 per unit, from bit 8 u_lo) and the pixel's
      // first value of unit u_lo inside the staged item
      const uint32_t m0 = pick4(mw, w0), m1 = pick4(mw, w0 + 1), m2 = pick4(mw, w0 + 2);
      const uint64_t m01 = ((uint64_t)m1 << 32) | m0;
      const uint64_t gmask = sh ? (m01 >> sh) | ((uint64_t)m2 << (64 - sh)) : m01;
      uint32_t first = po;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int nb = min(32, max(0, 8 * u_lo - 32 * w));  // bits of word w below unit u_lo
        first += __popc(nb == 32 ? mw[w] : (mw[w] & ((1u << nb) - 1u)));
      }
      const int b = i & 1;
      bool okw = true;
      if (lane == 0) {
        okw = tc::mbar_wait_abortable(&stg_full[b], (uint32_t)((i >> 1) & 1), abort_v, kWaitNs);
        if (okw)
          okw = tc::mbar_wait_abortable(&tfull[b], (uint32_t)((i >> 1) & 1), abort_v, kWaitNs);
      }
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      __syncwarp();
      tc::fence_after_sync();
      float *dv = vals(b);
      // this item's A tile for the next synthesis (dense BF16 codes)
      uint8_t *const atile = abuf + (size_t)q * kStrip * Kp * 2;
      uint32_t g[32];  // accumulator columns of up to 4 units (32 filters)
      // running address of the pixel's next sampled value (filter order)
      uint32_t a_run = tc::smem_u32(dv) + 4u * first;
      // two batches of at most 4 units, one wait each; a unit of the second
      // batch is loaded into the registers of the first batch's unit j as
      // soon as that unit is done, so its load overlaps the rest of the batch
      auto load_unit = [&](int jj) {
        tc::tmem_ld8_nowait(lane_base + b * 128 + 8 * (u_lo + jj),
                            *reinterpret_cast<uint32_t(*)[8]>(&g[8 * (jj & 3)]));
      };
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < nu) load_unit(j);
      tc::tmem_ld_wait();
      tc::reg_fence(g);
#pragma unroll
      for (int bt = 0; bt < 2; ++bt) {
        if (4 * bt >= nu) break;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = 4 * bt + j;
          if (jj >= nu) break;
          const uint32_t mu = (uint32_t)(gmask >> (8 * jj)) & 0xFFu;
          // slot of filter e2 = the running address: all loads are
          // independent, then all stores.  Loads are unconditional (an
          // unsampled filter's address still lies inside the staged item) and
          // stores predicated, so the loop has no branches.
          float zv[8], res[8];
          uint32_t ad[8];
#pragma unroll
          for (int e2 = 0; e2 < 8; ++e2) {
            ad[e2] = a_run;
            a_run += ((mu >> e2) & 1u) << 2;
          }
#pragma unroll
          for (int e2 = 0; e2 < 8; ++e2) zv[e2] = tc::ld_shared(ad[e2]);
#pragma unroll
          for (int e2 = 0; e2 < 8; ++e2) {
            const float gv = __uint_as_float(g[8 * j + e2]);
            const float v = zv[e2] - alpha * gv;  // soft threshold as v - clamp(v, -thr, thr)
            res[e2] = v - fminf(fmaxf(v, -thr), thr);
            tc::st_shared_if(ad[e2], res[e2], (mu >> e2) & 1u);
          }
          // the pixel's 8 filters of the A tile: the new codes in BF16, zero
          // off the sample (K-major core of 8 pixels x 8 filters)
#pragma unroll
          for (int e2 = 0; e2 < 8; ++e2) res[e2] = ((mu >> e2) & 1u) ? res[e2] : 0.0f;
          *reinterpret_cast<uint4 *>(atile + (size_t)(u_lo + jj) * 2048 + (px >> 3) * 128 +
                                     (px & 7) * 16) =
              make_uint4(pack_bf16x2(res[0], res[1]), pack_bf16x2(res[2], res[3]),
                         pack_bf16x2(res[4], res[5]), pack_bf16x2(res[6], res[7]));
          if (bt == 0 && jj + 4 < nu) {
            __syncwarp();
            load_unit(jj + 4);
          }
        }
        if (bt == 0 && nu > 4) {
          tc::tmem_ld_wait();
          tc::reg_fence(g);
        }
      }
      tc::fence_before_sync();
      tc::fence_proxy_async();  // the updated codes, to the copy warp's bulk write-back
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
#pragma unroll
      for (int w = 0; w < 4; ++w) mw[w] = mwn[w];
      po = pon;
      if (i + 2 < n_items) nxt = next_item(im, nxt);
    }
  } else if (lane == 0) {
    // ------------------------------------------------ copy warp: staging and write-back
    // Item i's packed codes come into buffer i & 1 by one bulk copy
    // (stg_full[i & 1]); once every epilogue warp has arrived on tempty for
    // item i, they go back to HBM by one bulk copy, and when that copy has
    // read the buffer, item i + 2 is staged into it.
    const int n_items = q_end - q_begin;
    int staged = 0;  // items whose staging copy was issued: [0, staged)
    for (; staged < 2 && staged < n_items; ++staged)
      stage_item(seg_base[q_begin + staged], seg_base[q_begin + staged + 1], packed,
                 vals(staged), &stg_full[staged]);
    int i = 0;
    for (; i < n_items; ++i) {
      const int b = i & 1;
      if (!tc::mbar_wait_abortable(&tempty[b], (uint32_t)((i >> 1) & 1), abort_v, kWaitNs)) break;
      const uint64_t beg = seg_base[q_begin + i], end = seg_base[q_begin + i + 1];
      if (end > beg) {
        tc::bulk_s2g(packed + beg, vals(b), (uint32_t)(end - beg) * 4u);
        tc::bulk_commit();
      }
      if (i + 2 < n_items) {
        tc::bulk_wait_read0();  // the write-back has read the buffer
        stage_item(seg_base[q_begin + i + 2], seg_base[q_begin + i + 3], packed, vals(b),
                   &stg_full[b]);
        staged = i + 3;
      }
    }
    // staging copies issued but not consumed (after an abort) land, and the
    // write-backs complete, before the CTA exits
    for (int j = i; j < staged; ++j)
      tc::mbar_wait_bounded(&stg_full[j & 1], (uint32_t)((j >> 1) & 1), kWaitNs);
    tc::bulk_wait0();
  }

  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 256);
  }
  if (tid == 0 && abort_flag) atomicExch(err, 1);
}

// ================================================================== synthesis

constexpr int kMaxAb = 4;  // A-operand buffers of the synthesis, at most

template <int S>
struct Syn2 {
  static constexpr int C = (S - 1) / 2;
  static constexpr int N = 16 * S;
  static constexpr int kThreads = 160;  // warps 0-3 fold and issue, warp 4 copies
  __host__ __device__ static size_t a_bytes(int Kp) { return (size_t)kStrip * Kp * 2; }
  __host__ __device__ static size_t b_bytes(int Kp) { return (size_t)N * Kp * 2; }
  // nab A-operand buffers (dense BF16 code tiles, filled by bulk copies)
  __host__ __device__ static size_t total(int Kp, int nab) {
    return 1024 + (size_t)nab * a_bytes(Kp) + b_bytes(Kp) + (size_t)2 * 4 * 2 * S * S * 4;
  }
  // as many A buffers as fit, up to kMaxAb (0 if not even one fits)
  static int pick(int Kp, int max_smem) {
    int nab = kMaxAb;
    while (nab > 0 && total(Kp, nab) > (size_t)max_smem) --nab;
    return nab;
  }
};

// Code rows a synthesis CTA visits: per segment, rows max(0, o0-c) ..
// min(H, o1+c) - 1 of the segment's strip.
struct CodeRowGen {
  SegIter sg;
  int a, a_end;
  bool live;
  int C;
  __device__ void init(int q0, int q1, int c) {
    sg.q = q0;
    sg.q_end = q1;
    live = false;
    C = c;
    a = a_end = 0;
  }
  __device__ bool next(const ItemMap &im) {
    if (live) ++a;
    while (!live || a >= a_end) {
      if (!sg.next(im)) return false;
      live = true;
      a = max(0, sg.o0 - C);
      a_end = min(sg.it.H, sg.o1 + C);
    }
    return true;
  }
  __device__ int q() const { return sg.it.q_row0 + a; }
};

template <int S>
__global__ void __launch_bounds__(Syn2<S>::kThreads, 1) syn2_kernel(
    ItemMap im, int K, int Kp, int nab, const uint8_t *__restrict__ abuf,
    const uint4 *__restrict__ bsyn, float *__restrict__ xcore, float *__restrict__ spill,
    int *err) {
  using L = Syn2<S>;
  constexpr int C = L::C, N = L::N;
  const int NC = Kp / 16;
  const uint32_t tile_bytes = (uint32_t)L::a_bytes(Kp);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *const As = smem;  // nab A tiles
  uint8_t *Bs = As + (size_t)nab * tile_bytes;
  float *Pu = reinterpret_cast<float *>(Bs + L::b_bytes(Kp));  // col2im edge exchange [2][4][2c][S]

  __shared__ uint64_t tfull[2], tempty[2], a_full[kMaxAb], a_free[kMaxAb], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], 4);  // one arrival per folding warp
    }
    for (int i = 0; i < kMaxAb; ++i) {
      tc::mbar_init(&a_full[i], 1);  // the copy's expect-tx arrival
      tc::mbar_init(&a_free[i], 1);  // the MMA commit
    }
    tc::mbar_init(&done_bar, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  {
    const int n16 = (int)(L::b_bytes(Kp) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(Bs);
    for (int i = tid; i < n16; i += blockDim.x) dst[i] = bsyn[i];
    for (int i = tid; i < 2 * 4 * 2 * S * S; i += blockDim.x) Pu[i] = 0.0f;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const int Q = im.total;
  const int q_begin = (int)((int64_t)Q * blockIdx.x / gridDim.x);
  const int q_end = (int)((int64_t)Q * (blockIdx.x + 1) / gridDim.x);
  volatile int *abort_v = &abort_flag;

  auto a_buf = [&](int r) { return As + (size_t)(r % nab) * tile_bytes; };
  if (warp == 4) {
    // ------------------------------------------------ A tiles and MMA issue
    // Code row r's dense BF16 codes (written by the adjoint's epilogue in
    // the A-operand layout) arrive by one bulk copy into buffer r % nab, up
    // to nab rows ahead, once the MMAs of row r - nab have released it; then
    // P = Z D^T of row r goes into TMEM buffer r & 1 once the folding group
    // has emptied it (row r - 2).
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(128, N);
      const uint32_t b_base = tc::smem_u32(Bs);
      const uint32_t b_lbo = 2 * S * 128;
      CodeRowGen g;  // the next row to copy
      g.init(q_begin, q_end, C);
      bool more = g.next(im);
      int copied = 0;
      bool ok = true;
      for (int r = 0; ok; ++r) {
        while (more && copied < r + nab) {
          const int ab = copied % nab;
          if (copied >= nab &&
              !tc::mbar_wait_abortable(&a_free[ab], (uint32_t)(((copied - nab) / nab) & 1),
                                       abort_v, kWaitNs)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&a_full[ab], tile_bytes);
          tc::bulk_g2s(a_buf(copied), abuf + (size_t)g.q() * tile_bytes, tile_bytes,
                       &a_full[ab]);
          ++copied;
          more = g.next(im);
        }
        if (!ok || r >= copied) break;  // every row copied has been multiplied
        const int ab = r % nab, b = r & 1;
        ok = tc::mbar_wait_abortable(&a_full[ab], (uint32_t)((r / nab) & 1), abort_v, kWaitNs) &&
             tc::mbar_wait_abortable(&tempty[b], (uint32_t)(((r >> 1) & 1) ^ 1), abort_v,
                                     kWaitNs);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t a_base = tc::smem_u32(a_buf(r));
#pragma unroll 1
        for (int kk = 0; kk < NC; ++kk) {
          uint64_t ad = tc::smem_desc(a_base + kk * 2 * 2048, 2048, 128);
          uint64_t bd = tc::smem_desc(b_base + kk * 2 * b_lbo, b_lbo, 128);
          tc::mma_bf16(taddr + b * 256, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
        tc::mma_commit(&tfull[b]);
        tc::mma_commit(&a_free[ab]);
      }
      // the last copies have landed and the MMAs issued are complete before
      // the CTA may exit (normally already so; this matters after an abort)
      for (int r = copied > nab ? copied - nab : 0; r < copied; ++r)
        tc::mbar_wait_bounded(&a_full[r % nab], (uint32_t)((r / nab) & 1), kWaitNs);
      tc::mma_commit(&done_bar);
      tc::mbar_wait_bounded(&done_bar, 0, kWaitNs);
    }
  } else {
    // ------------------------------------------------ epilogue: col2im
    // Output column L of this warp gets sum_v P[L + c - v][(u, v)] by one warp
    // shuffle per tap from lane (L + c - v) mod 32.  A source index that wraps
    // around the warp delivers a contribution to the neighbouring warp's
    // column L (the left neighbour's when L + c - v >= 32, the right one's when
    // it is < 0): those land on the c right-edge and c left-edge lanes, are
    // exchanged once per code row, and at the strip's outer edges accumulate
    // the spill columns.
    const int e = tid, ew = e >> 5;
    const uint32_t lane_base = taddr + ((uint32_t)(32 * ew) << 16);
    const bool left_edge = lane < C, right_edge = lane >= 32 - C;
    // taps v whose source lane L + c - v lies inside the warp (bit v)
    uint32_t own_taps = 0u;
#pragma unroll
    for (int v = 0; v < S; ++v)
      if ((unsigned)(lane + C - v) < 32u) own_taps |= 1u << v;
    // spill slots: j < c = column b0 - c + j (warp 0, lane 32 - c + j),
    // c + j = column b0 + 128 + j (warp 3, lane j)
    const bool spill_lane = (ew == 0 && right_edge) || (ew == 3 && left_edge);
    const int spill_slot = ew == 0 ? lane - (32 - C) : C + lane;
    bool ok = true;
    SegIter sg{q_begin, q_end};
    int i = 0;
    while (ok && sg.next(im)) {
      const int a_start = max(0, sg.o0 - C), a_end = min(sg.it.H, sg.o1 + C);
      const int b0 = sg.it.js * kStrip;
      const Item &it = sg.it;
      float acc[S], acch[S];
#pragma unroll
      for (int u = 0; u < S; ++u) acc[u] = acch[u] = 0.0f;
      for (int a = a_start; a < a_end; ++a, ++i) {
        const int b = i & 1;
        bool okw = true;
        if (e == 0)
          okw = tc::mbar_wait_abortable(&tfull[b], (uint32_t)((i >> 1) & 1), abort_v, kWaitNs);
        if (tc::named_sync_or(2, 128, !okw)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        // tap rows in batches of kB TMEM loads (one wait per batch)
        constexpr int kB = 4;
        uint32_t pr[kB][16];
        float hacc[S];
#pragma unroll
        for (int u = 0; u < S; ++u) {
          if (u % kB == 0) {
            __syncwarp();
#pragma unroll
            for (int w2 = 0; w2 < kB; ++w2)
              if (u + w2 < S) tc::tmem_ld16_nowait(lane_base + b * 256 + 16 * (u + w2), pr[w2]);
            tc::tmem_ld_wait();
          }
          float own0 = 0.0f, own1 = 0.0f, hal = 0.0f;
#pragma unroll
          for (int v = 0; v < S; ++v) {
            const float pvv = __uint_as_float(pr[u % kB][v]);
            const float t = __shfl_sync(0xffffffffu, pvv, (lane + C - v) & 31);
            if ((own_taps >> v) & 1u) {
              if (v & 1) own1 += t;
              else own0 += t;
            } else {
              hal += t;
            }
          }
          acc[u] += own0 + own1;
          hacc[u] = hal;
        }
        // TMEM reads of this row are done: the MMA thread may refill the
        // buffer (row i + 2)
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[b]);
        if (C > 0) {
          // edge partial sums of warp ew: slot j < c = its left neighbour's
          // column 32 - c + j (lane 32 - c + j), slot c + j = its right
          // neighbour's column j (lane j)
          float *xb = Pu + (i & 1) * (4 * 2 * C * S);
          if (left_edge || right_edge) {
            const int slot = right_edge ? lane - (32 - C) : C + lane;
#pragma unroll
            for (int u = 0; u < S; ++u) xb[(ew * 2 * C + slot) * S + u] = hacc[u];
          }
          tc::named_sync(2, 128);
          if (left_edge && ew > 0) {
#pragma unroll
            for (int u = 0; u < S; ++u) acc[u] += xb[((ew - 1) * 2 * C + C + lane) * S + u];
          }
          if (right_edge && ew < 3) {
#pragma unroll
            for (int u = 0; u < S; ++u) acc[u] += xb[((ew + 1) * 2 * C + lane - (32 - C)) * S + u];
          }
          if (spill_lane) {
#pragma unroll
            for (int u = 0; u < S; ++u) acch[u] += hacc[u];
          }
        }
        const int o = a - C;
        if (o >= sg.o0 && o < sg.o1) {
          if (b0 + e < it.W) xcore[it.base + (int64_t)o * it.W + b0 + e] = acc[0];
          if (spill_lane) spill[(int64_t)(it.q_row0 + o) * (2 * C) + spill_slot] = acch[0];
        }
#pragma unroll
        for (int u = 0; u < S - 1; ++u) {
          acc[u] = acc[u + 1];
          acch[u] = acch[u + 1];
        }
        acc[S - 1] = acch[S - 1] = 0.0f;
      }
      if (!ok) break;
#pragma unroll
      for (int j = 0; j < S - 1; ++j) {
        const int o = a_end - C + j;
        if (o >= sg.o0 && o < sg.o1 && o < it.H) {
          if (b0 + e < it.W) xcore[it.base + (int64_t)o * it.W + b0 + e] = acc[j];
          if (spill_lane) spill[(int64_t)(it.q_row0 + o) * (2 * C) + spill_slot] = acch[j];
        }
      }
    }
  }

  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, 512);
  }
  if (tid == 0 && abort_flag) atomicExch(err, 1);
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

bool tc_pipe_supported(int K, int s, int max_smem) {
  const int Kp = (K + 15) / 16 * 16, KW = (K + 31) / 32;
  if (Kp > 128) return false;
  size_t need = 0;
  dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    need = Adj2<S>::total(Kp, KW);
    size_t syn = Syn2<S>::total(Kp, 1);
    if (syn > need) need = syn;
    return cudaSuccess;
  });
  return need > 0 && need <= (size_t)max_smem;
}

cudaError_t prepare_pipe(int K, int s, int max_smem) {
  const int Kp = (K + 15) / 16 * 16, KW = (K + 31) / 32;
  return dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    const int nab = Syn2<S>::pick(Kp, max_smem);
    cudaError_t e = cudaFuncSetAttribute(syn2_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Syn2<S>::total(Kp, nab));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(adj2_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Adj2<S>::total(Kp, KW));
  });
}

size_t tc_abuf_bytes(int K, int Q) { return (size_t)Q * kStrip * ((K + 15) / 16 * 16) * 2; }

cudaError_t launch_syn2(const tcitems::ItemMap &im, int K, int s, const uint8_t *abuf,
                        const uint4 *bsyn, float *xcore, float *spill, int *err, int grid,
                        int max_smem, cudaStream_t st) {
  const int Kp = (K + 15) / 16 * 16;
  return dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    const int nab = Syn2<S>::pick(Kp, max_smem);
    const size_t smem = Syn2<S>::total(Kp, nab);
    syn2_kernel<S><<<grid, Syn2<S>::kThreads, smem, st>>>(im, K, Kp, nab, abuf, bsyn, xcore,
                                                          spill, err);
    return cudaGetLastError();
  });
}

cudaError_t launch_adj2(const tcitems::ItemMap &im, int K, int s, const uint32_t *bits,
                        const uint64_t *seg_base, const uint16_t *pxoff, float *packed,
                        uint8_t *abuf, const uint4 *badj, const float *xcore, const float *spill,
                        const float *x, const uint8_t *obs, const StepParams *prm, int *err,
                        int grid, cudaStream_t st) {
  const int Kp = (K + 15) / 16 * 16, KW = (K + 31) / 32;
  return dispatch_s(s, [&](auto SC) -> cudaError_t {
    constexpr int S = decltype(SC)::value;
    const size_t smem = Adj2<S>::total(Kp, KW);
    adj2_kernel<S><<<grid, Adj2<S>::kThreads, smem, st>>>(im, K, Kp, KW, bits, seg_base, pxoff,
                                                          packed, abuf, badj, xcore, spill, x,
                                                          obs, prm, err);
    return cudaGetLastError();
  });
}

}  // namespace scsc
