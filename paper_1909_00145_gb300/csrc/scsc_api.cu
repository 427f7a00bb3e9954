// scsc_api.cu -- the C ABI (include/scsc.h): argument checking, workspace
// ownership, batch descriptors and the orchestration of the kernels for the
// code step (Eq. 3, Eq. 4), the dictionary steps (Eq. 5, Eq. 7-8), the
// objective (Eq. 1) and the differentiation primitives.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/scsc.h"
#include "../../include/scsc_diag.h"
#include "scsc_internal.cuh"
#include "profiler.cuh"
#include "scsc_tc.cuh"

using namespace scsc;

namespace {

constexpr int kPowerIters = 50;        // normalised applications before the Rayleigh quotient
constexpr double kSafety = 1.01;       // L = 1.01 x estimate
constexpr uint64_t kTagLz = 0x4C;      // start-vector tags of the three power iterations
constexpr uint64_t kTagLd = 0x44;
constexpr uint64_t kTagLc = 0x43;
constexpr int kRedBlocks = 1024;       // blocks of the FP64 reductions (fixed: deterministic)
// The ADMM and screening kernels launch one grid row per image (grid y, at
// most 65535).
constexpr int kMaxGridImages = 65535;
constexpr int kGradGroups = 304;       // block rows of the filter-gradient reduction (2 x 152 SMs)
constexpr uint32_t kStateMagic = 0x43534353u;  // "SCSC"

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t want = need + need / 8;
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Host copy of a batch descriptor plus its device image.
struct BatchCache {
  std::vector<unsigned char> host;  // serialised descriptor (compare key)
  void *pinned = nullptr;
  size_t pinned_bytes = 0;
  DevBuf dev;
  BatchDev view{};
  int maxH = 0, maxW = 0;
  cudaEvent_t copied = nullptr;
};

}  // namespace

struct scsc_ctx {
  scsc_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  BatchCache batch, domain;     // the call's batch; the step-size domain
  int domainH = -1, domainW = -1;
  DevBuf bits, r, pix2, prm, scal, partials, gpart, gsum, pu, pw, flag;
  DevBuf xkeep, zkeep, bits_off;  // unsampled-keep variant: x - D z_off, sampled codes, complement
  DevBuf ddtG, ddtA;  // tap Gram matrix and per-class stencils of D D^T
  DevBuf admm;        // ADMM vectors: y, u, b, A^T x, CG residual, direction, QP image
  DevBuf admm_partials;  // per-image FP64 partials of the CG dot products
  // screening: D^T r on the active set, per-filter tap prefix sums and norms,
  // per-image partials, per-image results and survivor counts
  DevBuf sg, spref, snrm, spart, simg, skept;
  // the code step size (stencils + power iteration, ~160 launches) as one
  // CUDA graph, captured once per key and replayed
  struct StepKey {
    const float *d;
    int K, s, H, W;
    const void *G, *A, *pu, *pw, *part, *scal, *prm;
    double lambda;
    uint64_t seed;
  } step_key{};
  cudaGraphExec_t step_exec = nullptr;
  // host-buffer entry: device copies of d and of two chunks of x and z, the
  // copy streams and the events that order them
  DevBuf hd, hx[2], hz[2];
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr};
  // tensor path
  TcWorkspace tc;
  // the dictionary step's index of the nonzero codes: counts, offsets,
  // pixel-major and filter-major entries (kernels_sparse.cu)
  DevBuf sp_cpx, sp_ckt, sp_row, sp_kt, sp_scan, sp_pk, sp_pv, sp_kpix, sp_kimg, sp_kv;
  DevBuf sp_T;  // cross-correlations of the code maps (online surrogate update)
  DevBuf sp_seg, sp_P;  // their segment offsets and per-segment slices
  int64_t sp_nnz = 0;   // entries of the index
  bool sp_use = false;
  // online surrogates
  DevBuf C, B, Cd;
  DevBuf Cpart;  // partial sums of the products with C
  uint64_t online_t = 0;
  Profiler prof;
};

namespace {

scsc_status fail(scsc_ctx *c, scsc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(expr)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SCSC_ENOMEM : SCSC_ECUDA,  \
                  "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define CKS(expr)                  \
  do {                             \
    scsc_status s_ = (expr);       \
    if (s_ != SCSC_OK) return s_;  \
  } while (0)

int64_t tiles_of(int H, int W) { return (int64_t)((H + 31) / 32) * ((W + 31) / 32); }

// Validate the host arrays of a batch and stage them on the device.
scsc_status upload_batch(scsc_ctx *ctx, BatchCache &bc, int n, const int64_t *off, const int *H,
                         const int *W, const int64_t *ids) {
  if (n < 1) return fail(ctx, SCSC_EINVAL, "batch: n_images must be >= 1 (got %d)", n);
  if (!off || !H || !W || !ids) return fail(ctx, SCSC_EINVAL, "batch: NULL array");
  std::vector<int64_t> o(n + 1);
  std::vector<int> t0(n + 1);
  int64_t pos = 0, tiles = 0;
  int mh = 0, mw = 0;
  for (int i = 0; i < n; ++i) {
    if (H[i] < 1 || W[i] < 1 || H[i] > 65536 || W[i] > 65536)
      return fail(ctx, SCSC_EINVAL, "batch: image %d has size %dx%d", i, H[i], W[i]);
    if (off[i] != pos)
      return fail(ctx, SCSC_EINVAL,
                  "batch: offsets[%d] = %lld, images must be packed back to back (expected %lld)",
                  i, (long long)off[i], (long long)pos);
    if (ids[i] < 0) return fail(ctx, SCSC_EINVAL, "batch: image_ids[%d] < 0", i);
    o[i] = pos;
    t0[i] = (int)tiles;
    pos += (int64_t)H[i] * W[i];
    tiles += tiles_of(H[i], W[i]);
    if (tiles > (int64_t)0x7fffffff) return fail(ctx, SCSC_EINVAL, "batch too large");
    mh = H[i] > mh ? H[i] : mh;
    mw = W[i] > mw ? W[i] : mw;
  }
  o[n] = pos;
  t0[n] = (int)tiles;
  // layout: off[n+1] i64 | ids[n] i64 | H[n] i32 | W[n] i32 | tile0[n+1] i32
  size_t bytes = (size_t)(n + 1) * 8 + (size_t)n * 8 + (size_t)n * 4 * 2 + (size_t)(n + 1) * 4;
  std::vector<unsigned char> ser(bytes);
  unsigned char *q = ser.data();
  memcpy(q, o.data(), (n + 1) * 8);
  q += (n + 1) * 8;
  memcpy(q, ids, n * 8);
  q += n * 8;
  memcpy(q, H, n * 4);
  q += n * 4;
  memcpy(q, W, n * 4);
  q += n * 4;
  memcpy(q, t0.data(), (n + 1) * 4);
  if (bc.host == ser && bc.dev.p) return SCSC_OK;  // unchanged: reuse the device copy
  if (!bc.copied) CK(cudaEventCreateWithFlags(&bc.copied, cudaEventDisableTiming));
  CK(cudaEventSynchronize(bc.copied));  // the previous staging copy has landed
  if (bc.pinned_bytes < bytes) {
    if (bc.pinned) cudaFreeHost(bc.pinned);
    bc.pinned = nullptr;
    bc.pinned_bytes = 0;
    CK(cudaMallocHost(&bc.pinned, bytes));
    bc.pinned_bytes = bytes;
  }
  memcpy(bc.pinned, ser.data(), bytes);
  CK(bc.dev.ensure(bytes));
  CK(cudaMemcpyAsync(bc.dev.p, bc.pinned, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaEventRecord(bc.copied, ctx->stream));
  bc.host.swap(ser);
  unsigned char *d = bc.dev.as<unsigned char>();
  bc.view.n = n;
  bc.view.off = reinterpret_cast<const int64_t *>(d);
  bc.view.ids = reinterpret_cast<const int64_t *>(d + (n + 1) * 8);
  bc.view.H = reinterpret_cast<const int *>(d + (n + 1) * 8 + n * 8);
  bc.view.W = reinterpret_cast<const int *>(d + (n + 1) * 8 + n * 8 + n * 4);
  bc.view.tile0 = reinterpret_cast<const int *>(d + (n + 1) * 8 + n * 8 + n * 8);
  bc.view.total_px = pos;
  bc.view.n_tiles = (int)tiles;
  bc.view.tile_base = 0;
  bc.maxH = mh;
  bc.maxW = mw;
  return SCSC_OK;
}

// Device view of image i alone (pointers into the batch's descriptor).
BatchDev image_view(const BatchCache &bc, int i) {
  const int n = bc.view.n;
  const int64_t *off = reinterpret_cast<const int64_t *>(bc.host.data());
  const int *t0 = reinterpret_cast<const int *>(bc.host.data() + (n + 1) * 8 + n * 8 + n * 8);
  BatchDev v = bc.view;
  v.n = 1;
  v.off = bc.view.off + i;
  v.ids = bc.view.ids + i;
  v.H = bc.view.H + i;
  v.W = bc.view.W + i;
  v.tile0 = bc.view.tile0 + i;
  v.total_px = off[i + 1] - off[i];
  v.n_tiles = t0[i + 1] - t0[i];
  v.tile_base = t0[i];
  return v;
}

scsc_status stage_batch(scsc_ctx *ctx, const scsc_batch *b) {
  if (!b) return fail(ctx, SCSC_EINVAL, "batch is NULL");
  return upload_batch(ctx, ctx->batch, b->n_images, b->offsets, b->H, b->W, b->image_ids);
}

int KW_of(const scsc_ctx *ctx) { return (ctx->cfg.K + 31) / 32; }
int M_of(const scsc_ctx *ctx) { return ctx->cfg.s * ctx->cfg.s; }

uint64_t threshold_T(const scsc_config &c) {
  return ((uint64_t)c.p_num << 32) / (uint64_t)c.p_den;
}

// Device word that the input checks set when a NaN or an infinity is found
// (zeroed when allocated and whenever it is reported).
int *nonfinite_word(scsc_ctx *ctx) {
  if (!ctx->flag.p) {
    if (ctx->flag.ensure(sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemsetAsync(ctx->flag.p, 0, sizeof(int), ctx->stream) != cudaSuccess) return nullptr;
  }
  return ctx->flag.as<int>();
}

// Enqueue the NaN / Inf check of n floats (a NULL pointer is skipped).
scsc_status check_finite(scsc_ctx *ctx, const float *a, int64_t n) {
  int *w = nonfinite_word(ctx);
  if (!w) return fail(ctx, SCSC_ENOMEM, "input check: flag allocation failed");
  CK(launch_check_finite(a, n, w, ctx->stream));
  return SCSC_OK;
}

// After the stream has been synchronised: SCSC_ENONFINITE (and the word
// cleared) if an input check has fired since the last report.
scsc_status report_nonfinite(scsc_ctx *ctx) {
  if (!ctx->flag.p) return SCSC_OK;
  int word = 0;
  CK(cudaMemcpy(&word, ctx->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (word == 0) return SCSC_OK;
  CK(cudaMemset(ctx->flag.p, 0, sizeof(int)));
  return fail(ctx, SCSC_ENONFINITE,
              "an input (image, codes or filters) held a NaN or an infinity; the results of the "
              "calls since the last report are undefined");
}

scsc_status build_mask(scsc_ctx *ctx, uint64_t t) {
  const BatchDev &b = ctx->batch.view;
  CK(ctx->bits.ensure((size_t)b.total_px * KW_of(ctx) * 4));
  int pr = ctx->prof.begin(KID_MASK, ctx->stream);
  CK(launch_mask_bits(b, ctx->cfg.K, ctx->cfg.seed, t, threshold_T(ctx->cfg),
                      ctx->bits.as<uint32_t>(), ctx->stream));
  ctx->prof.end(pr, ctx->stream);
  return SCSC_OK;
}

// Operator D D^T on the step-size domain: u (pixels) -> w (pixels), through
// the per-class stencils built from d by launch_ddt_prepare (the same linear
// map as the adjoint followed by the synthesis, in (2s-1)^2 multiply-adds per
// pixel instead of 2 K s^2).
scsc_status apply_ddt(scsc_ctx *ctx, const float *u, float *w) {
  CK(launch_ddt_apply(ctx->ddtA.as<float>(), ctx->cfg.s, ctx->domainH, ctx->domainW, u, w,
                      ctx->stream));
  return SCSC_OK;
}

// G = sum over the batch of Z^T r (filter gradient), FP64 [K*M] into gsum.
scsc_status filter_gradient(scsc_ctx *ctx, const float *r, const float *z, const uint32_t *bits) {
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K, M = M_of(ctx);
  CK(ctx->gpart.ensure((size_t)kGradGroups * K * M * 4));
  CK(ctx->gsum.ensure((size_t)K * M * 8));
  CK(launch_filter_grad_fp32(b, K, ctx->cfg.s, r, z, bits, ctx->gpart.as<float>(), kGradGroups,
                             ctx->stream));
  CK(launch_reduce_partials(ctx->gpart.as<float>(), kGradGroups, K * M, ctx->gsum.as<double>(),
                            ctx->stream));
  return SCSC_OK;
}

// Operator sum_n Z_n^T Z_n on filter space: v -> w (float), via synthesis
// with filters v and the filter gradient of the result.
scsc_status apply_ztz(scsc_ctx *ctx, const float *z, const float *v, float *w);

// Generic power iteration on a float vector of length n; writes
// L = 1.01 * <u, A u> to scal[slot] and, if prm != null, the step params.
template <typename Op>
scsc_status power_iteration(scsc_ctx *ctx, int64_t n, uint64_t tag, Op &&apply, int slot,
                            StepParams *prm, double fixed_step) {
  CK(ctx->pu.ensure((size_t)n * 4));
  CK(ctx->pw.ensure((size_t)n * 4));
  CK(ctx->partials.ensure((size_t)2 * kRedBlocks * 8));
  CK(ctx->scal.ensure(8 * 8));
  float *u = ctx->pu.as<float>(), *w = ctx->pw.as<float>();
  double *part = ctx->partials.as<double>();
  cudaStream_t st = ctx->stream;
  CK(launch_power_init(u, n, ctx->cfg.seed, tag, st));
  CK(launch_dot_partials(u, u, n, part, kRedBlocks, st));
  CK(launch_power_normalize(u, u, n, part, kRedBlocks, st));
  for (int it = 0; it < kPowerIters; ++it) {
    CKS(apply(u, w));
    CK(launch_dot_partials(w, w, n, part, kRedBlocks, st));
    CK(launch_power_normalize(w, u, n, part, kRedBlocks, st));
  }
  CKS(apply(u, w));
  CK(launch_dot_partials(u, w, n, part, kRedBlocks, st));
  CK(launch_power_finish(part, kRedBlocks, kSafety, ctx->scal.as<double>() + slot,
                         ctx->cfg.lambda, fixed_step, prm, st));
  return SCSC_OK;
}

constexpr int kSparseGroups = 8;  // partials per filter of the sparse gradient

// Build the index of z's nonzero codes for the dictionary step's operators
// and set ctx->sp_use.  The dense operators stay in use when the codes are
// denser than 1/16 (where they are the faster ones), when a pixel index would
// not fit in 32 bits, or inside a stream capture (the entry count is read
// back to size the index).
scsc_status build_sparse(scsc_ctx *ctx, const float *z) {
  ctx->sp_use = false;
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K;
  cudaStream_t st = ctx->stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone || b.total_px <= 0 || b.total_px >= INT32_MAX)
    return SCSC_OK;
  const int nt = sparse_tiles(b.total_px);
  const int64_t nkt = (int64_t)K * nt;
  CK(ctx->sp_cpx.ensure((size_t)b.total_px * 4));
  CK(ctx->sp_ckt.ensure((size_t)nkt * 4));
  CK(ctx->sp_row.ensure((size_t)(b.total_px + 1) * 8));
  CK(ctx->sp_kt.ensure((size_t)(nkt + 1) * 8));
  CK(ctx->sp_scan.ensure(std::max(sparse_scan_scratch(b.total_px), sparse_scan_scratch(nkt)) * 8));
  CK(launch_sparse_count(b, K, z, ctx->sp_cpx.as<int>(), ctx->sp_ckt.as<int>(), st));
  CK(launch_scan_counts(ctx->sp_cpx.as<int>(), b.total_px, ctx->sp_row.as<int64_t>(),
                        ctx->sp_scan.as<int64_t>(), st));
  CK(launch_scan_counts(ctx->sp_ckt.as<int>(), nkt, ctx->sp_kt.as<int64_t>(),
                        ctx->sp_scan.as<int64_t>(), st));
  int64_t nnz = 0;
  CK(cudaMemcpyAsync(&nnz, ctx->sp_row.as<int64_t>() + b.total_px, sizeof nnz,
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (nnz * 16 > b.total_px * (int64_t)K) return SCSC_OK;
  ctx->sp_nnz = nnz;
  const size_t n1 = (size_t)std::max<int64_t>(nnz, 1);
  CK(ctx->sp_pk.ensure(n1 * 4));
  CK(ctx->sp_pv.ensure(n1 * 4));
  CK(ctx->sp_kpix.ensure(n1 * 4));
  CK(ctx->sp_kimg.ensure(n1 * 4));
  CK(ctx->sp_kv.ensure(n1 * 4));
  CK(launch_sparse_fill(b, K, z, ctx->sp_row.as<int64_t>(), ctx->sp_kt.as<int64_t>(),
                        ctx->sp_pk.as<int>(), ctx->sp_pv.as<float>(), ctx->sp_kpix.as<int>(),
                        ctx->sp_kimg.as<int>(), ctx->sp_kv.as<float>(), st));
  ctx->sp_use = true;
  return SCSC_OK;
}

// out = D z (minus x when given) with filters d, on the index when it is in use.
scsc_status dict_synth(scsc_ctx *ctx, const float *d, const float *z, const float *x, float *out) {
  const BatchDev &b = ctx->batch.view;
  if (ctx->sp_use)
    CK(launch_sparse_synth(b, ctx->cfg.K, ctx->cfg.s, d, ctx->sp_row.as<int64_t>(),
                           ctx->sp_pk.as<int>(), ctx->sp_pv.as<float>(), x, out, ctx->stream));
  else
    CK(launch_synth_fp32(b, ctx->cfg.K, ctx->cfg.s, d, z, nullptr, x, out, ctx->stream));
  return SCSC_OK;
}

// gsum = Z^T r (FP64), on the index when it is in use.
scsc_status dict_gradient(scsc_ctx *ctx, const float *r, const float *z) {
  if (!ctx->sp_use) return filter_gradient(ctx, r, z, nullptr);
  const int K = ctx->cfg.K, M = M_of(ctx);
  CK(ctx->gpart.ensure((size_t)kSparseGroups * K * M * 4));
  CK(ctx->gsum.ensure((size_t)K * M * 8));
  CK(launch_sparse_grad(ctx->batch.view, K, ctx->cfg.s, r, ctx->sp_kt.as<int64_t>(),
                        ctx->sp_kpix.as<int>(), ctx->sp_kimg.as<int>(), ctx->sp_kv.as<float>(),
                        ctx->gpart.as<float>(), kSparseGroups, ctx->stream));
  CK(launch_reduce_partials(ctx->gpart.as<float>(), kSparseGroups, K * M, ctx->gsum.as<double>(),
                            ctx->stream));
  return SCSC_OK;
}

scsc_status apply_ztz(scsc_ctx *ctx, const float *z, const float *v, float *w) {
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K, M = M_of(ctx);
  if (ctx->sp_use) {
    CKS(dict_synth(ctx, v, z, nullptr, ctx->pix2.as<float>()));
    CKS(dict_gradient(ctx, ctx->pix2.as<float>(), z));
    CK(launch_double_to_float(ctx->gsum.as<double>(), w, K * M, ctx->stream));
    return SCSC_OK;
  }
  CK(launch_synth_fp32(b, K, ctx->cfg.s, v, z, nullptr, nullptr, ctx->pix2.as<float>(),
                       ctx->stream));
  CKS(filter_gradient(ctx, ctx->pix2.as<float>(), z, nullptr));
  CK(launch_double_to_float(ctx->gsum.as<double>(), w, K * M, ctx->stream));
  return SCSC_OK;
}

// Step size of the code update into ctx->prm (device).
scsc_status code_step_size(scsc_ctx *ctx, const float *d) {
  CK(ctx->prm.ensure(sizeof(StepParams)));
  CK(ctx->scal.ensure(8 * 8));
  StepParams *prm = ctx->prm.as<StepParams>();
  if (ctx->cfg.step > 0.0) {
    CK(launch_set_step(prm, ctx->cfg.step, ctx->cfg.lambda, ctx->stream));
    return SCSC_OK;
  }
  int H = ctx->batch.maxH, W = ctx->batch.maxW;
  if (H != ctx->domainH || W != ctx->domainW) {
    int64_t zero = 0, id = 0;
    CKS(upload_batch(ctx, ctx->domain, 1, &zero, &H, &W, &id));
    ctx->domainH = H;
    ctx->domainW = W;
  }
  const int sz = ctx->cfg.s;
  const int64_t n = (int64_t)H * W;
  CK(ctx->ddtG.ensure((size_t)sz * sz * sz * sz * 8));
  CK(ctx->ddtA.ensure(ddt_stencil_floats(sz, H, W) * 4));
  // every buffer of the power iteration exists before a capture starts
  CK(ctx->pu.ensure((size_t)n * 4));
  CK(ctx->pw.ensure((size_t)n * 4));
  CK(ctx->partials.ensure((size_t)2 * kRedBlocks * 8));
  cudaStream_t st = ctx->stream;
  auto enqueue = [&]() -> scsc_status {
    CK(launch_ddt_prepare(d, ctx->cfg.K, sz, H, W, ctx->ddtG.as<double>(), ctx->ddtA.as<float>(),
                          st));
    return power_iteration(
        ctx, n, kTagLz, [&](const float *u, float *w) { return apply_ddt(ctx, u, w); }, 0, prm,
        0.0);
  };
  int pr = ctx->prof.begin(KID_POWER, st);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  const bool use_graph = st != nullptr && cap == cudaStreamCaptureStatusNone &&
                         !(ctx->cfg.flags & SCSC_FLAG_NO_GRAPH);
  scsc_status status = SCSC_OK;
  if (!use_graph) {
    status = enqueue();
  } else {
    scsc_ctx::StepKey key{};  // zero-filled, so that memcmp sees no padding bytes
    key.d = d;
    key.K = ctx->cfg.K;
    key.s = sz;
    key.H = H;
    key.W = W;
    key.G = ctx->ddtG.p;
    key.A = ctx->ddtA.p;
    key.pu = ctx->pu.p;
    key.pw = ctx->pw.p;
    key.part = ctx->partials.p;
    key.scal = ctx->scal.p;
    key.prm = prm;
    key.lambda = ctx->cfg.lambda;
    key.seed = ctx->cfg.seed;
    if (!ctx->step_exec || std::memcmp(&key, &ctx->step_key, sizeof key) != 0) {
      if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
      ctx->step_exec = nullptr;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      status = enqueue();
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (status != SCSC_OK) {
        if (g) cudaGraphDestroy(g);
        return status;
      }
      CK(e);
      e = cudaGraphInstantiate(&ctx->step_exec, g, 0);
      cudaGraphDestroy(g);
      CK(e);
      ctx->step_key = key;
    }
    CK(cudaGraphLaunch(ctx->step_exec, st));
  }
  ctx->prof.end(pr, st);
  return status;
}

scsc_status check_cfg(scsc_ctx *ctx, const scsc_config *c) {
  if (!c) return fail(ctx, SCSC_EINVAL, "config is NULL");
  if (c->K < 1 || c->K > kMaxK) return fail(ctx, SCSC_EINVAL, "K = %d outside [1, %d]", c->K, kMaxK);
  if (c->s < 1 || c->s > kMaxS || c->s % 2 == 0)
    return fail(ctx, SCSC_EINVAL, "s = %d must be odd and in [1, %d]", c->s, kMaxS);
  if (!(c->lambda > 0.0) || !std::isfinite(c->lambda))
    return fail(ctx, SCSC_EINVAL, "lambda must be finite and > 0");
  if (c->p_den == 0 || c->p_num > c->p_den)
    return fail(ctx, SCSC_EINVAL, "p = %u/%u must satisfy 0 <= p <= 1", c->p_num, c->p_den);
  if (!(c->step >= 0.0) || !std::isfinite(c->step))
    return fail(ctx, SCSC_EINVAL, "step must be finite and >= 0");
  if (c->prec == SCSC_TF32)
    return fail(ctx, SCSC_EUNSUPPORTED,
                "TF32 operands are not built: the tensor path uses BF16 operands (kind::f16), "
                "and SCSC_FP32 is the full-precision path");
  if (c->prec != SCSC_FP32 && c->prec != SCSC_BF16)
    return fail(ctx, SCSC_EINVAL, "unknown precision %d", (int)c->prec);
  if (c->flags & ~(SCSC_FLAG_PER_IMAGE | SCSC_FLAG_NO_GRAPH | SCSC_FLAG_NO_AUTOTUNE |
                   SCSC_FLAG_UNSAMPLED_KEEP | SCSC_FLAG_TWO_KERNEL))
    return fail(ctx, SCSC_EINVAL, "unknown flags 0x%x", c->flags);
  return SCSC_OK;
}

}  // namespace

// ===================================================================== ABI

extern "C" {

scsc_status scsc_create(const scsc_config *cfg, void *cuda_stream, scsc_ctx **out) {
  if (!out) return SCSC_EINVAL;
  *out = nullptr;
  scsc_ctx tmp;
  scsc_ctx *ctx = &tmp;
  CKS(check_cfg(ctx, cfg));
  scsc_ctx *c = new (std::nothrow) scsc_ctx();
  if (!c) return SCSC_ENOMEM;
  c->cfg = *cfg;
  c->tc.prof = &c->prof;
  c->tc.graphs = (cfg->flags & SCSC_FLAG_NO_GRAPH) == 0;
  c->tc.autotune = (cfg->flags & SCSC_FLAG_NO_AUTOTUNE) == 0;
  c->tc.fused = (cfg->flags & SCSC_FLAG_TWO_KERNEL) == 0;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return SCSC_ECUDA;
  }
  *out = c;
  return SCSC_OK;
}

scsc_status scsc_destroy(scsc_ctx *ctx) {
  if (!ctx) return SCSC_OK;
  cudaStreamSynchronize(ctx->stream);
  for (DevBuf *b : {&ctx->bits, &ctx->r, &ctx->pix2, &ctx->prm, &ctx->scal, &ctx->partials,
                    &ctx->gpart, &ctx->gsum, &ctx->pu, &ctx->pw,
                    &ctx->flag, &ctx->ddtG, &ctx->ddtA, &ctx->admm, &ctx->admm_partials,
                    &ctx->xkeep, &ctx->zkeep, &ctx->bits_off,
                    &ctx->hd, &ctx->hx[0], &ctx->hx[1], &ctx->hz[0], &ctx->hz[1],
                    &ctx->C, &ctx->B, &ctx->Cd, &ctx->batch.dev, &ctx->domain.dev,
                    &ctx->sg, &ctx->spref, &ctx->snrm, &ctx->spart, &ctx->simg, &ctx->skept,
                    &ctx->sp_cpx, &ctx->sp_ckt, &ctx->sp_row, &ctx->sp_kt, &ctx->sp_scan,
                    &ctx->sp_pk, &ctx->sp_pv, &ctx->sp_kpix, &ctx->sp_kimg, &ctx->sp_kv,
                    &ctx->sp_T, &ctx->sp_seg, &ctx->sp_P, &ctx->Cpart})
    b->release();
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  for (BatchCache *bc : {&ctx->batch, &ctx->domain}) {
    if (bc->pinned) cudaFreeHost(bc->pinned);
    if (bc->copied) cudaEventDestroy(bc->copied);
  }
  tc_release(ctx->tc);
  ctx->prof.release();
  for (cudaStream_t *sp : {&ctx->s_in, &ctx->s_out})
    if (*sp) cudaStreamDestroy(*sp);
  for (int i = 0; i < 2; ++i)
    for (cudaEvent_t e : {ctx->ev_in[i], ctx->ev_done[i], ctx->ev_out[i]})
      if (e) cudaEventDestroy(e);
  delete ctx;
  return SCSC_OK;
}

const char *scsc_last_error(const scsc_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

scsc_status scsc_mask(scsc_ctx *ctx, const scsc_batch *batch, uint64_t t, uint32_t *bits_dev) {
  if (!ctx) return SCSC_EINVAL;
  if (!bits_dev) return fail(ctx, SCSC_EINVAL, "bits_dev is NULL");
  CKS(stage_batch(ctx, batch));
  const BatchDev &b = ctx->batch.view;
  CK(launch_mask_bits(b, ctx->cfg.K, ctx->cfg.seed, t, threshold_T(ctx->cfg), bits_dev,
                      ctx->stream));
  return SCSC_OK;
}

scsc_status scsc_lipschitz_codes(scsc_ctx *ctx, const scsc_batch *batch, const float *d_dev,
                                 double *out_host) {
  if (!ctx) return SCSC_EINVAL;
  if (!d_dev || !out_host) return fail(ctx, SCSC_EINVAL, "NULL pointer");
  CKS(stage_batch(ctx, batch));
  CKS(check_finite(ctx, d_dev, (int64_t)ctx->cfg.K * M_of(ctx)));
  scsc_config saved = ctx->cfg;
  ctx->cfg.step = 0.0;  // always run the power iteration here
  scsc_status s = code_step_size(ctx, d_dev);
  ctx->cfg = saved;
  if (s != SCSC_OK) return s;
  CK(cudaMemcpyAsync(out_host, ctx->scal.as<double>(), 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return report_nonfinite(ctx);
}

// scsc_code_step / scsc_code_step_observed (obs = NULL: every pixel observed).
// keep_step: use the step parameters already in ctx->prm (the host-buffer
// entry computes them once for the whole batch before its chunks).
// keep_mask: iterate on the active set already in ctx->bits (screened steps).
static scsc_status code_step_impl(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *d_dev, float *z_dev, const uint8_t *obs, uint64_t t,
                           int n_iters, bool keep_step = false, bool keep_mask = false) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_dev || !d_dev || !z_dev) return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  if (n_iters < 0) return fail(ctx, SCSC_EINVAL, "n_iters = %d < 0", n_iters);
  CKS(stage_batch(ctx, batch));
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K, s = ctx->cfg.s;
  cudaStream_t st = ctx->stream;
  const bool keep = (ctx->cfg.flags & SCSC_FLAG_UNSAMPLED_KEEP) != 0;
  if (keep && keep_mask)
    return fail(ctx, SCSC_EUNSUPPORTED, "the unsampled-keep variant has no screened step");
  CKS(check_finite(ctx, x_dev, b.total_px));
  CKS(check_finite(ctx, d_dev, (int64_t)K * M_of(ctx)));
  if (!keep_mask) CKS(build_mask(ctx, t));
  if (!keep_step) CKS(code_step_size(ctx, d_dev));
  const StepParams *prm = ctx->prm.as<StepParams>();
  const uint32_t *bits = ctx->bits.as<uint32_t>();
  if (keep) {
    // Sec. 3.1's other reading: the codes off the sampled set stay as they
    // are, so the sampled problem sees x' = x - D z_off (FP32, once per step)
    CK(ctx->xkeep.ensure((size_t)b.total_px * 4));
    CK(ctx->bits_off.ensure((size_t)b.total_px * KW_of(ctx) * 4));
    CK(launch_complement_bits(bits, ctx->bits_off.as<uint32_t>(), b.total_px, K, st));
    CK(launch_synth_fp32(b, K, s, d_dev, z_dev, ctx->bits_off.as<uint32_t>(), x_dev,
                         ctx->xkeep.as<float>(), st));
    CK(launch_negate(ctx->xkeep.as<float>(), b.total_px, st));
    x_dev = ctx->xkeep.as<float>();
  }
  if (ctx->cfg.prec == SCSC_BF16) {
    int *errw = tc_error_word(ctx->tc);
    if (!errw) return fail(ctx, SCSC_ENOMEM, "tensor path: error word allocation failed");
    int *nf = nonfinite_word(ctx);
    if (!nf) return fail(ctx, SCSC_ENOMEM, "input check: flag allocation failed");
    CK(cudaMemsetAsync(errw, 0, sizeof(int), st));
    ctx->tc.sample_p = (double)ctx->cfg.p_num / (double)ctx->cfg.p_den;
    cudaError_t e = tc_code_step(ctx->tc, b, batch->H, batch->W, K, s, x_dev, d_dev, z_dev,
                                 bits, obs, prm, n_iters, keep, nf, st);
    if (e == cudaErrorNotSupported)
      return fail(ctx, SCSC_EUNSUPPORTED, "tensor path: %s", tc_last_error(ctx->tc));
    if (e == cudaErrorTimeout)
      return fail(ctx, SCSC_ETIMEOUT, "tensor path: a bounded wait ran out (%s)",
                  tc_last_error(ctx->tc));
    CK(e);
    return SCSC_OK;
  }
  // Plain FP32 path.  Eq. 4 warm start: unsampled codes are zero (the keep
  // variant iterates on a copy holding the sampled codes, merged back below).
  CKS(check_finite(ctx, z_dev, b.total_px * K));
  float *const z_user = z_dev;
  if (keep) {
    CK(ctx->zkeep.ensure((size_t)b.total_px * K * 4));
    CK(cudaMemcpyAsync(ctx->zkeep.p, z_dev, (size_t)b.total_px * K * 4, cudaMemcpyDeviceToDevice,
                       st));
    z_dev = ctx->zkeep.as<float>();
  }
  CK(launch_apply_mask_dense(b, K, ctx->bits.as<uint32_t>(), z_dev, st));
  CK(ctx->r.ensure((size_t)b.total_px * 4));
  // views to launch over: the whole batch, or each image on its own
  std::vector<BatchDev> views;
  if (ctx->cfg.flags & SCSC_FLAG_PER_IMAGE) {
    for (int i = 0; i < b.n; ++i) views.push_back(image_view(ctx->batch, i));
  } else {
    views.push_back(b);
  }
  for (int it = 0; it < n_iters; ++it) {
    for (const BatchDev &v : views) {
      int p1 = ctx->prof.begin(KID_SYNTH_FP32, st);
      CK(launch_synth_fp32(v, K, s, d_dev, z_dev, nullptr, x_dev, ctx->r.as<float>(), st));
      ctx->prof.end(p1, st);
    }
    if (obs) CK(launch_mask_residual(ctx->r.as<float>(), obs, b.total_px, st));
    for (const BatchDev &v : views) {
      int p2 = ctx->prof.begin(KID_ADJ_FP32, st);
      CK(launch_adjoint_fp32(v, K, s, d_dev, ctx->r.as<float>(), ctx->bits.as<uint32_t>(), 1,
                             prm, z_dev, st));
      ctx->prof.end(p2, st);
    }
  }
  if (keep) CK(launch_merge_sampled(b, K, ctx->bits.as<uint32_t>(), z_dev, z_user, st));
  return SCSC_OK;
}

static scsc_status objective_impl(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *z_dev, const float *d_dev, const uint8_t *obs,
                           double *out_host) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_dev || !z_dev || !d_dev || !out_host) return fail(ctx, SCSC_EINVAL, "NULL pointer");
  CKS(stage_batch(ctx, batch));
  const BatchDev &b = ctx->batch.view;
  cudaStream_t st = ctx->stream;
  CKS(check_finite(ctx, x_dev, b.total_px));
  CKS(check_finite(ctx, z_dev, b.total_px * ctx->cfg.K));
  CKS(check_finite(ctx, d_dev, (int64_t)ctx->cfg.K * M_of(ctx)));
  CK(ctx->r.ensure((size_t)b.total_px * 4));
  CK(ctx->partials.ensure((size_t)2 * kRedBlocks * 8));
  CK(ctx->scal.ensure(8 * 8));
  CK(launch_synth_fp32(b, ctx->cfg.K, ctx->cfg.s, d_dev, z_dev, nullptr, x_dev, ctx->r.as<float>(),
                       st));
  if (obs) CK(launch_mask_residual(ctx->r.as<float>(), obs, b.total_px, st));
  CK(launch_sum_sq_abs(ctx->r.as<float>(), b.total_px, z_dev, b.total_px * ctx->cfg.K,
                       ctx->partials.as<double>(), kRedBlocks, st));
  CK(launch_finish_sum(ctx->partials.as<double>(), kRedBlocks, 0.5, ctx->cfg.lambda,
                       ctx->scal.as<double>() + 4, st));
  CK(cudaMemcpyAsync(out_host, ctx->scal.as<double>() + 4, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return report_nonfinite(ctx);
}

scsc_status scsc_code_step(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *d_dev, float *z_dev, uint64_t t, int n_iters) {
  return code_step_impl(ctx, batch, x_dev, d_dev, z_dev, nullptr, t, n_iters);
}

scsc_status scsc_code_step_host(scsc_ctx *ctx, const scsc_batch *batch, const float *x_host,
                                const float *d_host, float *z_host, uint64_t t, int n_iters) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_host || !d_host || !z_host) return fail(ctx, SCSC_EINVAL, "NULL host pointer");
  if (n_iters < 0) return fail(ctx, SCSC_EINVAL, "n_iters = %d < 0", n_iters);
  if (!batch || batch->n_images < 1) return fail(ctx, SCSC_EINVAL, "batch: n_images must be >= 1");
  const int K = ctx->cfg.K, M = M_of(ctx), n = batch->n_images;
  cudaStream_t st = ctx->stream;
  if (!ctx->s_in) {
    CK(cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CK(cudaEventCreateWithFlags(&ctx->ev_in[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_out[i], cudaEventDisableTiming));
    }
  }
  // the step size of the whole batch (max H x max W domain), once
  CK(ctx->hd.ensure((size_t)K * M * 4));
  CK(cudaMemcpyAsync(ctx->hd.p, d_host, (size_t)K * M * 4, cudaMemcpyHostToDevice, st));
  const float *d_dev = ctx->hd.as<float>();
  CKS(stage_batch(ctx, batch));
  CKS(code_step_size(ctx, d_dev));
  // chunks: contiguous image ranges of about equal pixel counts, at least
  // 2^20 pixels each, at most 3 (the first chunk's copy in and the last one's
  // copy out are the parts that do not overlap; more chunks add per-call work
  // and, for the fused kernel, more recomputed boundary rows per owned row:
  // on 64 x 256^2, 3 chunks measured 520 Gpix*filter/s end to end, 4 chunks
  // 482-490, 2 chunks 451-502)
  int64_t total = 0;
  for (int i = 0; i < n; ++i) total += (int64_t)batch->H[i] * batch->W[i];
  const int want = (int)std::max<int64_t>(1, std::min<int64_t>({3, n, total >> 20}));
  std::vector<int> first{0};  // chunk c = images [first[c], first[c + 1])
  {
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
      acc += (int64_t)batch->H[i] * batch->W[i];
      if (i + 1 < n && (int)first.size() < want && acc * want >= total * (int64_t)first.size())
        first.push_back(i + 1);
    }
    first.push_back(n);
  }
  const int nch = (int)first.size() - 1;
  int64_t max_px = 0;
  for (int c = 0; c < nch; ++c) max_px = std::max(max_px, batch->offsets[first[c + 1] - 1] +
                                                              (int64_t)batch->H[first[c + 1] - 1] *
                                                                  batch->W[first[c + 1] - 1] -
                                                              batch->offsets[first[c]]);
  for (int i = 0; i < 2 && i < nch; ++i) {
    CK(ctx->hx[i].ensure((size_t)max_px * 4));
    CK(ctx->hz[i].ensure((size_t)max_px * K * 4));
  }
  // Chunk c uses slot c % 2: copy in on s_in (after the slot's previous
  // chunk has been copied out), compute on the context stream, copy out on
  // s_out; chunk c + 1's copy in overlaps chunk c's compute.
  std::vector<int64_t> off_c;
  scsc_status status = SCSC_OK;
  for (int c = 0; c < nch && status == SCSC_OK; ++c) {
    const int i0 = first[c], i1 = first[c + 1], slot = c & 1;
    const int64_t o = batch->offsets[i0];
    const int64_t px = batch->offsets[i1 - 1] + (int64_t)batch->H[i1 - 1] * batch->W[i1 - 1] - o;
    if (c >= 2) CK(cudaStreamWaitEvent(ctx->s_in, ctx->ev_out[slot], 0));
    CK(cudaMemcpyAsync(ctx->hx[slot].p, x_host + o, (size_t)px * 4, cudaMemcpyHostToDevice,
                       ctx->s_in));
    CK(cudaMemcpyAsync(ctx->hz[slot].p, z_host + o * K, (size_t)px * K * 4,
                       cudaMemcpyHostToDevice, ctx->s_in));
    CK(cudaEventRecord(ctx->ev_in[slot], ctx->s_in));
    CK(cudaStreamWaitEvent(st, ctx->ev_in[slot], 0));
    off_c.assign(i1 - i0, 0);
    for (int i = i0; i < i1; ++i) off_c[i - i0] = batch->offsets[i] - o;
    const scsc_batch cb{i1 - i0, off_c.data(), batch->H + i0, batch->W + i0, batch->image_ids + i0};
    status = code_step_impl(ctx, &cb, ctx->hx[slot].as<float>(), d_dev, ctx->hz[slot].as<float>(),
                            nullptr, t, n_iters, /*keep_step=*/true);
    if (status != SCSC_OK) break;
    CK(cudaEventRecord(ctx->ev_done[slot], st));
    CK(cudaStreamWaitEvent(ctx->s_out, ctx->ev_done[slot], 0));
    CK(cudaMemcpyAsync(z_host + o * K, ctx->hz[slot].p, (size_t)px * K * 4,
                       cudaMemcpyDeviceToHost, ctx->s_out));
    CK(cudaEventRecord(ctx->ev_out[slot], ctx->s_out));
  }
  CK(cudaStreamSynchronize(ctx->s_out));
  CK(cudaStreamSynchronize(st));
  if (status != SCSC_OK) return status;
  return report_nonfinite(ctx);
}

scsc_status scsc_code_step_observed(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                    const float *d_dev, float *z_dev,
                                    const uint8_t *observed_dev, uint64_t t, int n_iters) {
  return code_step_impl(ctx, batch, x_dev, d_dev, z_dev, observed_dev, t, n_iters);
}

scsc_status scsc_objective(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *z_dev, const float *d_dev, double *out_host) {
  return objective_impl(ctx, batch, x_dev, z_dev, d_dev, nullptr, out_host);
}

scsc_status scsc_code_step_admm(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                const float *d_dev, float *z_dev, uint64_t t, int n_iters,
                                int cg_iters, double rho, double alpha_r) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_dev || !d_dev || !z_dev) return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  if (n_iters < 0 || cg_iters < 0)
    return fail(ctx, SCSC_EINVAL, "n_iters = %d, cg_iters = %d must be >= 0", n_iters, cg_iters);
  if (rho <= 0.0) rho = 10.0 * ctx->cfg.lambda;
  if (alpha_r <= 0.0) alpha_r = 1.8;
  if (!std::isfinite(rho) || !std::isfinite(alpha_r) || alpha_r >= 2.0)
    return fail(ctx, SCSC_EINVAL, "rho = %g, alpha = %g outside rho > 0, 0 < alpha < 2", rho,
                alpha_r);
  if (ctx->cfg.flags & SCSC_FLAG_UNSAMPLED_KEEP)
    return fail(ctx, SCSC_EUNSUPPORTED, "the unsampled-keep variant has no ADMM step");
  CKS(stage_batch(ctx, batch));
  CKS(check_finite(ctx, x_dev, ctx->batch.view.total_px));
  CKS(check_finite(ctx, z_dev, ctx->batch.view.total_px * ctx->cfg.K));
  CKS(check_finite(ctx, d_dev, (int64_t)ctx->cfg.K * M_of(ctx)));
  if (ctx->batch.view.n > kMaxGridImages)
    return fail(ctx, SCSC_EINVAL, "ADMM: at most %d images per call", kMaxGridImages);
  CKS(build_mask(ctx, t));
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K, s = ctx->cfg.s;
  cudaStream_t st = ctx->stream;
  const int64_t DK = b.total_px * K;
  const size_t np = (size_t)b.n * kAdmmBlocks;  // partials per dot product
  CK(ctx->admm.ensure((size_t)7 * DK * 4));
  CK(ctx->r.ensure((size_t)b.total_px * 4));
  CK(ctx->admm_partials.ensure(4 * np * 8));
  float *const base = ctx->admm.as<float>();
  float *const y = base, *const u = base + DK, *const bv = base + 2 * DK, *const atx = base + 3 * DK,
              *const res = base + 4 * DK, *const pv = base + 5 * DK, *const Ap = base + 6 * DK;
  double *rr = ctx->admm_partials.as<double>(), *rr2 = rr + np, *pap = rr + 2 * np,
         *bb = rr + 3 * np;
  float *const pix = ctx->r.as<float>();
  const uint32_t *bits = ctx->bits.as<uint32_t>();
  const float frho = (float)rho;
  // Every image runs its own CG (per-image scalars, as in the per-image solver
  // of the paper); each launch covers the whole batch.
  // QP operator: out = m (D^T D (m in)) + rho m in
  auto apply_qp = [&](const float *in, float *out) -> scsc_status {
    int p1 = ctx->prof.begin(KID_SYNTH_FP32, st);
    CK(launch_synth_fp32(b, K, s, d_dev, in, bits, nullptr, pix, st));
    ctx->prof.end(p1, st);
    int p2 = ctx->prof.begin(KID_ADJ_FP32, st);
    CK(launch_adjoint_fp32(b, K, s, d_dev, pix, bits, 0, nullptr, out, st));
    ctx->prof.end(p2, st);
    CK(launch_admm_qp_finish(b, K, in, out, bits, frho, st));
    return SCSC_OK;
  };
  CK(launch_admm_init(b, K, z_dev, y, u, bits, st));
  CK(launch_adjoint_fp32(b, K, s, d_dev, x_dev, nullptr, 0, nullptr, atx, st));
  for (int it = 0; it < n_iters; ++it) {
    CK(launch_admm_rhs(b, K, atx, y, u, bv, bits, frho, st));
    CKS(apply_qp(z_dev, Ap));
    CK(launch_cg_init(b, K, bv, Ap, res, pv, st));
    CK(launch_seg_dot(b, K, res, res, rr, st));
    CK(launch_seg_dot(b, K, bv, bv, bb, st));
    for (int k = 0; k < cg_iters; ++k) {
      CKS(apply_qp(pv, Ap));
      CK(launch_seg_dot(b, K, pv, Ap, pap, st));
      CK(launch_cg_step(b, K, z_dev, res, pv, Ap, rr, pap, bb, st));
      CK(launch_seg_dot(b, K, res, res, rr2, st));
      CK(launch_cg_direction(b, K, pv, res, rr2, rr, bb, st));
      std::swap(rr, rr2);
    }
    CK(launch_admm_shrink(b, K, z_dev, y, u, bits, (float)alpha_r,
                          (float)(ctx->cfg.lambda / rho), st));
  }
  CK(launch_admm_final(b, K, z_dev, y, bits, st));
  return SCSC_OK;
}

// The screening test on the staged batch's active set `bits` (enqueued only):
// z <- z on the set (skipped when the caller knows z is zero off the set);
// r = D z - x; g = D^T r on the set; per-image gap and radius; bits and codes
// of the removed coordinates cleared; survivors counted into skept.
static scsc_status screen_enqueue(scsc_ctx *ctx, const float *x_dev, const float *d_dev,
                                  float *z_dev, uint32_t *bits, bool zero_off_set = true) {
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K, s = ctx->cfg.s;
  cudaStream_t st = ctx->stream;
  CK(ctx->r.ensure((size_t)b.total_px * 4));
  CK(ctx->sg.ensure((size_t)b.total_px * K * 4));
  CK(ctx->spref.ensure((size_t)K * (s + 1) * (s + 1) * 8));
  CK(ctx->snrm.ensure((size_t)K * 4));
  CK(ctx->spart.ensure((size_t)b.n * kScreenBlocks * 5 * 8));
  CK(ctx->simg.ensure((size_t)b.n * sizeof(ScreenImage)));
  CK(ctx->skept.ensure((size_t)b.n * 8));
  float *r = ctx->r.as<float>(), *g = ctx->sg.as<float>();
  if (zero_off_set) CK(launch_apply_mask_dense(b, K, bits, z_dev, st));
  CK(launch_screen_prepare(d_dev, K, s, ctx->spref.as<double>(), ctx->snrm.as<float>(), st));
  int p1 = ctx->prof.begin(KID_SYNTH_FP32, st);
  CK(launch_synth_fp32(b, K, s, d_dev, z_dev, nullptr, x_dev, r, st));
  ctx->prof.end(p1, st);
  int p2 = ctx->prof.begin(KID_ADJ_FP32, st);
  CK(launch_adjoint_fp32(b, K, s, d_dev, r, bits, 0, nullptr, g, st));
  ctx->prof.end(p2, st);
  int p3 = ctx->prof.begin(KID_SCREEN, st);
  CK(launch_screen_stats(b, K, x_dev, r, z_dev, g, bits, ctx->spart.as<double>(), st));
  CK(launch_screen_finish(b.n, ctx->spart.as<double>(), ctx->cfg.lambda,
                          ctx->simg.as<ScreenImage>(), st));
  CK(cudaMemsetAsync(ctx->skept.p, 0, (size_t)b.n * 8, st));
  CK(launch_screen_test(b, K, s, g, bits, z_dev, ctx->simg.as<ScreenImage>(),
                        ctx->spref.as<double>(), ctx->snrm.as<float>(),
                        ctx->skept.as<unsigned long long>(), st));
  ctx->prof.end(p3, st);
  return SCSC_OK;
}

// Per-image gaps and survivor counts of the last test, to the host.
static scsc_status screen_outputs(scsc_ctx *ctx, double *gap_host, int64_t *n_active_host) {
  const int n = ctx->batch.view.n;
  cudaStream_t st = ctx->stream;
  if (!gap_host && !n_active_host) return SCSC_OK;
  std::vector<ScreenImage> img(n);
  CK(cudaMemcpyAsync(img.data(), ctx->simg.p, (size_t)n * sizeof(ScreenImage),
                     cudaMemcpyDeviceToHost, st));
  if (n_active_host)
    CK(cudaMemcpyAsync(n_active_host, ctx->skept.p, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (gap_host)
    for (int i = 0; i < n; ++i) gap_host[i] = img[i].gap;
  return SCSC_OK;
}

scsc_status scsc_screen(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                        const float *d_dev, float *z_dev, uint32_t *bits_dev, double *gap_host,
                        int64_t *n_active_host) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_dev || !d_dev || !z_dev || !bits_dev) return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  CKS(stage_batch(ctx, batch));
  if (ctx->batch.view.n > kMaxGridImages)
    return fail(ctx, SCSC_EINVAL, "screening: at most %d images per call", kMaxGridImages);
  CKS(screen_enqueue(ctx, x_dev, d_dev, z_dev, bits_dev));
  return screen_outputs(ctx, gap_host, n_active_host);
}

scsc_status scsc_code_step_screened(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                    const float *d_dev, float *z_dev, uint64_t t, int n_iters,
                                    int screen_every, double *gap_host, int64_t *n_active_host) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_dev || !d_dev || !z_dev) return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  if (n_iters < 0) return fail(ctx, SCSC_EINVAL, "n_iters = %d < 0", n_iters);
  if (screen_every < 1) return fail(ctx, SCSC_EINVAL, "screen_every = %d < 1", screen_every);
  if (ctx->cfg.flags & SCSC_FLAG_UNSAMPLED_KEEP)
    return fail(ctx, SCSC_EUNSUPPORTED, "the unsampled-keep variant has no screened step");
  CKS(stage_batch(ctx, batch));
  if (ctx->batch.view.n > kMaxGridImages)
    return fail(ctx, SCSC_EINVAL, "screening: at most %d images per call", kMaxGridImages);
  CKS(build_mask(ctx, t));
  CKS(code_step_size(ctx, d_dev));
  uint32_t *bits = ctx->bits.as<uint32_t>();
  if (n_iters == 0) CK(launch_apply_mask_dense(ctx->batch.view, ctx->cfg.K, bits, z_dev,
                                               ctx->stream));
  for (int it = 0; it < n_iters; it += screen_every) {
    // after the first proximal-gradient chunk the codes are zero off the set
    CKS(screen_enqueue(ctx, x_dev, d_dev, z_dev, bits, /*zero_off_set=*/it == 0));
    const int chunk = std::min(screen_every, n_iters - it);
    CKS(code_step_impl(ctx, batch, x_dev, d_dev, z_dev, nullptr, t, chunk, /*keep_step=*/true,
                       /*keep_mask=*/true));
  }
  if (n_iters == 0) {
    if (gap_host || n_active_host)
      return fail(ctx, SCSC_EINVAL, "n_iters = 0: no screening test ran");
    return SCSC_OK;
  }
  return screen_outputs(ctx, gap_host, n_active_host);
}

scsc_status scsc_objective_observed(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                                    const float *z_dev, const float *d_dev,
                                    const uint8_t *observed_dev, double *out_host) {
  return objective_impl(ctx, batch, x_dev, z_dev, d_dev, observed_dev, out_host);
}

scsc_status scsc_synth(scsc_ctx *ctx, const scsc_batch *batch, const float *z_dev,
                       const float *d_dev, uint64_t t, int masked, float *xhat_dev) {
  if (!ctx) return SCSC_EINVAL;
  if (!z_dev || !d_dev || !xhat_dev) return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  CKS(stage_batch(ctx, batch));
  CKS(check_finite(ctx, z_dev, ctx->batch.view.total_px * ctx->cfg.K));
  CKS(check_finite(ctx, d_dev, (int64_t)ctx->cfg.K * M_of(ctx)));
  const uint32_t *bits = nullptr;
  if (masked) {
    CKS(build_mask(ctx, t));
    bits = ctx->bits.as<uint32_t>();
  }
  CK(launch_synth_fp32(ctx->batch.view, ctx->cfg.K, ctx->cfg.s, d_dev, z_dev, bits, nullptr,
                       xhat_dev, ctx->stream));
  return SCSC_OK;
}

scsc_status scsc_synth_backward(scsc_ctx *ctx, const scsc_batch *batch, const float *grad_dev,
                                const float *z_dev, const float *d_dev, uint64_t t, int masked,
                                float *grad_z_dev, float *grad_d_dev) {
  if (!ctx) return SCSC_EINVAL;
  if (!grad_dev || !d_dev || (grad_d_dev && !z_dev))
    return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  CKS(stage_batch(ctx, batch));
  CKS(check_finite(ctx, grad_dev, ctx->batch.view.total_px));
  if (grad_d_dev) CKS(check_finite(ctx, z_dev, ctx->batch.view.total_px * ctx->cfg.K));
  CKS(check_finite(ctx, d_dev, (int64_t)ctx->cfg.K * M_of(ctx)));
  const uint32_t *bits = nullptr;
  if (masked) {
    CKS(build_mask(ctx, t));
    bits = ctx->bits.as<uint32_t>();
  }
  const BatchDev &b = ctx->batch.view;
  if (grad_z_dev)
    CK(launch_adjoint_fp32(b, ctx->cfg.K, ctx->cfg.s, d_dev, grad_dev, bits, 0, nullptr,
                           grad_z_dev, ctx->stream));
  if (grad_d_dev) {
    CKS(filter_gradient(ctx, grad_dev, z_dev, bits));
    CK(launch_double_to_float(ctx->gsum.as<double>(), grad_d_dev, ctx->cfg.K * M_of(ctx),
                              ctx->stream));
  }
  return SCSC_OK;
}

scsc_status scsc_dict_step(scsc_ctx *ctx, const scsc_batch *batch, const float *x_dev,
                           const float *z_dev, float *d_dev, scsc_dict_mode mode, uint64_t t) {
  if (!ctx) return SCSC_EINVAL;
  if (!x_dev || !z_dev || !d_dev) return fail(ctx, SCSC_EINVAL, "NULL device pointer");
  if (mode != SCSC_DICT_BATCH && mode != SCSC_DICT_ONLINE && mode != SCSC_DICT_BATCH_GS)
    return fail(ctx, SCSC_EINVAL, "unknown dictionary mode %d", (int)mode);
  CKS(stage_batch(ctx, batch));
  const BatchDev &b = ctx->batch.view;
  const int K = ctx->cfg.K, s = ctx->cfg.s, M = M_of(ctx);
  CKS(check_finite(ctx, x_dev, b.total_px));
  CKS(check_finite(ctx, z_dev, b.total_px * K));
  CKS(check_finite(ctx, d_dev, (int64_t)K * M));
  cudaStream_t st = ctx->stream;
  CK(ctx->scal.ensure(8 * 8));
  if (mode == SCSC_DICT_BATCH) {
    CK(ctx->r.ensure((size_t)b.total_px * 4));
    CK(ctx->pix2.ensure((size_t)b.total_px * 4));
    CK(ctx->gsum.ensure((size_t)K * M * 8));
    CK(ctx->Cd.ensure((size_t)K * M * 8));
    // the operators on the nonzero codes where they are sparse enough
    CKS(build_sparse(ctx, z_dev));
    // r = D z - x, G = Z^T r (kept aside while the power iteration reuses gsum)
    scsc_status stt = dict_synth(ctx, d_dev, z_dev, x_dev, ctx->r.as<float>());
    if (stt == SCSC_OK) stt = dict_gradient(ctx, ctx->r.as<float>(), z_dev);
    if (stt == SCSC_OK &&
        cudaMemcpyAsync(ctx->Cd.p, ctx->gsum.p, (size_t)K * M * 8, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
      stt = fail(ctx, SCSC_ECUDA, "copy of the gradient failed");
    if (stt == SCSC_OK)
      stt = power_iteration(
          ctx, (int64_t)K * M, kTagLd,
          [&](const float *u, float *w) { return apply_ztz(ctx, z_dev, u, w); }, 1, nullptr, 0.0);
    ctx->sp_use = false;
    CKS(stt);
    CK(launch_project_step(d_dev, nullptr, ctx->Cd.as<double>(), ctx->scal.as<double>() + 1, K, M,
                           st));
    return SCSC_OK;
  }
  if (mode == SCSC_DICT_BATCH_GS) {
    CK(ctx->r.ensure((size_t)b.total_px * 4));
    CK(ctx->pix2.ensure((size_t)b.total_px * 4));
    CK(ctx->gpart.ensure((size_t)(kGradGroups + 1) * M * 4));
    CKS(build_sparse(ctx, z_dev));
    scsc_status stt = power_iteration(
        ctx, (int64_t)K * M, kTagLd,
        [&](const float *u, float *w) { return apply_ztz(ctx, z_dev, u, w); }, 1, nullptr, 0.0);
    ctx->sp_use = false;
    CKS(stt);
    // r = D z - x, then the blocks in order; the residual follows each block
    CK(launch_synth_fp32(b, K, s, d_dev, z_dev, nullptr, x_dev, ctx->r.as<float>(), st));
    float *partial = ctx->gpart.as<float>(), *delta = partial + (size_t)kGradGroups * M;
    for (int k = 0; k < K; ++k)
      CK(launch_gs_block(b, K, s, k, d_dev, z_dev, ctx->r.as<float>(), ctx->scal.as<double>() + 1,
                         partial, kGradGroups, delta, st));
    return SCSC_OK;
  }
  // Online (Eq. 7, Eq. 8)
  if (t < 1) return fail(ctx, SCSC_EINVAL, "online dictionary step needs t >= 1");
  if (t != ctx->online_t + 1)
    return fail(ctx, SCSC_EINVAL, "online step t = %llu does not follow the state's t = %llu",
                (unsigned long long)t, (unsigned long long)ctx->online_t);
  const int64_t KM = (int64_t)K * M;
  CK(ctx->C.ensure((size_t)KM * KM * 4));
  CK(ctx->B.ensure((size_t)KM * 8));
  CK(ctx->Cd.ensure((size_t)KM * 8));
  if (ctx->online_t == 0) {
    CK(cudaMemsetAsync(ctx->C.p, 0, (size_t)KM * KM * 4, st));
    CK(cudaMemsetAsync(ctx->B.p, 0, (size_t)KM * 8, st));
  }
  // on the nonzero codes where they are sparse enough, else the dense
  // implicit GEMM over every pixel
  CKS(build_sparse(ctx, z_dev));
  const double decay = (double)(t - 1) / (double)t, w_new = 1.0 / ((double)t * b.n);
  float *sp_corr = nullptr;  // the correlation buffer of the sparse update
  CorrSegments segs{};
  if (ctx->sp_use) {
    CK(ctx->sp_T.ensure(surrogate_corr_floats(K, s) * 4));
    sp_corr = ctx->sp_T.as<float>();
    surrogate_corr_segments(K, s, ctx->sp_nnz, &segs.seg_len, &segs.max_segments);
    CK(ctx->sp_seg.ensure((size_t)(K + 1) * 4));
    CK(ctx->sp_P.ensure((size_t)segs.max_segments * (surrogate_corr_floats(K, s) / K) * 4));
    segs.seg_off = ctx->sp_seg.as<int>();
    segs.P = ctx->sp_P.as<float>();
  }
  cudaError_t e =
      ctx->sp_use
          ? launch_surrogate_update_sparse(
                b, K, s, x_dev, ctx->sp_row.as<int64_t>(), ctx->sp_pk.as<int>(),
                ctx->sp_pv.as<float>(), ctx->sp_kt.as<int64_t>(), ctx->sp_kpix.as<int>(),
                ctx->sp_kimg.as<int>(), ctx->sp_kv.as<float>(), decay, w_new, ctx->C.as<float>(),
                ctx->B.as<double>(), sp_corr, &segs, st)
          : launch_surrogate_update(b, K, s, z_dev, x_dev, decay, w_new, ctx->C.as<float>(),
                                    ctx->B.as<double>(), st);
  ctx->sp_use = false;
  CK(e);
  CK(ctx->Cpart.ensure((size_t)symv_panels(KM) * KM * 4));
  float *cpart = ctx->Cpart.as<float>();
  CKS(power_iteration(ctx, KM, kTagLc,
                      [&](const float *u, float *w) -> scsc_status {
                        CK(launch_symv(ctx->C.as<float>(), KM, u, w, cpart, ctx->stream));
                        return SCSC_OK;
                      },
                      2, nullptr, 0.0));
  // grad = C d - B (FP64 accumulation), then the projected step
  CK(launch_symv_grad(ctx->C.as<float>(), KM, d_dev, ctx->B.as<double>(), ctx->Cd.as<double>(),
                      cpart, st));
  CK(launch_project_step(d_dev, nullptr, ctx->Cd.as<double>(), ctx->scal.as<double>() + 2, K, M, st));
  ctx->online_t = t;
  return SCSC_OK;
}

scsc_status scsc_sync(scsc_ctx *ctx) {
  if (!ctx) return SCSC_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->tc.err.p) {
    int word = 0;
    CK(cudaMemcpy(&word, ctx->tc.err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (word != 0)
      return fail(ctx, SCSC_ETIMEOUT, "a tensor-core kernel's bounded wait ran out");
  }
  return report_nonfinite(ctx);
}

scsc_status scsc_diag_profile(scsc_ctx *ctx, int enable) {
  if (!ctx) return SCSC_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.reset();
  ctx->prof.on = enable != 0;
  ctx->tc.prof = &ctx->prof;
  return SCSC_OK;
}

scsc_status scsc_diag_kernel_time(scsc_ctx *ctx, const char *name, double *total_ms,
                                  int *launches) {
  if (!ctx || !name || !total_ms || !launches) return SCSC_EINVAL;
  int id = kernel_id(name);
  if (id < 0) return fail(ctx, SCSC_EINVAL, "unknown kernel name '%s'", name);
  *total_ms = ctx->prof.total_ms(id, launches);
  return SCSC_OK;
}

scsc_status scsc_diag_tc_gemm(int N, const float *A_dev, const float *B_dev, float *D_dev) {
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return SCSC_ENOMEM;
  scsc_status s = SCSC_OK;
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
      tc_selftest_gemm(N, A_dev, B_dev, D_dev, err, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    s = SCSC_ECUDA;
  } else {
    int word = 0;
    if (cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) s = SCSC_ECUDA;
    else if (word) s = SCSC_ETIMEOUT;
  }
  cudaFree(err);
  return s;
}

scsc_status scsc_diag_tc_gemm_mn(int N, const float *A_dev, const float *B_dev, float *D_dev,
                                 int swap) {
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return SCSC_ENOMEM;
  scsc_status s = SCSC_OK;
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
      tc_selftest_gemm_mn(N, A_dev, B_dev, D_dev, swap != 0, err, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    s = SCSC_ECUDA;
  } else {
    int word = 0;
    if (cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) s = SCSC_ECUDA;
    else if (word) s = SCSC_ETIMEOUT;
  }
  cudaFree(err);
  return s;
}

scsc_status scsc_diag_mma_rate(int N, int layout, double *issue_cycles, double *complete_cycles) {
  if (!complete_cycles || N < 16 || N > 256 || N % 16 != 0 || layout < 0 || layout > 2)
    return SCSC_EINVAL;
  const int reps = 64;
  int *err = nullptr;
  long long *out = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return SCSC_ENOMEM;
  if (cudaMalloc(&out, 2 * sizeof(long long)) != cudaSuccess) {
    cudaFree(err);
    return SCSC_ENOMEM;
  }
  scsc_status s = SCSC_OK;
  long long h[2] = {0, 0};
  int word = 0;
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
      tc_selftest_mma_rate(N, layout, reps, out, err, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(h, out, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) {
    s = SCSC_ECUDA;
  } else if (word) {
    s = SCSC_ETIMEOUT;
  } else {
    if (issue_cycles) *issue_cycles = (double)h[0] / reps;
    *complete_cycles = (double)h[1] / reps;
  }
  cudaFree(out);
  cudaFree(err);
  return s;
}

scsc_status scsc_diag_wait_timeout(double limit_ms) {
  if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) return SCSC_EINVAL;
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return SCSC_ENOMEM;
  scsc_status s = SCSC_OK;
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
      tc_selftest_wait((uint64_t)(limit_ms * 1e6), err, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    s = SCSC_ECUDA;
  } else {
    int word = 0;
    if (cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) s = SCSC_ECUDA;
    else if (word) s = SCSC_ETIMEOUT;
  }
  cudaFree(err);
  return s;
}

scsc_status scsc_online_reset(scsc_ctx *ctx) {
  if (!ctx) return SCSC_EINVAL;
  ctx->online_t = 0;
  return SCSC_OK;
}

scsc_status scsc_online_state_size(scsc_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return SCSC_EINVAL;
  size_t KM = (size_t)ctx->cfg.K * M_of(ctx);
  *bytes = 4 * 4 + 8 + KM * KM * 4 + KM * 8;
  return SCSC_OK;
}

scsc_status scsc_online_save(scsc_ctx *ctx, void *host_buf, size_t bytes) {
  if (!ctx) return SCSC_EINVAL;
  size_t need;
  scsc_online_state_size(ctx, &need);
  if (!host_buf || bytes < need) return fail(ctx, SCSC_EINVAL, "state buffer needs %zu bytes", need);
  size_t KM = (size_t)ctx->cfg.K * M_of(ctx);
  unsigned char *q = static_cast<unsigned char *>(host_buf);
  uint32_t hdr[4] = {kStateMagic, (uint32_t)ctx->cfg.K, (uint32_t)ctx->cfg.s, 0};
  memcpy(q, hdr, 16);
  memcpy(q + 16, &ctx->online_t, 8);
  if (ctx->online_t == 0) {
    memset(q + 24, 0, KM * KM * 4 + KM * 8);
    return SCSC_OK;
  }
  CK(cudaMemcpyAsync(q + 24, ctx->C.p, KM * KM * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(q + 24 + KM * KM * 4, ctx->B.p, KM * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SCSC_OK;
}

scsc_status scsc_online_load(scsc_ctx *ctx, const void *host_buf, size_t bytes) {
  if (!ctx) return SCSC_EINVAL;
  size_t need;
  scsc_online_state_size(ctx, &need);
  if (!host_buf || bytes < need) return fail(ctx, SCSC_EINVAL, "state buffer needs %zu bytes", need);
  const unsigned char *q = static_cast<const unsigned char *>(host_buf);
  uint32_t hdr[4];
  memcpy(hdr, q, 16);
  if (hdr[0] != kStateMagic || (int)hdr[1] != ctx->cfg.K || (int)hdr[2] != ctx->cfg.s)
    return fail(ctx, SCSC_EINVAL, "state was saved for another K or s");
  uint64_t t;
  memcpy(&t, q + 16, 8);
  size_t KM = (size_t)ctx->cfg.K * M_of(ctx);
  CK(ctx->C.ensure(KM * KM * 4));
  CK(ctx->B.ensure(KM * 8));
  CK(cudaMemcpyAsync(ctx->C.p, q + 24, KM * KM * 4, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->B.p, q + 24 + KM * KM * 4, KM * 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->online_t = t;
  return SCSC_OK;
}

}  // extern "C"
