// scsc_tc.cuh -- the tensor-core (tcgen05, BF16 operands, FP32 accumulation)
// code-update path and the small helpers shared with the plain path.
#pragma once
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "profiler.cuh"
#include "scsc_internal.cuh"

namespace scsc {

// Autotuner key: device, K, s, log2 of the number of row items.
struct TuneKey {
  int dev, K, s, qclass;
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, K, s, qclass) < std::tie(o.dev, o.K, o.s, o.qclass);
  }
};

// Everything a captured iteration graph depends on (the buffers it names and
// the by-value launch arguments that follow from the batch shape).
struct GraphKey {
  const void *bits, *seg_base, *pxoff, *packed, *bsyn, *badj, *xcore, *spill, *r, *err, *x, *prm,
      *item0, *off, *obs, *abuf;
  const void *v16a, *v16b, *idx16, *xcore2, *spill2;  // fused path
  int64_t total_px;
  int n_images, K, s, Q, variant, iters;
  int a_chunks, stage_s, stage_a;  // shared-memory layout of the single-stage kernels
};

// A few captured graphs, reused while their key matches (the host-buffer
// entry alternates between two chunk buffers).
struct GraphSlot {
  GraphKey key{};
  cudaGraphExec_t exec = nullptr;
  uint64_t used = 0;
};
constexpr int kGraphSlots = 4;

// Workspace of the tensor path, owned by the context.
struct TcWorkspace {
  struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
  };
  Buf item0, seg_count, seg_base, pxoff, scan_blocks, packed, xcore, spill, r, badj, bsyn, err;
  Buf abuf;  // dense BF16 code tiles in the synthesis A-operand layout (pipelined kernels)
  // fused path: BF16 packed codes (input / output iterate), their A-tile
  // indices, and the second set of synthesis buffers
  Buf v16[2], idx16, xcore2, spill2;
  std::vector<int> host_item0;  // cached row-item map of the last batch
  std::vector<int> host_H, host_W;
  int n_items = 0;
  int sm_count = 0;
  int max_smem = 0;
  int smem_sm = 0;  // shared memory per SM
  Profiler *prof = nullptr;  // the owning context's profiler
  bool autotune = true, graphs = true, fused = true;
  // sampling rate p of the code step (set by the caller before each call):
  // the fused kernel is chosen only while an item's expected sampled codes,
  // 128 K p, fit one of its staging chunks (4096 values); at higher p the
  // two-kernel path is the faster one (C3 at p = 1/4: 632 vs 509
  // Gpix*filter/s; inpainting at p = 1: 141 vs 277)
  double sample_p = 1.0;
  std::map<TuneKey, int> tune;                       // chosen variant per key
  std::map<TuneKey, std::pair<float, float>> tune_ms;  // timings that chose it
  GraphSlot graphs_cached[kGraphSlots];
  uint64_t graph_clock = 0;
  std::string last_error;
};

// One outer iteration of the code update on the tensor path (see
// scsc_code_step): pack the warm start on the sampled set, n_iters
// proximal-gradient iterations on packed FP32 codes with BF16 tcgen05
// synthesis and adjoint, unpack to dense codes (Eq. 4).
// H_host / W_host are the batch's host arrays (n images).
// obs: one byte per pixel, nonzero = observed (data term on observed pixels
// only); NULL = every pixel observed.  keep_unsampled: codes off the sampled
// set are left as they are instead of zeroed (x must then already exclude
// their contribution).  *nonfinite |= 1 when a warm-start code is NaN or Inf.
cudaError_t tc_code_step(TcWorkspace &ws, const BatchDev &b, const int *H_host, const int *W_host,
                         int K, int s, const float *x, const float *d, float *z,
                         const uint32_t *bits, const uint8_t *obs, const StepParams *prm,
                         int n_iters, bool keep_unsampled, int *nonfinite, cudaStream_t st);
// Device error word of the tensor kernels (0 = ok, 1 = bounded wait ran out).
int *tc_error_word(TcWorkspace &ws);
void tc_release(TcWorkspace &ws);
const char *tc_last_error(const TcWorkspace &ws);

// D[128 x N] = A[128 x 64] * B[N x 64]^T through one tcgen05 pipeline (BF16
// operands rounded from the float inputs, FP32 accumulation); device buffers.
cudaError_t tc_selftest_gemm(int N, const float *A, const float *B, float *D, int *err,
                             cudaStream_t st);
// The same product with B stored MN-major (swap: which descriptor field holds
// the K-direction core stride).
cudaError_t tc_selftest_gemm_mn(int N, const float *A, const float *B, float *D, int swap,
                                int *err, cudaStream_t st);
// One bounded mbarrier wait that nothing completes: sets *err after limit_ns.
cudaError_t tc_selftest_wait(uint64_t limit_ns, int *err, cudaStream_t st);
cudaError_t tc_selftest_mma_rate(int N, int layout, int reps, long long *out, int *err,
                                 cudaStream_t st);

// Pipelined tensor kernels (kernels_tc_pipe.cu): K <= 128 and shared memory
// within `max_smem` bytes per block.
bool tc_pipe_supported(int K, int s, int max_smem);

// Helpers implemented in kernels_online.cu.
cudaError_t launch_surrogate_update(const BatchDev &b, int K, int s, const float *z, const float *x,
                                    double alpha, double beta, float *Cm, double *Bv,
                                    cudaStream_t st);
// The correlations walk each filter's nonzeros in segments of seg_len, each
// into its own slice of P (max_segments slices of K * (2s-1)^2 floats);
// seg_off holds K + 1 ints.
struct CorrSegments {
  int seg_len;
  int64_t max_segments;
  int *seg_off;
  float *P;
};
void surrogate_corr_segments(int K, int s, int64_t nnz, int *seg_len, int64_t *max_segments);
// The same update from the index of the nonzero codes (dictionary-step index
// of kernels_sparse.cu) in the correlation form: O(nnz * (2s-1)^2 * nonzeros
// per pixel) plus the patches centred outside the image.  T holds
// surrogate_corr_floats(K, s) floats.
cudaError_t launch_surrogate_update_sparse(const BatchDev &b, int K, int s, const float *x,
                                           const int64_t *row_ptr, const int *pk, const float *pv,
                                           const int64_t *kt_off, const int *kpix,
                                           const int *kimg, const float *kv, double alpha,
                                           double beta, float *Cm, double *Bv, float *T,
                                           const CorrSegments *segs, cudaStream_t st);
// Floats of the correlation buffer T of that update (K * K * (2s-1)^2).
size_t surrogate_corr_floats(int K, int s);
// out = C v (FP32 out) and out = C d - B (FP64 out) for the symmetric C of
// order n, from its upper block triangle; part holds symv_panels(n) * n
// floats of partial sums.
int symv_panels(int64_t n);
cudaError_t launch_symv(const float *Cm, int64_t n, const float *v, float *out, float *part,
                        cudaStream_t st);
cudaError_t launch_symv_grad(const float *Cm, int64_t n, const float *d, const double *Bv,
                             double *out, float *part, cudaStream_t st);
cudaError_t launch_double_to_float(const double *in, float *out, int n, cudaStream_t st);
cudaError_t launch_set_step(StepParams *prm, double step, double lambda, cudaStream_t st);

}  // namespace scsc
