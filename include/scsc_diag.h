/*
 * scsc_diag.h -- diagnostic entry points of the SCSC library.
 *
 * scsc_diag_tc_gemm runs one tcgen05 matrix multiply through the same
 * shared-memory descriptor, instruction descriptor and TMEM read-back code
 * that the tensor-core code update uses, so that their encodings can be
 * checked on the device against a plain product:
 *     D[128 x N] = A[128 x 64] * B[N x 64]^T,
 * A, B float32 row-major device arrays whose values are rounded to BF16,
 * D float32 row-major [128][N] device array, N a multiple of 16 in [16, 256].
 * Runs on the legacy default stream and synchronises the device.  Returns
 * SCSC_OK, SCSC_ENOMEM if its one-word error flag cannot be allocated,
 * SCSC_ECUDA on an invalid N or a launch error, SCSC_ETIMEOUT if the MMA's
 * completion barrier was not reached within one second.  The paper has no
 * counterpart: this checks the build's instruction encodings.
 */
#ifndef SCSC_DIAG_H
#define SCSC_DIAG_H
#include "scsc.h"

#ifdef __cplusplus
extern "C" {
#endif

scsc_status scsc_diag_tc_gemm(int N, const float *A_dev, const float *B_dev, float *D_dev);

/* scsc_diag_tc_gemm_mn: the same product with B held MN-major in shared
 * memory (the N index contiguous inside each core matrix), the layout in
 * which the synthesis reads the adjoint's filter image.  swap = 0 puts the
 * K-direction core stride in the descriptor's leading-dimension offset field
 * and the N-direction stride in the stride-dimension field; swap = 1 the
 * other way round.  Returns as scsc_diag_tc_gemm. */
scsc_status scsc_diag_tc_gemm_mn(int N, const float *A_dev, const float *B_dev, float *D_dev,
                                 int swap);

/* scsc_diag_wait_timeout launches one block whose thread waits on a
 * shared-memory mbarrier that nothing arrives on, through the bounded wait
 * every tensor kernel uses, with a limit of limit_ms milliseconds (0 <
 * limit_ms <= 1000).  The wait gives up at the limit and raises the kernel's
 * error word, which the host reads.  Returns SCSC_ETIMEOUT when the wait ran
 * out (the expected outcome), SCSC_OK if it did not, SCSC_EINVAL for a bad
 * limit, SCSC_ENOMEM / SCSC_ECUDA as scsc_diag_tc_gemm.  Runs on the legacy
 * default stream and synchronises the device; the context stays usable. */
scsc_status scsc_diag_wait_timeout(double limit_ms);

/* Per-kernel timing.  scsc_diag_profile(ctx, 1) synchronises the context's
 * stream, clears the records and from then on brackets every launch of the
 * library's kernels with a pair of CUDA events on that stream; 0 turns it
 * off.  scsc_diag_kernel_time() waits for the recorded events and returns the
 * summed device time and the launch count of one kernel, named "mask",
 * "power", "synth_fp32", "adjoint_fp32", "pack", "synth_tc", "finalize_r",
 * "adj_tc", "unpack" or "screen" (SCSC_EINVAL for another name). */
scsc_status scsc_diag_profile(scsc_ctx *ctx, int enable);
scsc_status scsc_diag_kernel_time(scsc_ctx *ctx, const char *name, double *total_ms,
                                  int *launches);

/* scsc_diag_mma_rate times 64 back-to-back tcgen05 MMAs of shape M = 128,
 * K = 16 and the given N (a multiple of 16 in [16, 256]) issued by one
 * thread of one CTA, on zero BF16 operands in shared memory, after one
 * untimed round.  layout 0: both operands K-major (no swizzle); 1: A is the
 * overlapping Toeplitz view the adjoint uses (core-matrix strides of 128
 * bytes in both directions), B K-major; 2: A K-major, B MN-major (the
 * synthesis's filter operand).  *issue_cycles (may be NULL) receives the SM
 * cycles per MMA until the last one was issued, *complete_cycles the cycles
 * per MMA until their completion barrier.  Runs on the legacy default stream
 * and synchronises the device.  Returns SCSC_OK, SCSC_EINVAL for a bad N,
 * layout or NULL complete_cycles, SCSC_ENOMEM, SCSC_ECUDA, or SCSC_ETIMEOUT
 * if the completion barrier was not reached within one second.  The paper
 * has no counterpart: this measures the tensor core's rate for the MMA
 * shapes the code update issues. */
scsc_status scsc_diag_mma_rate(int N, int layout, double *issue_cycles, double *complete_cycles);

/* scsc_diag_ffma_peak measures the FP32 fused multiply-add rate of the
 * current device: a SIMT kernel of independent FMA chains (4 blocks of 512
 * threads per SM), the fastest of five launches timed with CUDA events after
 * one warm-up launch on the legacy default stream.  *tflops receives
 * 2 x FMAs / time in TFLOP/s, *ms (may be NULL) the kernel time.  This is the
 * denominator of the plain FP32 path's roofline fraction, whose synthesis and
 * adjoint are FMA-bound.  Returns SCSC_OK, SCSC_EINVAL for a NULL tflops,
 * SCSC_ENOMEM if its output buffer cannot be allocated, SCSC_ECUDA on a CUDA
 * error.  The paper has no counterpart: this measures the hardware. */
scsc_status scsc_diag_ffma_peak(double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif
