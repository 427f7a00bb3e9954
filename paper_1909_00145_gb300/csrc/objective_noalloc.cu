// objective_noalloc.cu -- the objective of Eq. 1 for a batch of equal-size
// images, computed without allocating device memory.
//
// Some callers cannot call cudaMalloc: code running inside stream capture,
// services whose memory pool already reserves the whole device, and loops that
// cannot afford the implicit synchronisation of an allocation.  This entry
// point serves them.  Its scratch (the per-tile partial sums) lives in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.  Calls share that array: calls that overlap on the
// GPU race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/scsc.h"
#include "scsc_internal.cuh"

namespace {

constexpr int kTile = 32;
constexpr int kMaxTiles = 65536;       // 32x32 tiles: up to 67,108,864 pixels per call
constexpr int kAbsBlocks = 1024;
constexpr int kMaxDevices = 64;

// Partial sums of one call: [0, kMaxTiles) residual^2 per tile,
// [kMaxTiles, kMaxTiles + kAbsBlocks) |z| per block.
static __device__ __align__(256) double g_scratch[kMaxTiles + kAbsBlocks];

std::mutex g_mu;
// Cached address of g_scratch per device, with the id of the CUDA context it
// was looked up in: a device reset (or any new primary context) reloads the
// module, so an address from an older context is stale and is looked up anew.
struct ScratchSlot {
  double *ptr = nullptr;
  unsigned long long ctx_id = 0;
  bool have_id = false;
};
ScratchSlot g_slot[kMaxDevices];

// Per-tile sum of (D z - x)^2 over one 32x32 tile of image n = tile / tiles_per_image.
template <int S>
__global__ void __launch_bounds__(128) residual_sq_tiles_kernel(int K, int H, int W,
                                                                const float *__restrict__ d,
                                                                const float *__restrict__ z,
                                                                const float *__restrict__ x,
                                                                double *__restrict__ part) {
  constexpr int C = (S - 1) / 2;
  constexpr int HS = kTile + S - 1;
  constexpr int R = 8;
  constexpr int KC = 4;
  __shared__ float zs[KC][HS][HS + 1];
  __shared__ float ds[KC][S * S];
  __shared__ double red[4];
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  const int per_image = tiles_x * tiles_y;
  const int n = blockIdx.x / per_image, lt = blockIdx.x - n * per_image;
  const int y0 = (lt / tiles_x) * kTile, x0 = (lt % tiles_x) * kTile;
  const int64_t base = (int64_t)n * H * W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += KC) {
    __syncthreads();
    for (int i = threadIdx.x; i < HS * HS; i += blockDim.x) {
      int hy = i / HS, hx = i - hy * HS;
      int yy = y0 - C + hy, xx = x0 - C + hx;
      bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
      int64_t pix = base + (int64_t)yy * W + xx;
#pragma unroll
      for (int kk = 0; kk < KC; ++kk)
        zs[kk][hy][hx] = (in && k0 + kk < K) ? z[pix * K + k0 + kk] : 0.0f;
    }
    for (int i = threadIdx.x; i < KC * S * S; i += blockDim.x) {
      int kk = i / (S * S), m = i - kk * S * S;
      ds[kk][m] = (k0 + kk < K) ? d[(int64_t)(k0 + kk) * S * S + m] : 0.0f;
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
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int i = y0 + ty * R + r, j = x0 + tx;
    if (i < H && j < W) {
      double rv = (double)acc[r] - (double)x[base + (int64_t)i * W + j];
      s += rv * rv;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (tx == 0) red[ty] = s;
  __syncthreads();
  if (threadIdx.x == 0) part[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

__global__ void __launch_bounds__(256) abs_sum_kernel(const float *__restrict__ z, int64_t n,
                                                      double *__restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += fabs((double)z[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

__global__ void finish_kernel(const double *__restrict__ part, int n_tiles, double lambda,
                              double *__restrict__ out) {
  __shared__ double red[2][32];
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) s += part[i];
  for (int i = threadIdx.x; i < kAbsBlocks; i += blockDim.x) t += part[kMaxTiles + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    t += __shfl_down_sync(0xffffffffu, t, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)blockDim.x / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    *out = 0.5 * a + lambda * b;
  }
}

// Id of the CUDA context current on this thread (driver entry points fetched
// through the runtime, so the library does not link the driver library).
// False when no context is current or the entry points are unavailable.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
bool current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    looked_up = true;
  }
  if (!get_current || !get_id) return false;
  void *ctx = nullptr;
  if (get_current(&ctx) != 0 || ctx == nullptr) return false;
  return get_id(ctx, id) == 0;
}

// Address of the scratch array on the current device.  Looked up with that
// device current on the first call, and again whenever the device's current
// context is not the one of the cached address (after a device reset), or on
// every call where the context id cannot be read.
scsc_status scratch_for_current_device(double **ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCSC_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return SCSC_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  ScratchSlot &slot = g_slot[dev];
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  if (slot.ptr == nullptr || !have_id || !slot.have_id || slot.ctx_id != id) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return SCSC_ECUDA;
    // the lookup makes the device's primary context current if none was
    if (!have_id) have_id = current_context_id(&id);
    slot.ptr = static_cast<double *>(p);
    slot.ctx_id = id;
    slot.have_id = have_id;
  }
  *ptr = slot.ptr;
  return SCSC_OK;
}

}  // namespace

extern "C" scsc_status scsc_objective_noalloc(const scsc_config *cfg, int n_images, int H, int W,
                                              const float *x_dev, const float *z_dev,
                                              const float *d_dev, double *out_dev,
                                              void *cuda_stream) {
  if (!cfg || !x_dev || !z_dev || !d_dev || !out_dev) return SCSC_EINVAL;
  const int K = cfg->K, s = cfg->s;
  if (K < 1 || K > scsc::kMaxK || s < 1 || s > scsc::kMaxS || s % 2 == 0) return SCSC_EINVAL;
  if (!(cfg->lambda > 0.0)) return SCSC_EINVAL;
  if (n_images < 1 || H < 1 || W < 1) return SCSC_EINVAL;
  const int64_t tiles =
      (int64_t)n_images * ((H + kTile - 1) / kTile) * (int64_t)((W + kTile - 1) / kTile);
  if (tiles > kMaxTiles) return SCSC_EINVAL;  // beyond the static scratch: see scsc.h
  double *part = nullptr;
  scsc_status st = scratch_for_current_device(&part);
  if (st != SCSC_OK) return st;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int64_t npx = (int64_t)n_images * H * W;
  switch (s) {
#define SCSC_CASE(SV)                                                                        \
  case SV:                                                                                   \
    residual_sq_tiles_kernel<SV><<<(unsigned)tiles, 128, 0, stream>>>(K, H, W, d_dev, z_dev, \
                                                                      x_dev, part);          \
    break;
    SCSC_CASE(1)
    SCSC_CASE(3)
    SCSC_CASE(5)
    SCSC_CASE(7)
    SCSC_CASE(9)
    SCSC_CASE(11)
#undef SCSC_CASE
    default: return SCSC_EINVAL;
  }
  if (cudaGetLastError() != cudaSuccess) return SCSC_ECUDA;
  abs_sum_kernel<<<kAbsBlocks, 256, 0, stream>>>(z_dev, npx * K, part + kMaxTiles);
  if (cudaGetLastError() != cudaSuccess) return SCSC_ECUDA;
  finish_kernel<<<1, 256, 0, stream>>>(part, (int)tiles, cfg->lambda, out_dev);
  if (cudaGetLastError() != cudaSuccess) return SCSC_ECUDA;
  return SCSC_OK;
}
