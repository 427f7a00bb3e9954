// profiler.cuh -- optional per-kernel timing with CUDA events recorded on the
// launching stream around each launch (diagnostic; off by default).
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

namespace scsc {

enum KernelId {
  KID_MASK = 0,
  KID_POWER,
  KID_SYNTH_FP32,
  KID_ADJ_FP32,
  KID_PACK,
  KID_SYNTH_TC,
  KID_FINALIZE,
  KID_ADJ_TC,
  KID_UNPACK,
  KID_SCREEN,
  KID_FUSED,
  KID_COUNT
};

inline const char *kernel_name(int id) {
  static const char *names[KID_COUNT] = {"mask",     "power",    "synth_fp32", "adjoint_fp32",
                                         "pack",     "synth_tc", "finalize_r", "adj_tc",
                                         "unpack",   "screen",   "fused"};
  return (id >= 0 && id < KID_COUNT) ? names[id] : "";
}

inline int kernel_id(const char *name) {
  for (int i = 0; i < KID_COUNT; ++i)
    if (std::strcmp(name, kernel_name(i)) == 0) return i;
  return -1;
}

struct Profiler {
  bool on = false;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;

  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  // Returns the record index, or -1 when profiling is off.
  int begin(int id, cudaStream_t st) {
    if (!on) return -1;
    Rec r{id, take(), take()};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, st);
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(recs[idx].b, st);
  }
  void reset() {
    recs.clear();
    used = 0;
  }
  double total_ms(int id, int *count) {
    double t = 0.0;
    int n = 0;
    for (const Rec &r : recs) {
      if (r.id != id) continue;
      float ms = 0.0f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        t += ms;
        ++n;
      }
    }
    if (count) *count = n;
    return t;
  }
  void release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    recs.clear();
    used = 0;
  }
};

}  // namespace scsc
