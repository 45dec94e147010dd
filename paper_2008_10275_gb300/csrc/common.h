// Internal helpers shared by the lrfsi translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lrfsi.h"

namespace lrfsi {

// ---- error reporting -------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define LRFSI_CUDA(call)                                        \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::lrfsi::cuda_fail(e_, #call); \
  } while (0)

#define LRFSI_TRY(call)              \
  do {                               \
    int s_ = (call);                 \
    if (s_ != LRFSI_OK) return s_;   \
  } while (0)

// per-class accounting (see lrfsi_stats); timed_begin/timed_end bracket a
// launch with events when timing is enabled
// KC_LU, KC_LUSOLVE and KC_SVD time whole regions that contain launches of
// other classes (they overlap those classes); the rest time single launches.
// KC_GEMM_TC / KC_GRAM_TC time the whole tensor-core pipelines of FP64 GEMMs
// and Gram products (exponents, slices, slice products, combination) and
// count their FP64 algorithmic FLOPs; KC_TCMMA times the slice-product
// kernels inside them and counts the BF16 MMA FLOPs they issue.
enum KClass {
  KC_GEMM = 0, KC_SPMM = 1, KC_GRAM = 2, KC_LU = 3, KC_FE = 4, KC_GEMM32 = 5, KC_SPMM32 = 6, KC_TRUNC = 7,
  KC_LUPANEL = 8, KC_LUTRSM = 9, KC_LUSOLVE = 10, KC_SVD = 11, KC_TCMMA = 12, KC_GEMM_TC = 13, KC_GRAM_TC = 14
};
constexpr int kNumKClasses = 15;
void account(int cls, double flops, double bytes);
struct TimedLaunch {
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedLaunch(int c, cudaStream_t s);
  void end(cudaStream_t s);
};

// every kernel launch goes through count_launch() so that the process-wide
// launch counter (lrfsi_kernel_launches) is exact
void count_launch(uint64_t n = 1);
inline int check_launch(const char* name) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, name);
  return LRFSI_OK;
}

// ---- device-side run conditions ---------------------------------------------
// A batched descriptor's work runs only if each non-null flag is nonzero: the
// per-subset "still iterating" flag of a solve whose launch sequence is fixed
// (and captured in a CUDA graph), and optional passes of the truncation that
// the device decides on.  A gated-off descriptor leaves its outputs untouched.
struct Gate {
  const int* a = nullptr;
  const int* b = nullptr;
};
#ifdef __CUDACC__
__host__ __device__ inline bool gate_open(const Gate& g) { return (!g.a || *g.a) && (!g.b || *g.b); }
#endif
// While kernel timing is on (lrfsi_timing), the algorithmic work of a gated
// descriptor is counted only if its gate is open: the flags are read back
// (synchronising the stream).  Without timing every descriptor counts.
bool timing_enabled();
bool gate_counts(const Gate& g, cudaStream_t s);

// ---- device buffers --------------------------------------------------------
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    release();
    if (count == 0) return LRFSI_OK;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(LRFSI_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    n = count;
    return LRFSI_OK;
  }
  int upload(const std::vector<T>& h, cudaStream_t s = 0) {
    LRFSI_TRY(alloc(h.size()));
    if (!h.empty()) LRFSI_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return LRFSI_OK;
  }
  size_t bytes() const { return n * sizeof(T); }
  void swap(DevBuf& o) {
    T* tp = p; p = o.p; o.p = tp;
    size_t tn = n; n = o.n; o.n = tn;
  }
};

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace lrfsi
