// lrfsi_residual_batch_noalloc: the batched nonlinear residual and its column
// norms without any device allocation.
//
// Some callers cannot let a library allocate device memory: applications
// whose device memory is owned by their own pool allocator (a framework's
// caching allocator, a serving process with a fixed memory budget) must not
// have memory taken or returned behind that allocator's back, and a
// cudaMalloc or cudaFree in the middle of their stream work would also
// synchronise the device.  lrfsi_residual_batch allocates a temporary block
// for the per-row-block partial sums of the column norms on every call; this
// variant keeps those partial sums in a file-scope device array instead and
// requires the caller to pass the residual output.
#include <mutex>

#include "mesh.h"

namespace lrfsi {

// Partial sums of the column norms: colnorm_work_len(M, m) = ceil(M / 256) x m
// doubles per call.
constexpr size_t kNoallocScratch = size_t(1) << 21;  // doubles (16 MiB per device, held until exit)
static __device__ __align__(256) double g_norm_partials[kNoallocScratch];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[128] = {nullptr};

// Device address of the scratch array for the current device, looked up once
// per device (with that device current) and cached for the life of the
// process.  Host code may not use the symbol itself: on the host it names a
// stand-in, not device memory.  The cached address belongs to the device's
// primary context, so the library must not be used across cudaDeviceReset.
static int noalloc_scratch(double** out) {
  int dev = 0;
  LRFSI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(LRFSI_EINVAL, "lrfsi_residual_batch_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_norm_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_norm_partials)");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return LRFSI_OK;
}

}  // namespace lrfsi

using namespace lrfsi;

extern "C" int lrfsi_residual_batch_noalloc(lrfsi_mesh_h m, const double* X, int ldx, int ncol, const double* mu,
                                            const double* nu, double* R, int ldr, double* norm2,
                                            lrfsi_stream_t stream) {
  if (!m || !X || !mu || !nu || !R || ncol < 0 || ldx < ncol || ldr < ncol)
    return fail(LRFSI_EINVAL, "lrfsi_residual_batch_noalloc: bad argument (R is required, ldx, ldr >= ncol)");
  if (ncol == 0) return LRFSI_OK;
  const size_t need = colnorm_work_len(m->h.M, ncol);
  if (norm2 && need > kNoallocScratch)
    return fail(LRFSI_EINVAL, "lrfsi_residual_batch_noalloc: ceil(M/256) * ncol exceeds the 2^21-double scratch; "
                              "use lrfsi_residual_batch or fewer columns per call");
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  LRFSI_TRY(noalloc_scratch(&scratch));
  LRFSI_TRY(launch_residual(m, X, ldx, ncol, nullptr, mu, nu, R, ldr, s));
  // every partial read below is written by this call's first kernel, so the
  // scratch needs no clearing
  if (norm2) LRFSI_TRY(launch_colnorm2(R, m->h.M, ncol, ldr, norm2, scratch, kNoallocScratch, s));
  return LRFSI_OK;
}
