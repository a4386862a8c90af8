// numa_rhs_static_scratch: the right-hand side with its scratch (primitive
// fields and element residuals) in a fixed, library-owned device array
// instead of the caller's workspace.
//
// Who needs this: callers that cannot allocate device memory themselves --
// code that runs while a CUDA graph is being captured, real-time loops that
// forbid allocation after start-up, or plug-ins whose host application owns
// all device memory and hands them only input and output buffers.  Such a
// caller cannot make room for a second residual scratch next to the one in
// the bound workspace (which numa_rk_step and numa_run use), so this entry
// point evaluates R = dq/dt on the caller's own buffers with a scratch array
// that is part of the library image: nothing is allocated per call.
//
// The array is 16 MiB: 40 bytes per global node of primitive fields plus 40
// (FP64) or 20 (FP32-mixed) bytes per element node of residuals, about 2,200
// elements at N=4.  Every GPU that loads this library keeps it until the
// process exits.  All calls share it: two calls whose work overlaps on the
// GPU (different streams, or different contexts) race on it.  Nothing in it
// needs clearing between calls: each call overwrites every primitive and
// residual entry before the next kernel reads it.
#include <mutex>
#include <string>

#include "numa_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = NUMA_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) double g_static_re[kStaticScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of g_static_re on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must not be passed to a
// kernel).
cudaError_t static_scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_re);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

namespace numa {
// Implemented in numa_api.cu: the two RHS launches with a given residual buffer.
int rhs_with_scratch(numa_ctx* ctx, const double* q_dev, double* r_dev, double* re_scratch,
                     long long scratch_doubles);
}  // namespace numa

extern "C" int numa_rhs_static_scratch(numa_ctx* ctx, const double* q_dev, double* r_dev) {
  if (!ctx || !q_dev || !r_dev) return NUMA_EINVAL;
  double* re = nullptr;
  cudaError_t e = static_scratch_address(&re);
  if (e != cudaSuccess) return NUMA_ECUDA;
  return numa::rhs_with_scratch(ctx, q_dev, r_dev, re, (long long)(kStaticScratchBytes / sizeof(double)));
}
