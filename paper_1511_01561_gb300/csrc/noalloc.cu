// numa_rhs_static_scratch: the right-hand side with its scratch (primitive
// fields and element residuals) in a fixed, library-owned device array
// instead of the caller's workspace.
//
// Who needs this: callers that cannot allocate device memory themselves --
// real-time loops that forbid allocation after start-up, or plug-ins whose
// host application owns all device memory and hands them only input and
// output buffers.  Such a caller cannot make room for a second residual
// scratch next to the one in the bound workspace (which numa_rk_step and
// numa_run use), so this entry point evaluates R = dq/dt on the caller's own
// buffers with a scratch array that is part of the library image: nothing
// is allocated per call.
//
// The array is 16 MiB.  Per global node the primitive fields take 72 bytes
// (FP64: nine flux components), 32 (FP32-mixed) or 64 (FP64-pairs); per
// element node the residuals take 40 (FP64, pairs) or 20 (FP32-mixed).  At
// N=4 the largest cubic boxes that fit are 11^3 elements in FP64, 12^3 in
// the pairs mode and 15^3 in FP32-mixed.  Every GPU that loads this library keeps the array until the
// process exits.  All calls share it: two calls whose work overlaps on the
// GPU (different streams, or different contexts on one device) race on it.
// Nothing in it needs clearing between calls: each call overwrites every
// primitive and residual entry before the next kernel reads it.
//
// The host-side name of the array is only a stand-in; the kernels get its
// device address, which cudaGetSymbolAddress returns for the CUDA context
// that is current.  That address belongs to the module as loaded in that
// context, so it is cached per context, keyed by the context's unique id
// (cuCtxGetId: ids are never reused within a process, so a context created
// after a device reset gets a new entry).  The first call in each context
// does the lookup.
#include <cuda.h>

#include <mutex>
#include <string>

#include "numa_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = NUMA_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) double g_static_re[kStaticScratchBytes / sizeof(double)];

// Driver calls that name the current context, resolved through the runtime
// (the library does not link the driver library directly).
using GetCurrentFn = CUresult (*)(CUcontext*);
using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);

constexpr int kCacheEntries = 64;
struct CacheEntry {
  unsigned long long ctx_id;
  double* addr;
};

std::mutex g_mu;
GetCurrentFn g_get_current = nullptr;
GetIdFn g_get_id = nullptr;
CacheEntry g_cache[kCacheEntries];
int g_cache_n = 0, g_cache_next = 0;

// Resolve the two driver entry points (once; caller holds g_mu).
cudaError_t resolve_driver_calls() {
  if (g_get_current && g_get_id) return cudaSuccess;
  void* a = nullptr;
  void* b = nullptr;
  cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
  if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
  if (e != cudaSuccess) return e;
  if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
    return cudaErrorSymbolNotFound;
  g_get_current = reinterpret_cast<GetCurrentFn>(a);
  g_get_id = reinterpret_cast<GetIdFn>(b);
  return cudaSuccess;
}

// Device address of g_static_re in the current CUDA context.
cudaError_t static_scratch_address(double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = resolve_driver_calls();
  if (e != cudaSuccess) return e;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  if (g_get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  for (int t = 0; t < g_cache_n; ++t)
    if (g_cache[t].ctx_id == id) {
      *out = g_cache[t].addr;
      return cudaSuccess;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_static_re);
  if (e != cudaSuccess) return e;
  // a small ring: the oldest context's entry makes room for a new one
  g_cache[g_cache_next] = {id, static_cast<double*>(p)};
  g_cache_next = (g_cache_next + 1) % kCacheEntries;
  if (g_cache_n < kCacheEntries) ++g_cache_n;
  *out = static_cast<double*>(p);
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
  if (e != cudaSuccess) {
    ctx->err = std::string("numa_rhs_static_scratch: device address of the static array: ") + cudaGetErrorString(e);
    return NUMA_ECUDA;
  }
  return numa::rhs_with_scratch(ctx, q_dev, r_dev, re, (long long)(kStaticScratchBytes / sizeof(double)));
}
