// Throughput probes of the arithmetic units the element kernels could run
// on (measurement helper, not part of the method): register-only FP64 and
// FP32 FMA chains, and warp-level mma.sync in FP64 (m8n8k4) and TF32
// (m16n8k8).  They give the ALU ceilings against which the FP64 element
// kernels are judged, and decide whether a tensor-core variant of the D
// contraction could win.
//
// Every kernel keeps its operands in registers (no memory traffic inside the
// loop), runs independent dependency chains per thread or warp so that the
// pipes stay full, and writes one value per thread at the end so that no
// work is dead.  Grids are whole multiples of the SM count.
#include <cuda_runtime.h>

#include <cstdint>

#include "numa.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kAcc = 4;         // independent mma accumulators per warp
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + C, A 8x4, B 4x8, C/D 8x8, FP64: one A, one B and two C/D
// values per thread.
__device__ __forceinline__ void dmma_884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kThreads) dmma_chains(double* out, int iters) {
  double acc[kAcc][2];
#pragma unroll
  for (int c = 0; c < kAcc; ++c) acc[c][0] = acc[c][1] = 0.0;
  const double a = 1e-3 * (1 + (threadIdx.x & 3)), b = 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kAcc; ++c) dmma_884(acc[c][0], acc[c][1], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kAcc; ++c) s += acc[c][0] + acc[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + C, A 16x8, B 8x8 (TF32 operands held in 32-bit registers), C/D
// 16x8 FP32: four A, two B and four C/D registers per thread.
__device__ __forceinline__ void tf32_1688(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                          uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kThreads) tf32_chains(float* out, int iters) {
  float acc[kAcc][4];
#pragma unroll
  for (int c = 0; c < kAcc; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.0f;
  const uint32_t a = __float_as_uint(1e-3f * (1 + (threadIdx.x & 3))), b = __float_as_uint(1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kAcc; ++c) tf32_1688(acc[c], a, a, a, a, b, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kAcc; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Half of the warps run FP64 FMA chains, the other half FP64 mma.sync: shows
// whether the two FP64 paths share one pipe (the total stays near either
// rate alone) or run side by side (it approaches their sum).
__global__ void __launch_bounds__(kThreads) fp64_fma_and_mma(double* out, int iters_fma, int iters_mma) {
  double s = 0.0;
  if ((threadIdx.x >> 5) & 1) {
    double acc[kAcc][2];
#pragma unroll
    for (int c = 0; c < kAcc; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double a = 1e-3 * (1 + (threadIdx.x & 3)), b = 1e-3;
    for (int i = 0; i < iters_mma; ++i) {
#pragma unroll
      for (int c = 0; c < kAcc; ++c) dmma_884(acc[c][0], acc[c][1], a, b);
    }
#pragma unroll
    for (int c = 0; c < kAcc; ++c) s += acc[c][0] + acc[c][1];
  } else {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = double(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters_fma; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], 0.999999, 1e-6);
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int numa_probe_peak(int kind, int iters, void* dev_out, size_t out_bytes, void* stream, double* ms,
                               double* tflops) {
  if (!ms || !tflops || !dev_out || iters < 1 || kind < 0 || kind > 4) return NUMA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NUMA_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NUMA_ECUDA;
  const unsigned blocks = (unsigned)(sms * kBlocksPerSM);
  const size_t threads = (size_t)blocks * kThreads;
  const size_t elem = (kind == 1 || kind == 3) ? 4 : 8;
  // kind 4: an FMA thread does 16 flops per iteration, an mma thread 64; with
  // the rates of each path alone (1.26 and 1.10 TFLOP/s) both halves take the
  // same time when the mma warps run 16/64 * 1.10/1.26 of the iterations
  const int iters_fma = iters;
  const int iters_mma = (int)(iters * 0.2186) > 1 ? (int)(iters * 0.2186) : 1;
  if (out_bytes < threads * elem) return NUMA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    switch (kind) {
      case 0: fma_chains<double><<<blocks, kThreads, 0, s>>>((double*)dev_out, iters, 0.999999, 1e-6); break;
      case 1: fma_chains<float><<<blocks, kThreads, 0, s>>>((float*)dev_out, iters, 0.9999f, 1e-4f); break;
      case 2: dmma_chains<<<blocks, kThreads, 0, s>>>((double*)dev_out, iters); break;
      case 3: tf32_chains<<<blocks, kThreads, 0, s>>>((float*)dev_out, iters); break;
      default: fp64_fma_and_mma<<<blocks, kThreads, 0, s>>>((double*)dev_out, iters_fma, iters_mma); break;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return NUMA_ECUDA;
  // flops per thread and iteration: an FMA is 2 flops; an mma is issued by
  // the 32 threads of a warp together (m*n*k multiply-adds)
  double per_thread_iter;
  switch (kind) {
    case 0:
    case 1: per_thread_iter = 2.0 * kChains; break;
    case 2: per_thread_iter = 2.0 * 8 * 8 * 4 * kAcc / 32.0; break;
    case 3: per_thread_iter = 2.0 * 16 * 8 * 8 * kAcc / 32.0; break;
    default:  // half the threads each way, flops of both halves over the one kernel time
      per_thread_iter = 0.5 * (2.0 * kChains + 2.0 * 8 * 8 * 4 * kAcc / 32.0 * iters_mma / (double)iters_fma);
      break;
  }
  *ms = t;
  *tflops = per_thread_iter * (double)iters * (double)threads / (t * 1e-3) / 1e12;
  return NUMA_OK;
}
