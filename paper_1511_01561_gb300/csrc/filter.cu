// Element part of the Boyd-Vandeven filter (Sec. 2.3), applied after a time
// step as in the time loop of Sec. 7: per element the tensor product
// F x F x F of the 1D modal filter on the five state variables.  The kernel
// writes the Jw-weighted correction Jw ((F x F x F) q - q) into the residual
// buffer; mode 3 of the update kernel then forms q + M^-1 DSS(correction),
// which for a continuous q equals M^-1 DSS(Jw (F x F x F) q) because
// DSS(Jw q) = M q.  The correction form lets the FP32 form keep its FP32
// residual buffer while the state stays FP64.
#include "kernels_common.cuh"

namespace numa {
namespace {

// One CTA per element, one thread per element node; three passes along xi,
// eta and zeta through shared memory.  T = double: FP64 (also the pairs
// mode); T = float: the FP32 form (the correction in FP32).
template <int N, typename T>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32) filter_kernel(FilterArgs a) {
  constexpr int P = N + 1, NP = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);  // [5][NP]
  T* W = U + 5 * NP;                        // [5][NP]
  T* Fs = W + 5 * NP;                       // [P][P]
  const T* Fg = static_cast<const T*>(a.F);
  const int l = threadIdx.x;
  for (int t = l; t < P * P; t += blockDim.x) Fs[t] = Fg[t];
  const long long e = blockIdx.x, Ng = a.Ng, Nl = a.Nl, n = e * NP + l;
  const int i = l % P, j = (l / P) % P, k = l / (P * P);
  T qv[5];
  if (l < NP) {
    const int g = a.l2g[n];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double x = a.q[v * Ng + g];
      if constexpr (sizeof(T) == 8) qv[v] = x;
      else qv[v] = d2f(x);
      U[v * NP + l] = qv[v];
    }
  }
  __syncthreads();
  if (l < NP) {  // along xi
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < P; ++m) s = fma(Fs[i * P + m], U[v * NP + m + P * (j + P * k)], s);
      W[v * NP + l] = s;
    }
  }
  __syncthreads();
  if (l < NP) {  // along eta (U is free again)
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < P; ++m) s = fma(Fs[j * P + m], W[v * NP + i + P * (m + P * k)], s);
      U[v * NP + l] = s;
    }
  }
  __syncthreads();
  if (l < NP) {  // along zeta, then the weighted correction
    T jw;
    if (a.met64) jw = T(a.met64[9 * Nl + n]);
    else if (a.met2) {
      const float2 p = a.met2[9 * Nl + n];
      jw = T(join64(Pairs{p.x, p.y}));
    } else {
      if constexpr (sizeof(T) == 8) jw = f2d(a.met32[9 * Nl + n]);
      else jw = a.met32[9 * Nl + n];
    }
    T* re = static_cast<T*>(a.re);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < P; ++m) s = fma(Fs[k * P + m], U[v * NP + i + P * (j + P * m)], s);
      re[v * Nl + n] = jw * (s - qv[v]);
    }
  }
}

template <int N, typename T>
cudaError_t launch_filter_t(const FilterArgs& a, cudaStream_t s) {
  constexpr int P = N + 1, NP = P * P * P;
  constexpr int NT = (NP + 31) / 32 * 32;
  constexpr size_t smem = sizeof(T) * (10 * NP + P * P);
  static DeviceFlags attr_set;
  if (!attr_set.has()) {
    cudaError_t e = cudaFuncSetAttribute(filter_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set.set();
  }
  if (a.Ne == 0) return cudaSuccess;
  filter_kernel<N, T><<<a.Ne, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_filter_p(int N, const FilterArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_filter_t<1, T>(a, s);
    case 2: return launch_filter_t<2, T>(a, s);
    case 3: return launch_filter_t<3, T>(a, s);
    case 4: return launch_filter_t<4, T>(a, s);
    case 5: return launch_filter_t<5, T>(a, s);
    case 6: return launch_filter_t<6, T>(a, s);
    case 7: return launch_filter_t<7, T>(a, s);
    case 8: return launch_filter_t<8, T>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_filter(int N, int precision, const FilterArgs& a, cudaStream_t s) {
  if (precision == NUMA_FP32_MIXED) return launch_filter_p<float>(N, a, s);
  return launch_filter_p<double>(N, a, s);
}

}  // namespace numa
