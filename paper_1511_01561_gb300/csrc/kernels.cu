// CUDA kernels of the GB300 NUMA hot path (sm_103a):
//   volume_kernel : per-element create_rhs of Eq. 4 / Eq. 5 (fluxes, tensor-
//                   product derivatives with D, chain rule with the metric
//                   terms, -Jw div F), one CTA per element, flux fields
//                   staged in shared memory;
//   update_kernel : per global node, deterministic direct stiffness
//                   summation over a precomputed inverse map (fixed order, no
//                   atomics), inverse mass matrix, sources, wall condition and
//                   the SSP-RK3 stage combination.
#include <cstdint>

#include "numa_internal.h"

namespace numa {
namespace {

template <typename T>
struct Arith;

template <>
struct Arith<double> {
  // p' = p0 ((1+x)^gamma - 1), x = Theta'/(rho theta)_0, without cancellation
  static __device__ __forceinline__ double pprime(double p0, double Tp, double Th0, double gam) {
    return p0 * expm1(gam * log1p(Tp / Th0));
  }
};

template <>
struct Arith<float> {
  // Mixed form: the reference values stay FP64 and are combined with the
  // state in FP64; the cancellation-free factor expm1(gamma log1p(x)) is
  // evaluated in FP32, where it keeps full FP32 relative accuracy.
  static __device__ __forceinline__ float pprime(double p0, double Tp, double Th0, double gam) {
    float x = (float)(Tp / Th0);
    return (float)p0 * expm1f((float)gam * log1pf(x));
  }
};

// Field slots of the 13 unique flux components staged per element node.
enum : int { kUx = 0, kUy, kUz, kTxx, kTxy, kTxz, kTyy, kTyz, kTzz, kPp, kHx, kHy, kHz, kNF };

template <int N, typename T>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    volume_kernel(VolumeArgs a) {
  constexpr int P = N + 1, NP = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* F = reinterpret_cast<T*>(smem_raw);  // [kNF][NP]
  T* Ds = F + kNF * NP;                     // [P][P]
  const T* Dg;
  const T* met;
  if constexpr (sizeof(T) == 8) {
    Dg = reinterpret_cast<const T*>(a.D64);
    met = reinterpret_cast<const T*>(a.met64);
  } else {
    Dg = reinterpret_cast<const T*>(a.D32);
    met = reinterpret_cast<const T*>(a.met32);
  }
  const int e = blockIdx.x;
  const int l = threadIdx.x;
  for (int t = l; t < P * P; t += blockDim.x) Ds[t] = Dg[t];
  const long long n = (long long)e * NP + l;
  const long long Ng = a.Ng, Nl = a.Nl;
  if (l < NP) {
    // primitive variables at this element node (the state is FP64)
    const int g = a.l2g[n];
    const double rp = a.q[g];
    const double Ux = a.q[Ng + g], Uy = a.q[2 * Ng + g], Uz = a.q[3 * Ng + g];
    const double Tp = a.q[4 * Ng + g];
    const double rho0 = a.ref[g], Th0 = a.ref[Ng + g], p0 = a.ref[2 * Ng + g];
    const double rho = rho0 + rp;
    const double Th = Th0 + Tp;
    const T pp = Arith<T>::pprime(p0, Tp, Th0, a.gamma);
    const T rinv = T(1) / T(rho);
    const T ux = T(Ux) * rinv, uy = T(Uy) * rinv, uz = T(Uz) * rinv;
    const T th = T(Th) * rinv;
    // F_rho = U, F_U = U (x) u + p' I (symmetric part stored once), F_Theta = theta U
    F[kUx * NP + l] = T(Ux);
    F[kUy * NP + l] = T(Uy);
    F[kUz * NP + l] = T(Uz);
    F[kTxx * NP + l] = T(Ux) * ux;
    F[kTxy * NP + l] = T(Ux) * uy;
    F[kTxz * NP + l] = T(Ux) * uz;
    F[kTyy * NP + l] = T(Uy) * uy;
    F[kTyz * NP + l] = T(Uy) * uz;
    F[kTzz * NP + l] = T(Uz) * uz;
    F[kPp * NP + l] = pp;
    F[kHx * NP + l] = th * T(Ux);
    F[kHy * NP + l] = th * T(Uy);
    F[kHz * NP + l] = th * T(Uz);
  }
  __syncthreads();
  if (l >= NP) return;
  const int i = l % P, j = (l / P) % P, k = l / (P * P);
  T dx[P], dy[P], dz[P];
#pragma unroll
  for (int m = 0; m < P; ++m) {
    dx[m] = Ds[i * P + m];
    dy[m] = Ds[j * P + m];
    dz[m] = Ds[k * P + m];
  }
  // metric terms B[3d+c] = d xi_d / d x_c and Jw (Eq. 5)
  T B[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) B[t] = met[t * Nl + n];
  const T jw = met[9 * Nl + n];
  const int bx = P * (j + P * k), by = i + P * P * k, bz = i + P * j;
  // reference-space derivatives of field f along xi, eta, zeta (Eq. 5)
  auto dref = [&](int f, T& s0, T& s1, T& s2) {
    const T* Ff = F + f * NP;
    s0 = s1 = s2 = T(0);
#pragma unroll
    for (int m = 0; m < P; ++m) {
      s0 = fma(dx[m], Ff[bx + m], s0);
      s1 = fma(dy[m], Ff[by + P * m], s1);
      s2 = fma(dz[m], Ff[bz + P * P * m], s2);
    }
  };
  // physical derivative along x_c by the chain rule
  auto phys = [&](int c, T s0, T s1, T s2) { return fma(s0, B[c], fma(s1, B[3 + c], s2 * B[6 + c])); };
  T s0, s1, s2;
  T div_r, div_x, div_y, div_z, div_t;
  dref(kUx, s0, s1, s2); div_r = phys(0, s0, s1, s2);
  dref(kUy, s0, s1, s2); div_r += phys(1, s0, s1, s2);
  dref(kUz, s0, s1, s2); div_r += phys(2, s0, s1, s2);
  dref(kTxx, s0, s1, s2); div_x = phys(0, s0, s1, s2);
  dref(kTxy, s0, s1, s2); div_x += phys(1, s0, s1, s2); div_y = phys(0, s0, s1, s2);
  dref(kTxz, s0, s1, s2); div_x += phys(2, s0, s1, s2); div_z = phys(0, s0, s1, s2);
  dref(kTyy, s0, s1, s2); div_y += phys(1, s0, s1, s2);
  dref(kTyz, s0, s1, s2); div_y += phys(2, s0, s1, s2); div_z += phys(1, s0, s1, s2);
  dref(kTzz, s0, s1, s2); div_z += phys(2, s0, s1, s2);
  dref(kPp, s0, s1, s2);
  div_x += phys(0, s0, s1, s2);
  div_y += phys(1, s0, s1, s2);
  div_z += phys(2, s0, s1, s2);
  dref(kHx, s0, s1, s2); div_t = phys(0, s0, s1, s2);
  dref(kHy, s0, s1, s2); div_t += phys(1, s0, s1, s2);
  dref(kHz, s0, s1, s2); div_t += phys(2, s0, s1, s2);
  // element residual -Jw div F (Eq. 4); the sources are added per global node
  a.re[n] = -(double)(jw * div_r);
  a.re[Nl + n] = -(double)(jw * div_x);
  a.re[2 * Nl + n] = -(double)(jw * div_y);
  a.re[3 * Nl + n] = -(double)(jw * div_z);
  a.re[4 * Nl + n] = -(double)(jw * div_t);
}

template <int MODE, bool SHELL>
__global__ void __launch_bounds__(256) update_kernel(UpdateArgs a) {
  const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= a.Ng) return;
  const long long Ng = a.Ng, Nl = a.Nl;
  // direct stiffness summation in ascending element-node order (Eq. 4)
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
  const int t0 = a.off[I], t1 = a.off[I + 1];
  for (int t = t0; t < t1; ++t) {
    const long long n = a.idx[t];
    s0 += a.re[n];
    s1 += a.re[Nl + n];
    s2 += a.re[2 * Nl + n];
    s3 += a.re[3 * Nl + n];
    s4 += a.re[4 * Nl + n];
  }
  const double minv = a.Minv[I];
  double R0 = s0 * minv, R1 = s1 * minv, R2 = s2 * minv, R3 = s3 * minv, R4 = s4 * minv;
  // sources at the global node: buoyancy of rho' (and Coriolis on the shell)
  const double rp = a.qk[I];
  const uint8_t w = a.wall[I];
  if constexpr (SHELL) {
    const double gx = a.gvec[I], gy = a.gvec[Ng + I], gz = a.gvec[2 * Ng + I];
    R1 = fma(-rp, gx, R1) + a.two_omega * a.qk[2 * Ng + I];
    R2 = fma(-rp, gy, R2) - a.two_omega * a.qk[Ng + I];
    R3 = fma(-rp, gz, R3);
    if (w & 8) {  // remove the radial momentum tendency at the bottom and lid
      const double nx = a.nrm[I], ny = a.nrm[Ng + I], nz = a.nrm[2 * Ng + I];
      const double dot = R1 * nx + R2 * ny + R3 * nz;
      R1 -= dot * nx;
      R2 -= dot * ny;
      R3 -= dot * nz;
    }
  } else {
    R3 = fma(-rp, a.g, R3);
    if (w & 1) R1 = 0.0;
    if (w & 2) R2 = 0.0;
    if (w & 4) R3 = 0.0;
  }
  if constexpr (MODE == 0) {
    a.out[I] = R0;
    a.out[Ng + I] = R1;
    a.out[2 * Ng + I] = R2;
    a.out[3 * Ng + I] = R3;
    a.out[4 * Ng + I] = R4;
  } else {
    const double bdt = a.b * a.dt;
    double y[5];
    const double R[5] = {R0, R1, R2, R3, R4};
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double qk = a.qk[v * Ng + I];
      double t = fma(a.b, qk, bdt * R[v]);
      if (a.a != 0.0) t = fma(a.a, a.qn[v * Ng + I], t);
      y[v] = t;
    }
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a.out[v * Ng + I] = y[v];
      bad |= !isfinite(y[v]);
    }
    if (bad) atomicOr(a.flag, 1);
  }
}

template <int N, typename T>
cudaError_t launch_volume_t(const VolumeArgs& a, cudaStream_t s) {
  constexpr int P = N + 1, NP = P * P * P;
  constexpr int NT = (NP + 31) / 32 * 32;
  const size_t smem = sizeof(T) * (kNF * NP + P * P);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(volume_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (a.Ne == 0) return cudaSuccess;
  volume_kernel<N, T><<<a.Ne, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_volume_p(int N, const VolumeArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_volume_t<1, T>(a, s);
    case 2: return launch_volume_t<2, T>(a, s);
    case 3: return launch_volume_t<3, T>(a, s);
    case 4: return launch_volume_t<4, T>(a, s);
    case 5: return launch_volume_t<5, T>(a, s);
    case 6: return launch_volume_t<6, T>(a, s);
    case 7: return launch_volume_t<7, T>(a, s);
    case 8: return launch_volume_t<8, T>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_volume(int N, int precision, const VolumeArgs& a, cudaStream_t s) {
  if (precision == NUMA_FP32_MIXED) return launch_volume_p<float>(N, a, s);
  return launch_volume_p<double>(N, a, s);
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  if (a.Ng == 0) return cudaSuccess;
  const int nt = 256;
  const unsigned nb = (unsigned)((a.Ng + nt - 1) / nt);
  const bool shell = a.gvec != nullptr;
  if (a.mode == 0) {
    if (shell) update_kernel<0, true><<<nb, nt, 0, s>>>(a);
    else update_kernel<0, false><<<nb, nt, 0, s>>>(a);
  } else {
    if (shell) update_kernel<1, true><<<nb, nt, 0, s>>>(a);
    else update_kernel<1, false><<<nb, nt, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace numa
