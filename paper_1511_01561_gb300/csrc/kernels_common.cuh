// Device code shared by the kernel translation units of the GB300 NUMA hot
// path (sm_103a): FP64-pipe-free conversions, float-pair arithmetic, the
// equation of state, the element kernels of Eq. 4 / Eq. 5 (per-node, affine
// and line forms), the per-node DSS / inverse-mass / RK-stage update, the
// ragged multi-member kernels, and their launch templates.  Everything is in
// an anonymous namespace: each translation unit instantiates the templates
// it launches.
//
// GB300 executes FP64 at 1/64 of the FP32 rate, so everything that does not
// need FP64 stays off the FP64 pipe: float<->double conversions and the
// finiteness test are done with integer operations on the bit patterns.
#pragma once

#include <atomic>
#include <cstdint>
#include <type_traits>

#include "numa_internal.h"

namespace numa {
namespace {

// ---- FP64-pipe-free conversions -------------------------------------------
// The rare cases (subnormal, infinite, NaN) go through out-of-line functions:
// an inline fallback would be predicated into every call and issue its FP64
// conversion on every lane whether taken or not.

__device__ __noinline__ double f2d_rare(float f) { return (double)f; }
__device__ __noinline__ float d2f_rare(double d) { return __double2float_rn(d); }

// Exact float -> double.  Subnormal, infinite and NaN inputs take the
// hardware conversion (zeros, common in a state at rest, do not).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (ex == 0u || ex == 0xffu) return f2d_rare(f);
  const unsigned hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// double -> float, round to nearest even.  Results that are subnormal,
// infinite or NaN take the hardware conversion; zeros do not.
__device__ __forceinline__ float d2f(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(hi & 0x80000000u);
  const int ex = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (ex <= 0 || ex >= 255) return d2f_rare(d);
  // 52-bit fraction = (hi & 0xfffff) : lo; keep the top 23 bits, round on the other 29
  const unsigned keep = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  unsigned bits = (hi & 0x80000000u) | ((unsigned)ex << 23) | keep;
  const unsigned half = 0x10000000u;
  bits += (rest > half || (rest == half && (keep & 1u))) ? 1u : 0u;  // carries into the exponent
  return __uint_as_float(bits);
}

__device__ __forceinline__ bool nonfinite(double d) {
  return ((((unsigned)__double2hiint(d)) >> 20) & 0x7ffu) == 0x7ffu;
}

// 1/x in FP64 for a positive density: FP32 reciprocal seed (conversions by
// integer ops), two Newton steps.
__device__ __forceinline__ double rcp64(double x) {
  double r = f2d(__frcp_rn(d2f(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// ---- FP64 accuracy on the FP32 units ("pairs") ------------------------------
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2:
// about 48 significant bits.  Products are formed with the FMA-based exact
// product split (Dekker's two-product via FMA), sums with Knuth's TwoSum.

struct Pairs {
  float h, l;
};

// double -> pair with integer operations: h = the double's top 24 significant
// bits (truncated), l = the next bits rounded to a float.  Values outside
// float range (below 2^-74 the low part vanishes; zeros excepted) take the
// FP64 path.
__device__ __noinline__ Pairs split64_rare(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ Pairs split64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ffu);  // biased FP64 exponent
  // zeros (common at walls and in a state at rest) inline, with their sign
  if (((hi & 0x7fffffffu) | lo) == 0u) return {__uint_as_float(hi & 0x80000000u), 0.0f};
  if (E < 1023 - 74 || E > 1023 + 127) return split64_rare(x);
  const unsigned sign = hi & 0x80000000u;
  const float h = __uint_as_float(sign | ((unsigned)(E - 1023 + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  // remainder: the low 29 fraction bits, weight 2^(E-1023-52)
  const unsigned rem = lo & 0x1fffffffu;
  const float r = __uint2float_rn(rem);  // rounds 29 -> 24 bits
  const float scale = __uint_as_float((unsigned)(E - 1023 - 52 + 127) << 23);
  const float l = r * scale;
  return {h, sign ? -l : l};
}

// (h, l) pair -> double (exact: the pair fits in 53 bits).
__device__ __forceinline__ double join64(Pairs a) { return f2d(a.h) + f2d(a.l); }

__device__ __forceinline__ Pairs pp_mul(Pairs a, Pairs b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = p + e;
  return {s, e - (s - p)};
}

// Unnormalised accumulator (sh, sl) += a * b.
__device__ __forceinline__ void pp_fma(float& sh, float& sl, Pairs a, Pairs b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = sh + p;
  const float bb = s - sh;
  const float t = (sh - (s - bb)) + (p - bb);
  sl += t + e;
  sh = s;
}

// First term of an accumulation: (sh, sl) = a * b.
__device__ __forceinline__ void pp_first(float& sh, float& sl, Pairs a, Pairs b) {
  sh = a.h * b.h;
  float e = fmaf(a.h, b.h, -sh);
  e = fmaf(a.h, b.l, e);
  sl = fmaf(a.l, b.h, e);
}

__device__ __forceinline__ Pairs pp_norm(float sh, float sl) {
  const float s = sh + sl;
  return {s, sl - (s - sh)};
}

// a + b (TwoSum of the high parts, low parts added in).
__device__ __forceinline__ Pairs pp_add(Pairs a, Pairs b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float t = (a.h - (s - bb)) + (b.h - bb) + (a.l + b.l);
  return pp_norm(s, t);
}

// a - b (TwoSum of the high parts, low parts added in).
__device__ __forceinline__ Pairs pp_sub(Pairs a, Pairs b) {
  const float s = a.h - b.h;
  const float bb = s - a.h;
  const float t = (a.h - (s - bb)) - (b.h + bb) + (a.l - b.l);
  return pp_norm(s, t);
}

__device__ __noinline__ double eos_ratio_rare(double x, double gamma) { return expm1(gamma * log1p(x)); }

// (1+x)^gamma - 1 with full relative accuracy: the binomial series
// sum_k C(gamma,k) x^k (Horner) for |x| <= 2^-5, else expm1(gamma log1p(x)).
// For 1 < gamma < 2 every |C(gamma,k+1) / C(gamma,1)| <= 1, so the relative
// truncation after K terms is below |x|^K; K is the least count that keeps
// it below 2^-60 (2^-30 for a result stored as a float, F32OUT): 2, 3, 4, 5,
// 6 or 12 terms for |x| <= 2^-30, 2^-20, 2^-15, 2^-12, 2^-10, 2^-5 (F32OUT:
// 1, 2, 3, 6 for 2^-30, 2^-15, 2^-10, 2^-5).  The term count is a loop bound,
// not a branch, so a warp runs the series once, to its largest count.
template <bool F32OUT = false>
__device__ __forceinline__ double eos_ratio(double x, const PrimArgs& a) {
  const unsigned hx = ((unsigned)__double2hiint(x)) & 0x7fffffffu;  // |x| by its high word
  if (hx > 0x3fa00000u) return eos_ratio_rare(x, a.gamma);          // |x| > 2^-5
  // thresholds 2^-e as high words: (1023 - e) << 20
  int K;
  if constexpr (F32OUT)
    K = hx <= 0x3e100000u ? 1 : hx <= 0x3f000000u ? 2 : hx <= 0x3f500000u ? 3 : 6;
  else
    K = hx <= 0x3e100000u ? 2 : hx <= 0x3eb00000u ? 3 : hx <= 0x3f000000u ? 4 : hx <= 0x3f300000u ? 5
      : hx <= 0x3f500000u ? 6 : kEosTerms;
  double t = a.eos[K - 1];
  for (int k = K - 2; k >= 0; --k) t = fma(t, x, a.eos[k]);
  return t * x;
}

// Primitive fields of state (rp, U, Tp) at global node I (reference from a.ref):
// rho = rho0 + rho', u = U / rho, theta = (Theta0 + Theta') / rho,
// p' = p0 ((1 + Theta'/Theta0)^gamma - 1); in FP64 the flux components
// built from them (the element kernels' gathered input).
// F32: the FP32-mixed form (known at compile time, so that its kernels carry
// none of the FP64 form's code); otherwise FP64 or pairs by a.precision.
template <bool F32>
__device__ __forceinline__ void write_prim(const PrimArgs& a, long long I, double rp, double Ux, double Uy,
                                           double Uz, double Tp) {
  const long long Ng = a.Ng;
  const double rho0 = a.ref[I], Th0 = a.ref[Ng + I], p0 = a.ref[2 * Ng + I], iTh0 = a.ref[3 * Ng + I];
  if constexpr (F32) {
    // u and theta are FP32 fields, so rho and Theta are summed in FP32; p'
    // (the reference-state subtraction of the equation of state) in FP64, to
    // the accuracy of the float it is stored as
    // node-interleaved: two float4 per node, one 32-byte sector
    float4* w = static_cast<float4*>(a.prim);
    const float rf = 1.0f / (d2f(rho0) + d2f(rp));
    const float Uxf = d2f(Ux), Uyf = d2f(Uy), Uzf = d2f(Uz);
    w[2 * I] = make_float4(Uxf, Uyf, Uzf, Uxf * rf);
    w[2 * I + 1] = make_float4(Uyf * rf, Uzf * rf, (d2f(Th0) + d2f(Tp)) * rf, d2f(p0 * eos_ratio<true>(Tp * iTh0, a)));
    return;
  } else {
  const double rho = rho0 + rp;
  const double Th = Th0 + Tp;
  if (a.precision == NUMA_FP64_PAIRS) {
    // FP64 primitives, stored as (hi, lo) pairs for the element kernel
    Pairs* w = static_cast<Pairs*>(a.prim);
    const double r = rcp64(rho);
    w[I] = split64(Ux);
    w[Ng + I] = split64(Uy);
    w[2 * Ng + I] = split64(Uz);
    w[3 * Ng + I] = split64(Ux * r);
    w[4 * Ng + I] = split64(Uy * r);
    w[5 * Ng + I] = split64(Uz * r);
    w[6 * Ng + I] = split64(Th * r);
    w[7 * Ng + I] = split64(p0 * eos_ratio(Tp * iTh0, a));
  } else {
    // FP64: the nine flux components the element kernels need besides U,
    // formed once per global node (kFlux64 slots): U_c u_c + p' on the
    // diagonal, the symmetric U_c u_d once, and theta U = Theta u
    double* w = static_cast<double*>(a.prim);
    const double r = rcp64(rho);
    const double ux = Ux * r, uy = Uy * r, uz = Uz * r;
    const double pp = p0 * eos_ratio(Tp * iTh0, a);
    w[I] = fma(Ux, ux, pp);
    w[Ng + I] = fma(Uy, uy, pp);
    w[2 * Ng + I] = fma(Uz, uz, pp);
    w[3 * Ng + I] = Ux * uy;
    w[4 * Ng + I] = Ux * uz;
    w[5 * Ng + I] = Uy * uz;
    w[6 * Ng + I] = Th * ux;
    w[7 * Ng + I] = Th * uy;
    w[8 * Ng + I] = Th * uz;
  }
  }
}


// Field slots of the 13 unique flux components staged per element node.
enum : int { kUx = 0, kUy, kUz, kTxx, kTxy, kTxz, kTyy, kTyz, kTzz, kPp, kHx, kHy, kHz, kNF };

// Momentum and primitive fields of the global node behind element node n
// (CG storage: gathered through l2g), FP32 form.
template <typename T>
struct NodeState {
  T Ux, Uy, Uz, ux, uy, uz, th, pp;
};

template <typename T>
__device__ __forceinline__ NodeState<T> gather_node(const VolumeArgs& a, long long n) {
  static_assert(sizeof(T) == 4, "the FP64 kernels gather flux components (gather_fluxes64)");
  const int g = a.l2g[n];
  NodeState<T> z;
  {
    const float4* w = static_cast<const float4*>(a.prim);
    const float4 p = w[2 * g], r = w[2 * g + 1];
    z.Ux = p.x;
    z.Uy = p.y;
    z.Uz = p.z;
    z.ux = p.w;
    z.uy = r.x;
    z.uz = r.y;
    z.th = r.z;
    z.pp = r.w;
  }
  return z;
}

// The 13 unique flux components of element node l (index n) into the shared
// tile F[kNF][NP]: F_rho = U, F_U = U (x) u + p' I (symmetric part stored
// once), F_Theta = theta U.
template <int N, typename T>
__device__ __forceinline__ void stage_fluxes(const VolumeArgs& a, long long n, int l, T* F) {
  constexpr int P = N + 1, NP = P * P * P;
  const NodeState<T> z = gather_node<T>(a, n);
  F[kUx * NP + l] = z.Ux;
  F[kUy * NP + l] = z.Uy;
  F[kUz * NP + l] = z.Uz;
  F[kTxx * NP + l] = z.Ux * z.ux;
  F[kTxy * NP + l] = z.Ux * z.uy;
  F[kTxz * NP + l] = z.Ux * z.uz;
  F[kTyy * NP + l] = z.Uy * z.uy;
  F[kTyz * NP + l] = z.Uy * z.uz;
  F[kTzz * NP + l] = z.Uz * z.uz;
  F[kPp * NP + l] = z.pp;
  F[kHx * NP + l] = z.th * z.Ux;
  F[kHy * NP + l] = z.th * z.Uy;
  F[kHz * NP + l] = z.th * z.Uz;
}

// Affine elements (every element of a box without warp) have the same metric
// terms B[3d+c] = d xi_d / d x_c at all their nodes, so the chain rule of
// Eq. 5 commutes with the derivative:
//   sum_c B_dc dF_vc/d xi_d = d/d xi_d (sum_c B_dc F_vc).
// Node l stages the contravariant fluxes G[3v+d] = sum_c B_dc F_vc of the
// five equations v along the three directions d (15 values):
//   mass      G = B_d . U
//   momentum  G_x = U_x (B_d . u) + B_dx p'   (and y, z)
//   Theta     G = theta (B_d . U)
template <int N, typename T>
__device__ __forceinline__ void stage_fluxes_affine(const VolumeArgs& a, long long n, int l, const T (&B)[9], T* G) {
  constexpr int P = N + 1, NP = P * P * P;
  const NodeState<T> z = gather_node<T>(a, n);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T b0 = B[3 * d], b1 = B[3 * d + 1], b2 = B[3 * d + 2];
    const T ud = fma(b0, z.ux, fma(b1, z.uy, b2 * z.uz));
    const T Gr = fma(b0, z.Ux, fma(b1, z.Uy, b2 * z.Uz));
    G[d * NP + l] = Gr;
    G[(3 + d) * NP + l] = fma(z.Ux, ud, b0 * z.pp);
    G[(6 + d) * NP + l] = fma(z.Uy, ud, b1 * z.pp);
    G[(9 + d) * NP + l] = fma(z.Uz, ud, b2 * z.pp);
    G[(12 + d) * NP + l] = z.th * Gr;
  }
}

// The 12 flux fields of the FP64 (and pairs) kernels: F_rho = U, F_U =
// U (x) u + p' I with the pressure in the diagonal components (the
// symmetric part stored once), F_Theta = theta U.
enum : int { lUx = 0, lUy, lUz, lTxx, lTyy, lTzz, lTxy, lTxz, lTyz, lHx, lHy, lHz, kLF };

// The 12 flux fields at the global node behind element node n, FP64: U from
// the state, the other nine as the update kernel formed them (write_prim).
struct FluxState64 {
  double f[kLF];
};

__device__ __forceinline__ FluxState64 gather_fluxes64(const VolumeArgs& a, long long n) {
  const long long Ng = a.Ng;
  const int g = a.l2g[n];
  const double* w = static_cast<const double*>(a.prim);
  FluxState64 z;
  z.f[lUx] = a.q[Ng + g];
  z.f[lUy] = a.q[2 * Ng + g];
  z.f[lUz] = a.q[3 * Ng + g];
  z.f[lTxx] = w[g];
  z.f[lTyy] = w[Ng + g];
  z.f[lTzz] = w[2 * Ng + g];
  z.f[lTxy] = w[3 * Ng + g];
  z.f[lTxz] = w[4 * Ng + g];
  z.f[lTyz] = w[5 * Ng + g];
  z.f[lHx] = w[6 * Ng + g];
  z.f[lHy] = w[7 * Ng + g];
  z.f[lHz] = w[8 * Ng + g];
  return z;
}

// D of every order N = 1..8 in FP32 ([N][(N+1)^2], row-major), read by the
// FP32 line kernel as instruction operands.  Written at bind time; every
// mesh of one order writes the same values.
__constant__ float c_D32[9 * 81];

template <int N>
__device__ __forceinline__ float cD32(int i, int m) {
  return c_D32[N * 81 + i * (N + 1) + m];
}

// Directions of the line kernel: lines of one direction per work group of
// W threads (whole warps when three of them fit in the CTA, so that each
// warp reads one direction's lines without conflicts between directions).
template <int N>
__host__ __device__ constexpr int line_group() {
  constexpr int P2 = (N + 1) * (N + 1), NT = ((N + 1) * P2 + 31) / 32 * 32, W32 = (P2 + 31) / 32 * 32;
  return 3 * W32 <= NT ? W32 : P2;
}

// ---- FP64 element kernels with fewer FP64 instructions ---------------------
// GB300 issues 2 FP64 FMAs per SM per clock, so the FP64 element kernels are
// bound by their FP64 instruction count.  Exact rearrangements cut it:
//
// (1) Per-node form (any element): the pressure is added into the diagonal
//     momentum fluxes before they are differentiated (12 fields instead of
//     13) and the metric terms are stored pre-multiplied by -Jw, so the chain
//     rule is three FMAs per use of a field and no final weighting remains.
// (2) Rectilinear affine elements (every element of an unwarped box): the
//     metric terms dxi_d/dx_c vanish for c != d and J is constant over the
//     element, so -Jw div F at node (i,j,k) is w_i w_j w_k sum_d K_d (D F_d)
//     along xi_d, with K_d = -J dxi_d/dx_d per element.  Folding K_d into the
//     direction's copy of D (formed per element in shared memory) leaves the
//     12 unweighted flux fields of (1) and 15 contractions, with no metric or
//     Jw load per node.  The weight w_i w_j w_k is the same at every element
//     node of a global node (the Lobatto weights are symmetric and the box's
//     elements meet face to face), so it moves out of the element kernel
//     into the inverse mass of the DSS: the kernel writes
//     sum_d K_d (D F_d), and the update multiplies the sum over element
//     nodes by w_i w_j w_k / M (Minv_r) instead of 1 / M.
// (3) Both forms: the nine flux components besides U (U_c u_c + p', the
//     symmetric U_c u_d, Theta u) are formed once per global node by the
//     update that writes the state (write_prim) and gathered as they are, not
//     formed again at each of the global node's element nodes.

// create_rhs of element e in FP64, per-node form of Eq. 5 (any element,
// curved included), one thread per element node.  The metric terms arrive
// pre-multiplied by -Jw (rows 0..8 of met64 hold -Jw dxi_d/dx_c for this
// form), and the pressure sits in the diagonal momentum fluxes, so each of
// the 12 staged flux fields (kLF) is differentiated along xi, eta and zeta
// (15 FMAs) and folded into the divergence of every equation that uses it
// with three FMAs: 180 + 45 FP64 operations per node at N = 4 (the update
// formed the flux components once per global node).  The
// result is the weighted residual -Jw div F of Eq. 4.  smem_raw holds
// 12 (N+1)^3 + (N+1)^2 doubles.
template <int N>
__device__ __forceinline__ void volume_element_nodal64(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  constexpr int P = N + 1, NP = P * P * P;
  double* F = reinterpret_cast<double*>(smem_raw);  // [kLF][NP]
  double* Ds = F + kLF * NP;                         // [P][P]
  const double* met = a.met64;
  const int l = threadIdx.x;
  for (int t = l; t < P * P; t += blockDim.x) Ds[t] = a.D64[t];
  const long long Nl = a.Nl, n = (long long)e * NP + l;
  double B[9];  // -Jw dxi_d/dx_c at this node, [3d + c]
  if (l < NP) {
#pragma unroll
    for (int t = 0; t < 9; ++t) B[t] = met[t * Nl + n];
    const FluxState64 z = gather_fluxes64(a, n);
#pragma unroll
    for (int f = 0; f < kLF; ++f) F[f * NP + l] = z.f[f];
  }
  __syncthreads();
  if (l >= NP) return;
  const int i = l % P, j = (l / P) % P, k = l / (P * P);
  double dx[P], dy[P], dz[P];
#pragma unroll
  for (int m = 0; m < P; ++m) {
    dx[m] = Ds[i * P + m];
    dy[m] = Ds[j * P + m];
    dz[m] = Ds[k * P + m];
  }
  const int bx = P * (j + P * k), by = i + P * P * k, bz = i + P * j;
  // reference-space derivatives of field f along xi, eta, zeta (Eq. 5)
  auto dref = [&](int f, double& s0, double& s1, double& s2) {
    const double* Ff = F + f * NP;
    s0 = dx[0] * Ff[bx];
    s1 = dy[0] * Ff[by];
    s2 = dz[0] * Ff[bz];
#pragma unroll
    for (int m = 1; m < P; ++m) {
      s0 = fma(dx[m], Ff[bx + m], s0);
      s1 = fma(dy[m], Ff[by + P * m], s1);
      s2 = fma(dz[m], Ff[bz + P * P * m], s2);
    }
  };
  // chain rule into the weighted divergence: acc += -Jw d/dx_c of the field
  auto first = [&](int c, double s0, double s1, double s2) { return fma(s2, B[6 + c], fma(s1, B[3 + c], s0 * B[c])); };
  auto add = [&](double& acc, int c, double s0, double s1, double s2) {
    acc = fma(s2, B[6 + c], fma(s1, B[3 + c], fma(s0, B[c], acc)));
  };
  double s0, s1, s2, dr, dxm, dym, dzm, dt;
  dref(lUx, s0, s1, s2); dr = first(0, s0, s1, s2);
  dref(lUy, s0, s1, s2); add(dr, 1, s0, s1, s2);
  dref(lUz, s0, s1, s2); add(dr, 2, s0, s1, s2);
  dref(lTxx, s0, s1, s2); dxm = first(0, s0, s1, s2);
  dref(lTyy, s0, s1, s2); dym = first(1, s0, s1, s2);
  dref(lTzz, s0, s1, s2); dzm = first(2, s0, s1, s2);
  dref(lTxy, s0, s1, s2); add(dxm, 1, s0, s1, s2); add(dym, 0, s0, s1, s2);
  dref(lTxz, s0, s1, s2); add(dxm, 2, s0, s1, s2); add(dzm, 0, s0, s1, s2);
  dref(lTyz, s0, s1, s2); add(dym, 2, s0, s1, s2); add(dzm, 1, s0, s1, s2);
  dref(lHx, s0, s1, s2); dt = first(0, s0, s1, s2);
  dref(lHy, s0, s1, s2); add(dt, 1, s0, s1, s2);
  dref(lHz, s0, s1, s2); add(dt, 2, s0, s1, s2);
  double* re = static_cast<double*>(a.re);
  re[n] = dr;
  re[Nl + n] = dxm;
  re[2 * Nl + n] = dym;
  re[3 * Nl + n] = dzm;
  re[4 * Nl + n] = dt;
}

// create_rhs of a rectilinear affine element in FP64 (see (2) above), one
// thread per element node: 75 FP64 operations per node at N = 4 (the flux
// components come from the update, formed once per global node).  It
// writes the residual without its weight w_i w_j w_k, which the update
// applies with the inverse mass.  a.affk holds K_d per element [3][Ne].
// Shared memory: 12 (N+1)^3 + 3 (N+1)^2 doubles.
template <int N>
__device__ __forceinline__ void volume_element_rect(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  constexpr int P = N + 1, PP = P * P, NP = PP * P;
  double* F = reinterpret_cast<double*>(smem_raw);  // [kLF][NP]
  double* Dk = F + kLF * NP;                         // [3][P][P]: K_d D
  const int l = threadIdx.x;
  for (int t = l; t < 3 * PP; t += blockDim.x) {
    const int d = t / PP;
    Dk[t] = a.affk[d * (long long)a.Ne + e] * a.D64[t - d * PP];
  }
  const long long Nl = a.Nl, n = (long long)e * NP + l;
  if (l < NP) {
    const FluxState64 z = gather_fluxes64(a, n);
#pragma unroll
    for (int f = 0; f < kLF; ++f) F[f * NP + l] = z.f[f];
  }
  __syncthreads();
  if (l >= NP) return;
  const int i = l % P, j = (l / P) % P, k = l / PP;
  double dx[P], dy[P], dz[P];
#pragma unroll
  for (int m = 0; m < P; ++m) {
    dx[m] = Dk[i * P + m];
    dy[m] = Dk[PP + j * P + m];
    dz[m] = Dk[2 * PP + k * P + m];
  }
  const int bx = P * (j + P * k), by = i + PP * k, bz = i + P * j;
  // K_x D F_x along xi + K_y D F_y along eta + K_z D F_z along zeta
  auto div = [&](int fx, int fy, int fz) {
    const double* gx = F + fx * NP;
    const double* gy = F + fy * NP;
    const double* gz = F + fz * NP;
    double t = dx[0] * gx[bx];
#pragma unroll
    for (int m = 1; m < P; ++m) t = fma(dx[m], gx[bx + m], t);
#pragma unroll
    for (int m = 0; m < P; ++m) t = fma(dy[m], gy[by + P * m], t);
#pragma unroll
    for (int m = 0; m < P; ++m) t = fma(dz[m], gz[bz + PP * m], t);
    return t;
  };
  double* re = static_cast<double*>(a.re);
  re[n] = div(lUx, lUy, lUz);
  re[Nl + n] = div(lTxx, lTxy, lTxz);
  re[2 * Nl + n] = div(lTxy, lTyy, lTyz);
  re[3 * Nl + n] = div(lTxz, lTyz, lTzz);
  re[4 * Nl + n] = div(lHx, lHy, lHz);
}

// create_rhs of element e in the FP32 form, organised by 1D lines of nodes
// (Eq. 5 is a contraction along xi, eta and zeta).  Thread t < 3W takes one
// line along one reference direction d; for each field it reads the line's
// N+1 values once (distinct addresses, no broadcast) and applies the whole
// of D to them.
//   general element: the 13 flux fields, each derivative folded into the
//     divergence of its equation at the line's nodes with row d of the
//     metric (d xi_d / d x_c, read before the barrier);
//   affine element (AFF): the 5 contravariant fluxes G[3v+d] of direction d
//     (stage_fluxes_affine), whose derivatives are the partial sums.
// The partial sums go to shared memory over the no longer needed flux tile;
// one thread per element node then adds the three directions and weights by
// -Jw.  Shared memory: 15 (N+1)^3 floats.
template <int N, bool AFF>
__device__ __forceinline__ void volume_element_lines(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  constexpr int P = N + 1, P2 = P * P, NP = P2 * P;
  constexpr int W = line_group<N>();
  static_assert(3 * W <= (NP + 31) / 32 * 32, "one line per thread");
  float* F = reinterpret_cast<float*>(smem_raw);  // [kNF or 15][NP], then [3][5][NP]
  const float* met = a.met32;
  const long long Nl = a.Nl, e0 = (long long)e * NP;
  const int l = threadIdx.x;
  const int d = l / W, r = l - (l / W) * W;
  const bool act = d < 3 && r < P2;
  int base = 0, stride = 0;
  if (d == 0) {  // along xi: line (j, k)
    base = P * r;
    stride = 1;
  } else if (d == 1) {  // along eta: line (i, k)
    base = r % P + P2 * (r / P);
    stride = P;
  } else {  // along zeta: line (i, j)
    base = r;
    stride = P2;
  }
  float part[5][P];
  if constexpr (AFF) {
    if (l < NP) {
      float B[9];  // the element's metric terms, at its first node
#pragma unroll
      for (int t = 0; t < 9; ++t) B[t] = met[t * Nl + e0];
      stage_fluxes_affine<N, float>(a, e0 + l, l, B, F);
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const float* Gv = F + (3 * v + d) * NP + base;
        float x[P];
#pragma unroll
        for (int m = 0; m < P; ++m) x[m] = Gv[m * stride];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          float t = 0.0f;
#pragma unroll
          for (int m = 0; m < P; ++m) t = fmaf(cD32<N>(p, m), x[m], t);
          part[v][p] = t;
        }
      }
    }
  } else {
    float B[3][P];  // d xi_d / d x_c at the line's nodes
    if (act) {
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) B[c][p] = met[(3 * d + c) * Nl + e0 + base + p * stride];
    }
    if (l < NP) stage_fluxes<N, float>(a, e0 + l, l, F);
    __syncthreads();
    if (act) {
      // s[p] = d F_f / d xi_d at node p of the line
      auto deriv = [&](int f, float (&s)[P]) {
        const float* Ff = F + f * NP + base;
        float x[P];
#pragma unroll
        for (int m = 0; m < P; ++m) x[m] = Ff[m * stride];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          float t = 0.0f;
#pragma unroll
          for (int m = 0; m < P; ++m) t = fmaf(cD32<N>(p, m), x[m], t);
          s[p] = t;
        }
      };
      float s[P];
      // mass: div U
      deriv(kUx, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[0][p] = s[p] * B[0][p];
      deriv(kUy, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[0][p] = fmaf(s[p], B[1][p], part[0][p]);
      deriv(kUz, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[0][p] = fmaf(s[p], B[2][p], part[0][p]);
      // momentum: div (U (x) u + p' I)
      deriv(kPp, s);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        part[1][p] = s[p] * B[0][p];
        part[2][p] = s[p] * B[1][p];
        part[3][p] = s[p] * B[2][p];
      }
      deriv(kTxx, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[1][p] = fmaf(s[p], B[0][p], part[1][p]);
      deriv(kTxy, s);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        part[1][p] = fmaf(s[p], B[1][p], part[1][p]);
        part[2][p] = fmaf(s[p], B[0][p], part[2][p]);
      }
      deriv(kTxz, s);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        part[1][p] = fmaf(s[p], B[2][p], part[1][p]);
        part[3][p] = fmaf(s[p], B[0][p], part[3][p]);
      }
      deriv(kTyy, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[2][p] = fmaf(s[p], B[1][p], part[2][p]);
      deriv(kTyz, s);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        part[2][p] = fmaf(s[p], B[2][p], part[2][p]);
        part[3][p] = fmaf(s[p], B[1][p], part[3][p]);
      }
      deriv(kTzz, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[3][p] = fmaf(s[p], B[2][p], part[3][p]);
      // potential temperature: div (theta U)
      deriv(kHx, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[4][p] = s[p] * B[0][p];
      deriv(kHy, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[4][p] = fmaf(s[p], B[1][p], part[4][p]);
      deriv(kHz, s);
#pragma unroll
      for (int p = 0; p < P; ++p) part[4][p] = fmaf(s[p], B[2][p], part[4][p]);
    }
  }
  __syncthreads();  // every flux value has been read: the tile now takes the partial sums
  if (act) {
    float* acc = F + d * 5 * NP + base;
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int p = 0; p < P; ++p) acc[v * NP + p * stride] = part[v][p];
  }
  __syncthreads();
  if (l < NP) {
    const long long n = e0 + l;
    const float jw = met[9 * Nl + n];
    float* re = static_cast<float*>(a.re);
#pragma unroll
    for (int v = 0; v < 5; ++v) re[v * Nl + n] = -(jw * ((F[v * NP + l] + F[(5 + v) * NP + l]) + F[(10 + v) * NP + l]));
  }
}

// create_rhs of element e in the pairs mode: the steps of
// volume_element_nodal64 (12 flux fields with the pressure on the diagonal,
// metric terms pre-multiplied by -Jw: rows 0..8 of met2 hold -Jw dxi_d/dx_c
// for this form), every value and product carried as a (hi, lo) float pair.
// The fluxes are differentiated less their values at element node 0, and
// p' enters less its node-0 value, so that the 48-bit products round at the
// level of the fields' variation, not of their common level.  smem_raw
// holds 12 (N+1)^3 + (N+1)^2 + 12 pairs.
template <int N>
__device__ __forceinline__ void volume_element_pairs(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  constexpr int P = N + 1, NP = P * P * P;
  Pairs* F = reinterpret_cast<Pairs*>(smem_raw);  // [kLF][NP]
  Pairs* Ds = F + kLF * NP;                         // [P][P]
  Pairs* base = Ds + P * P;                         // [kLF]: the fluxes at element node 0
  const Pairs* Dg = reinterpret_cast<const Pairs*>(a.D2);
  const Pairs* met = reinterpret_cast<const Pairs*>(a.met2);
  const int l = threadIdx.x;
  for (int t = l; t < P * P; t += blockDim.x) Ds[t] = Dg[t];
  const long long e0 = e * NP, n = e0 + l;
  const long long Ng = a.Ng, Nl = a.Nl;
  if (l < NP) {
    const int g = a.l2g[n];
    const Pairs* w = static_cast<const Pairs*>(a.prim);
    const Pairs Ux = w[g], Uy = w[Ng + g], Uz = w[2 * Ng + g];
    const Pairs ux = w[3 * Ng + g], uy = w[4 * Ng + g], uz = w[5 * Ng + g];
    const Pairs th = w[6 * Ng + g];
    const Pairs pp = pp_sub(w[7 * Ng + g], w[7 * Ng + a.l2g[e0]]);
    Pairs v[kLF];
    v[lUx] = Ux;
    v[lUy] = Uy;
    v[lUz] = Uz;
    v[lTxx] = pp_add(pp_mul(Ux, ux), pp);
    v[lTyy] = pp_add(pp_mul(Uy, uy), pp);
    v[lTzz] = pp_add(pp_mul(Uz, uz), pp);
    v[lTxy] = pp_mul(Ux, uy);
    v[lTxz] = pp_mul(Ux, uz);
    v[lTyz] = pp_mul(Uy, uz);
    v[lHx] = pp_mul(th, Ux);
    v[lHy] = pp_mul(th, Uy);
    v[lHz] = pp_mul(th, Uz);
#pragma unroll
    for (int f = 0; f < kLF; ++f) F[f * NP + l] = v[f];
    if (l == 0) {
#pragma unroll
      for (int f = 0; f < kLF; ++f) base[f] = v[f];
    }
  }
  __syncthreads();
  // D annihilates constants, so the derivatives of F and of F - F(node 0)
  // are the same; the differences keep their full relative accuracy in the
  // contractions (no cancellation against the fields' common level).  Each
  // thread rewrites only its own node's entries.
  if (l < NP) {
#pragma unroll
    for (int f = 0; f < kLF; ++f) F[f * NP + l] = pp_sub(F[f * NP + l], base[f]);
  }
  __syncthreads();
  if (l >= NP) return;
  const int i = l % P, j = (l / P) % P, k = l / (P * P);
  Pairs B[9];  // -Jw dxi_d/dx_c at this node, [3d + c]
#pragma unroll
  for (int t = 0; t < 9; ++t) B[t] = met[t * Nl + n];
  const int bx = P * (j + P * k), by = i + P * P * k, bz = i + P * j;
  // reference-space derivatives (Eq. 5) as normalised pairs
  auto dref = [&](int f, Pairs& s0, Pairs& s1, Pairs& s2) {
    const Pairs* Ff = F + f * NP;
    float h0, l0, h1, l1, h2, l2;
    pp_first(h0, l0, Ds[i * P], Ff[bx]);
    pp_first(h1, l1, Ds[j * P], Ff[by]);
    pp_first(h2, l2, Ds[k * P], Ff[bz]);
#pragma unroll
    for (int m = 1; m < P; ++m) {
      pp_fma(h0, l0, Ds[i * P + m], Ff[bx + m]);
      pp_fma(h1, l1, Ds[j * P + m], Ff[by + P * m]);
      pp_fma(h2, l2, Ds[k * P + m], Ff[bz + P * P * m]);
    }
    s0 = pp_norm(h0, l0);
    s1 = pp_norm(h1, l1);
    s2 = pp_norm(h2, l2);
  };
  // chain rule into the weighted divergence: (dh, dl) += -Jw d/dx_c of a field
  auto phys = [&](float& dh, float& dl, bool first, int c, Pairs s0, Pairs s1, Pairs s2) {
    if (first) pp_first(dh, dl, s0, B[c]);
    else pp_fma(dh, dl, s0, B[c]);
    pp_fma(dh, dl, s1, B[3 + c]);
    pp_fma(dh, dl, s2, B[6 + c]);
  };
  Pairs s0, s1, s2;
  float rh, rl, xh, xl, yh, yl, zh, zl, th_, tl;
  dref(lUx, s0, s1, s2); phys(rh, rl, true, 0, s0, s1, s2);
  dref(lUy, s0, s1, s2); phys(rh, rl, false, 1, s0, s1, s2);
  dref(lUz, s0, s1, s2); phys(rh, rl, false, 2, s0, s1, s2);
  dref(lTxx, s0, s1, s2); phys(xh, xl, true, 0, s0, s1, s2);
  dref(lTyy, s0, s1, s2); phys(yh, yl, true, 1, s0, s1, s2);
  dref(lTzz, s0, s1, s2); phys(zh, zl, true, 2, s0, s1, s2);
  dref(lTxy, s0, s1, s2); phys(xh, xl, false, 1, s0, s1, s2); phys(yh, yl, false, 0, s0, s1, s2);
  dref(lTxz, s0, s1, s2); phys(xh, xl, false, 2, s0, s1, s2); phys(zh, zl, false, 0, s0, s1, s2);
  dref(lTyz, s0, s1, s2); phys(yh, yl, false, 2, s0, s1, s2); phys(zh, zl, false, 1, s0, s1, s2);
  dref(lHx, s0, s1, s2); phys(th_, tl, true, 0, s0, s1, s2);
  dref(lHy, s0, s1, s2); phys(th_, tl, false, 1, s0, s1, s2);
  dref(lHz, s0, s1, s2); phys(th_, tl, false, 2, s0, s1, s2);
  // the weighted residual -Jw div F of Eq. 4 in FP64 (the pair is exact in a double)
  double* re = static_cast<double*>(a.re);
  re[n] = join64(pp_norm(rh, rl));
  re[Nl + n] = join64(pp_norm(xh, xl));
  re[2 * Nl + n] = join64(pp_norm(yh, yl));
  re[3 * Nl + n] = join64(pp_norm(zh, zl));
  re[4 * Nl + n] = join64(pp_norm(th_, tl));
}

// create_rhs of an affine element in the pairs mode: the contravariant
// fluxes of stage_fluxes_affine in (hi, lo) float pairs, less their values
// at element node 0, and three contractions with D per equation.  smem_raw
// holds 15 (N+1)^3 + (N+1)^2 + 15 pairs.
template <int N>
__device__ __forceinline__ void volume_element_pairs_affine(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  constexpr int P = N + 1, NP = P * P * P;
  Pairs* G = reinterpret_cast<Pairs*>(smem_raw);  // [15][NP]
  Pairs* Ds = G + 15 * NP;                         // [P][P]
  Pairs* base = Ds + P * P;                        // [15]: the fluxes at element node 0
  const Pairs* Dg = reinterpret_cast<const Pairs*>(a.D2);
  const Pairs* met = reinterpret_cast<const Pairs*>(a.met2);
  const int l = threadIdx.x;
  for (int t = l; t < P * P; t += blockDim.x) Ds[t] = Dg[t];
  const long long e0 = e * NP, n = e0 + l;
  const long long Ng = a.Ng, Nl = a.Nl;
  if (l < NP) {
    Pairs B[9];  // the element's metric terms, at its first node
#pragma unroll
    for (int t = 0; t < 9; ++t) B[t] = met[t * Nl + e0];
    const int g = a.l2g[n];
    const Pairs* w = static_cast<const Pairs*>(a.prim);
    const Pairs Ux = w[g], Uy = w[Ng + g], Uz = w[2 * Ng + g];
    const Pairs ux = w[3 * Ng + g], uy = w[4 * Ng + g], uz = w[5 * Ng + g];
    const Pairs th = w[6 * Ng + g];
    // p' relative to its value at element node 0: B_dc p'(node 0) is constant
    // over the element and D annihilates it, and the difference keeps the
    // pressure term's rounding at the level of its variation, not of p'
    const Pairs pp = pp_sub(w[7 * Ng + g], w[7 * Ng + a.l2g[e0]]);
    Pairs v[15];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float h, lo;
      pp_first(h, lo, B[3 * d], ux);
      pp_fma(h, lo, B[3 * d + 1], uy);
      pp_fma(h, lo, B[3 * d + 2], uz);
      const Pairs ud = pp_norm(h, lo);  // B_d . u
      pp_first(h, lo, B[3 * d], Ux);
      pp_fma(h, lo, B[3 * d + 1], Uy);
      pp_fma(h, lo, B[3 * d + 2], Uz);
      const Pairs Gr = pp_norm(h, lo);  // B_d . U
      v[d] = Gr;
      pp_first(h, lo, Ux, ud);
      pp_fma(h, lo, B[3 * d], pp);
      v[3 + d] = pp_norm(h, lo);
      pp_first(h, lo, Uy, ud);
      pp_fma(h, lo, B[3 * d + 1], pp);
      v[6 + d] = pp_norm(h, lo);
      pp_first(h, lo, Uz, ud);
      pp_fma(h, lo, B[3 * d + 2], pp);
      v[9 + d] = pp_norm(h, lo);
      v[12 + d] = pp_mul(th, Gr);
    }
#pragma unroll
    for (int f = 0; f < 15; ++f) G[f * NP + l] = v[f];
    if (l == 0) {
#pragma unroll
      for (int f = 0; f < 15; ++f) base[f] = v[f];
    }
  }
  __syncthreads();
  // D annihilates constants: differentiate G - G(node 0), as in the per-node form
  if (l < NP) {
#pragma unroll
    for (int f = 0; f < 15; ++f) G[f * NP + l] = pp_sub(G[f * NP + l], base[f]);
  }
  __syncthreads();
  if (l >= NP) return;
  const int i = l % P, j = (l / P) % P, k = l / (P * P);
  const int bx = P * (j + P * k), by = i + P * P * k, bz = i + P * j;
  const Pairs jw = met[9 * Nl + n];
  double* re = static_cast<double*>(a.re);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const Pairs* g0 = G + (3 * v) * NP;
    const Pairs* g1 = g0 + NP;
    const Pairs* g2 = g1 + NP;
    float h, lo;
    pp_first(h, lo, Ds[i * P], g0[bx]);
#pragma unroll
    for (int m = 1; m < P; ++m) pp_fma(h, lo, Ds[i * P + m], g0[bx + m]);
#pragma unroll
    for (int m = 0; m < P; ++m) pp_fma(h, lo, Ds[j * P + m], g1[by + P * m]);
#pragma unroll
    for (int m = 0; m < P; ++m) pp_fma(h, lo, Ds[k * P + m], g2[bz + P * P * m]);
    re[v * Nl + n] = -join64(pp_mul(jw, pp_norm(h, lo)));
  }
}

// create_rhs of a rectilinear affine element in the pairs mode: the folded
// form of volume_element_rect (K_d D per direction, the weight w_i w_j w_k
// left to the update's inverse mass, no metric or Jw per node) in (hi, lo)
// float pairs.  The 12 unweighted fields are differentiated less their values at
// element node 0 (K_d D annihilates constants as D does), and p' enters less
// its node-0 value (as in volume_element_pairs_affine).  smem_raw holds
// 12 (N+1)^3 + 3 (N+1)^2 + 12 pairs.
template <int N>
__device__ __forceinline__ void volume_element_pairs_rect(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  constexpr int P = N + 1, PP = P * P, NP = PP * P;
  Pairs* F = reinterpret_cast<Pairs*>(smem_raw);  // [kLF][NP]
  Pairs* Dk = F + kLF * NP;                        // [3][P][P]: K_d D
  Pairs* base = Dk + 3 * PP;                       // [kLF]: the fluxes at element node 0
  const int l = threadIdx.x;
  for (int t = l; t < 3 * PP; t += blockDim.x) {
    const int d = t / PP;
    Dk[t] = split64(a.affk[d * (long long)a.Ne + e] * a.D64[t - d * PP]);
  }
  const long long e0 = e * NP, n = e0 + l;
  const long long Ng = a.Ng, Nl = a.Nl;
  if (l < NP) {
    const int g = a.l2g[n];
    const Pairs* w = static_cast<const Pairs*>(a.prim);
    const Pairs Ux = w[g], Uy = w[Ng + g], Uz = w[2 * Ng + g];
    const Pairs ux = w[3 * Ng + g], uy = w[4 * Ng + g], uz = w[5 * Ng + g];
    const Pairs th = w[6 * Ng + g];
    const Pairs pp = pp_sub(w[7 * Ng + g], w[7 * Ng + a.l2g[e0]]);
    Pairs v[kLF];
    v[lUx] = Ux;
    v[lUy] = Uy;
    v[lUz] = Uz;
    v[lTxx] = pp_add(pp_mul(Ux, ux), pp);
    v[lTyy] = pp_add(pp_mul(Uy, uy), pp);
    v[lTzz] = pp_add(pp_mul(Uz, uz), pp);
    v[lTxy] = pp_mul(Ux, uy);
    v[lTxz] = pp_mul(Ux, uz);
    v[lTyz] = pp_mul(Uy, uz);
    v[lHx] = pp_mul(th, Ux);
    v[lHy] = pp_mul(th, Uy);
    v[lHz] = pp_mul(th, Uz);
#pragma unroll
    for (int f = 0; f < kLF; ++f) F[f * NP + l] = v[f];
    if (l == 0) {
#pragma unroll
      for (int f = 0; f < kLF; ++f) base[f] = v[f];
    }
  }
  __syncthreads();
  if (l < NP) {
#pragma unroll
    for (int f = 0; f < kLF; ++f) F[f * NP + l] = pp_sub(F[f * NP + l], base[f]);
  }
  __syncthreads();
  if (l >= NP) return;
  const int i = l % P, j = (l / P) % P, k = l / PP;
  const int bx = P * (j + P * k), by = i + PP * k, bz = i + P * j;
  double* re = static_cast<double*>(a.re);
  auto div = [&](int fx, int fy, int fz) {
    const Pairs* gx = F + fx * NP;
    const Pairs* gy = F + fy * NP;
    const Pairs* gz = F + fz * NP;
    float h, lo;
    pp_first(h, lo, Dk[i * P], gx[bx]);
#pragma unroll
    for (int m = 1; m < P; ++m) pp_fma(h, lo, Dk[i * P + m], gx[bx + m]);
#pragma unroll
    for (int m = 0; m < P; ++m) pp_fma(h, lo, Dk[PP + j * P + m], gy[by + P * m]);
#pragma unroll
    for (int m = 0; m < P; ++m) pp_fma(h, lo, Dk[2 * PP + k * P + m], gz[bz + PP * m]);
    return join64(pp_norm(h, lo));
  };
  re[n] = div(lUx, lUy, lUz);
  re[Nl + n] = div(lTxx, lTxy, lTxz);
  re[2 * Nl + n] = div(lTxy, lTyy, lTyz);
  re[3 * Nl + n] = div(lTxz, lTyz, lTzz);
  re[4 * Nl + n] = div(lHx, lHy, lHz);
}

// Dynamic shared memory of one element: the staged fluxes, D and (pairs
// mode) the node-0 base values.
template <int N, typename T, bool AFF>
constexpr size_t element_smem_bytes() {
  constexpr int P = N + 1, NP = P * P * P;
  if constexpr (std::is_same<T, float>::value) return sizeof(float) * (kNF > 15 ? kNF : 15) * NP;
  if constexpr (AFF && std::is_same<T, double>::value) return sizeof(T) * (kLF * NP + 3 * P * P);
  if constexpr (std::is_same<T, double>::value) return sizeof(T) * (kLF * NP + P * P);
  if constexpr (AFF) return sizeof(T) * (15 * NP + P * P + 15);
  return sizeof(T) * (kLF * NP + P * P + kLF);
}

// Element kernel of one precision; AFF selects the affine-element form.
template <int N, typename T, bool AFF>
__device__ __forceinline__ void element_rhs(const VolumeArgs& a, long long e, unsigned char* smem_raw) {
  if constexpr (std::is_same<T, Pairs>::value) {
    if constexpr (AFF) {
      // uniform over the CTA: rectilinear elements take the folded form
      if (a.affine == 2) volume_element_pairs_rect<N>(a, e, smem_raw);
      else volume_element_pairs_affine<N>(a, e, smem_raw);
    } else {
      volume_element_pairs<N>(a, e, smem_raw);
    }
  } else if constexpr (std::is_same<T, float>::value) {
    volume_element_lines<N, AFF>(a, e, smem_raw);
  } else if constexpr (AFF) {
    // FP64 launches the affine instantiation for rectilinear elements only
    // (volume_form); other affine meshes take the per-node form
    volume_element_rect<N>(a, e, smem_raw);
  } else {
    volume_element_nodal64<N>(a, e, smem_raw);
  }
}

template <int N, typename T, bool AFF>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    volume_kernel(VolumeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  element_rhs<N, T, AFF>(a, a.ebeg + (long long)blockIdx.x, smem_raw);
}

template <typename RT>
__device__ __forceinline__ double re_load(const void* re, long long idx) {
  if constexpr (sizeof(RT) == 8) return static_cast<const double*>(re)[idx];
  else return f2d(static_cast<const float*>(re)[idx]);
}

// DSS, inverse mass, sources, walls and the stage update at global node I of
// one mesh (shared by the single-mesh and the ragged kernels).  MODE 0 writes
// the tendency R; MODE 1 a general RK stage; MODE 2 the first stage (a = 0,
// b = 1: no q^n read, no q^n term); MODE 3 the DSS of the filter correction,
// q + M^-1 DSS(Jw ((F x F x F) q - q)), with the wall-normal momentum left as
// it was; MODE 4 a stage of the low-storage scheme, MODE 5 its first stage.
// Direct stiffness summation at global node I in ascending element-node
// order (Eq. 4), FP64; every global node has at least one element node.
template <typename RT>
__device__ __forceinline__ void dss_node(const UpdateArgs& a, long long I, double (&s)[5]) {
  const long long Nl = a.Nl;
  const int t0 = a.off[I], t1 = a.off[I + 1];
  const long long n0 = a.idx[t0];
#pragma unroll
  for (int v = 0; v < 5; ++v) s[v] = re_load<RT>(a.re, v * Nl + n0);
  for (int t = t0 + 1; t < t1; ++t) {
    const long long n = a.idx[t];
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += re_load<RT>(a.re, v * Nl + n);
  }
}

// Element nodes at lattice index x along one axis of a CG box with ne
// elements of order N along it: one (element, local index) pair inside an
// element, two on a face between elements (and at a periodic seam), sorted by
// element, then local index; returned as their parts se*e + sl*i of the
// element-node index.
__device__ __forceinline__ int axis_nodes(unsigned x, unsigned N, unsigned ne, int per, unsigned se, unsigned sl,
                                          unsigned (&o)[2]) {
  const unsigned q = x / N, r = x - q * N;
  if (r != 0) {
    o[0] = q * se + r * sl;
    return 1;
  }
  if (!per) {
    if (q == 0) {
      o[0] = 0;
      return 1;
    }
    if (q == ne) {  // the far wall
      o[0] = (ne - 1) * se + N * sl;
      return 1;
    }
    o[0] = (q - 1) * se + N * sl;
    o[1] = q * se;
    return 2;
  }
  const unsigned qm = q == 0 ? ne - 1 : q - 1;  // periodic: x < ne N, the seam wraps
  if (qm < q) {
    o[0] = qm * se + N * sl;
    o[1] = q * se;
  } else {  // qm > q, or qm == q (one element along the axis): (q, 0) first
    o[0] = q * se;
    o[1] = qm * se + N * sl;
  }
  return 2;
}

// Direct stiffness summation at global node I of a CG box, with the element
// nodes found from the structured numbering (g = ix + nx (iy + ny iz), element
// e = ex + nex (ey + ney ez), local l = i + P (j + P k), element node
// n = e (N+1)^3 + l) instead of the inverse map: the same terms summed in the
// same ascending element-node order as dss_node, so the sums are identical.
// Where the axis-by-axis order is not ascending overall (possible only with
// single-element periodic axes) the node falls back to the inverse map.  The
// host enables this only for meshes with fewer than 2^31 element nodes.
template <typename RT>
__device__ __forceinline__ void dss_box(const UpdateArgs& a, long long I, double (&s)[5]) {
  const unsigned N = (unsigned)a.box_N, P = N + 1, NP = P * P * P;
  const unsigned nex = (unsigned)a.box_ne[0], ney = (unsigned)a.box_ne[1];
  const unsigned nx = (unsigned)a.box_n[0], ny = (unsigned)a.box_n[1];
  const unsigned u = (unsigned)I, t = u / nx, ix = u - t * nx, iz = t / ny, iy = t - iz * ny;
  unsigned xo[2], yo[2], zo[2];
  const int cx = axis_nodes(ix, N, nex, a.box_per[0], NP, 1, xo);
  const int cy = axis_nodes(iy, N, ney, a.box_per[1], nex * NP, P, yo);
  const int cz = axis_nodes(iz, N, (unsigned)a.box_ne[2], a.box_per[2], nex * ney * NP, P * P, zo);
  bool ascending = true;
  unsigned prev = 0;
  bool any = false;
  for (int zc = 0; zc < cz; ++zc)
    for (int yc = 0; yc < cy; ++yc)
      for (int xc = 0; xc < cx; ++xc) {
        const unsigned n = zo[zc] + yo[yc] + xo[xc];
        ascending &= !any || n > prev;
        prev = n;
        any = true;
      }
  if (!ascending) {
    dss_node<RT>(a, I, s);
    return;
  }
  const long long Nl = a.Nl;
  bool first = true;
  for (int zc = 0; zc < cz; ++zc)
    for (int yc = 0; yc < cy; ++yc)
      for (int xc = 0; xc < cx; ++xc) {
        const long long n = zo[zc] + yo[yc] + xo[xc];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double r = re_load<RT>(a.re, v * Nl + n);
          s[v] = first ? r : s[v] + r;
        }
        first = false;
      }
}

// Everything after the DSS at global node I, given its sums s0..s4.
template <int MODE, bool SHELL, bool F32>
__device__ __forceinline__ void update_node_sums(const UpdateArgs& a, long long I, double s0, double s1, double s2,
                                                 double s3, double s4) {
  const long long Ng = a.Ng;
  const double minv = a.Minv[I];
  const double rp = a.qk[I];
  const uint8_t w = a.wall[I];
  if constexpr (MODE == 3) {
    double c1 = s1 * minv, c2 = s2 * minv, c3 = s3 * minv;
    if constexpr (SHELL) {
      if (w & 8) {  // no radial correction at the bottom and lid
        const double nx = a.nrm[I], ny = a.nrm[Ng + I], nz = a.nrm[2 * Ng + I];
        const double dot = c1 * nx + c2 * ny + c3 * nz;
        c1 -= dot * nx;
        c2 -= dot * ny;
        c3 -= dot * nz;
      }
    } else {
      if (w & 1) c1 = 0.0;
      if (w & 2) c2 = 0.0;
      if (w & 4) c3 = 0.0;
    }
    const double y0 = fma(s0, minv, rp), y1 = a.qk[Ng + I] + c1, y2 = a.qk[2 * Ng + I] + c2;
    const double y3 = a.qk[3 * Ng + I] + c3, y4 = fma(s4, minv, a.qk[4 * Ng + I]);
    a.out[I] = y0;
    a.out[Ng + I] = y1;
    a.out[2 * Ng + I] = y2;
    a.out[3 * Ng + I] = y3;
    a.out[4 * Ng + I] = y4;
    if (nonfinite(y0) | nonfinite(y1) | nonfinite(y2) | nonfinite(y3) | nonfinite(y4)) atomicOr(a.flag, 1);
    write_prim<F32>(a.pa, I, y0, y1, y2, y3, y4);
    return;
  }
  if constexpr (MODE == 0 || MODE >= 4 || SHELL) {
    // R = M^-1 DSS(r_e) + S, then the wall condition
    double R0 = s0 * minv, R1 = s1 * minv, R2 = s2 * minv, R3 = s3 * minv, R4 = s4 * minv;
    if constexpr (SHELL) {
      // buoyancy of rho' along g(r) r_hat and Coriolis -2 Omega z x U
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
      return;
    }
    s0 = R0;  // the stage combination below takes the full tendency
    s1 = R1;
    s2 = R2;
    s3 = R3;
    s4 = R4;
  }
  if constexpr (MODE >= 4) {
    // low-storage stage (MODE 5: the first, A = 0): dq <- A dq + dt R,
    // q <- q + B dq, in place
    double y[5];
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double Rv = v == 0 ? s0 : v == 1 ? s1 : v == 2 ? s2 : v == 3 ? s3 : s4;
      double dqv;
      if constexpr (MODE == 5) dqv = a.dt * Rv;
      else dqv = fma(a.a, a.dq[v * Ng + I], a.dt * Rv);
      a.dq[v * Ng + I] = dqv;
      y[v] = fma(a.b, dqv, v == 0 ? rp : a.qk[v * Ng + I]);
      a.out[v * Ng + I] = y[v];
      bad |= nonfinite(y[v]);
    }
    if (bad) atomicOr(a.flag, 1);
    write_prim<F32>(a.pa, I, y[0], y[1], y[2], y[3], y[4]);
  } else if constexpr (MODE >= 1) {
    // q^{k+1} = a q^n + b q^k + b dt R with, in the box, the inverse mass
    // folded into one coefficient: b dt R_v = c s_v (+ b dt S_v), c = b dt / M
    const double c = SHELL ? a.bdt : a.bdt * minv;
    double y[5];
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double qk = (v == 0) ? rp : a.qk[v * Ng + I];
      // first stage (MODE 2: a = 0, b = 1): t = q^k; otherwise a q^n + b q^k
      double t;
      if constexpr (MODE == 2) t = qk;
      else t = fma(a.a, a.qn[v * Ng + I], a.b * qk);
      const double sv = v == 0 ? s0 : v == 1 ? s1 : v == 2 ? s2 : v == 3 ? s3 : s4;
      if constexpr (!SHELL) {
        // a wall removes the whole normal momentum tendency, source included
        const bool walled = (v >= 1 && v <= 3) && (w & (1 << (v - 1)));
        if (v == 3 && !walled) t = fma(-rp, a.bdtg, t);  // buoyancy -rho' g
        y[v] = walled ? t : fma(c, sv, t);
      } else {
        y[v] = fma(c, sv, t);
      }
      a.out[v * Ng + I] = y[v];
      bad |= nonfinite(y[v]);
    }
    if (bad) atomicOr(a.flag, 1);
    write_prim<F32>(a.pa, I, y[0], y[1], y[2], y[3], y[4]);
  }
}

template <int MODE, bool SHELL, typename RT>
__device__ __forceinline__ void update_node(const UpdateArgs& a, long long I) {
  double s[5];
  dss_node<RT>(a, I, s);
  update_node_sums<MODE, SHELL, std::is_same<RT, float>::value>(a, I, s[0], s[1], s[2], s[3], s[4]);
}

// One block per kDssBlock consecutive global nodes.  The DSS runs in the
// block's precomputed order (nodes sorted by their number of element nodes,
// so that the lanes of a warp loop equally often) and leaves the sums in
// shared memory; the rest runs in natural order (coalesced).  Each node's
// sum is the same as update_node's, bit for bit.  BOX: a CG box, whose DSS
// finds the element nodes from the structured numbering (dss_box).
template <int MODE, bool SHELL, typename RT, bool BOX = false>
__global__ void __launch_bounds__(kDssBlock) update_kernel(UpdateArgs a) {
  __shared__ double sums[5][kDssBlock];
  const long long base = a.ibeg + (long long)blockIdx.x * kDssBlock;
  {
    const int lt = a.order[base + threadIdx.x];
    const long long IA = base + lt;
    if (IA < a.iend) {
      double s[5];
      if constexpr (BOX) dss_box<RT>(a, IA, s);
      else dss_node<RT>(a, IA, s);
#pragma unroll
      for (int v = 0; v < 5; ++v) sums[v][lt] = s[v];
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  const long long I = base + t;
  if (I < a.iend)
    update_node_sums<MODE, SHELL, std::is_same<RT, float>::value>(a, I, sums[0][t], sums[1][t], sums[2][t], sums[3][t],
                                                                  sums[4][t]);
}

// ---- ragged multi-member kernels (serving) ---------------------------------
// Persistent kernels over the concatenated elements (or global nodes) of the
// members of one group (same N, precision and mesh kind); the group table
// maps a position in the concatenation to (member, local index).  Each
// member's work is done by the same element / node functions as above.

__device__ __forceinline__ int ragged_find(const long long* prefix, int n, long long w) {
  int lo = 0, hi = n - 1;  // last m with prefix[m] <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int N, typename T, bool AFF>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    volume_ragged(const MemberDesc* __restrict__ d, const RaggedGroup* __restrict__ g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_m;
  __shared__ long long s_e;
  const int n = g->n;
  const long long total = n > 0 ? g->elem_prefix[n] : 0;
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    if (threadIdx.x == 0) {
      const int m = ragged_find(g->elem_prefix, n, w);
      s_m = g->member[m];
      s_e = w - g->elem_prefix[m];
    }
    __syncthreads();
    // (uniform across the CTA) guard against a table that disagrees with the member
    if (s_m >= 0 && s_m < kMaxMembers && s_e >= 0 && s_e < d[s_m].va.Ne)
      element_rhs<N, T, AFF>(d[s_m].va, s_e, smem_raw);
    __syncthreads();
  }
}

// One block of kDssBlock global nodes of one member per iteration, as in
// update_kernel: the member's DSS order within the block (sorted by entry
// count), the structured box DSS on CG boxes, then the rest in natural
// order.  Members' node ranges are padded to whole blocks in the table.
template <int MODE, bool SHELL, typename RT>
__global__ void __launch_bounds__(kDssBlock) update_ragged(const MemberDesc* __restrict__ d,
                                                           const RaggedGroup* __restrict__ g, int stage) {
  __shared__ double sums[5][kDssBlock];
  __shared__ int s_slot;
  __shared__ long long s_base;
  const int n = g->n;
  const long long total = n > 0 ? g->block_prefix[n] : 0;
  for (long long b = blockIdx.x; b < total; b += gridDim.x) {
    if (threadIdx.x == 0) {
      const int m = ragged_find(g->block_prefix, n, b);
      s_slot = g->member[m];
      s_base = (b - g->block_prefix[m]) * kDssBlock;
    }
    __syncthreads();
    const int slot = s_slot;
    const long long base = s_base;
    // (uniform across the CTA) guard against a table that disagrees with the member
    if (slot >= 0 && slot < kMaxMembers && base >= 0 && base < d[slot].ua[stage].iend) {
      const UpdateArgs& a = d[slot].ua[stage];
      const int lt = a.order[base + threadIdx.x];
      const long long IA = base + lt;
      if (IA < a.iend) {
        double s[5];
        if constexpr (SHELL) {
          dss_node<RT>(a, IA, s);
        } else {
          if (a.box_N) dss_box<RT>(a, IA, s);
          else dss_node<RT>(a, IA, s);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) sums[v][lt] = s[v];
      }
      __syncthreads();
      const int t = threadIdx.x;
      const long long I = base + t;
      if (I < a.iend)
        update_node_sums<MODE, SHELL, std::is_same<RT, float>::value>(a, I, sums[0][t], sums[1][t], sums[2][t],
                                                                      sums[3][t], sums[4][t]);
    }
    __syncthreads();  // the block's slot, base and sums are rewritten in the next iteration
  }
}

// Kernel attributes (the dynamic shared-memory limit) apply per device, so a
// launch template records per device (one bit each, up to 64) that it has
// set them there.  The bit is set after the attribute call succeeds: two
// host threads may both set an attribute, but none launches before it is set.
class DeviceFlags {
 public:
  bool has() const { return (bits_.load() >> device()) & 1ull; }
  void set() { bits_.fetch_or(1ull << device()); }

 private:
  static int device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return dev & 63;
  }
  std::atomic<unsigned long long> bits_{0};
};

// A per-device value computed once (SM count, persistent grid size).
class DeviceInts {
 public:
  int get() const { return v_[device()].load(); }
  void put(int x) { v_[device()].store(x); }

 private:
  static int device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return dev & 63;
  }
  std::atomic<int> v_[64] = {};
};

template <int N, typename T, bool AFF>
cudaError_t launch_volume_t(const VolumeArgs& a, cudaStream_t s) {
  constexpr int P = N + 1, NP = P * P * P;
  constexpr int NT = (NP + 31) / 32 * 32;
  const size_t smem = element_smem_bytes<N, T, AFF>();
  static DeviceFlags attr_set;
  if (!attr_set.has()) {
    cudaError_t e =
        cudaFuncSetAttribute(volume_kernel<N, T, AFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set.set();
  }
  if (a.ecnt <= 0) return cudaSuccess;
  volume_kernel<N, T, AFF><<<a.ecnt, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, bool AFF>
cudaError_t launch_volume_p(int N, const VolumeArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_volume_t<1, T, AFF>(a, s);
    case 2: return launch_volume_t<2, T, AFF>(a, s);
    case 3: return launch_volume_t<3, T, AFF>(a, s);
    case 4: return launch_volume_t<4, T, AFF>(a, s);
    case 5: return launch_volume_t<5, T, AFF>(a, s);
    case 6: return launch_volume_t<6, T, AFF>(a, s);
    case 7: return launch_volume_t<7, T, AFF>(a, s);
    case 8: return launch_volume_t<8, T, AFF>(a, s);
    default: return cudaErrorInvalidValue;
  }
}



// SMs of the current device.
int sm_count() {
  static DeviceInts count;
  int n = count.get();
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 1;
    count.put(n);
  }
  return n;
}

// Persistent launch: as many CTAs as fit on the GPU at once.
template <int N, typename T, bool AFF>
cudaError_t launch_volume_ragged_t(const MemberDesc* d, const RaggedGroup* g, cudaStream_t s) {
  constexpr int P = N + 1, NP = P * P * P;
  constexpr int NT = (NP + 31) / 32 * 32;
  const size_t smem = element_smem_bytes<N, T, AFF>();
  static DeviceInts grids;  // per device, set up at its first launch there
  int grid = grids.get();
  if (!grid) {
    cudaError_t e =
        cudaFuncSetAttribute(volume_ragged<N, T, AFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, volume_ragged<N, T, AFF>, NT, smem);
    if (e != cudaSuccess) return e;
    grid = (per_sm > 0 ? per_sm : 1) * sm_count();
    grids.put(grid);
  }
  volume_ragged<N, T, AFF><<<grid, NT, smem, s>>>(d, g);
  return cudaGetLastError();
}

template <typename T, bool AFF>
cudaError_t launch_volume_ragged_p(int N, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s) {
  switch (N) {
    case 1: return launch_volume_ragged_t<1, T, AFF>(d, g, s);
    case 2: return launch_volume_ragged_t<2, T, AFF>(d, g, s);
    case 3: return launch_volume_ragged_t<3, T, AFF>(d, g, s);
    case 4: return launch_volume_ragged_t<4, T, AFF>(d, g, s);
    case 5: return launch_volume_ragged_t<5, T, AFF>(d, g, s);
    case 6: return launch_volume_ragged_t<6, T, AFF>(d, g, s);
    case 7: return launch_volume_ragged_t<7, T, AFF>(d, g, s);
    case 8: return launch_volume_ragged_t<8, T, AFF>(d, g, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace numa
