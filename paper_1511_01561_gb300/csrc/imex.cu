// Column part of the 1D-IMEX leapfrog step (Sec. 2.2: an explicit leapfrog
// step, then implicit corrections along each vertical column of grid points;
// the IMEX line of the time loop in Sec. 7), for the z-columns of a box and
// the radial columns of the cubed-sphere shell.
//
// With the explicit tendency R = R(q^n) already in memory, per column:
//   q*  = qprev + cR R                      (cR = 2 dt; dt on the start step)
//   s   = 2 q^n - qprev                     (q^0 on the start step)
//   solve (I - tau L) x = q* - tau L s for rho', W, Theta'; U, V take q*.
// L couples rho', W (the momentum along the column) and Theta' through the
// column derivative Dz and the divergence G = Dz + 2/r (G = Dz in the box);
// eliminating rho' and Theta' leaves the Schur system H x_W = f in W,
//   H = I - tau^2 (Dz C2 G T0 + g G)        (identity rows at the walls),
// which in the increment y = x_W - s reads
//   H y = q*_W - s_W - tau g (q*_rho - s_rho) + tau Dz(c2 (s_Theta - q*_Theta))
// (q*_W - s_W at the walls), after which
//   x_W = s_W + y,  x_rho = q*_rho - tau G y,  x_Theta = q*_Theta - tau G(theta0 y).
// The Robert-Asselin filter gives qbar^n = q^n + nu (qprev - 2 q^n + x).
//
// One block holds cols_per_block consecutive columns.  Shared memory keeps
// the two vectors whose neighbours the column derivative reads ([2][nz][cols]
// doubles); values needed only at their own node (q*_rho, s_W, q*_Theta) go
// back into R, which the same thread reads at the end.  The derivative
// applications run over all (level, column) pairs of the block; one thread
// per column runs the banded LU sweeps.
#include "kernels_common.cuh"

namespace numa {
namespace {

constexpr int kImexThreads = 128;
constexpr size_t kImexSmemMax = 200 * 1024;

// Band entries [j0, j1] of row k of Dz that can be nonzero: the row of a node
// inside element e couples to that element's N+1 nodes; a node shared by two
// elements (k a multiple of N) to both elements' nodes.
__device__ __forceinline__ void dz_row_range(int k, int N, int nz, int& j0, int& j1) {
  const int i = k % N;
  if (i == 0) {
    j0 = max(0, N - k);
    j1 = min(2 * N, nz - 1 - k + N);
  } else {
    j0 = N - i;  // column k - i, the element's first node
    j1 = 2 * N - i;
  }
}

// Column c, level k is global node c + ncol k.  RADIAL = false: z-columns of
// the box (W = U_z); RADIAL = true: radial columns of the shell (W = U . r_hat,
// U^{n+1} = U* + (x_W - W*) r_hat).
template <bool RADIAL>
__global__ void __launch_bounds__(kImexThreads) imex_column_kernel(ImexArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int nz = a.nz, CPB = a.cols_per_block, N = a.N, W2 = 2 * a.N + 1, kl = a.kl, US = 1 + 4 * a.N;
  const long long Ng = a.Ng, ncol = a.ncol;
  const size_t plane = (size_t)nz * CPB;
  double* UT = sm;          // c2 (s_Theta - q*_Theta), then theta0 y
  double* EY = sm + plane;  // e, then r (right-hand side of H y = r), then y
  // the factors, read on the serial path of the sweeps, staged once per block
  double* Ls = EY + plane;                   // [nz][kl]
  double* Us = Ls + (size_t)nz * kl;         // [nz][1 + 4N]
  int* Ps = reinterpret_cast<int*>(Us + (size_t)nz * US);  // [nz][3]
  for (int t = threadIdx.x; t < nz * kl; t += blockDim.x) Ls[t] = a.Lf[t];
  for (int t = threadIdx.x; t < nz * US; t += blockDim.x) Us[t] = a.Uf[t];
  for (int t = threadIdx.x; t < 3 * nz; t += blockDim.x) Ps[t] = a.piv[t];
  double* R = a.R;
  const long long col0 = (long long)blockIdx.x * CPB;
  const double nu = a.nu, tau = a.tau;
  const int items = nz * CPB;
  auto node = [&](long long col, int k) -> long long { return col + ncol * k; };

  // explicit step, the filter's first part; U and V finished in the box,
  // U* parked in q on the shell
  for (int t = threadIdx.x; t < items; t += blockDim.x) {
    const int k = t / CPB, cl = t - k * CPB;
    const long long col = col0 + cl;
    if (col >= ncol) continue;
    const long long g = node(col, k);
    double qst[5], sv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double qn = a.q[v * Ng + g], qp = a.qprev[v * Ng + g];
      qst[v] = fma(a.cR, R[v * Ng + g], qp);
      sv[v] = fma(2.0, qn, -qp);  // s = 2 q^n - qprev, so qprev - 2 q^n = -s
      if (!RADIAL && (v == 1 || v == 2)) {
        a.q[v * Ng + g] = qst[v];
        a.qs[v * Ng + g] = fma(nu, qst[v] - sv[v], qn);  // x = q* for U and V
      } else {
        if (RADIAL && v >= 1 && v <= 3) a.q[v * Ng + g] = qst[v];
        a.qs[v * Ng + g] = fma(-nu, sv[v], qn);  // q^n + nu (qprev - 2 q^n)
      }
    }
    double wst = qst[3], swv = sv[3];
    if constexpr (RADIAL) {
      const double nx = a.nrm[g], ny = a.nrm[Ng + g], nz_ = a.nrm[2 * Ng + g];
      wst = fma(qst[1], nx, fma(qst[2], ny, qst[3] * nz_));
      swv = fma(sv[1], nx, fma(sv[2], ny, sv[3] * nz_));
      R[Ng + g] = wst;
    }
    R[g] = qst[0];
    R[3 * Ng + g] = swv;
    R[4 * Ng + g] = qst[4];
    const size_t o = (size_t)k * CPB + cl;
    UT[o] = a.c2[k] * (sv[4] - qst[4]);
    const double e = wst - swv;
    EY[o] = (k == 0 || k == nz - 1) ? e : fma(-tau * a.gl[k], qst[0] - sv[0], e);
  }
  __syncthreads();

  // r = e + tau Dz(c2 (s_Theta - q*_Theta)) on the interior rows
  for (int t = threadIdx.x; t < items; t += blockDim.x) {
    const int k = t / CPB, cl = t - k * CPB;
    if (k == 0 || k == nz - 1) continue;
    int j0, j1;
    dz_row_range(k, N, nz, j0, j1);
    double acc = 0.0;
    for (int j = j0; j <= j1; ++j) acc = fma(a.Dz[k * W2 + j], UT[(size_t)(k - N + j) * CPB + cl], acc);
    EY[(size_t)k * CPB + cl] = fma(tau, acc, EY[(size_t)k * CPB + cl]);
  }
  __syncthreads();

  // H y = r: forward elimination with the recorded row swaps, back substitution
  for (int cl = threadIdx.x; cl < CPB; cl += blockDim.x) {
    if (col0 + cl >= ncol) break;
    for (int k = 0; k < nz; ++k) {
      const int p = Ps[3 * k];
      double yk = EY[(size_t)k * CPB + cl];
      if (p != k) {
        const double yp = EY[(size_t)p * CPB + cl];
        EY[(size_t)p * CPB + cl] = yk;
        EY[(size_t)k * CPB + cl] = yp;
        yk = yp;
      }
      const int imax = Ps[3 * k + 1];
      for (int i = 1; i <= imax; ++i)
        EY[(size_t)(k + i) * CPB + cl] = fma(-Ls[k * kl + i - 1], yk, EY[(size_t)(k + i) * CPB + cl]);
    }
    for (int k = nz - 1; k >= 0; --k) {
      double acc = EY[(size_t)k * CPB + cl];
      const int jmax = Ps[3 * k + 2];
      for (int j = 1; j <= jmax; ++j) acc = fma(-Us[k * US + j], EY[(size_t)(k + j) * CPB + cl], acc);
      EY[(size_t)k * CPB + cl] = acc * Us[k * US];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < items; t += blockDim.x) UT[t] = a.th0[t / CPB] * EY[t];
  __syncthreads();

  // x_rho = q*_rho - tau G y, x_Theta = q*_Theta - tau G(theta0 y), x_W = s_W + y
  // (G = Dz + 2/r); q^{n+1}, the filtered q^n and the primitive fields of q^{n+1}
  for (int t = threadIdx.x; t < items; t += blockDim.x) {
    const int k = t / CPB, c = t - k * CPB;
    const long long col = col0 + c;
    if (col >= ncol) continue;
    const long long g = node(col, k);
    int j0, j1;
    dz_row_range(k, N, nz, j0, j1);
    double dy = 0.0, dty = 0.0;
    for (int j = j0; j <= j1; ++j) {
      const double d = a.Dz[k * W2 + j];
      const size_t o = (size_t)(k - N + j) * CPB + c;
      dy = fma(d, EY[o], dy);
      dty = fma(d, UT[o], dty);
    }
    const size_t o = (size_t)k * CPB + c;
    const double yk = EY[o];
    if constexpr (RADIAL) {
      dy = fma(a.r2[k], yk, dy);
      dty = fma(a.r2[k], UT[o], dty);
    }
    const double xr = fma(-tau, dy, R[g]);
    const double xw = R[3 * Ng + g] + yk;
    const double xt = fma(-tau, dty, R[4 * Ng + g]);
    a.q[g] = xr;
    a.q[4 * Ng + g] = xt;
    a.qs[g] = fma(nu, xr, a.qs[g]);
    a.qs[4 * Ng + g] = fma(nu, xt, a.qs[4 * Ng + g]);
    double xu, xv, xz;
    if constexpr (RADIAL) {
      const double dw = xw - R[Ng + g];  // x_W - W*
      xu = fma(dw, a.nrm[g], a.q[Ng + g]);
      xv = fma(dw, a.nrm[Ng + g], a.q[2 * Ng + g]);
      xz = fma(dw, a.nrm[2 * Ng + g], a.q[3 * Ng + g]);
      a.q[Ng + g] = xu;
      a.q[2 * Ng + g] = xv;
      a.qs[Ng + g] = fma(nu, xu, a.qs[Ng + g]);
      a.qs[2 * Ng + g] = fma(nu, xv, a.qs[2 * Ng + g]);
    } else {
      xu = a.q[Ng + g];
      xv = a.q[2 * Ng + g];
      xz = xw;
    }
    a.q[3 * Ng + g] = xz;
    a.qs[3 * Ng + g] = fma(nu, xz, a.qs[3 * Ng + g]);
    if (nonfinite(xr) | nonfinite(xu) | nonfinite(xv) | nonfinite(xz) | nonfinite(xt)) atomicOr(a.flag, 1);
    write_prim<false>(a.pa, g, xr, xu, xv, xz, xt);  // FP64 or pairs
  }
}

DeviceFlags imex_attr;

template <bool RADIAL>
cudaError_t set_imex_attr() {
  return cudaFuncSetAttribute(imex_column_kernel<RADIAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kImexSmemMax);
}

}  // namespace

// Columns per block: kImexColsTarget while a block's shared memory stays
// under kImexSmemMax / 2, fewer for tall columns.
constexpr int kImexColsTarget = 32;

int imex_cols_per_block(int nz, int N) {
  for (int c = kImexColsTarget; c >= 32; c /= 2)
    if (imex_smem_bytes(nz, N, c) <= kImexSmemMax / 2) return c;
  for (int c = 16; c >= 1; c /= 2)
    if (imex_smem_bytes(nz, N, c) <= kImexSmemMax) return c;
  return 0;
}

// Two column vectors per column, the factors of one Schur matrix (rows of
// 2N multipliers and 1 + 4N U entries) and the pivot rows.
size_t imex_smem_bytes(int nz, int N, int cols_per_block) {
  return sizeof(double) * (size_t)nz * (2 * (size_t)cols_per_block + 2 * N + 1 + 4 * N) + 3 * sizeof(int) * (size_t)nz;
}

cudaError_t imex_kernel_setup() {
  if (imex_attr.has()) return cudaSuccess;
  cudaError_t e = set_imex_attr<false>();
  if (e == cudaSuccess) e = set_imex_attr<true>();
  if (e == cudaSuccess) imex_attr.set();
  return e;
}

cudaError_t launch_imex(const ImexArgs& a, cudaStream_t s) {
  if (a.cols_per_block < 1 || a.cols_per_block > kImexThreads || a.nz < 2 || a.N < 1 || a.kl > 2 * a.N ||
      a.ku > 4 * a.N)
    return cudaErrorInvalidValue;
  const size_t smem = imex_smem_bytes(a.nz, a.N, a.cols_per_block);
  if (smem > kImexSmemMax || !imex_attr.has()) return cudaErrorInvalidValue;
  if (a.ncol == 0) return cudaSuccess;
  const long long blocks = (a.ncol + a.cols_per_block - 1) / a.cols_per_block;
  if (a.nrm) imex_column_kernel<true><<<(unsigned)blocks, kImexThreads, smem, s>>>(a);
  else imex_column_kernel<false><<<(unsigned)blocks, kImexThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace numa
