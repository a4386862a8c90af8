// Column part of the 1D-IMEX leapfrog step (Sec. 2.2: an explicit leapfrog
// step, then implicit corrections along each vertical column of grid points;
// the IMEX line of the time loop in Sec. 6).
//
// With the explicit tendency R = R(q^n) already in memory, per column:
//   q*  = qprev + cR R                      (cR = 2 dt; dt on the start step)
//   s   = 2 q^n - qprev                     (q^0 on the start step)
//   solve (I - tau L) x = q* - tau L s for rho', W, Theta'; U, V take q*.
// L couples rho', W and Theta' through the column derivative Dz; eliminating
// rho' and Theta' leaves the Schur system H x_W = f in W,
//   H = I - tau^2 (Dz C2 Dz T0 + g Dz)      (identity rows at the walls),
// which in the increment y = x_W - s reads
//   H y = q*_W - s_W - tau g (q*_rho - s_rho) + tau Dz(c2 (s_Theta - q*_Theta))
// (q*_W - s_W at the walls), after which
//   x_W = s_W + y,  x_rho = q*_rho - tau Dz y,  x_Theta = q*_Theta - tau Dz(theta0 y).
// The Robert-Asselin filter gives qbar^n = q^n + nu (qprev - 2 q^n + x).
//
// One block holds cols_per_block consecutive columns in shared memory
// ([5][nz][cols] doubles); all threads load and store (coalesced along the
// columns), one thread per column runs the banded solves.
#include "kernels_common.cuh"

namespace numa {
namespace {

constexpr int kImexThreads = 128;
constexpr size_t kImexSmemMax = 200 * 1024;

__global__ void __launch_bounds__(kImexThreads) imex_column_kernel(ImexArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int nz = a.nz, CPB = a.cols_per_block, N = a.N, W2 = 2 * a.N + 1;
  const long long Ng = a.Ng, ncol = a.ncol;
  const size_t plane = (size_t)nz * CPB;
  double* QR = sm;              // q*_rho, then x_rho
  double* QT = sm + plane;      // q*_Theta, then x_Theta
  double* SW = sm + 2 * plane;  // s_W, then x_W
  double* UT = sm + 3 * plane;  // c2 (s_Theta - q*_Theta), then theta0 y
  double* EY = sm + 4 * plane;  // right-hand side of H y = r, then y
  const long long col0 = (long long)blockIdx.x * CPB;
  const double nu = a.nu, tau = a.tau;

  // explicit step, the filter's first part, U and V finished
  for (int t = threadIdx.x; t < nz * CPB; t += blockDim.x) {
    const int k = t / CPB, cl = t - k * CPB;
    const long long col = col0 + cl;
    if (col >= ncol) continue;
    const long long g = col + ncol * k;
    double qs_[5], qn_[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double qn = a.q[v * Ng + g], qp = a.qprev[v * Ng + g];
      const double qst = fma(a.cR, a.R[v * Ng + g], qp);
      qs_[v] = qst;
      qn_[v] = fma(-2.0, qn, qp);  // qprev - 2 q^n
      if (v == 1 || v == 2) {
        a.q[v * Ng + g] = qst;
        a.qs[v * Ng + g] = fma(nu, qn_[v] + qst, qn);
      } else {
        a.qs[v * Ng + g] = fma(nu, qn_[v], qn);  // q^n + nu (qprev - 2 q^n)
      }
      qn_[v] = fma(2.0, qn, -qp);  // s = 2 q^n - qprev
    }
    const size_t o = (size_t)k * CPB + cl;
    QR[o] = qs_[0];
    QT[o] = qs_[4];
    SW[o] = qn_[3];
    UT[o] = a.c2[k] * (qn_[4] - qs_[4]);
    const double e = qs_[3] - qn_[3];
    EY[o] = (k == 0 || k == nz - 1) ? e : fma(-tau * a.g, qs_[0] - qn_[0], e);
  }
  __syncthreads();

  const int cl = threadIdx.x;
  if (cl < CPB && col0 + cl < ncol) {
    // r = e + tau Dz(c2 (s_Theta - q*_Theta)) on the interior rows
    for (int k = 1; k < nz - 1; ++k) {
      const int j0 = max(0, N - k), j1 = min(W2 - 1, nz - 1 - k + N);
      double acc = 0.0;
      for (int j = j0; j <= j1; ++j) acc = fma(a.Dz[k * W2 + j], UT[(size_t)(k - N + j) * CPB + cl], acc);
      EY[(size_t)k * CPB + cl] = fma(tau, acc, EY[(size_t)k * CPB + cl]);
    }
    // forward elimination with the recorded row swaps, then back substitution
    for (int k = 0; k < nz; ++k) {
      const int p = a.piv[k];
      double yk = EY[(size_t)k * CPB + cl];
      if (p != k) {
        const double yp = EY[(size_t)p * CPB + cl];
        EY[(size_t)p * CPB + cl] = yk;
        EY[(size_t)k * CPB + cl] = yp;
        yk = yp;
      }
      const int imax = min(a.kl, nz - 1 - k);
      for (int i = 1; i <= imax; ++i)
        EY[(size_t)(k + i) * CPB + cl] = fma(-a.Lf[k * a.kl + i - 1], yk, EY[(size_t)(k + i) * CPB + cl]);
    }
    const int US = 1 + 4 * N;
    for (int k = nz - 1; k >= 0; --k) {
      double acc = EY[(size_t)k * CPB + cl];
      const int jmax = min(a.ku, nz - 1 - k);
      for (int j = 1; j <= jmax; ++j) acc = fma(-a.Uf[k * US + j], EY[(size_t)(k + j) * CPB + cl], acc);
      EY[(size_t)k * CPB + cl] = acc * a.Uf[k * US];
    }
    for (int k = 0; k < nz; ++k) UT[(size_t)k * CPB + cl] = a.th0[k] * EY[(size_t)k * CPB + cl];
    // x_rho = q*_rho - tau Dz y, x_Theta = q*_Theta - tau Dz(theta0 y), x_W = s_W + y
    for (int k = 0; k < nz; ++k) {
      const int j0 = max(0, N - k), j1 = min(W2 - 1, nz - 1 - k + N);
      double dy = 0.0, dty = 0.0;
      for (int j = j0; j <= j1; ++j) {
        const double d = a.Dz[k * W2 + j];
        const size_t o = (size_t)(k - N + j) * CPB + cl;
        dy = fma(d, EY[o], dy);
        dty = fma(d, UT[o], dty);
      }
      const size_t o = (size_t)k * CPB + cl;
      QR[o] = fma(-tau, dy, QR[o]);
      QT[o] = fma(-tau, dty, QT[o]);
      SW[o] += EY[o];
    }
  }
  __syncthreads();

  // q^{n+1}, the filtered q^n and the primitive fields of q^{n+1}
  for (int t = threadIdx.x; t < nz * CPB; t += blockDim.x) {
    const int k = t / CPB, c = t - k * CPB;
    const long long col = col0 + c;
    if (col >= ncol) continue;
    const long long g = col + ncol * k;
    const size_t o = (size_t)k * CPB + c;
    const double xr = QR[o], xw = SW[o], xt = QT[o];
    a.q[g] = xr;
    a.q[3 * Ng + g] = xw;
    a.q[4 * Ng + g] = xt;
    a.qs[g] = fma(nu, xr, a.qs[g]);
    a.qs[3 * Ng + g] = fma(nu, xw, a.qs[3 * Ng + g]);
    a.qs[4 * Ng + g] = fma(nu, xt, a.qs[4 * Ng + g]);
    const double xu = a.q[Ng + g], xv = a.q[2 * Ng + g];
    if (nonfinite(xr) | nonfinite(xu) | nonfinite(xv) | nonfinite(xw) | nonfinite(xt)) atomicOr(a.flag, 1);
    write_prim(a.pa, g, xr, xu, xv, xw, xt);
  }
}

DeviceFlags imex_attr;

}  // namespace

int imex_cols_per_block(int nz) {
  for (int c = 32; c >= 1; c /= 2)
    if (imex_smem_bytes(nz, c) <= kImexSmemMax) return c;
  return 0;
}

size_t imex_smem_bytes(int nz, int cols_per_block) { return 5 * sizeof(double) * (size_t)nz * cols_per_block; }

cudaError_t imex_kernel_setup() {
  if (imex_attr.has()) return cudaSuccess;
  cudaError_t e =
      cudaFuncSetAttribute(imex_column_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kImexSmemMax);
  if (e == cudaSuccess) imex_attr.set();
  return e;
}

cudaError_t launch_imex(const ImexArgs& a, cudaStream_t s) {
  if (a.cols_per_block < 1 || a.cols_per_block > kImexThreads || a.nz < 2 || a.N < 1 || a.kl > 2 * a.N ||
      a.ku > 4 * a.N)
    return cudaErrorInvalidValue;
  const size_t smem = imex_smem_bytes(a.nz, a.cols_per_block);
  if (smem > kImexSmemMax || !imex_attr.has()) return cudaErrorInvalidValue;
  if (a.ncol == 0) return cudaSuccess;
  const long long blocks = (a.ncol + a.cols_per_block - 1) / a.cols_per_block;
  imex_column_kernel<<<(unsigned)blocks, kImexThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace numa
