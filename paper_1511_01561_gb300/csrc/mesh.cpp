// Host-side mesh and geometry setup of the GB300 NUMA hot path (not timed):
// Lobatto basis, box and cubed-sphere shell meshes, isoparametric metric
// terms, element-to-global maps and their inverse, mass matrix, hydrostatic
// reference state and initial conditions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "numa_internal.h"

namespace numa {
namespace {

constexpr double kPi = 3.14159265358979323846;

// P_N and P_{N-1} at x (three-term recurrence).
void legendre_pair(int N, double x, double& pn, double& pnm1) {
  double a = 1.0, b = x;
  if (N == 0) {
    pn = 1.0;
    pnm1 = 0.0;
    return;
  }
  for (int k = 2; k <= N; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  pn = b;
  pnm1 = a;
}

// Sec. 2.1 Lobatto points: the N+1 roots of f(x) = x P_N(x) - P_{N-1}(x)
// (which equals -(1-x^2) P_N'(x) / N), found by Newton's method with
// f'(x) = (N+1) P_N(x); weights 2 / (N (N+1) P_N^2).
void lobatto(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  for (int i = 0; i <= N; ++i) {
    double t = -std::cos(kPi * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 200; ++it) {
        double pn, pm;
        legendre_pair(N, t, pn, pm);
        double step = (t * pn - pm) / ((N + 1) * pn);
        t -= step;
        if (std::fabs(step) <= 1e-17) break;
      }
    }
    x[i] = t;
  }
  for (int i = 0; i <= N / 2; ++i) {  // exact mirror symmetry
    double s = 0.5 * (x[N - i] - x[i]);
    x[i] = -s;
    x[N - i] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 0; i <= N; ++i) {
    double pn, pm;
    legendre_pair(N, x[i], pn, pm);
    w[i] = 2.0 / (N * (N + 1.0) * pn * pn);
  }
}

// Eq. 5 derivative matrix D_ij = psi_j'(xi_i) from barycentric weights
// lambda_j = 1 / prod_{k != j} (x_j - x_k); diagonal = -(row sum) so D 1 = 0.
void diffmat(const std::vector<double>& x, std::vector<double>& D) {
  int P = (int)x.size();
  std::vector<double> lam(P, 1.0);
  for (int j = 0; j < P; ++j)
    for (int k = 0; k < P; ++k)
      if (k != j) lam[j] *= (x[j] - x[k]);
  for (int j = 0; j < P; ++j) lam[j] = 1.0 / lam[j];
  D.assign(P * P, 0.0);
  for (int i = 0; i < P; ++i) {
    double s = 0.0;
    for (int j = 0; j < P; ++j) {
      if (j == i) continue;
      D[i * P + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * P + j];
    }
    D[i * P + i] = -s;
  }
}

// Right-handed cube-panel frames (e_a, e_b, e_n) of the gnomonic cubed sphere.
const int kFrame[6][3][3] = {
    {{0, 1, 0}, {0, 0, 1}, {1, 0, 0}},  {{-1, 0, 0}, {0, 0, 1}, {0, 1, 0}},
    {{0, -1, 0}, {0, 0, 1}, {-1, 0, 0}}, {{1, 0, 0}, {0, 0, 1}, {0, -1, 0}},
    {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}}, {{0, 1, 0}, {1, 0, 0}, {0, 0, -1}},
};

// Structured box: element e = ex + nex (ey + ney ez), local l = i + P (j + P k).
void box_nodes(const numa_config& c, HostMesh& m, std::vector<double>& X) {
  const int N = m.N, P = m.P;
  const long long nx = (long long)c.nex * N + (c.periodic[0] ? 0 : 1);
  const long long ny = (long long)c.ney * N + (c.periodic[1] ? 0 : 1);
  const long long nz = (long long)c.nez * N + (c.periodic[2] ? 0 : 1);
  m.Ne = (long long)c.nex * c.ney * c.nez;
  m.Nl = m.Ne * m.Np;
  m.Ng = nx * ny * nz;
  X.assign(3 * m.Nl, 0.0);
  m.l2g.assign(m.Nl, 0);
  for (int ez = 0; ez < c.nez; ++ez)
    for (int ey = 0; ey < c.ney; ++ey)
      for (int ex = 0; ex < c.nex; ++ex) {
        long long e = ex + (long long)c.nex * (ey + (long long)c.ney * ez);
        for (int k = 0; k < P; ++k)
          for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
              long long n = e * m.Np + i + P * (j + P * k);
              double u = (ex + 0.5 * (1.0 + m.xi[i])) / c.nex;
              double v = (ey + 0.5 * (1.0 + m.xi[j])) / c.ney;
              double t = (ez + 0.5 * (1.0 + m.xi[k])) / c.nez;
              double su = std::sin(kPi * u), sv = std::sin(kPi * v), st = std::sin(kPi * t);
              X[n] = c.Lx * (u + c.warp * su * sv * st);
              X[m.Nl + n] = c.Ly * (v + c.warp * std::sin(2.0 * kPi * u) * sv * st);
              X[2 * m.Nl + n] = c.Lz * (t + c.warp * su * std::sin(2.0 * kPi * v) * st);
              long long ix = (long long)ex * N + i, iy = (long long)ey * N + j, iz = (long long)ez * N + k;
              if (ix == nx) ix = 0;
              if (iy == ny) iy = 0;
              if (iz == nz) iz = 0;
              m.l2g[n] = (int32_t)(ix + nx * (iy + ny * iz));
            }
      }
  m.wall.assign(m.Ng, 0);
  for (long long iz = 0; iz < nz; ++iz)
    for (long long iy = 0; iy < ny; ++iy)
      for (long long ix = 0; ix < nx; ++ix) {
        uint8_t b = 0;
        if (!c.periodic[0] && (ix == 0 || ix == nx - 1)) b |= 1;
        if (!c.periodic[1] && (iy == 0 || iy == ny - 1)) b |= 2;
        if (!c.periodic[2] && (iz == 0 || iz == nz - 1)) b |= 4;
        m.wall[ix + nx * (iy + ny * iz)] = b;
      }
}

// Cubed-sphere shell: element e = il + nl (ia + np (ib + np p)) so that each
// radial column is contiguous, bottom to top (Sec. 4, p6est layers).  A
// surface point is identified exactly by its integer point on the cube
// lattice K e_n + (2 ta - K) e_a + (2 tb - K) e_b (K = np N), which is the
// same from every panel that shares it.  Global nodes are numbered level by
// level: node = column + ncol * level, with the ncol surface points (radial
// columns) numbered by first appearance in element-node order and
// level = il N + k from the bottom, so that a radial column is the same
// stride-ncol sequence as a z-column of the box.
void shell_nodes(const numa_config& c, HostMesh& m, std::vector<double>& X) {
  const int N = m.N, P = m.P, np = c.npanel, nl = c.nlayer;
  const long long K = (long long)np * N, W = 2 * K + 1, NR = (long long)nl * N + 1;
  m.Ne = 6LL * np * np * nl;
  m.Nl = m.Ne * m.Np;
  X.assign(3 * m.Nl, 0.0);
  m.hgt.assign(m.Nl, 0.0);
  std::vector<long long> key(m.Nl);
  std::vector<int> level(m.Nl);
  const double dA = 0.5 * kPi / np, dR = (c.r_outer - c.r_inner) / nl;
  for (int p = 0; p < 6; ++p)
    for (int ib = 0; ib < np; ++ib)
      for (int ia = 0; ia < np; ++ia)
        for (int il = 0; il < nl; ++il) {
          long long e = il + (long long)nl * (ia + (long long)np * (ib + (long long)np * p));
          for (int k = 0; k < P; ++k)
            for (int j = 0; j < P; ++j)
              for (int i = 0; i < P; ++i) {
                long long n = e * m.Np + i + P * (j + P * k);
                double al = -0.25 * kPi + (ia + 0.5 * (1.0 + m.xi[i])) * dA;
                double be = -0.25 * kPi + (ib + 0.5 * (1.0 + m.xi[j])) * dA;
                const double h = (il + 0.5 * (1.0 + m.xi[k])) * dR;
                double r = c.r_inner + h;
                m.hgt[n] = h;
                double ta = std::tan(al), tb = std::tan(be), v[3], nn = 0.0;
                for (int d = 0; d < 3; ++d) {
                  v[d] = kFrame[p][2][d] + ta * kFrame[p][0][d] + tb * kFrame[p][1][d];
                  nn += v[d] * v[d];
                }
                double s = r / std::sqrt(nn);
                for (int d = 0; d < 3; ++d) X[d * m.Nl + n] = s * v[d];
                long long la = (long long)ia * N + i, lb = (long long)ib * N + j;
                long long L[3];
                for (int d = 0; d < 3; ++d)
                  L[d] = K * kFrame[p][2][d] + (2 * la - K) * kFrame[p][0][d] + (2 * lb - K) * kFrame[p][1][d];
                key[n] = ((L[0] + K) * W + (L[1] + K)) * W + (L[2] + K);  // the surface point
                level[n] = (int)((long long)il * N + k);
              }
        }
  // columns: the unique surface points, numbered by first appearance
  std::vector<long long> order(m.Nl);
  std::iota(order.begin(), order.end(), 0LL);
  std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return key[a] < key[b]; });
  std::vector<long long> first(m.Nl, -1);  // per element node: first node with its surface point
  std::vector<long long> firsts;
  for (long long t = 0; t < m.Nl; ++t) {
    if (t == 0 || key[order[t]] != key[order[t - 1]]) firsts.push_back(order[t]);
    first[order[t]] = firsts.back();
  }
  std::vector<long long> f_sorted = firsts;
  std::sort(f_sorted.begin(), f_sorted.end());
  std::vector<int32_t> col_of_first(m.Nl, -1);
  for (size_t t = 0; t < f_sorted.size(); ++t) col_of_first[f_sorted[t]] = (int32_t)t;
  const long long ncol = (long long)f_sorted.size();
  m.Ng = ncol * NR;
  m.l2g.assign(m.Nl, 0);
  for (long long n = 0; n < m.Nl; ++n) m.l2g[n] = (int32_t)(col_of_first[first[n]] + ncol * level[n]);
  m.wall.assign(m.Ng, 0);
  for (long long c = 0; c < ncol; ++c) {  // the bottom and the lid
    m.wall[c] = 8;
    m.wall[c + ncol * (NR - 1)] = 8;
  }
}

// DSS order: within each block of kDssBlock consecutive global nodes, the
// nodes sorted (stably) by their number of element nodes, so that the lanes
// of a warp of the update kernel sum the same number of contributions.
void build_dss_order(HostMesh& m) {
  const long long Ng = m.Ng;
  const long long nb = (Ng + kDssBlock - 1) / kDssBlock;
  m.dss_order.assign(nb * kDssBlock, 0);
  std::vector<int> loc(kDssBlock);
  for (long long b = 0; b < nb; ++b) {
    const long long I0 = b * kDssBlock;
    const int n = (int)std::min<long long>(kDssBlock, Ng - I0);
    std::iota(loc.begin(), loc.end(), 0);
    std::stable_sort(loc.begin(), loc.begin() + n, [&](int x, int y) {
      return m.csr_off[I0 + x + 1] - m.csr_off[I0 + x] < m.csr_off[I0 + y + 1] - m.csr_off[I0 + y];
    });
    for (int t = 0; t < kDssBlock; ++t) m.dss_order[I0 + t] = (uint8_t)loc[t];
  }
}

}  // namespace

// Boyd-Vandeven filter (Sec. 2.3).  Weight of Legendre mode k: 1 below the
// first damped mode s; above it Vandeven's filter of order p in Boyd's
// erfc-log form, 1/2 erfc(2 sqrt(p) chi(O) O) with O = theta - 1/2,
// theta = (k - s)/(N - s) and chi(O)^2 = -log(1 - 4 O^2) / (4 O^2), which is 1
// at theta = 0 and 0 at theta = 1; blended with the identity by mu.
// The matrix F = V diag(sigma) V^-1 uses V_ik = P_k(xi_i) and its inverse from
// the discrete orthogonality of the Legendre polynomials under Lobatto
// quadrature: sum_i w_i P_j(xi_i) P_k(xi_i) = delta_jk g_k with g_k = 2/(2k+1)
// for k < N and g_N = 2/N (the quadrature is exact up to degree 2N-1), so
// (V^-1)_ki = w_i P_k(xi_i) / g_k.
void filter_matrix_host(int N, const double* xi, const double* w, int s, double p, double mu, double* F) {
  const int P = N + 1;
  std::vector<double> sigma(P), V(P * P);
  for (int k = 0; k < P; ++k) {
    double sg = 1.0;
    if (k >= s) {
      const double theta = s >= N ? 1.0 : double(k - s) / double(N - s);
      const double o = theta - 0.5;
      if (theta >= 1.0) sg = 0.0;
      else if (theta > 0.0) sg = o == 0.0 ? 0.5 : 0.5 * std::erfc(2.0 * std::sqrt(p) * std::sqrt(-std::log(1.0 - 4.0 * o * o) / (4.0 * o * o)) * o);
    }
    sigma[k] = 1.0 - mu * (1.0 - sg);
  }
  for (int i = 0; i < P; ++i) {
    double a = 1.0, b = xi[i];
    V[i * P] = 1.0;
    if (P > 1) V[i * P + 1] = b;
    for (int k = 2; k < P; ++k) {
      const double c = ((2 * k - 1) * xi[i] * b - (k - 1) * a) / k;
      a = b;
      b = c;
      V[i * P + k] = c;
    }
  }
  for (int i = 0; i < P; ++i)
    for (int m = 0; m < P; ++m) {
      double acc = 0.0;
      for (int k = 0; k < P; ++k) {
        const double gk = k < N ? 2.0 / (2.0 * k + 1.0) : 2.0 / N;
        acc += V[i * P + k] * sigma[k] * (w[m] * V[m * P + k] / gk);
      }
      F[i * P + m] = acc;
    }
}

bool build_host_mesh(const numa_config& c, HostMesh& m, std::string& err) {
  if (c.N < 1 || c.N > kMaxN) {
    err = "N must be in 1..8";
    return false;
  }
  m.N = c.N;
  m.P = c.N + 1;
  m.Np = m.P * m.P * m.P;
  lobatto(m.N, m.xi, m.w);
  diffmat(m.xi, m.D);
  std::vector<double> X;
  // element nodes from the configuration alone, so that a mesh beyond the
  // 32-bit indices is refused before any of its arrays is built (each global
  // node belongs to at least one element node, so Nl bounds Ng as well)
  {
    const double np = (double)(c.N + 1) * (c.N + 1) * (c.N + 1);
    double ne = 0.0;
    if (c.mesh_kind == NUMA_MESH_BOX) ne = (double)c.nex * c.ney * c.nez;
    else if (c.mesh_kind == NUMA_MESH_SHELL) ne = 6.0 * c.npanel * c.npanel * c.nlayer;
    if (ne * np >= 2147483648.0) {
      err = "mesh too large for 32-bit node indices";
      return false;
    }
  }
  if (c.mesh_kind == NUMA_MESH_BOX) {
    if (c.nex < 1 || c.ney < 1 || c.nez < 1 || !(c.Lx > 0) || !(c.Ly > 0) || !(c.Lz > 0)) {
      err = "box needs positive element counts and extents";
      return false;
    }
    box_nodes(c, m, X);
  } else if (c.mesh_kind == NUMA_MESH_SHELL) {
    if (c.npanel < 1 || c.nlayer < 1 || !(c.r_outer > c.r_inner) || !(c.r_inner > 0)) {
      err = "shell needs npanel, nlayer >= 1 and 0 < r_inner < r_outer";
      return false;
    }
    shell_nodes(c, m, X);
  } else {
    err = "unknown mesh_kind";
    return false;
  }
  if (m.Ng >= (1LL << 31) || m.Nl >= (1LL << 31)) {
    err = "mesh too large for 32-bit node indices";
    return false;
  }
  const int P = m.P, Np = m.Np;
  const long long Nl = m.Nl, Ng = m.Ng;
  // global coordinates: first element node that maps to each global node
  m.gxyz.assign(3 * Ng, 0.0);
  std::vector<double> gh;  // shell: node height above r_inner, from the layer construction
  if (c.mesh_kind == NUMA_MESH_SHELL) gh.assign(Ng, 0.0);
  {
    std::vector<uint8_t> seen(Ng, 0);
    for (long long n = 0; n < Nl; ++n) {
      int32_t g = m.l2g[n];
      if (seen[g]) continue;
      seen[g] = 1;
      for (int d = 0; d < 3; ++d) m.gxyz[d * Ng + g] = X[d * Nl + n];
      if (!gh.empty()) gh[g] = m.hgt[n];
    }
  }
  std::vector<double>().swap(m.hgt);
  // Eq. 5 metric terms: dx_c/dxi_d = sum_m D x_c along direction d, then the
  // analytic inverse of the 3x3 Jacobian matrix; Jw = det * w_i w_j w_k.
  m.met.assign(10 * Nl, 0.0);
  for (long long e = 0; e < m.Ne; ++e) {
    const long long b = e * Np;
    for (int l = 0; l < Np; ++l) {
      const int i = l % P, j = (l / P) % P, k = l / (P * P);
      double A[3][3];
      for (int cc = 0; cc < 3; ++cc) {
        // coordinates relative to the first node of each 1D line: D
        // annihilates constants, and the differences keep full precision even
        // for 9e6 m wide elements on a 6.4e6 m radius shell
        const double* xc = &X[cc * Nl + b];
        const double lx = xc[P * (j + P * k)], ly = xc[i + P * P * k], lz = xc[i + P * j];
        double s0 = 0, s1 = 0, s2 = 0;
        for (int q = 0; q < P; ++q) {
          s0 += m.D[i * P + q] * (xc[q + P * (j + P * k)] - lx);
          s1 += m.D[j * P + q] * (xc[i + P * (q + P * k)] - ly);
          s2 += m.D[k * P + q] * (xc[i + P * (j + P * q)] - lz);
        }
        A[cc][0] = s0;
        A[cc][1] = s1;
        A[cc][2] = s2;
      }
      double C00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
      double C01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
      double C02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
      double det = A[0][0] * C00 + A[0][1] * C01 + A[0][2] * C02;
      if (!(det > 0.0)) {
        err = "non-positive element Jacobian";
        return false;
      }
      double inv = 1.0 / det;
      double Bi[3][3];  // Bi[d][c] = d xi_d / d x_c
      Bi[0][0] = C00 * inv;
      Bi[1][0] = C01 * inv;
      Bi[2][0] = C02 * inv;
      Bi[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * inv;
      Bi[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * inv;
      Bi[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * inv;
      Bi[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * inv;
      Bi[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * inv;
      Bi[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * inv;
      for (int d = 0; d < 3; ++d)
        for (int cc = 0; cc < 3; ++cc) m.met[(3 * d + cc) * Nl + b + l] = Bi[d][cc];
      m.met[9 * Nl + b + l] = det * m.w[i] * m.w[j] * m.w[k];
    }
  }
  // inverse map (CSR, ascending element node) and the mass matrix of Eq. 4
  m.csr_off.assign(Ng + 1, 0);
  for (long long n = 0; n < Nl; ++n) m.csr_off[m.l2g[n] + 1]++;
  for (long long g = 0; g < Ng; ++g) m.csr_off[g + 1] += m.csr_off[g];
  m.csr_idx.assign(Nl, 0);
  {
    std::vector<int32_t> fill(m.csr_off.begin(), m.csr_off.end() - 1);
    for (long long n = 0; n < Nl; ++n) m.csr_idx[fill[m.l2g[n]]++] = (int32_t)n;
  }
  m.nentries = Nl;
  build_dss_order(m);
  m.Minv.assign(Ng, 0.0);
  for (long long g = 0; g < Ng; ++g) {
    double s = 0.0;
    for (int32_t t = m.csr_off[g]; t < m.csr_off[g + 1]; ++t) s += m.met[9 * Nl + m.csr_idx[t]];
    m.Minv[g] = 1.0 / s;
  }
  // hydrostatic reference state from the geopotential Phi (g z in the box,
  // g0 a (1 - a/r) on the shell) and, on the shell, the gravity vectors
  m.ref.assign(4 * Ng, 0.0);
  if (c.mesh_kind == NUMA_MESH_SHELL) {
    m.gvec.assign(3 * Ng, 0.0);
    m.nrm.assign(3 * Ng, 0.0);
  }
  for (long long g = 0; g < Ng; ++g) {
    double x = m.gxyz[g], y = m.gxyz[Ng + g], z = m.gxyz[2 * Ng + g], phi;
    if (c.mesh_kind == NUMA_MESH_BOX) {
      phi = c.g * z;
    } else {
      double r = std::sqrt(x * x + y * y + z * z);
      // potential of g(r) = g0 (a/r)^2: g0 a (1 - a/r) = g0 a h / (a + h),
      // with the height h taken from the layer construction (no cancellation)
      phi = c.g * c.r_inner * gh[g] / (c.r_inner + gh[g]);
      double gr = c.g * (c.r_inner / r) * (c.r_inner / r);
      m.gvec[g] = gr * x / r;
      m.gvec[Ng + g] = gr * y / r;
      m.gvec[2 * Ng + g] = gr * z / r;
      m.nrm[g] = x / r;
      m.nrm[Ng + g] = y / r;
      m.nrm[2 * Ng + g] = z / r;
    }
    double p0, Th0, rho0;
    if (c.ref_kind == NUMA_REF_ISENTROPIC) {
      double exner = 1.0 - phi / (c.cp * c.theta0);
      if (!(exner > 0.0)) {
        err = "isentropic reference reaches zero Exner pressure inside the domain";
        return false;
      }
      p0 = c.P00 * std::pow(exner, c.cp / c.Rd);
      Th0 = p0 / (c.Rd * exner);
      rho0 = Th0 / c.theta0;
    } else if (c.ref_kind == NUMA_REF_ISOTHERMAL) {
      p0 = c.P00 * std::exp(-phi / (c.Rd * c.T0));
      rho0 = p0 / (c.Rd * c.T0);
      Th0 = (c.P00 / c.Rd) * std::pow(p0 / c.P00, c.cv / c.cp);
    } else {
      err = "unknown ref_kind";
      return false;
    }
    m.ref[g] = rho0;
    m.ref[Ng + g] = Th0;
    m.ref[2 * Ng + g] = p0;
    m.ref[3 * Ng + g] = 1.0 / Th0;
  }
  return true;
}

// DG storage (the paper's Sec. 6 comparison of CG, DG and CG/DG storage):
// every element node keeps its own copy of the node data.  The expanded mesh
// has Nl storage nodes, l2g the identity, and per-node arrays (coordinates,
// reference state, M^-1, wall flags, shell vectors) copied from each element
// node's global node.  Storage node n's DSS entries are those of its global
// node g = l2g[n] (all element nodes at g, ascending), so every copy forms the
// same sum, in the same order, as CG storage forms at g.
void expand_to_dg_storage(HostMesh& m) {
  const long long Nl = m.Nl, Ng = m.Ng;
  const std::vector<int32_t> g_of = m.l2g;
  auto expand = [&](std::vector<double>& v, int rows) {
    if (v.empty()) return;
    std::vector<double> out((size_t)rows * Nl);
    for (int r = 0; r < rows; ++r)
      for (long long n = 0; n < Nl; ++n) out[r * Nl + n] = v[r * Ng + g_of[n]];
    v.swap(out);
  };
  expand(m.gxyz, 3);
  expand(m.ref, 4);
  expand(m.Minv, 1);
  expand(m.gvec, 3);
  expand(m.nrm, 3);
  {
    std::vector<uint8_t> w(Nl);
    for (long long n = 0; n < Nl; ++n) w[n] = m.wall[g_of[n]];
    m.wall.swap(w);
  }
  std::vector<int32_t> off(Nl + 1, 0), idx;
  for (long long n = 0; n < Nl; ++n) off[n + 1] = off[n] + (m.csr_off[g_of[n] + 1] - m.csr_off[g_of[n]]);
  idx.resize(off[Nl]);
  for (long long n = 0; n < Nl; ++n) {
    const int32_t t0 = m.csr_off[g_of[n]], t1 = m.csr_off[g_of[n] + 1];
    std::copy(m.csr_idx.begin() + t0, m.csr_idx.begin() + t1, idx.begin() + off[n]);
  }
  m.csr_off.swap(off);
  m.csr_idx.swap(idx);
  m.nentries = (long long)m.csr_idx.size();
  std::iota(m.l2g.begin(), m.l2g.end(), 0);
  m.Ng = Nl;
  build_dss_order(m);
}

bool init_state_host(const numa_config& c, const HostMesh& m, int kind, const double* prm, int nprm,
                     double* q, std::string& err) {
  const long long Ng = m.Ng;
  double p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = 0; t < nprm && t < 8; ++t) p[t] = prm[t];
  if (kind == NUMA_IC_JETWAVE && c.mesh_kind != NUMA_MESH_SHELL) {
    err = "JETWAVE needs a shell mesh";
    return false;
  }
  if (kind < NUMA_IC_REST || kind > NUMA_IC_JETWAVE) {
    err = "unknown initial condition";
    return false;
  }
  for (long long g = 0; g < Ng; ++g) {
    const double x = m.gxyz[g], y = m.gxyz[Ng + g], z = m.gxyz[2 * Ng + g];
    const double rho0 = m.ref[g], Th0 = m.ref[Ng + g];
    double rp = 0.0, U[3] = {0.0, 0.0, 0.0};
    if (kind == NUMA_IC_BUBBLE) {
      // cosine bubble in potential temperature with rho theta unchanged
      double dx = x - p[2], dy = y - p[3], dz = z - p[4];
      double r = std::sqrt(dx * dx + dy * dy + dz * dz);
      double dth = r <= p[1] ? 0.5 * p[0] * (1.0 + std::cos(kPi * r / p[1])) : 0.0;
      rp = Th0 / (Th0 / rho0 + dth) - rho0;
    } else if (kind == NUMA_IC_UNIFORM) {
      for (int a = 0; a < 3; ++a) U[a] = rho0 * p[a];
    } else if (kind == NUMA_IC_JETWAVE) {
      double rr = std::sqrt(x * x + y * y + z * z);
      double lat = std::asin(z / rr), lon = std::atan2(y, x);
      double cd = std::sin(p[4]) * std::sin(lat) + std::cos(p[4]) * std::cos(lat) * std::cos(lon - p[3]);
      cd = std::min(1.0, std::max(-1.0, cd));
      double d = std::acos(cd) / p[2];
      double s2 = std::sin(2.0 * lat);
      double u = p[0] * s2 * s2 + p[1] * std::exp(-d * d);
      U[0] = -rho0 * u * std::sin(lon);
      U[1] = rho0 * u * std::cos(lon);
    }
    q[g] = rp;
    q[Ng + g] = U[0];
    q[2 * Ng + g] = U[1];
    q[3 * Ng + g] = U[2];
    q[4 * Ng + g] = 0.0;
  }
  return true;
}

}  // namespace numa
