// Host tables of the 1D-IMEX column correction (Sec. 2.2): the CG
// derivative along a vertical column, the linearisation coefficients of the
// reference state, and the banded LU factors (partial pivoting) of the Schur
// matrix H = I - tau^2 (Dz C2 G T0 + g G) that the column kernel solves, with
// G = Dz + 2/r the divergence along the column (G = Dz in the box).
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "numa_internal.h"

namespace numa {

bool imex_supported(const numa_config& c, long long* ncol, int* nz, std::string* why) {
  auto no = [&](const char* w) {
    if (why) *why = w;
    return false;
  };
  // R is parked in the primitive buffer: 40 B per node, which the FP32 form's 32 B do not hold
  if (c.precision != NUMA_FP64 && c.precision != NUMA_FP64_PAIRS) return no("1D-IMEX runs in FP64 or FP64-pairs");
  if (c.storage != NUMA_STORAGE_CG) return no("1D-IMEX runs with CG storage");
  long long cols = 0, h = 0;
  if (c.mesh_kind == NUMA_MESH_BOX) {
    if (c.periodic[2]) return no("1D-IMEX needs walls at the bottom and top (not periodic in z)");
    if (c.warp != 0.0) return no("1D-IMEX needs straight columns (warp = 0)");
    if (c.N < 1 || c.nex < 1 || c.ney < 1 || c.nez < 1) return no("bad mesh");
    cols = ((long long)c.nex * c.N + (c.periodic[0] ? 0 : 1)) * ((long long)c.ney * c.N + (c.periodic[1] ? 0 : 1));
    h = (long long)c.nez * c.N + 1;
  } else if (c.mesh_kind == NUMA_MESH_SHELL) {
    if (c.N < 1 || c.npanel < 1 || c.nlayer < 1) return no("bad mesh");
    const long long K = (long long)c.npanel * c.N;
    cols = 6 * K * K + 2;
    h = (long long)c.nlayer * c.N + 1;
  } else {
    return no("unknown mesh kind");
  }
  if (h > 4097 || imex_cols_per_block((int)h, c.N) == 0) return no("columns too tall for the column kernel");
  if (ncol) *ncol = cols;
  if (nz) *nz = (int)h;
  return true;
}

size_t imex_table_doubles(int nz, int N) {
  const size_t n = (size_t)nz;
  return n * (2 * N + 1) + 4 * n + 2 * (n * 2 * N + n * (1 + 4 * N));
}

namespace {

// Radial columns of the shell: the mesh numbers global nodes level by level
// (node = column + ncol * level, level = il N + k from the bottom), so a
// radial column is the same stride-ncol sequence as a z-column of the box.
// Check that structure: walk the element columns (layers are the fastest
// element index) and require every node of the column above bottom node c
// to be c + ncol * level.
bool check_shell_columns(const numa_config& c, const HostMesh& m, long long ncol, int nz, std::string& err) {
  const int N = m.N, P = m.P, nl = c.nlayer;
  const long long ecols = m.Ne / nl;
  for (long long ec = 0; ec < ecols; ++ec)
    for (int j = 0; j < P; ++j)
      for (int i = 0; i < P; ++i) {
        const long long col = m.l2g[(ec * nl) * m.Np + i + P * j];
        if (col < 0 || col >= ncol) {
          err = "1D-IMEX: a bottom node is not on level 0";
          return false;
        }
        for (int il = 0; il < nl; ++il)
          for (int k = 0; k < P; ++k)
            if (m.l2g[(ec * nl + il) * m.Np + i + P * (j + P * k)] != col + ncol * (il * N + k)) {
              err = "1D-IMEX: radial columns are not numbered level by level";
              return false;
            }
      }
  if ((long long)nz * ncol != m.Ng) {
    err = "1D-IMEX: radial columns do not cover the nodes";
    return false;
  }
  return true;
}

}  // namespace

bool imex_operator(const numa_config& c, const HostMesh& m, ImexTables& t, std::string& err) {
  long long ncol = 0;
  int nz = 0;
  if (!imex_supported(c, &ncol, &nz, &err)) return false;
  const int N = m.N, P = m.P, W2 = 2 * N + 1;
  const long long Ng = m.Ng;
  if (ncol * nz != Ng) {
    err = "1D-IMEX: unexpected node count";
    return false;
  }
  const bool shell = c.mesh_kind == NUMA_MESH_SHELL;
  if (shell && !check_shell_columns(c, m, ncol, nz, err)) return false;
  auto node = [&](long long col, int k) -> long long { return col + (long long)k * ncol; };
  // the reference state must be the same in every column (it depends on the height only)
  for (int v = 0; v < 3; ++v)
    for (int k = 0; k < nz; ++k) {
      const double r = m.ref[v * Ng + node(0, k)];
      for (long long col = 1; col < ncol; ++col)
        if (m.ref[v * Ng + node(col, k)] != r) {
          err = "1D-IMEX: the reference state varies along a level";
          return false;
        }
    }
  // heights of the levels: box z; shell the layer construction, uniform
  // layers with Lobatto points inside each
  std::vector<double> z(nz);
  const int nez = shell ? c.nlayer : c.nez;
  if (shell) {
    const double dR = (c.r_outer - c.r_inner) / c.nlayer;
    for (int il = 0; il < c.nlayer; ++il)
      for (int k = 0; k < N; ++k) z[il * N + k] = (il + 0.5 * (1.0 + m.xi[k])) * dR;
    z[nz - 1] = c.nlayer * dR;
  } else {
    for (int k = 0; k < nz; ++k) z[k] = m.gxyz[2 * Ng + node(0, k)];
  }
  // A_KM = sum_e w_k D_km (the Jacobian dz/2 cancels against dxi/dz), mass_K = sum_e w_k dz_e / 2
  std::vector<double> A((size_t)nz * W2, 0.0), mass(nz, 0.0);
  for (int e = 0; e < nez; ++e) {
    const double h = z[(e + 1) * N] - z[e * N];
    for (int k = 0; k < P; ++k) {
      const int K = e * N + k;
      mass[K] += m.w[k] * (0.5 * h);
      for (int j = 0; j < P; ++j) A[(size_t)K * W2 + (j - k + N)] += m.w[k] * m.D[k * P + j];
    }
  }
  t.nz = nz;
  t.N = N;
  t.kl = 2 * N;
  t.Dz.assign((size_t)nz * W2, 0.0);
  for (int K = 0; K < nz; ++K)
    for (int j = 0; j < W2; ++j) t.Dz[(size_t)K * W2 + j] = A[(size_t)K * W2 + j] / mass[K];
  const double gamma = c.cp / c.cv;
  t.c2.resize(nz);
  t.th0.resize(nz);
  t.gl.resize(nz);
  t.r2.resize(nz);
  for (int k = 0; k < nz; ++k) {
    const long long g = node(0, k);
    t.c2[k] = gamma * m.ref[2 * Ng + g] / m.ref[Ng + g];
    t.th0[k] = m.ref[Ng + g] / m.ref[g];
    if (shell) {
      const double r = c.r_inner + z[k];
      t.gl[k] = c.g * (c.r_inner / r) * (c.r_inner / r);
      t.r2[k] = 2.0 / r;
    } else {
      t.gl[k] = c.g;
      t.r2[k] = 0.0;
    }
  }
  return true;
}

bool imex_factor(const ImexTables& t, double tau, std::vector<double>& Lf, std::vector<double>& Uf,
                 std::vector<int>& piv, int* ku, std::string& err) {
  const int nz = t.nz, N = t.N, W2 = 2 * N + 1, kl = 2 * N, US = 1 + 4 * N;
  auto dz = [&](int i, int j) -> double {
    const int d = j - i + N;
    return (d >= 0 && d < W2) ? t.Dz[(size_t)i * W2 + d] : 0.0;
  };
  // G = Dz + diag(2/r): the divergence along the column
  auto gd = [&](int i, int j) -> double { return i == j ? dz(i, j) + t.r2[i] : dz(i, j); };
  // H = I - tau^2 (Dz C2 G T0 + g G) on the interior rows, identity rows at the walls
  std::vector<double> H((size_t)nz * nz, 0.0);
  for (int i = 0; i < nz; ++i) {
    H[(size_t)i * nz + i] = 1.0;
    if (i == 0 || i == nz - 1) continue;
    for (int j = std::max(0, i - kl); j <= std::min(nz - 1, i + kl); ++j) {
      double s = 0.0;
      for (int l = std::max(0, i - N); l <= std::min(nz - 1, i + N); ++l) s += dz(i, l) * t.c2[l] * gd(l, j);
      s = s * t.th0[j] + t.gl[i] * gd(i, j);
      H[(size_t)i * nz + j] -= tau * tau * s;
    }
  }
  // Gaussian elimination with partial pivoting inside the band; the row swap
  // of step k acts on the unfinished columns, so the solve applies swap k and
  // then the multipliers of step k, in that order
  Lf.assign((size_t)nz * kl, 0.0);
  Uf.assign((size_t)nz * US, 0.0);
  piv.assign(3 * (size_t)nz, 0);
  int kumax = 0;
  for (int k = 0; k < nz; ++k) {
    const int last = std::min(nz - 1, k + kl);
    int p = k;
    for (int i = k + 1; i <= last; ++i)
      if (std::fabs(H[(size_t)i * nz + k]) > std::fabs(H[(size_t)p * nz + k])) p = i;
    piv[3 * k] = p;
    if (p != k)
      for (int j = k; j < nz; ++j) std::swap(H[(size_t)k * nz + j], H[(size_t)p * nz + j]);
    const double d = H[(size_t)k * nz + k];
    if (!(std::fabs(d) > 0.0) || !std::isfinite(d)) {
      err = "1D-IMEX: singular column matrix";
      return false;
    }
    const int jend = std::min(nz - 1, k + 4 * N);
    int lused = 0, uused = 0;
    for (int i = k + 1; i <= last; ++i) {
      const double f = H[(size_t)i * nz + k] / d;
      Lf[(size_t)k * kl + (i - k - 1)] = f;
      if (f == 0.0) continue;
      lused = i - k;
      for (int j = k; j <= jend; ++j) H[(size_t)i * nz + j] -= f * H[(size_t)k * nz + j];
    }
    Uf[(size_t)k * US] = 1.0 / d;
    for (int j = 1; j <= 4 * N && k + j < nz; ++j) {
      Uf[(size_t)k * US + j] = H[(size_t)k * nz + k + j];
      if (H[(size_t)k * nz + k + j] != 0.0) uused = j;
    }
    piv[3 * k + 1] = lused;
    piv[3 * k + 2] = uused;
    kumax = std::max(kumax, uused);
    for (int j = k + 4 * N + 1; j < nz; ++j)
      if (H[(size_t)k * nz + j] != 0.0) {
        err = "1D-IMEX: fill outside the band";
        return false;
      }
  }
  *ku = kumax;
  return true;
}

}  // namespace numa
