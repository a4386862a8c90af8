/*
 * numa_oracle.c -- plain FP64 CPU oracle of the NUMA CG spectral-element
 * right-hand side, direct stiffness summation, inverse mass matrix and
 * SSP-RK3 stage (Mueller et al., Sec. 2 "Numerical Methods", Eqs. 1-5, and
 * the main loop of code example 1 in Sec. 7).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
 * It shares no code with the GPU library and is never called by it.
 *
 * Readings of the paper taken here (the paper gives Eq. 1 only in generic
 * flux form):
 *  - inviscid Euler equations in perturbation form about a hydrostatic
 *    reference state: q = (rho', U, Theta') with U = rho u, Theta = rho theta;
 *    F_rho = U, F_U = U (x) u + p' I, F_Theta = theta U;
 *    S_U = -rho' g e_up  (- 2 Omega x U on the rotating shell);
 *  - strong form with chain-rule physical derivatives, Eq. 4 and Eq. 5 (Eq. 5
 *    read with the eta-term using d(eta)/dx and each 1D derivative taken along
 *    its own index);
 *  - DSS "weighted by the volume of the elements" read as the Jw-weighted sum
 *    divided by M = sum_e Jw (Eq. 4);
 *  - no-normal-flow walls: the wall-normal momentum tendency is removed at
 *    wall nodes;
 *  - three-stage SSP-RK3 (Shu-Osher) for the explicit stages of Sec. 2.2.
 * All of these are listed with their reasons in the design notes.
 *
 * Build without fast-math and without FMA contraction so that the results
 * are the same on x86-64 and aarch64 hosts.
 */
#include "numa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_MAXP 9 /* N <= 8 */

struct orc_mesh {
  orc_config c;
  int N, P;
  long Np, Ne, Nl, Ng;
  double xi[ORC_MAXP], w[ORC_MAXP], D[ORC_MAXP * ORC_MAXP];
  double *ex, *ey, *ez; /* element-node coordinates [Nl] */
  long* l2g;            /* element node -> global node [Nl] */
  double *gx, *gy, *gz; /* global-node coordinates [Ng] */
  double* gh;           /* shell: height of the global node above r_inner [Ng] */
  double* dxi;          /* dxi_d/dx_c at [n*9 + d*3 + c] */
  double* J;            /* Jacobian determinant [Nl] */
  double* Jw;           /* J w_i w_j w_k [Nl] */
  double* M;            /* diagonal mass matrix [Ng] */
  double *rho0, *Th0, *p0;
  unsigned char* wall;
};

/* ---------------------------------------------------------------------- */
/* 1D basis: Lobatto points, quadrature weights, differentiation matrix.    */
/* ---------------------------------------------------------------------- */

/* Legendre P_N(x) and P_{N-1}(x) by the three-term (Bonnet) recurrence. */
static void legendre(int N, double x, double* PN, double* PNm1) {
  double pm = 1.0, p = x;
  if (N == 0) {
    *PN = 1.0;
    *PNm1 = 0.0;
    return;
  }
  for (int k = 1; k < N; ++k) {
    double pn = ((2.0 * k + 1.0) * x * p - k * pm) / (k + 1.0);
    pm = p;
    p = pn;
  }
  *PN = p;
  *PNm1 = pm;
}

/* Sec. 2.1: N+1 Lobatto points per direction.  The interior points are the
 * roots of P_N'; Newton's method on P_N' with P_N'' taken from the Legendre
 * differential equation, started from the Chebyshev-Lobatto points.
 * Weights w_i = 2 / (N (N+1) P_N(xi_i)^2). */
void orc_lgl(int N, double* xi, double* w) {
  xi[0] = -1.0;
  xi[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double x = -cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre(N, x, &P, &Pm1);
      double dP = N * (x * P - Pm1) / (x * x - 1.0);
      double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    xi[i] = x;
  }
  /* the node set is symmetric about 0 */
  for (int i = 0; i < (N + 1) / 2; ++i) {
    double a = 0.5 * (xi[N - i] - xi[i]);
    xi[i] = -a;
    xi[N - i] = a;
  }
  if (N % 2 == 0) xi[N / 2] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double P, Pm1;
    legendre(N, xi[i], &P, &Pm1);
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
}

/* Eq. 5: D_ij = d psi_j / d xi evaluated at xi_i.  Off-diagonal entries from
 * the Lobatto identity psi_j'(xi_i) = P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j));
 * each diagonal entry is minus its row's off-diagonal sum, so that D 1 = 0. */
void orc_dmatrix(int N, const double* xi, double* D) {
  int P = N + 1;
  double PN[ORC_MAXP];
  for (int i = 0; i < P; ++i) {
    double Pm1;
    legendre(N, xi[i], &PN[i], &Pm1);
  }
  for (int i = 0; i < P; ++i) {
    double s = 0.0;
    for (int j = 0; j < P; ++j) {
      if (j == i) continue;
      D[i * P + j] = PN[i] / (PN[j] * (xi[i] - xi[j]));
      s += D[i * P + j];
    }
    D[i * P + i] = -s;
  }
}

/* ---------------------------------------------------------------------- */
/* Mesh                                                                     */
/* ---------------------------------------------------------------------- */

static void* xalloc(size_t n) { return calloc(n ? n : 1, 1); }

void orc_free(orc_mesh* m) {
  if (!m) return;
  free(m->ex); free(m->ey); free(m->ez); free(m->l2g);
  free(m->gx); free(m->gy); free(m->gz); free(m->gh); free(m->dxi); free(m->J); free(m->Jw);
  free(m->M); free(m->rho0); free(m->Th0); free(m->p0); free(m->wall);
  free(m);
}

void orc_sizes(const orc_mesh* m, long* Ne, long* Nl, long* Ng) {
  *Ne = m->Ne;
  *Nl = m->Nl;
  *Ng = m->Ng;
}

/* Box: affine map of each element plus an optional smooth warp that vanishes
 * on every face; the global node is the structured index of the node in the
 * (nex N [+1]) x (ney N [+1]) x (nez N [+1]) lattice, wrapped on periodic axes. */
static int build_box(orc_mesh* m) {
  const orc_config* c = &m->c;
  int N = m->N, P = m->P;
  long nx = (long)c->nex * N + (c->periodic[0] ? 0 : 1);
  long ny = (long)c->ney * N + (c->periodic[1] ? 0 : 1);
  long nz = (long)c->nez * N + (c->periodic[2] ? 0 : 1);
  m->Ne = (long)c->nex * c->ney * c->nez;
  m->Nl = m->Ne * m->Np;
  m->Ng = nx * ny * nz;
  m->ex = xalloc(sizeof(double) * m->Nl);
  m->ey = xalloc(sizeof(double) * m->Nl);
  m->ez = xalloc(sizeof(double) * m->Nl);
  m->l2g = xalloc(sizeof(long) * m->Nl);
  m->gx = xalloc(sizeof(double) * m->Ng);
  m->gy = xalloc(sizeof(double) * m->Ng);
  m->gz = xalloc(sizeof(double) * m->Ng);
  unsigned char* seen = xalloc(m->Ng);
  if (!m->ex || !m->ey || !m->ez || !m->l2g || !m->gx || !m->gy || !m->gz || !seen) {
    free(seen);
    return -2;
  }
  for (int ez = 0; ez < c->nez; ++ez)
    for (int ey = 0; ey < c->ney; ++ey)
      for (int ex = 0; ex < c->nex; ++ex) {
        long e = ex + (long)c->nex * (ey + (long)c->ney * ez);
        for (int k = 0; k < P; ++k)
          for (int j = 0; j < P; ++j)
            for (int i = 0; i < P; ++i) {
              long n = e * m->Np + i + P * (j + P * k);
              double X = (ex + 0.5 * (m->xi[i] + 1.0)) / c->nex;
              double Y = (ey + 0.5 * (m->xi[j] + 1.0)) / c->ney;
              double Z = (ez + 0.5 * (m->xi[k] + 1.0)) / c->nez;
              double sx = sin(M_PI * X), sy = sin(M_PI * Y), sz = sin(M_PI * Z);
              double s2x = sin(2.0 * M_PI * X), s2y = sin(2.0 * M_PI * Y);
              m->ex[n] = c->Lx * (X + c->warp * sx * sy * sz);
              m->ey[n] = c->Ly * (Y + c->warp * s2x * sy * sz);
              m->ez[n] = c->Lz * (Z + c->warp * sx * s2y * sz);
              long ix = ((long)ex * N + i) % nx;
              long iy = ((long)ey * N + j) % ny;
              long iz = ((long)ez * N + k) % nz;
              long g = ix + nx * (iy + ny * iz);
              m->l2g[n] = g;
              if (!seen[g]) {
                seen[g] = 1;
                m->gx[g] = m->ex[n];
                m->gy[g] = m->ey[n];
                m->gz[g] = m->ez[n];
              }
            }
      }
  free(seen);
  m->wall = xalloc(m->Ng);
  if (!m->wall) return -2;
  for (long iz = 0; iz < nz; ++iz)
    for (long iy = 0; iy < ny; ++iy)
      for (long ix = 0; ix < nx; ++ix) {
        unsigned char b = 0;
        if (!c->periodic[0] && (ix == 0 || ix == nx - 1)) b |= 1;
        if (!c->periodic[1] && (iy == 0 || iy == ny - 1)) b |= 2;
        if (!c->periodic[2] && (iz == 0 || iz == nz - 1)) b |= 4;
        m->wall[ix + nx * (iy + ny * iz)] = b;
      }
  return 0;
}

/* Union-find over element nodes, used to identify coincident shell nodes. */
static long uf_find(long* par, long a) {
  while (par[a] != a) {
    par[a] = par[par[a]];
    a = par[a];
  }
  return a;
}
static void uf_union(long* par, long a, long b) {
  a = uf_find(par, a);
  b = uf_find(par, b);
  if (a == b) return;
  if (a < b) par[b] = a; else par[a] = b;
}

typedef struct {
  long kx, ky, kz, n;
} qkey;
static int qkey_cmp(const void* pa, const void* pb) {
  const qkey* a = pa;
  const qkey* b = pb;
  if (a->kx != b->kx) return a->kx < b->kx ? -1 : 1;
  if (a->ky != b->ky) return a->ky < b->ky ? -1 : 1;
  if (a->kz != b->kz) return a->kz < b->kz ? -1 : 1;
  return a->n < b->n ? -1 : (a->n > b->n);
}

/* Shell: equiangular gnomonic cubed sphere (six panels, npanel x npanel
 * columns each) times nlayer uniform radial layers from r_inner to r_outer,
 * columns stored bottom to top (Sec. 4, p6est columns).  Element nodes that
 * coincide in space are the same global node; they are found by brute-force
 * coordinate matching (eight half-cell-shifted quantisation grids joined by
 * union-find), numbered by first appearance in element-node order. */
static const double panel_frame[6][3][3] = {
    /* e_a, e_b, e_n (right-handed: e_a x e_b = e_n) */
    {{0, 1, 0}, {0, 0, 1}, {1, 0, 0}},
    {{-1, 0, 0}, {0, 0, 1}, {0, 1, 0}},
    {{0, -1, 0}, {0, 0, 1}, {-1, 0, 0}},
    {{1, 0, 0}, {0, 0, 1}, {0, -1, 0}},
    {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 0}, {0, 0, -1}},
};

static int build_shell(orc_mesh* m) {
  const orc_config* c = &m->c;
  int N = m->N, P = m->P, np = c->npanel, nl = c->nlayer;
  m->Ne = 6L * np * np * nl;
  m->Nl = m->Ne * m->Np;
  m->ex = xalloc(sizeof(double) * m->Nl);
  m->ey = xalloc(sizeof(double) * m->Nl);
  m->ez = xalloc(sizeof(double) * m->Nl);
  m->l2g = xalloc(sizeof(long) * m->Nl);
  if (!m->ex || !m->ey || !m->ez || !m->l2g) return -2;
  double dA = 0.5 * M_PI / np;
  double dR = (c->r_outer - c->r_inner) / nl;
  for (int p = 0; p < 6; ++p)
    for (int ib = 0; ib < np; ++ib)
      for (int ia = 0; ia < np; ++ia)
        for (int il = 0; il < nl; ++il) {
          long e = il + (long)nl * (ia + (long)np * (ib + (long)np * p));
          for (int k = 0; k < P; ++k)
            for (int j = 0; j < P; ++j)
              for (int i = 0; i < P; ++i) {
                long n = e * m->Np + i + P * (j + P * k);
                double al = -0.25 * M_PI + (ia + 0.5 * (m->xi[i] + 1.0)) * dA;
                double be = -0.25 * M_PI + (ib + 0.5 * (m->xi[j] + 1.0)) * dA;
                double r = c->r_inner + (il + 0.5 * (m->xi[k] + 1.0)) * dR;
                double ta = tan(al), tb = tan(be);
                double v[3];
                for (int d = 0; d < 3; ++d)
                  v[d] = panel_frame[p][2][d] + ta * panel_frame[p][0][d] + tb * panel_frame[p][1][d];
                double s = r / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                m->ex[n] = s * v[0];
                m->ey[n] = s * v[1];
                m->ez[n] = s * v[2];
              }
        }
  long Nl = m->Nl;
  long* par = xalloc(sizeof(long) * Nl);
  qkey* keys = xalloc(sizeof(qkey) * Nl);
  if (!par || !keys) {
    free(par);
    free(keys);
    return -2;
  }
  for (long n = 0; n < Nl; ++n) par[n] = n;
  double qstep = 1e-7 * c->r_outer;
  for (int off = 0; off < 8; ++off) {
    double sx = 0.5 * (off & 1), sy = 0.5 * ((off >> 1) & 1), sz = 0.5 * ((off >> 2) & 1);
    for (long n = 0; n < Nl; ++n) {
      keys[n].kx = (long)floor(m->ex[n] / qstep + sx);
      keys[n].ky = (long)floor(m->ey[n] / qstep + sy);
      keys[n].kz = (long)floor(m->ez[n] / qstep + sz);
      keys[n].n = n;
    }
    qsort(keys, Nl, sizeof(qkey), qkey_cmp);
    for (long t = 1; t < Nl; ++t)
      if (keys[t].kx == keys[t - 1].kx && keys[t].ky == keys[t - 1].ky && keys[t].kz == keys[t - 1].kz)
        uf_union(par, keys[t].n, keys[t - 1].n);
  }
  free(keys);
  long* id = xalloc(sizeof(long) * Nl);
  if (!id) {
    free(par);
    return -2;
  }
  for (long n = 0; n < Nl; ++n) id[n] = -1;
  long Ng = 0;
  for (long n = 0; n < Nl; ++n) {
    long r = uf_find(par, n);
    if (id[r] < 0) id[r] = Ng++;
    m->l2g[n] = id[r];
  }
  free(id);
  free(par);
  m->Ng = Ng;
  m->gx = xalloc(sizeof(double) * Ng);
  m->gy = xalloc(sizeof(double) * Ng);
  m->gz = xalloc(sizeof(double) * Ng);
  m->gh = xalloc(sizeof(double) * Ng);
  m->wall = xalloc(Ng);
  unsigned char* seen = xalloc(Ng);
  if (!m->gx || !m->gy || !m->gz || !m->gh || !m->wall || !seen) {
    free(seen);
    return -2;
  }
  for (long e = 0; e < m->Ne; ++e) {
    int il = (int)(e % nl);
    for (int k = 0; k < P; ++k)
      for (int j = 0; j < P; ++j)
        for (int i = 0; i < P; ++i) {
          long n = e * m->Np + i + P * (j + P * k);
          long g = m->l2g[n];
          if (!seen[g]) {
            seen[g] = 1;
            m->gx[g] = m->ex[n];
            m->gy[g] = m->ey[n];
            m->gz[g] = m->ez[n];
            m->gh[g] = (il + 0.5 * (m->xi[k] + 1.0)) * (c->r_outer - c->r_inner) / nl;
          }
          if ((il == 0 && k == 0) || (il == nl - 1 && k == N)) m->wall[g] = 8;
        }
  }
  free(seen);
  return 0;
}

/* Eq. 5 metric terms: x_xi etc. by the isoparametric derivative of the node
 * coordinates with D, then J = det(dx/dxi) and dxi/dx as the 3x3 inverse.
 * D annihilates constants (D 1 = 0), so along each 1D line of nodes the
 * coordinates are differentiated relative to the line's first node: the same
 * metric terms, without the rounding of large absolute coordinates (6.4e6 m
 * on the shell, 9e6 m across one element of a coarse cubed sphere). */
static int build_metrics(orc_mesh* m) {
  int P = m->P;
  long Np = m->Np;
  m->dxi = xalloc(sizeof(double) * 9 * m->Nl);
  m->J = xalloc(sizeof(double) * m->Nl);
  m->Jw = xalloc(sizeof(double) * m->Nl);
  if (!m->dxi || !m->J || !m->Jw) return -2;
  const double* X[3] = {m->ex, m->ey, m->ez};
  for (long e = 0; e < m->Ne; ++e)
    for (int k = 0; k < P; ++k)
      for (int j = 0; j < P; ++j)
        for (int i = 0; i < P; ++i) {
          long n = e * Np + i + P * (j + P * k);
          double A[3][3]; /* A[c][d] = d x_c / d xi_d */
          for (int cc = 0; cc < 3; ++cc) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            const double* xe = &X[cc][e * Np];
            double x0 = xe[P * (j + P * k)], y0 = xe[i + P * P * k], z0 = xe[i + P * j];
            for (int mm = 0; mm < P; ++mm) {
              s0 += m->D[i * P + mm] * (xe[mm + P * (j + P * k)] - x0);
              s1 += m->D[j * P + mm] * (xe[i + P * (mm + P * k)] - y0);
              s2 += m->D[k * P + mm] * (xe[i + P * (j + P * mm)] - z0);
            }
            A[cc][0] = s0;
            A[cc][1] = s1;
            A[cc][2] = s2;
          }
          double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
          if (!(det > 0.0)) return -1;
          /* inverse: B[d][c] = cof(A)[c][d] / det */
          double B[3][3];
          B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
          B[0][1] = -(A[0][1] * A[2][2] - A[0][2] * A[2][1]) / det;
          B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
          B[1][0] = -(A[1][0] * A[2][2] - A[1][2] * A[2][0]) / det;
          B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
          B[1][2] = -(A[0][0] * A[1][2] - A[0][2] * A[1][0]) / det;
          B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
          B[2][1] = -(A[0][0] * A[2][1] - A[0][1] * A[2][0]) / det;
          B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
          for (int d = 0; d < 3; ++d)
            for (int cc = 0; cc < 3; ++cc) m->dxi[n * 9 + d * 3 + cc] = B[d][cc];
          m->J[n] = det;
          m->Jw[n] = det * m->w[i] * m->w[j] * m->w[k];
        }
  return 0;
}

/* Geopotential of the node: g z in the box; on the shell the potential of
 * the deep-atmosphere gravity g(r) = g0 (a/r)^2, g0 a (1 - a/r), written as
 * g0 a h / (a + h) with the node height h = r - a taken from the layer
 * construction (no cancellation of 1 - a/r). */
static double geopotential(const orc_mesh* m, long g) {
  const orc_config* c = &m->c;
  if (c->kind == ORC_BOX) return c->g * m->gz[g];
  double h = m->gh[g];
  return c->g * c->r_inner * h / (c->r_inner + h);
}

/* Hydrostatic reference state per global node.
 * Isentropic (constant theta0): Exner pi0 = 1 - Phi/(cp theta0),
 *   p0 = P00 pi0^(cp/R), (rho theta)_0 = p0/(R pi0), rho0 = (rho theta)_0/theta0.
 * Isothermal (T0): p0 = P00 exp(-Phi/(R T0)), rho0 = p0/(R T0),
 *   (rho theta)_0 = (P00/R) (p0/P00)^(cv/cp). */
static int build_reference(orc_mesh* m) {
  const orc_config* c = &m->c;
  m->rho0 = xalloc(sizeof(double) * m->Ng);
  m->Th0 = xalloc(sizeof(double) * m->Ng);
  m->p0 = xalloc(sizeof(double) * m->Ng);
  m->M = xalloc(sizeof(double) * m->Ng);
  if (!m->rho0 || !m->Th0 || !m->p0 || !m->M) return -2;
  for (long g = 0; g < m->Ng; ++g) {
    double Phi = geopotential(m, g);
    if (c->ref_kind == ORC_REF_ISENTROPIC) {
      double pi0 = 1.0 - Phi / (c->cp * c->theta0);
      if (!(pi0 > 0.0)) return -1;
      m->p0[g] = c->P00 * pow(pi0, c->cp / c->Rd);
      m->Th0[g] = m->p0[g] / (c->Rd * pi0);
      m->rho0[g] = m->Th0[g] / c->theta0;
    } else {
      m->p0[g] = c->P00 * exp(-Phi / (c->Rd * c->T0));
      m->rho0[g] = m->p0[g] / (c->Rd * c->T0);
      m->Th0[g] = (c->P00 / c->Rd) * pow(m->p0[g] / c->P00, c->cv / c->cp);
    }
  }
  /* Eq. 4: M_I = sum over the element nodes at I of Jw */
  for (long n = 0; n < m->Nl; ++n) m->M[m->l2g[n]] += m->Jw[n];
  return 0;
}

int orc_build(const orc_config* cfg, orc_mesh** out) {
  *out = NULL;
  if (cfg->N < 1 || cfg->N > 8) return -1;
  if (cfg->kind == ORC_BOX && (cfg->nex < 1 || cfg->ney < 1 || cfg->nez < 1)) return -1;
  if (cfg->kind == ORC_SHELL && (cfg->npanel < 1 || cfg->nlayer < 1 || !(cfg->r_outer > cfg->r_inner)))
    return -1;
  if (cfg->kind != ORC_BOX && cfg->kind != ORC_SHELL) return -1;
  orc_mesh* m = xalloc(sizeof(orc_mesh));
  if (!m) return -2;
  m->c = *cfg;
  m->N = cfg->N;
  m->P = cfg->N + 1;
  m->Np = (long)m->P * m->P * m->P;
  orc_lgl(m->N, m->xi, m->w);
  orc_dmatrix(m->N, m->xi, m->D);
  int rc = cfg->kind == ORC_BOX ? build_box(m) : build_shell(m);
  if (!rc) rc = build_metrics(m);
  if (!rc) rc = build_reference(m);
  if (rc) {
    orc_free(m);
    return rc;
  }
  *out = m;
  return 0;
}

void orc_get_coords(const orc_mesh* m, double* xyz) {
  memcpy(xyz, m->gx, sizeof(double) * m->Ng);
  memcpy(xyz + m->Ng, m->gy, sizeof(double) * m->Ng);
  memcpy(xyz + 2 * m->Ng, m->gz, sizeof(double) * m->Ng);
}
void orc_get_elem_coords(const orc_mesh* m, double* xyz) {
  memcpy(xyz, m->ex, sizeof(double) * m->Nl);
  memcpy(xyz + m->Nl, m->ey, sizeof(double) * m->Nl);
  memcpy(xyz + 2 * m->Nl, m->ez, sizeof(double) * m->Nl);
}
void orc_get_l2g(const orc_mesh* m, long* l2g) { memcpy(l2g, m->l2g, sizeof(long) * m->Nl); }
void orc_get_metrics(const orc_mesh* m, double* met) {
  for (long n = 0; n < m->Nl; ++n) {
    for (int t = 0; t < 9; ++t) met[t * m->Nl + n] = m->dxi[n * 9 + t];
    met[9 * m->Nl + n] = m->J[n];
  }
}
void orc_get_jw(const orc_mesh* m, double* jw) { memcpy(jw, m->Jw, sizeof(double) * m->Nl); }
void orc_get_mass(const orc_mesh* m, double* M) { memcpy(M, m->M, sizeof(double) * m->Ng); }
void orc_get_ref(const orc_mesh* m, double* ref) {
  memcpy(ref, m->rho0, sizeof(double) * m->Ng);
  memcpy(ref + m->Ng, m->Th0, sizeof(double) * m->Ng);
  memcpy(ref + 2 * m->Ng, m->p0, sizeof(double) * m->Ng);
}
void orc_get_wall(const orc_mesh* m, unsigned char* wall) { memcpy(wall, m->wall, m->Ng); }

/* ---------------------------------------------------------------------- */
/* Equation of state                                                       */
/* ---------------------------------------------------------------------- */

/* p = P00 (R rho theta / P00)^gamma, gamma = cp/cv, so with x = Theta'/(rho theta)_0
 * the perturbation is p' = p - p0 = p0 ((1+x)^gamma - 1) = p0 expm1(gamma log1p(x)),
 * which keeps full relative accuracy when Theta' is small. */
double orc_pprime(double Th_pert, double Th0, double p0, double gamma) {
  return p0 * expm1(gamma * log1p(Th_pert / Th0));
}

/* The same quantity as a plain difference of two pressures; used only as a
 * cross-check of orc_pprime. */
double orc_pprime_naive(double Th_pert, double Th0, double p0, const orc_config* c) {
  double p = c->P00 * pow(c->Rd * (Th0 + Th_pert) / c->P00, c->cp / c->cv);
  return p - p0;
}

/* ---------------------------------------------------------------------- */
/* Initial conditions                                                       */
/* ---------------------------------------------------------------------- */

int orc_init_state(const orc_mesh* m, int kind, const double* prm, double* q) {
  const orc_config* c = &m->c;
  long Ng = m->Ng;
  for (long g = 0; g < Ng; ++g) {
    double x = m->gx[g], y = m->gy[g], z = m->gz[g];
    double rp = 0.0, U[3] = {0.0, 0.0, 0.0}, Tp = 0.0;
    if (kind == ORC_IC_REST) {
    } else if (kind == ORC_IC_BUBBLE) {
      /* theta' = (A/2)(1 + cos(pi r / r_c)) inside r <= r_c; pressure (hence
       * rho theta) unperturbed, so Theta' = 0 and the density absorbs theta'. */
      double A = prm[0], rc = prm[1];
      double dx = x - prm[2], dy = y - prm[3], dz = z - prm[4];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      double thp = r <= rc ? 0.5 * A * (1.0 + cos(M_PI * r / rc)) : 0.0;
      double thref = m->Th0[g] / m->rho0[g];
      rp = m->Th0[g] / (thref + thp) - m->rho0[g];
    } else if (kind == ORC_IC_UNIFORM) {
      U[0] = m->rho0[g] * prm[0];
      U[1] = m->rho0[g] * prm[1];
      U[2] = m->rho0[g] * prm[2];
    } else if (kind == ORC_IC_JETWAVE) {
      if (c->kind != ORC_SHELL) return -1;
      /* zonal jet u = U_jet sin^2(2 phi) plus a Gaussian zonal-wind bump of
       * amplitude pert_amp and radius pert_radius_frac * r_inner centred at
       * (lambda_c, phi_c), great-circle distance on the unit sphere. */
      double Uj = prm[0], amp = prm[1], rad = prm[2], lc = prm[3], pc = prm[4];
      double rr = sqrt(x * x + y * y + z * z);
      double phi = asin(z / rr), lam = atan2(y, x);
      double cosd = sin(pc) * sin(phi) + cos(pc) * cos(phi) * cos(lam - lc);
      if (cosd > 1.0) cosd = 1.0;
      if (cosd < -1.0) cosd = -1.0;
      double d = acos(cosd);
      double s2 = sin(2.0 * phi);
      double u = Uj * s2 * s2 + amp * exp(-(d / rad) * (d / rad));
      U[0] = -m->rho0[g] * u * sin(lam);
      U[1] = m->rho0[g] * u * cos(lam);
      U[2] = 0.0;
    } else {
      return -1;
    }
    q[0 * Ng + g] = rp;
    q[1 * Ng + g] = U[0];
    q[2 * Ng + g] = U[1];
    q[3 * Ng + g] = U[2];
    q[4 * Ng + g] = Tp;
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Right-hand side                                                          */
/* ---------------------------------------------------------------------- */

/* Per element (Eq. 4, Eq. 5):
 *   primitives at each element node from the global state,
 *   the 15 flux components F_vc (v in rho, U_x, U_y, U_z, Theta; c in x,y,z),
 *   dF_vc/dxi_d = sum_m D F along direction d,
 *   div_v = sum_c sum_d dF_vc/dxi_d * dxi_d/dx_c,
 *   source S_v,
 *   r_e = -Jw (div_v - S_v). */
void orc_rhs_elem(const orc_mesh* m, const double* q, double* re) {
  const orc_config* c = &m->c;
  int P = m->P;
  long Np = m->Np, Ng = m->Ng, Nl = m->Nl;
  double gamma = c->cp / c->cv;
#pragma omp parallel for schedule(static)
  for (long e = 0; e < m->Ne; ++e) {
    double F[5][3][ORC_MAXP * ORC_MAXP * ORC_MAXP];
    for (long l = 0; l < Np; ++l) {
      long g = m->l2g[e * Np + l];
      double rho = m->rho0[g] + q[g];
      double U[3] = {q[Ng + g], q[2 * Ng + g], q[3 * Ng + g]};
      double Th = m->Th0[g] + q[4 * Ng + g];
      double u[3] = {U[0] / rho, U[1] / rho, U[2] / rho};
      double theta = Th / rho;
      double pp = orc_pprime(q[4 * Ng + g], m->Th0[g], m->p0[g], gamma);
      for (int cc = 0; cc < 3; ++cc) {
        F[0][cc][l] = U[cc];
        for (int a = 0; a < 3; ++a) F[1 + a][cc][l] = U[a] * u[cc] + (a == cc ? pp : 0.0);
        F[4][cc][l] = theta * U[cc];
      }
    }
    for (int k = 0; k < P; ++k)
      for (int j = 0; j < P; ++j)
        for (int i = 0; i < P; ++i) {
          long l = i + P * (j + P * k);
          long n = e * Np + l;
          long g = m->l2g[n];
          const double* B = &m->dxi[n * 9];
          double div[5];
          for (int v = 0; v < 5; ++v) {
            double s = 0.0;
            for (int cc = 0; cc < 3; ++cc) {
              const double* f = F[v][cc];
              double d0 = 0.0, d1 = 0.0, d2 = 0.0;
              for (int mm = 0; mm < P; ++mm) {
                d0 += m->D[i * P + mm] * f[mm + P * (j + P * k)];
                d1 += m->D[j * P + mm] * f[i + P * (mm + P * k)];
                d2 += m->D[k * P + mm] * f[i + P * (j + P * mm)];
              }
              s += d0 * B[0 * 3 + cc] + d1 * B[1 * 3 + cc] + d2 * B[2 * 3 + cc];
            }
            div[v] = s;
          }
          /* source: buoyancy of the density perturbation, plus Coriolis on the shell */
          double rp = q[g];
          double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
          if (c->kind == ORC_BOX) {
            S[3] = -rp * c->g;
          } else {
            double x = m->gx[g], y = m->gy[g], z = m->gz[g];
            double r = sqrt(x * x + y * y + z * z);
            double gr = c->g * (c->r_inner / r) * (c->r_inner / r);
            S[1] = -rp * gr * x / r + 2.0 * c->Omega * q[2 * Ng + g];
            S[2] = -rp * gr * y / r - 2.0 * c->Omega * q[1 * Ng + g];
            S[3] = -rp * gr * z / r;
          }
          for (int v = 0; v < 5; ++v) re[v * Nl + n] = -m->Jw[n] * (div[v] - S[v]);
        }
  }
}

/* Eq. 4 assembled: R_I = (sum of r_e over the element nodes at I, in
 * ascending element-node order) / M_I, then the no-normal-flow wall condition
 * on the momentum tendency. */
void orc_rhs(const orc_mesh* m, const double* q, double* R) {
  long Nl = m->Nl, Ng = m->Ng;
  double* re = malloc(sizeof(double) * 5 * Nl);
  if (!re) {
    for (long t = 0; t < 5 * Ng; ++t) R[t] = NAN;
    return;
  }
  orc_rhs_elem(m, q, re);
  for (long t = 0; t < 5 * Ng; ++t) R[t] = 0.0;
  for (int v = 0; v < 5; ++v)
    for (long n = 0; n < Nl; ++n) R[v * Ng + m->l2g[n]] += re[v * Nl + n];
  free(re);
  for (int v = 0; v < 5; ++v)
    for (long g = 0; g < Ng; ++g) R[v * Ng + g] /= m->M[g];
  for (long g = 0; g < Ng; ++g) {
    unsigned char b = m->wall[g];
    if (b & 1) R[1 * Ng + g] = 0.0;
    if (b & 2) R[2 * Ng + g] = 0.0;
    if (b & 4) R[3 * Ng + g] = 0.0;
    if (b & 8) {
      double x = m->gx[g], y = m->gy[g], z = m->gz[g];
      double r = sqrt(x * x + y * y + z * z);
      double n3[3] = {x / r, y / r, z / r};
      double dot = R[1 * Ng + g] * n3[0] + R[2 * Ng + g] * n3[1] + R[3 * Ng + g] * n3[2];
      for (int a = 0; a < 3; ++a) R[(1 + a) * Ng + g] -= dot * n3[a];
    }
  }
}

/* ---------------------------------------------------------------------- */
/* Time integration                                                         */
/* ---------------------------------------------------------------------- */

/* Three-stage, third-order strong-stability-preserving Runge-Kutta
 * (Shu-Osher form) for the explicit stages of Sec. 2.2:
 *   q1      = q^n + dt R(q^n)
 *   q2      = 3/4 q^n + 1/4 (q1 + dt R(q1))
 *   q^{n+1} = 1/3 q^n + 2/3 (q2 + dt R(q2))
 * work holds 3n doubles. */
void orc_ssprk3_step(long n, double* q, double dt, orc_rhs_fn f, void* ctx, double* work) {
  static const double a[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double b[3] = {1.0, 0.25, 2.0 / 3.0};
  double* qn = work;
  double* qk = work + n;
  double* r = work + 2 * n;
  memcpy(qn, q, sizeof(double) * n);
  memcpy(qk, q, sizeof(double) * n);
  for (int s = 0; s < 3; ++s) {
    f(ctx, qk, r);
    for (long t = 0; t < n; ++t) qk[t] = a[s] * qn[t] + b[s] * (qk[t] + dt * r[t]);
  }
  memcpy(q, qk, sizeof(double) * n);
}

/* Five-stage, low-storage ("2N") explicit Runge-Kutta of Carpenter and
 * Kennedy (1994): the paper's integrator has five stages and third order
 * (Sec. 2.2) but names no coefficients; this scheme has five stages and
 * order four.  With dq = 0 on entry, for i = 1..5:
 *   dq <- A_i dq + dt R(q);   q <- q + B_i dq
 * (A_1 = 0).  work holds 2n doubles. */
static const double kLsA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double kLsB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};

void orc_lsrk54_coefficients(double* A, double* B) {
  for (int i = 0; i < 5; ++i) {
    A[i] = kLsA[i];
    B[i] = kLsB[i];
  }
}

void orc_lsrk54_step(long n, double* q, double dt, orc_rhs_fn f, void* ctx, double* work) {
  double* dq = work;
  double* r = work + n;
  for (long t = 0; t < n; ++t) dq[t] = 0.0;
  for (int s = 0; s < 5; ++s) {
    f(ctx, q, r);
    for (long t = 0; t < n; ++t) {
      dq[t] = kLsA[s] * dq[t] + dt * r[t];
      q[t] += kLsB[s] * dq[t];
    }
  }
}

static void numa_rhs_cb(void* ctx, const double* q, double* r) { orc_rhs((const orc_mesh*)ctx, q, r); }

int orc_run_lsrk54(const orc_mesh* m, double* q, double dt, int nsteps) {
  long n = 5 * m->Ng;
  double* work = malloc(sizeof(double) * 2 * n);
  if (!work) return -2;
  for (int s = 0; s < nsteps; ++s) orc_lsrk54_step(n, q, dt, numa_rhs_cb, (void*)m, work);
  free(work);
  return 0;
}

int orc_run(const orc_mesh* m, double* q, double dt, int nsteps) {
  long n = 5 * m->Ng;
  double* work = malloc(sizeof(double) * 3 * n);
  if (!work) return -2;
  for (int s = 0; s < nsteps; ++s) orc_ssprk3_step(n, q, dt, numa_rhs_cb, (void*)m, work);
  free(work);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Filter (Sec. 2.3 and the time loop of Sec. 7)                            */
/* ---------------------------------------------------------------------- */

/* Boyd-Vandeven filter weights of the Legendre modes k = 0..N: Vandeven's
 * filter of order p in Boyd's erfc-log form (J. P. Boyd, 1996).  Modes below
 * s are kept; for s <= k <= N, with theta = (k - s) / (N - s) and
 * Omega = theta - 1/2,
 *   sigma_k = 1/2 erfc(2 sqrt(p) chi Omega),
 *   chi = sqrt(-log(1 - 4 Omega^2) / (4 Omega^2))   (chi -> 1 as Omega -> 0),
 * which runs from 1 at theta = 0 to 0 at theta = 1.  A strength mu blends the
 * filtered and unfiltered values: the applied weight is 1 - mu (1 - sigma_k).
 * s = N damps only the top mode (theta = 1 there). */
void orc_filter_weights(int N, int s, double p, double mu, double* sigma) {
  for (int k = 0; k <= N; ++k) {
    double sg = 1.0;
    if (k >= s) {
      double theta = (s >= N) ? 1.0 : (double)(k - s) / (double)(N - s);
      double om = theta - 0.5;
      if (theta <= 0.0) {
        sg = 1.0;
      } else if (theta >= 1.0) {
        sg = 0.0;
      } else if (om == 0.0) {
        sg = 0.5;
      } else {
        double chi = sqrt(-log(1.0 - 4.0 * om * om) / (4.0 * om * om));
        sg = 0.5 * erfc(2.0 * sqrt(p) * chi * om);
      }
    }
    sigma[k] = 1.0 - mu * (1.0 - sg);
  }
}

/* Invert the n x n matrix A (row-major) by Gauss-Jordan elimination with
 * partial pivoting.  Returns 0, or -1 if A is singular. */
static int invert(int n, const double* A, double* Ainv) {
  double* W = malloc(sizeof(double) * n * 2 * n);
  if (!W) return -1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) W[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(W[r * 2 * n + c]) > fabs(W[piv * 2 * n + c])) piv = r;
    if (W[piv * 2 * n + c] == 0.0) {
      free(W);
      return -1;
    }
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        double t = W[c * 2 * n + j];
        W[c * 2 * n + j] = W[piv * 2 * n + j];
        W[piv * 2 * n + j] = t;
      }
    double d = W[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) W[c * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = W[r * 2 * n + c];
      if (f != 0.0)
        for (int j = 0; j < 2 * n; ++j) W[r * 2 * n + j] -= f * W[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i * 2 * n + n + j];
  free(W);
  return 0;
}

/* The 1D filter matrix F = V diag(sigma) V^-1 on the N+1 Lobatto points, with
 * the Legendre Vandermonde matrix V_ik = P_k(xi_i): nodal values to modal
 * coefficients, weights on the modes, back to nodal values.  Row-major
 * F[i * (N+1) + m].  Returns 0, or -1 on failure. */
int orc_filter_matrix(int N, int s, double p, double mu, double* F) {
  int P = N + 1;
  double xi[ORC_MAXP], w[ORC_MAXP], sigma[ORC_MAXP];
  double V[ORC_MAXP * ORC_MAXP], Vi[ORC_MAXP * ORC_MAXP];
  if (N < 1 || N >= ORC_MAXP) return -1;
  orc_lgl(N, xi, w);
  for (int i = 0; i < P; ++i) {
    /* P_0 .. P_N at xi_i by the three-term recurrence */
    double pkm1 = 1.0, pk = xi[i];
    V[i * P + 0] = 1.0;
    if (N >= 1) V[i * P + 1] = xi[i];
    for (int k = 1; k < N; ++k) {
      double pkp1 = ((2.0 * k + 1.0) * xi[i] * pk - k * pkm1) / (k + 1.0);
      pkm1 = pk;
      pk = pkp1;
      V[i * P + k + 1] = pk;
    }
  }
  if (invert(P, V, Vi) != 0) return -1;
  orc_filter_weights(N, s, p, mu, sigma);
  for (int i = 0; i < P; ++i)
    for (int m = 0; m < P; ++m) {
      double acc = 0.0;
      for (int k = 0; k < P; ++k) acc += V[i * P + k] * sigma[k] * Vi[k * P + m];
      F[i * P + m] = acc;
    }
  return 0;
}

/* One application of the filter to the global state q (in place), as the
 * time loop of Sec. 7 states it: per element, the tensor product F x F x F
 * on the element-node values of each variable; then DSS of the Jw-weighted
 * element values in ascending element-node order and division by M.  At wall
 * nodes the wall-normal momentum component keeps its value from before the
 * filter (the filter does not move mass through a wall).  Returns 0, or -1
 * / -2 on a bad filter or allocation failure. */
int orc_filter(const orc_mesh* m, double* q, int s, double p, double mu) {
  int N = m->N, P = N + 1;
  long NP = (long)P * P * P, Nl = m->Nl, Ng = m->Ng;
  double F[ORC_MAXP * ORC_MAXP];
  if (orc_filter_matrix(N, s, p, mu, F) != 0) return -1;
  double* acc = calloc((size_t)5 * Ng, sizeof(double));
  double* u = malloc(sizeof(double) * 2 * NP);
  if (!acc || !u) {
    free(acc);
    free(u);
    return -2;
  }
  double* t = u + NP;
  for (long e = 0; e < m->Ne; ++e) {
    for (int v = 0; v < 5; ++v) {
      for (long l = 0; l < NP; ++l) u[l] = q[v * Ng + m->l2g[e * NP + l]];
      /* along xi, then eta, then zeta; node l = i + P (j + P k) */
      for (int k = 0; k < P; ++k)
        for (int j = 0; j < P; ++j)
          for (int i = 0; i < P; ++i) {
            double a = 0.0;
            for (int mm = 0; mm < P; ++mm) a += F[i * P + mm] * u[mm + P * (j + P * k)];
            t[i + P * (j + P * k)] = a;
          }
      for (int k = 0; k < P; ++k)
        for (int j = 0; j < P; ++j)
          for (int i = 0; i < P; ++i) {
            double a = 0.0;
            for (int mm = 0; mm < P; ++mm) a += F[j * P + mm] * t[i + P * (mm + P * k)];
            u[i + P * (j + P * k)] = a;
          }
      for (int k = 0; k < P; ++k)
        for (int j = 0; j < P; ++j)
          for (int i = 0; i < P; ++i) {
            double a = 0.0;
            for (int mm = 0; mm < P; ++mm) a += F[k * P + mm] * u[i + P * (j + P * mm)];
            t[i + P * (j + P * k)] = a;
          }
      for (long l = 0; l < NP; ++l) acc[v * Ng + m->l2g[e * NP + l]] += m->Jw[e * NP + l] * t[l];
    }
  }
  free(u);
  /* the elements are visited in ascending order, so each global node sums its
   * element-node contributions in ascending element-node order */
  for (long g = 0; g < Ng; ++g) {
    double out[5];
    for (int v = 0; v < 5; ++v) out[v] = acc[v * Ng + g] / m->M[g];
    unsigned char b = m->wall[g];
    if (b & 1) out[1] = q[1 * Ng + g];
    if (b & 2) out[2] = q[2 * Ng + g];
    if (b & 4) out[3] = q[3 * Ng + g];
    if (b & 8) {
      double x = m->gx[g], y = m->gy[g], z = m->gz[g];
      double r = sqrt(x * x + y * y + z * z);
      double n3[3] = {x / r, y / r, z / r};
      double dn = 0.0, dq = 0.0;
      for (int a = 0; a < 3; ++a) {
        dn += out[1 + a] * n3[a];
        dq += q[(1 + a) * Ng + g] * n3[a];
      }
      for (int a = 0; a < 3; ++a) out[1 + a] += (dq - dn) * n3[a];
    }
    for (int v = 0; v < 5; ++v) q[v * Ng + g] = out[v];
  }
  free(acc);
  return 0;
}

/* nsteps SSP-RK3 steps with the filter applied after every `every`-th step
 * (counted from the first step of this call), in place on q. */
int orc_run_filtered(const orc_mesh* m, double* q, double dt, int nsteps, int every, int s, double p, double mu) {
  long n = 5 * m->Ng;
  double* work = malloc(sizeof(double) * 3 * n);
  if (!work) return -2;
  for (int st = 1; st <= nsteps; ++st) {
    orc_ssprk3_step(n, q, dt, numa_rhs_cb, (void*)m, work);
    if (every > 0 && st % every == 0) {
      int rc = orc_filter(m, q, s, p, mu);
      if (rc != 0) {
        free(work);
        return rc;
      }
    }
  }
  free(work);
  return 0;
}
