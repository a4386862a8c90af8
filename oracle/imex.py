"""1D-IMEX oracle: leapfrog steps with implicit corrections along vertical
columns (Sec. 2.2, the time loop of Sec. 7), in plain numpy, FP64.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module.  It shares no code
with the GPU library and never imports it.

The paper names the method (an explicit leapfrog step, then implicit
corrections along each vertical column of grid points, after Giraldo et al.
2013) without formulas.  This module implements one reading of it, written
from the definitions below:

* L is the linear vertical operator of Eq. 1 about the hydrostatic reference
  state (rho0, Theta0, p0): for rho', the vertical momentum W and Theta',
      (L q)_rho   = -dz W
      (L q)_W     = -dz(c2 Theta') - g rho'     (zero at the bottom and top walls)
      (L q)_Theta = -dz(theta0 W)
  with c2 = gamma p0 / Theta0 (p' linearised in Theta') and theta0 =
  Theta0 / rho0, products taken at the nodes; U and V have no L terms.
  dz is the CG derivative along a column: the element derivatives weighted
  by the quadrature weights and Jacobians, summed at shared nodes and divided
  by the summed weights (the vertical part of Eq. 4's DSS and M^-1).
* the step is semi-implicit leapfrog: everything explicit at t^n except L,
  which the trapezoidal rule takes over [t^{n-1}, t^{n+1}]:
      q^{n+1} = q^{n-1} + 2 dt (R(q^n) - L q^n) + dt L (q^{n+1} + q^{n-1}),
  i.e. q* = q^{n-1} + 2 dt R(q^n) (the explicit step), then the correction
      (I - dt L) q^{n+1} = q* - dt L (2 q^n - q^{n-1});
  a Robert-Asselin filter of strength nu follows:
      qbar^n = q^n + nu (qbar^{n-1} - 2 q^n + q^{n+1});
* the first step from q^0 is the same with q^{-1} = q^0 and dt/2, which is
  forward Euler for R - L and the trapezoidal rule for L:
      (I - dt/2 L) q^1 = q^0 + dt R(q^0) - dt/2 L q^0,
  and q^0 itself is left unfiltered.

Meshes: boxes with walls at the bottom and top, without warp (straight
vertical columns), and the cubed-sphere shell (radial columns).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


# ---- the scheme, for any R, L and solve ------------------------------------

def lf_imex_start(R, Lop, solve, q0: np.ndarray, dt: float) -> np.ndarray:
    """q^1 from q^0: forward Euler for R - L, trapezoidal rule for L."""
    b = q0 + dt * R(q0) - 0.5 * dt * Lop(q0)
    return solve(0.5 * dt, b)


def lf_imex_step(R, Lop, solve, q_prev: np.ndarray, q_cur: np.ndarray, dt: float, nu: float):
    """One leapfrog step with the implicit correction and the Robert-Asselin
    filter.  q_prev is the filtered q^{n-1}, q_cur is q^n.  Returns
    (q^{n+1}, filtered q^n)."""
    q_star = q_prev + 2.0 * dt * R(q_cur)
    b = q_star - dt * Lop(2.0 * q_cur - q_prev)
    q_next = solve(dt, b)
    return q_next, q_cur + nu * (q_prev - 2.0 * q_cur + q_next)


def lf_imex_run(R, Lop, solve, q0: np.ndarray, dt: float, nsteps: int, nu: float):
    """nsteps steps from q^0 (the first is the start step).  Returns
    (q^nsteps, filtered q^{nsteps-1}); for nsteps = 0, (q^0, q^0)."""
    if nsteps == 0:
        return q0.copy(), q0.copy()
    prev, cur = q0.copy(), lf_imex_start(R, Lop, solve, q0, dt)
    for _ in range(nsteps - 1):
        nxt, prev = lf_imex_step(R, Lop, solve, prev, cur, dt, nu)
        cur = nxt
    return cur, prev


# ---- the vertical operator of a box mesh ------------------------------------

def cg_derivative_1d(z: np.ndarray, N: int) -> np.ndarray:
    """The CG derivative matrix along one column of nodes z (ascending,
    N per element, shared end nodes): element derivatives (2/dz_e) D weighted
    by w_k dz_e/2, summed at shared nodes, divided by the summed weights."""
    xi, w = O.lgl(N)
    D = O.dmatrix(N)
    nz = z.size
    ne = (nz - 1) // N
    assert ne * N + 1 == nz
    A = np.zeros((nz, nz))
    mass = np.zeros(nz)
    for e in range(ne):
        idx = np.arange(e * N, e * N + N + 1)
        h = z[idx[-1]] - z[idx[0]]
        jac = 0.5 * h
        # sum_m w_k jac (1/jac) D_km f_m: the Jacobian cancels in the derivative term
        A[np.ix_(idx, idx)] += (w * jac)[:, None] * (D / jac)
        mass[idx] += w * jac
    return A / mass[:, None]


class VerticalColumns:
    """The vertical columns of a mesh and the operator L on them.

    Box (unwarped, walls at the bottom and top): the z-lines; W = U_z.
    Shell: the radial lines; W = U . r_hat with r_hat = x / |x| at each node,
    and the divergence along the column carries the spherical term:
        (L q)_rho   = -(dr W + 2 W / r)
        (L q)_U     = r_hat (-dr(c2 Theta') - g(r) rho')   (zero at the bottom and lid)
        (L q)_Theta = -(dr(theta0 W) + 2 theta0 W / r)
    with g(r) = g0 (a / r)^2 and r, dr from the layer construction (uniform
    layers from r_inner to r_outer, Lobatto points inside each)."""

    def __init__(self, mesh: O.Mesh):
        cfg = mesh.cfg
        self.shell = cfg["kind"] == "shell"
        if not self.shell:
            assert cfg["kind"] == "box" and not cfg.get("periodic", (0, 0, 0))[2] and cfg.get("warp", 0.0) == 0.0
        self.mesh = mesh
        self.N = N = int(cfg["N"])
        gamma = float(cfg["cp"]) / float(cfg["cv"])
        xyz = mesh.coords()
        if self.shell:
            rad = np.sqrt((xyz ** 2).sum(axis=0))
            dirs = np.round(xyz / rad, 9)
            keyv, height = [tuple(d) for d in dirs.T], rad
        else:
            keyv, height = list(zip(xyz[0], xyz[1])), xyz[2]
        keys = {}
        for n, key in enumerate(keyv):
            keys.setdefault(key, []).append(n)
        cols = [sorted(v, key=lambda n: height[n]) for v in keys.values()]
        nz = len(cols[0])
        assert all(len(c) == nz for c in cols)
        self.cols = np.array(cols, dtype=np.int64)  # [ncol][nz] global nodes
        self.nz = nz
        rho0, Th0, p0 = mesh.ref()
        self.c2 = gamma * p0 / Th0
        self.theta0 = Th0 / rho0
        if self.shell:
            a, nl = float(cfg["r_inner"]), int(cfg["nlayer"])
            dR = (float(cfg["r_outer"]) - a) / nl
            xi, _ = O.lgl(N)
            h = np.array([(e + 0.5 * (xi[k] + 1.0)) * dR for e in range(nl) for k in range(N)] + [nl * dR])
            r = a + h
            self.Dz = [cg_derivative_1d(h, N)] * len(self.cols)
            self.glev = float(cfg["g"]) * (a / r) ** 2
            self.r2 = 2.0 / r
            self.nhat = xyz / rad
            self.zwall = (mesh.wall() & 8) != 0
        else:
            self.Dz = [cg_derivative_1d(xyz[2, c], N) for c in self.cols]
            self.glev = np.full(nz, float(cfg["g"]))
            self.r2 = np.zeros(nz)
            self.nhat = np.zeros_like(xyz)
            self.nhat[2] = 1.0
            # W rows vanish at the bottom and top walls (wall bit 2: normal to z)
            self.zwall = (mesh.wall() & 4) != 0

    def radial(self, q: np.ndarray) -> np.ndarray:
        """W = U . r_hat at every node."""
        return (q[1:4] * self.nhat).sum(axis=0)

    def apply(self, q: np.ndarray) -> np.ndarray:
        """L q for a state q [5][Ng]."""
        out = np.zeros_like(q)
        Wall = self.radial(q)
        for c, Dz in zip(self.cols, self.Dz):
            rho, W, Th = q[0, c], Wall[c], q[4, c]
            out[0, c] = -(Dz @ W + self.r2 * W)
            LW = np.where(self.zwall[c], 0.0, -Dz @ (self.c2[c] * Th) - self.glev * rho)
            out[1:4, c] = self.nhat[:, c] * LW
            tw = self.theta0[c] * W
            out[4, c] = -(Dz @ tw + self.r2 * tw)
        return out

    def block(self, c: int) -> np.ndarray:
        """L on column c as a dense [3 nz][3 nz] matrix over (rho', W, Theta')."""
        nodes, Dz, nz = self.cols[c], self.Dz[c], self.nz
        G = Dz + np.diag(self.r2)  # the divergence along the column
        keep = np.where(self.zwall[nodes], 0.0, 1.0)[:, None]
        Lc = np.zeros((3 * nz, 3 * nz))
        Lc[:nz, nz:2 * nz] = -G
        Lc[nz:2 * nz, :nz] = -np.diag(self.glev) * keep
        Lc[nz:2 * nz, 2 * nz:] = -(Dz * self.c2[nodes][None, :]) * keep
        Lc[2 * nz:, nz:2 * nz] = -G * self.theta0[nodes][None, :]
        return Lc

    def solve(self, tau: float, b: np.ndarray) -> np.ndarray:
        """x with (I - tau L) x = b: a dense solve per column for (rho', W,
        Theta'); the momentum keeps the part of b_U across the column,
        x_U = b_U + (x_W - b_U . r_hat) r_hat."""
        x = b.copy()
        nz = self.nz
        bW = self.radial(b)
        for c in range(len(self.cols)):
            nodes = self.cols[c]
            rhs = np.concatenate([b[0, nodes], bW[nodes], b[4, nodes]])
            sol = np.linalg.solve(np.eye(3 * nz) - tau * self.block(c), rhs)
            x[0, nodes], x[4, nodes] = sol[:nz], sol[2 * nz:]
            x[1:4, nodes] = b[1:4, nodes] + (sol[nz:2 * nz] - bW[nodes]) * self.nhat[:, nodes]
        return x


def run_imex(mesh: O.Mesh, q0: np.ndarray, dt: float, nsteps: int, nu: float, cols: VerticalColumns = None):
    """The 1D-IMEX leapfrog on a box mesh: (q^nsteps, filtered q^{nsteps-1})."""
    cols = cols or VerticalColumns(mesh)
    return lf_imex_run(mesh.rhs, cols.apply, cols.solve, np.ascontiguousarray(q0, dtype=np.float64), dt, nsteps, nu)


def run_imex_filtered(mesh: O.Mesh, q0: np.ndarray, dt: float, nsteps: int, nu: float, every: int, s: int,
                      p: float, mu: float, cols: VerticalColumns = None):
    """The 1D-IMEX leapfrog with the Boyd-Vandeven filter after every
    `every`-th step, as the time loop of Sec. 7 orders them: the IMEX
    correction (and the Robert-Asselin average, which takes the unfiltered
    q^{n+1}), then the filter of q^{n+1} with DSS and M^-1.  Returns
    (q^nsteps, filtered q^{nsteps-1})."""
    cols = cols or VerticalColumns(mesh)
    R, Lop, solve = mesh.rhs, cols.apply, cols.solve
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    if nsteps == 0:
        return q0.copy(), q0.copy()
    prev, cur = q0.copy(), lf_imex_start(R, Lop, solve, q0, dt)
    for n in range(1, nsteps + 1):
        if n > 1:
            cur, prev = lf_imex_step(R, Lop, solve, prev, cur, dt, nu)
        if every > 0 and n % every == 0:
            cur = mesh.filter(cur, s, p, mu)
    return cur, prev
