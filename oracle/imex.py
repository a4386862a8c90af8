"""1D-IMEX oracle: leapfrog steps with implicit corrections along vertical
columns (Sec. 2.2, the time loop of Sec. 6), in plain numpy, FP64.

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
vertical columns).
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
    """The columns of a walled, unwarped box and the operator L on them."""

    def __init__(self, mesh: O.Mesh):
        cfg = mesh.cfg
        assert cfg["kind"] == "box" and not cfg.get("periodic", (0, 0, 0))[2] and cfg.get("warp", 0.0) == 0.0
        self.mesh = mesh
        self.N = int(cfg["N"])
        self.g = float(cfg["g"])
        gamma = float(cfg["cp"]) / float(cfg["cv"])
        xyz = mesh.coords()
        # columns: nodes with the same (x, y), ordered by z
        keys = {}
        for n, (x, y) in enumerate(zip(xyz[0], xyz[1])):
            keys.setdefault((x, y), []).append(n)
        cols = [sorted(v, key=lambda n: xyz[2, n]) for v in keys.values()]
        nz = len(cols[0])
        assert all(len(c) == nz for c in cols)
        self.cols = np.array(cols, dtype=np.int64)  # [ncol][nz] global nodes
        self.nz = nz
        rho0, Th0, p0 = mesh.ref()
        self.Dz = [cg_derivative_1d(xyz[2, c], self.N) for c in self.cols]
        self.c2 = gamma * p0 / Th0
        self.theta0 = Th0 / rho0
        # W rows vanish at the bottom and top walls (wall bit 2: normal to z)
        self.zwall = (mesh.wall() & 4) != 0

    def apply(self, q: np.ndarray) -> np.ndarray:
        """L q for a state q [5][Ng]."""
        out = np.zeros_like(q)
        for c, Dz in zip(self.cols, self.Dz):
            rho, W, Th = q[0, c], q[3, c], q[4, c]
            out[0, c] = -Dz @ W
            out[3, c] = np.where(self.zwall[c], 0.0, -Dz @ (self.c2[c] * Th) - self.g * rho)
            out[4, c] = -Dz @ (self.theta0[c] * W)
        return out

    def block(self, c: int) -> np.ndarray:
        """L on column c as a dense [3 nz][3 nz] matrix over (rho', W, Theta')."""
        nodes, Dz, nz = self.cols[c], self.Dz[c], self.nz
        keep = np.where(self.zwall[nodes], 0.0, 1.0)[:, None]
        Lc = np.zeros((3 * nz, 3 * nz))
        Lc[:nz, nz:2 * nz] = -Dz
        Lc[nz:2 * nz, :nz] = -self.g * np.eye(nz) * keep
        Lc[nz:2 * nz, 2 * nz:] = -(Dz * self.c2[nodes][None, :]) * keep
        Lc[2 * nz:, nz:2 * nz] = -Dz * self.theta0[nodes][None, :]
        return Lc

    def solve(self, tau: float, b: np.ndarray) -> np.ndarray:
        """x with (I - tau L) x = b: a dense solve per column; U, V pass through."""
        x = b.copy()
        nz = self.nz
        for c in range(len(self.cols)):
            nodes = self.cols[c]
            rhs = np.concatenate([b[0, nodes], b[3, nodes], b[4, nodes]])
            sol = np.linalg.solve(np.eye(3 * nz) - tau * self.block(c), rhs)
            x[0, nodes], x[3, nodes], x[4, nodes] = sol[:nz], sol[nz:2 * nz], sol[2 * nz:]
        return x


def run_imex(mesh: O.Mesh, q0: np.ndarray, dt: float, nsteps: int, nu: float, cols: VerticalColumns = None):
    """The 1D-IMEX leapfrog on a box mesh: (q^nsteps, filtered q^{nsteps-1})."""
    cols = cols or VerticalColumns(mesh)
    return lf_imex_run(mesh.rhs, cols.apply, cols.solve, np.ascontiguousarray(q0, dtype=np.float64), dt, nsteps, nu)
