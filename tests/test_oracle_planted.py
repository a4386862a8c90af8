"""The oracle's right-hand-side pins against planted mistakes.

The pins of tests/test_oracle_basis.py, test_oracle_mesh.py,
test_oracle_rk.py and test_oracle_rhs.py fix the Lobatto basis, the metric
terms, the stage loop and the right-hand side of Eqs. 1, 4 and 5 by closed
forms, exact balances and convergence properties.  Here the box pins are
gathered into one set of normalised errors (value / bar: at most 1 for a
correct oracle) and run on copies of the oracle with a plausible mistake
planted in its C source: a wrong Lobatto weight or D entry, the metric
terms stored transposed, a weight missing from Jw or M, equidistant instead
of equiangular cubed-sphere coordinates, a wrong jet direction or profile
in the shell's initial state, a wrong exponent in
the reference state or the equation of state, a wrong SSP-RK3 or
low-storage coefficient, the low-storage stages in the wrong order, a transposed D or metric index in the RHS, a dropped or
misplaced pressure term, a wrong flux, a sign error in the buoyancy or the
weighting, an inverse mass left out, a wall condition on the wrong
component, a wrong density in the velocity.  Every planted mistake must
push at least one pin over its bar."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .test_oracle_rhs import _gamma, _jetwave_error, _manufactured

# plausible mistakes, each as textual edits of oracle/numa_oracle.c
PLANTED = {
    # D transposed in the eta contraction
    "d_transposed": [("d1 += m->D[j * P + mm] * f[i + P * (mm + P * k)];",
                      "d1 += m->D[mm * P + j] * f[i + P * (mm + P * k)];")],
    # chain rule with the metric terms transposed (dxi_c/dx_d for dxi_d/dx_c)
    "metric_transposed": [("s += d0 * B[0 * 3 + cc] + d1 * B[1 * 3 + cc] + d2 * B[2 * 3 + cc];",
                           "s += d0 * B[cc * 3 + 0] + d1 * B[cc * 3 + 1] + d2 * B[cc * 3 + 2];")],
    # p' left out of the momentum flux
    "pressure_dropped": [("F[1 + a][cc][l] = U[a] * u[cc] + (a == cc ? pp : 0.0);",
                          "F[1 + a][cc][l] = U[a] * u[cc];")],
    # p' in every component of the momentum flux, not only the diagonal
    "pressure_everywhere": [("F[1 + a][cc][l] = U[a] * u[cc] + (a == cc ? pp : 0.0);",
                             "F[1 + a][cc][l] = U[a] * u[cc] + pp;")],
    # Theta U (rho theta U) instead of theta U in the Theta flux
    "theta_flux": [("F[4][cc][l] = theta * U[cc];", "F[4][cc][l] = Th * U[cc];")],
    # buoyancy with the wrong sign
    "buoyancy_sign": [("S[3] = -rp * c->g;", "S[3] = rp * c->g;")],
    # residual weighted by +Jw
    "weight_sign": [("re[v * Nl + n] = -m->Jw[n] * (div[v] - S[v]);",
                     "re[v * Nl + n] = m->Jw[n] * (div[v] - S[v]);")],
    # the DSS sum not divided by the mass matrix
    "mass_missing": [("R[v * Ng + g] /= m->M[g];", "R[v * Ng + g] /= 1.0;")],
    # the z-wall condition applied to the y momentum
    "wall_component": [("if (b & 4) R[3 * Ng + g] = 0.0;", "if (b & 4) R[2 * Ng + g] = 0.0;")],
    # velocity from the reference density only
    "velocity_density": [("double u[3] = {U[0] / rho, U[1] / rho, U[2] / rho};",
                          "double u[3] = {U[0] / m->rho0[g], U[1] / m->rho0[g], U[2] / m->rho0[g]};")],
    # Lobatto weights with |P_N| instead of P_N^2
    "lgl_weight": [("w[i] = 2.0 / (N * (N + 1.0) * P * P);", "w[i] = 2.0 / (N * (N + 1.0) * fabs(P));")],
    # the diagonal of D left at zero (D 1 != 0)
    "d_diagonal": [("D[i * P + i] = -s;", "D[i * P + i] = 0.0;")],
    # off-diagonal D with P_N(xi_i) and P_N(xi_j) exchanged
    "d_offdiagonal": [("D[i * P + j] = PN[i] / (PN[j] * (xi[i] - xi[j]));",
                       "D[i * P + j] = PN[j] / (PN[i] * (xi[i] - xi[j]));")],
    # the inverse Jacobian stored transposed
    "metric_stored_transposed": [("m->dxi[n * 9 + d * 3 + cc] = B[d][cc];", "m->dxi[n * 9 + d * 3 + cc] = B[cc][d];")],
    # Jw missing the zeta weight
    "jw_weight": [("m->Jw[n] = det * m->w[i] * m->w[j] * m->w[k];", "m->Jw[n] = det * m->w[i] * m->w[j];")],
    # Exner exponent R/cp for cp/R in the isentropic reference pressure
    "exner_exponent": [("m->p0[g] = c->P00 * pow(pi0, c->cp / c->Rd);", "m->p0[g] = c->P00 * pow(pi0, c->Rd / c->cp);")],
    # exponent R/cp for cv/cp in the isothermal reference (rho theta)_0
    "isothermal_theta": [("m->Th0[g] = (c->P00 / c->Rd) * pow(m->p0[g] / c->P00, c->cv / c->cp);",
                          "m->Th0[g] = (c->P00 / c->Rd) * pow(m->p0[g] / c->P00, c->Rd / c->cp);")],
    # 1/gamma for gamma in the equation of state
    "eos_gamma": [("return p0 * expm1(gamma * log1p(Th_pert / Th0));", "return p0 * expm1(log1p(Th_pert / Th0) / gamma);")],
    # mass matrix from J without the quadrature weights
    "mass_weights": [("for (long n = 0; n < m->Nl; ++n) m->M[m->l2g[n]] += m->Jw[n];",
                      "for (long n = 0; n < m->Nl; ++n) m->M[m->l2g[n]] += m->J[n];")],
    # equidistant instead of equiangular panel coordinates on the cubed sphere
    "shell_equidistant": [("double ta = tan(al), tb = tan(be);",
                           "double ta = al * (4.0 / M_PI), tb = be * (4.0 / M_PI);")],
    # the jet along the radial-horizontal direction instead of eastward
    "jet_direction": [("U[0] = -m->rho0[g] * u * sin(lam);\n      U[1] = m->rho0[g] * u * cos(lam);",
                       "U[0] = m->rho0[g] * u * cos(lam);\n      U[1] = m->rho0[g] * u * sin(lam);")],
    # sin(2 phi) instead of sin^2(2 phi) in the jet profile
    "jet_profile": [("double u = Uj * s2 * s2 + amp * exp(-(d / rad) * (d / rad));",
                     "double u = Uj * s2 + amp * exp(-(d / rad) * (d / rad));")],
    # a digit dropped from one five-stage low-storage coefficient
    "ls54_coefficient": [("5161836677717.0 / 13612068292357.0", "516183667771.0 / 13612068292357.0")],
    # the low-storage update reading dq before it is refreshed
    "ls54_stage_order": [("      dq[t] = kLsA[s] * dq[t] + dt * r[t];\n      q[t] += kLsB[s] * dq[t];",
                          "      q[t] += kLsB[s] * dq[t];\n      dq[t] = kLsA[s] * dq[t] + dt * r[t];")],
    # SSP-RK3 with the second stage's q^n coefficient 1/4 instead of 3/4
    "rk3_coefficient": [("static const double a[3] = {0.0, 0.75, 1.0 / 3.0};",
                         "static const double a[3] = {0.0, 0.25, 1.0 / 3.0};")],
}


def _basis_error(orc):
    """The Lobatto closed forms (tests/golden/lgl_closed_forms.json),
    quadrature exactness to degree 2N-1 and D exact on polynomials of degree
    <= N (tests/test_oracle_basis.py), as one normalised error."""
    import json
    import math
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "lgl_closed_forms.json")) as f:
        cases = json.load(f)["cases"]
    e = 0.0
    for N, c in cases.items():
        xi, w = orc.lgl(int(N))
        ex_x = np.array([eval(v, {"math": math}) for v in c["nodes"]])
        ex_w = np.array([eval(v, {"math": math}) for v in c["weights"]])
        e = max(e, np.abs(xi - ex_x).max() / 2e-16, np.abs(w - ex_w).max() / 4e-16)
    for N in range(1, 9):
        xi, w = orc.lgl(N)
        D = orc.dmatrix(N)
        for k in range(0, 2 * N):
            e = max(e, abs(w @ xi**k - (0.0 if k % 2 else 2.0 / (k + 1))) / 1e-14)
        for k in range(0, N + 1):
            exact = k * xi ** (k - 1) if k else np.zeros_like(xi)
            e = max(e, np.abs(D @ xi**k - exact).max() / (1e-12 * max(1, N * N)))
    return e


def _metric_error(orc):
    """Box metric terms and Jw in closed form, and the box volume
    (tests/test_oracle_mesh.py)."""
    ne, L = (2, 3, 4), (1000.0, 600.0, 800.0)
    m = orc.Mesh(I.box(ne, 3, L=L))
    met = m.metrics()
    h = [L[a] / ne[a] for a in range(3)]
    e = 0.0
    for d in range(3):
        for c in range(3):
            exact = 2.0 / h[c] if c == d else 0.0
            e = max(e, np.abs(met[3 * d + c] - exact).max() / (1e-13 * 2.0 / min(h)))
    e = max(e, np.abs(met[9] / (h[0] * h[1] * h[2] / 8.0) - 1.0).max() / 1e-13)
    vol = L[0] * L[1] * L[2]
    e = max(e, abs(m.jw().sum() - vol) / (1e-12 * vol), abs(m.mass().sum() - vol) / (1e-12 * vol))
    return e


def _eos_error(orc):
    """p'(0) = 0; the log1p form against the plain difference of pressures
    and against the binomial series of (1 + x)^gamma - 1
    (tests/test_oracle_rhs.py)."""
    cfg = I.box(1, 1)
    gam = _gamma(cfg)
    th0 = 348.0
    p_ref = cfg["P00"] * (cfg["Rd"] * th0 / cfg["P00"]) ** gam
    e = 0.0 if orc.pprime(0.0, th0, p_ref, gam) == 0.0 else np.inf
    for x in (1e-4, -3e-3, 2e-2, -0.1, 0.3):
        a = orc.pprime(x * th0, th0, p_ref, gam)
        b = orc.pprime_naive(x * th0, th0, p_ref, cfg)
        s, term = 0.0, 1.0
        for k in range(1, 60):
            term *= (gam - k + 1) / k * x
            s += term
        e = max(e, abs(a - b) / (1e-10 * abs(a)), abs(a - p_ref * s) / (2e-15 * abs(a)))
    return e


def _reference_error(orc):
    """The box reference states in hydrostatic balance, dp0/dz = -rho0 g
    (a polynomial fit on a fine column), and p0 = p((rho theta)_0)
    (tests/test_oracle_rhs.py)."""
    e = 0.0
    for ref in ("isentropic", "isothermal"):
        cfg = I.box((1, 1, 16), 4, L=(100.0, 100.0, 10000.0), ref=ref, T0=250.0)
        m = orc.Mesh(cfg)
        xyz, (rho0, th0, p0) = m.coords(), m.ref()
        col = (np.abs(xyz[0]) < 1e-9) & (np.abs(xyz[1]) < 1e-9)
        z, p, r = xyz[2][col], p0[col], rho0[col]
        o = np.argsort(z)
        z, p, r = z[o], p[o], r[o]
        c = np.polynomial.polynomial.polyfit(z / 1e4, p / 1e5, 14)
        dpdz = np.polynomial.polynomial.polyval(z / 1e4, np.polynomial.polynomial.polyder(c)) * 1e5 / 1e4
        e = max(e, np.abs(dpdz / (-r * cfg["g"]) - 1.0).max() / 1e-7)
        peos = cfg["P00"] * (cfg["Rd"] * th0 / cfg["P00"]) ** _gamma(cfg)
        e = max(e, np.abs(peos / p0 - 1.0).max() / 1e-13)
    return e


def _mass_error(orc):
    """M = sum of Jw over each node's element nodes: its total is the box
    volume, and every node of a box with equal elements has the mass of its
    weights times J (tests/test_oracle_mesh.py)."""
    L = (1000.0, 600.0, 800.0)
    m = orc.Mesh(I.box((2, 3, 4), 3, L=L))
    vol = L[0] * L[1] * L[2]
    return abs(m.mass().sum() - vol) / (1e-12 * vol)


def _shell_error(orc):
    """The equiangular cubed sphere (tests/test_oracle_mesh.py): element
    boundaries equally spaced in angle along the equator, Lobatto points of
    the angle inside each element."""
    from .test_oracle_mesh import _equator_longitudes

    npanel, N = 2, 4
    lon = _equator_longitudes(orc, npanel, N)
    d = 0.5 * np.pi / npanel
    pos = (lon + np.pi) / d
    xi, _ = orc.lgl(N)
    frac = np.unique(np.round(pos % 1.0, 9) % 1.0)
    if frac.size != N:
        return np.inf
    e = np.abs(frac - np.sort((xi[:-1] + 1.0) / 2.0)).max() / 1e-9
    corners = np.sort(lon[np.abs(pos - np.round(pos)) < 1e-9])
    if corners.size != 4 * npanel:
        return np.inf
    return max(e, np.abs(np.diff(corners) - d).max() / 1e-11)


def _ls54_error(orc):
    """One five-stage low-storage step on a linear system agrees with
    exp(Z) through Z^4 (the rest O(dt^5): halving dt divides the
    difference by about 32; tests/test_oracle_rk.py)."""
    A = np.array([[-0.3, 1.2, 0.0], [-1.1, -0.2, 0.4], [0.1, 0.0, -0.9]])
    q0 = np.array([1.0, -2.0, 0.5])
    res = []
    for dt in (0.2, 0.1):
        Z = A * dt
        taylor4 = np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
        res.append(np.abs(orc.lsrk54_step(q0, dt, lambda q: A @ q) - taylor4 @ q0).max())
    ratio = res[0] / res[1]
    return 0.0 if 28.0 < ratio < 36.0 else np.inf


def _rk3_error(orc):
    """One SSP-RK3 step of dq/dt = lambda q multiplies q by the cubic
    Taylor polynomial of exp(z) (tests/test_oracle_rk.py)."""
    lam = np.array([-0.3, -1.7, 0.4, -2.5])
    z = lam * 0.8
    q = orc.ssprk3_step(np.ones(4), 0.8, lambda x: lam * x)
    return np.abs(q - (1 + z + z**2 / 2 + z**3 / 6)).max() / 1e-14


def _pin_errors(orc, manufactured_bar):
    """Normalised errors of the basis, metric, RK and box RHS pins: each at
    most 1 for a correct oracle (the bars of tests/test_oracle_*.py)."""
    out = {"basis": _basis_error(orc), "metric": _safe(_metric_error, orc), "rk3": _rk3_error(orc),
           "ls54": _ls54_error(orc),
           "eos": _eos_error(orc), "reference": _safe(_reference_error, orc), "mass": _safe(_mass_error, orc),
           "shell": _safe(_shell_error, orc), "jetwave": _safe(_jetwave_error, orc)}
    try:
        out.update(_rhs_pin_errors(orc, manufactured_bar))
    except ValueError:  # the oracle refused to build a mesh (e.g. a Jacobian <= 0)
        out["rhs"] = np.inf
    return out


def _safe(fn, orc):
    try:
        return fn(orc)
    except ValueError:  # the oracle refused to build a mesh
        return np.inf


def _rhs_pin_errors(orc, manufactured_bar):
    out = {}
    # a state at rest about its own reference: R = 0 bitwise (warped walls)
    m = orc.Mesh(I.box(2, 4, warp=0.05))
    out["rest"] = 0.0 if np.all(m.rhs(m.init_state("rest")) == 0.0) else np.inf
    # uniform flow without gravity, periodic and warped: R = 0 to roundoff
    cfg = I.box((3, 2, 2), 4, periodic=(1, 1, 1), warp=0.05, g=0.0)
    m = orc.Mesh(cfg)
    R = m.rhs(m.init_state("uniform", (10.0, -4.0, 2.5)))
    out["uniform"] = np.abs(R).max() / (1e-12 * m.ref()[0].max() * 100.0 / (1000.0 / 12))
    # linear p', U = 0 on a warped box: R_U = -grad p' exactly inside, R_rho = R_Theta = 0
    b = np.array([3.0e-3, -2.0e-3, 5.0e-3]) * 1e3
    cfg = I.box((2, 3, 2), 4, warp=0.06, g=0.0)
    m = orc.Mesh(cfg)
    xyz = m.coords()
    _, th0, p0 = m.ref()
    pp = b @ (xyz - xyz.mean(axis=1, keepdims=True))
    q = np.zeros((5, m.Ng))
    q[4] = th0 * ((1.0 + pp / p0) ** (1.0 / _gamma(cfg)) - 1.0)
    R = m.rhs(q)
    inner = m.wall() == 0
    e = max(np.abs(R[1 + a][inner] + b[a]).max() for a in range(3)) / (1e-9 * np.abs(b).max())
    out["linear_pressure"] = e if (np.all(R[0] == 0.0) and np.all(R[4] == 0.0)) else np.inf
    # a linear density carried by a uniform velocity, g = 0, p' = 0, on a
    # walled warped box: R_rho = -u0 . grad rho', R_U = -(u0 . grad rho') u0
    # exactly at every node, with the wall-normal components zeroed at the
    # walls, and R_Theta = 0 (Theta0 is uniform without gravity)
    out["linear_advection"] = _linear_advection_error(orc)
    # linear momentum: R_rho = -div U exactly
    G = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [-0.6, 0.9, 0.25]]) * 1e-2
    m = orc.Mesh(I.box((2, 2, 3), 4, warp=0.05, g=0.0))
    q = np.zeros((5, m.Ng))
    q[1:4] = G @ m.coords()
    out["linear_divergence"] = np.abs(m.rhs(q)[0] + np.trace(G)).max() / (1e-12 * 1e3 * np.abs(G).max())
    # discrete conservation of rho' and Theta' on a walled box
    m = orc.Mesh(I.box((3, 2, 2), 4))
    q = I.random_perturbation(m.Ng, seed=3)
    wall = m.wall()
    for a in range(3):
        q[1 + a][(wall >> a) & 1 == 1] = 0.0
    R = m.rhs(q)
    M = m.mass()
    out["conservation"] = max(abs(M @ R[v]) / (1e-13 * (M @ np.abs(R[v]))) for v in (0, 4))
    # the bubble's first RHS in closed form
    cfg = I.box(4, 4)
    m = orc.Mesh(cfg)
    q = m.init_state("bubble", I.BUBBLE_PARAMS)
    R = m.rhs(q)
    tb = (m.wall() & 4) != 0
    ok = np.all(R[[0, 1, 2, 4]] == 0.0) and np.all(R[3][tb] == 0.0)
    exact = -q[0] * cfg["g"]
    rel = np.abs(R[3][~tb] - exact[~tb]).max() / np.abs(exact[~tb]).max()
    out["bubble_closed_form"] = rel / 1e-14 if ok else np.inf
    # a smooth manufactured state: R close to -div F + S (one resolution)
    cfg = I.box(4, 4, L=(1000.0, 800.0, 600.0), warp=0.04)
    m = orc.Mesh(cfg)
    f_state, f_rhs = _manufactured(cfg)
    xyz = m.coords()
    q = np.array([np.broadcast_to(f, xyz[0].shape) for f in f_state(*xyz)])
    ex = np.array([np.broadcast_to(f, xyz[0].shape) for f in f_rhs(*xyz)])
    R = m.rhs(q)
    inner = m.wall() == 0
    err = max(np.abs(R[v][inner] - ex[v][inner]).max() / np.abs(ex[v]).max() for v in range(5))
    out["manufactured"] = err / manufactured_bar
    return out


def _linear_advection_error(orc):
    a = np.array([2.0e-6, -1.0e-6, 1.5e-6])  # grad rho' (kg/m^4)
    u0 = np.array([7.0, -3.0, 4.0])
    cfg = I.box((2, 3, 2), 4, warp=0.06, g=0.0)
    m = orc.Mesh(cfg)
    xyz = m.coords()
    rho0 = m.ref()[0]
    rp = a @ (xyz - xyz.mean(axis=1, keepdims=True))
    q = np.zeros((5, m.Ng))
    q[0] = rp
    q[1:4] = (rho0 + rp) * u0[:, None]
    R = m.rhs(q)
    adv = u0 @ a
    wall = m.wall()
    e = np.abs(R[0] + adv).max() / abs(adv)
    for c in range(3):
        expect = np.where((wall >> c) & 1 == 1, 0.0, -adv * u0[c])
        e = max(e, np.abs(R[1 + c] - expect).max() / abs(adv * np.abs(u0).max()))
    e = max(e, np.abs(R[4]).max() / abs(adv * m.ref()[1].max() / rho0.max()))
    return e / 1e-9


def test_linear_advection_exact(orc):
    """A linear density carried by a uniform velocity (p' = 0, g = 0) on a
    warped walled box: the fluxes are linear, so Eq. 5 differentiates them
    exactly, and the wall condition zeroes exactly the wall-normal momentum
    components."""
    assert _linear_advection_error(orc) <= 1.0


# The manufactured pin's bar at this one resolution: the correct oracle's
# error at 4^3 elements, N = 4 is below 1e-2 (test_oracle_rhs.py holds the
# convergence rate; 3e-3 at 8^3 elements).
MANUFACTURED_BAR = 1e-2


def test_correct_oracle_meets_every_bar(orc):
    errs = _pin_errors(orc, MANUFACTURED_BAR)
    assert all(v <= 1.0 for v in errs.values()), errs


@pytest.fixture(scope="module")
def variants(orc):
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = orc.build_variant(PLANTED[name], name)
        return cache[name]

    return get


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_planted_mistake_breaks_a_pin(orc, variants, mistake):
    with orc.using_library(variants(mistake)):
        errs = _pin_errors(orc, MANUFACTURED_BAR)
    broken = [k for k, v in errs.items() if not v <= 1.0]
    assert broken, (mistake, errs)


# ------------------------------------------------------------- the filter ----
# The pins of tests/test_oracle_filter.py (Sec. 2.3) as normalised errors, run
# on copies of the oracle with a mistake planted in the filter's C code.

FILTER_PLANTED = {
    # F transposed in the xi sweep of the tensor product
    "filter_transposed": [("for (int mm = 0; mm < P; ++mm) a += F[i * P + mm] * u[mm + P * (j + P * k)];",
                           "for (int mm = 0; mm < P; ++mm) a += F[mm * P + i] * u[mm + P * (j + P * k)];")],
    # the factor 2 dropped from the erfc argument
    "filter_erfc_factor": [("sg = 0.5 * erfc(2.0 * sqrt(p) * chi * om);", "sg = 0.5 * erfc(sqrt(p) * chi * om);")],
    # the DSS of the filtered values without the Jw weights
    "filter_unweighted_dss": [("acc[v * Ng + m->l2g[e * NP + l]] += m->Jw[e * NP + l] * t[l];",
                               "acc[v * Ng + m->l2g[e * NP + l]] += t[l];")],
    # the z walls' normal momentum filtered like the rest
    "filter_wall": [("if (b & 4) out[3] = q[3 * Ng + g];", "")],
    # the strength applied to the weight instead of to its damping
    "filter_strength": [("sigma[k] = 1.0 - mu * (1.0 - sg);", "sigma[k] = mu * sg;")],
    # the damped modes counted from s - 1
    "filter_first_mode": [("double theta = (s >= N) ? 1.0 : (double)(k - s) / (double)(N - s);",
                           "double theta = (s >= N) ? 1.0 : (double)(k - s + 1) / (double)(N - s);")],
}

P_ORDER = 12.0


def _filter_pin_errors(orc):
    from numpy.polynomial import legendre as L

    out = {}
    # closed forms of the weights: kept modes 1, theta = 1/2 gives 1/2, the
    # top mode 0, the erfc-log symmetry, the strength blend
    s = orc.filter_weights(4, 2, P_ORDER)
    s6 = orc.filter_weights(6, 2, P_ORDER)
    ok = (np.array_equal(s[:3], [1.0, 1.0, 1.0]) and s[3] == 0.5 and s[4] == 0.0 and s6[4] == 0.5
          and abs(s6[3] + s6[5] - 1.0) < 1e-15
          and np.allclose(orc.filter_weights(6, 2, P_ORDER, 0.3), 1.0 - 0.3 * (1.0 - s6), atol=1e-15, rtol=0))
    # Vandeven's filter 1 - I_theta(p, p) at p = 12, N = 8, s = 0, within 0.02
    # (its values from the regularised incomplete beta function, scipy)
    betainc = pytest.importorskip("scipy.special").betainc
    sig = orc.filter_weights(8, 0, P_ORDER)
    vand = 1.0 - betainc(P_ORDER, P_ORDER, np.arange(9) / 8.0)
    out["weights"] = 0.0 if ok and np.abs(sig - vand).max() < 0.02 else np.inf
    # F P_k = sigma_k P_k at the Lobatto points
    e = 0.0
    for N, sm in ((4, 2), (6, 3)):
        xi, _ = orc.lgl(N)
        F = orc.filter_matrix(N, sm, P_ORDER)
        sg = orc.filter_weights(N, sm, P_ORDER)
        for k in range(N + 1):
            pk = L.legval(xi, np.eye(N + 1)[k])
            e = max(e, np.abs(F @ pk - sg[k] * pk).max() / 5e-14)
    out["eigenvectors"] = e
    # one walled element: (F x F x F) q exactly
    N = 4
    m = orc.Mesh(I.box(1, N, L=(800.0, 900.0, 1000.0)))
    F = orc.filter_matrix(N, 2, P_ORDER)
    rng = np.random.default_rng(3)
    q = rng.standard_normal((5, m.Ng))
    res = m.filter(q, 2, P_ORDER)
    xyz = m.coords()
    K = np.kron(F, np.kron(F, F))
    order = np.lexsort((xyz[0], xyz[1], xyz[2]))
    ref = np.empty(m.Ng)
    ref[order] = K @ q[0][order]
    out["tensor_product"] = np.abs(res[0] - ref).max() / (1e-13 * np.abs(q[0]).max())
    # conservation of rho' and Theta' on a walled affine box, and the walls'
    # normal momentum kept
    m = orc.Mesh(I.box((3, 2, 2), 4))
    q = rng.standard_normal((5, m.Ng))
    M = m.mass()
    res = m.filter(q, 2, P_ORDER)
    e = max(abs(M @ res[v] - M @ q[v]) / (1e-12 * (M @ np.abs(q[v]))) for v in (0, 4))
    wall = m.wall()
    for a in range(3):
        w = (wall & (1 << a)) != 0
        if not np.array_equal(res[1 + a][w], q[1 + a][w]):
            e = np.inf
    out["conservation_walls"] = e
    # fields of degree < s per coordinate are kept (affine elements)
    m = orc.Mesh(I.box((3, 2, 2), 5, L=(900.0, 600.0, 700.0)))
    x, y, z = m.coords() / 1000.0
    f = 1.0 + x - 2 * y * y + 0.5 * x * z + x * x * y * z * z
    qf = np.stack([f, 2 * f, -f, 0.5 * f, 3 * f])
    out["low_degree"] = np.abs(m.filter(qf, 3, P_ORDER) - qf).max() / (1e-13 * np.abs(qf).max())
    return out


def test_correct_filter_meets_every_bar(orc):
    errs = _filter_pin_errors(orc)
    assert all(v <= 1.0 for v in errs.values()), errs


@pytest.mark.parametrize("mistake", sorted(FILTER_PLANTED))
def test_planted_filter_mistake_breaks_a_pin(orc, mistake):
    with orc.using_library(orc.build_variant(FILTER_PLANTED[mistake], mistake)):
        errs = _filter_pin_errors(orc)
    assert [k for k, v in errs.items() if not v <= 1.0], (mistake, errs)


# ------------------------------------------------------------- 1D-IMEX ----
# The pins of tests/test_oracle_imex.py (Sec. 2.2) as normalised errors, run on
# copies of the Python IMEX oracle (oracle/imex.py) with a mistake planted in
# its source: each copy is the module's text with one edit, executed as a
# fresh module of the oracle package.

IMEX_PLANTED = {
    # buoyancy with the wrong sign, in L and in its column blocks alike
    "gravity_sign": [("- self.glev * rho)", "+ self.glev * rho)"),
                     ("Lc[nz:2 * nz, :nz] = -np.diag(self.glev) * keep",
                      "Lc[nz:2 * nz, :nz] = np.diag(self.glev) * keep")],
    # the sound speed without gamma (p' linearised as p0 Theta' / Theta0)
    "gamma_dropped": [("self.c2 = gamma * p0 / Th0", "self.c2 = p0 / Th0")],
    # Theta0 for the potential temperature Theta0 / rho0
    "theta0_is_Theta0": [("self.theta0 = Th0 / rho0", "self.theta0 = Th0")],
    # theta0 taken out of the derivative of theta0 W (exact only where theta0
    # is constant, as in an isentropic reference state)
    "theta0_outside_derivative": [("out[4, c] = -(Dz @ tw + self.r2 * tw)",
                                   "out[4, c] = -(self.theta0[c] * (Dz @ W) + self.r2 * tw)")],
    # the vertical momentum rows of L kept at the bottom and top walls
    "wall_rows_kept": [("LW = np.where(self.zwall[c], 0.0, -Dz @ (self.c2[c] * Th) - self.glev * rho)",
                        "LW = -Dz @ (self.c2[c] * Th) - self.glev * rho")],
    # the column derivative assembled without the element Jacobians: an
    # unweighted mean of the one-sided derivatives at shared nodes (exact on
    # polynomials, wrong at a kink between elements of unequal height)
    "derivative_unweighted": [("A[np.ix_(idx, idx)] += (w * jac)[:, None] * (D / jac)",
                               "A[np.ix_(idx, idx)] += w[:, None] * (D / jac)"),
                              ("mass[idx] += w * jac", "mass[idx] += w")],
    # c2 taken out of the derivative in the column blocks (not in L itself)
    "block_c2_outside": [("Lc[nz:2 * nz, 2 * nz:] = -(Dz * self.c2[nodes][None, :]) * keep",
                          "Lc[nz:2 * nz, 2 * nz:] = -(self.c2[nodes][:, None] * Dz) * keep")],
    # the momentum left as b_U, without the implicit change of its radial part
    "momentum_uncorrected": [("x[1:4, nodes] = b[1:4, nodes] + (sol[nz:2 * nz] - bW[nodes]) * self.nhat[:, nodes]",
                              "x[1:4, nodes] = b[1:4, nodes]")],
    # the start step over dt instead of dt / 2 (backward Euler for L)
    "start_full_step": [("b = q0 + dt * R(q0) - 0.5 * dt * Lop(q0)\n    return solve(0.5 * dt, b)",
                         "b = q0 + dt * R(q0) - dt * Lop(q0)\n    return solve(dt, b)")],
    # the explicit L term removed from q^n alone, not from 2 q^n - q^{n-1}
    "correction_from_q_n": [("b = q_star - dt * Lop(2.0 * q_cur - q_prev)", "b = q_star - dt * Lop(q_cur)")],
    # the Robert-Asselin filter with the wrong sign
    "asselin_sign": [("return q_next, q_cur + nu * (q_prev - 2.0 * q_cur + q_next)",
                      "return q_next, q_cur - nu * (q_prev - 2.0 * q_cur + q_next)")],
    # no 2 W / r term in the divergence along a radial column
    "spherical_divergence_dropped": [("self.r2 = 2.0 / r", "self.r2 = np.zeros_like(r)")],
    # constant gravity g0 along a radial column instead of g0 (a / r)^2
    "flat_gravity": [("self.glev = float(cfg[\"g\"]) * (a / r) ** 2",
                      "self.glev = np.full_like(r, float(cfg[\"g\"]))")],
}


def _imex_variant(edits, tag):
    """oracle/imex.py with textual edits [(old, new), ...], each old snippet
    occurring exactly once, run as a new module of the oracle package (its
    relative import of the C oracle's binding resolves as in the original)."""
    import types

    from oracle import imex

    with open(imex.__file__) as f:
        src = f.read()
    for old, new in edits:
        n = src.count(old)
        if n != 1:
            raise ValueError(f"edit target occurs {n} times: {old!r}")
        src = src.replace(old, new)
    mod = types.ModuleType(f"oracle.imex_planted_{tag}")
    mod.__package__ = "oracle"
    exec(compile(src, f"<oracle/imex.py, {tag}>", "exec"), mod.__dict__)
    return mod


IMEX_ISOTHERMAL = I.box((2, 2, 3), 4, L=(3000.0, 3000.0, 1500.0), periodic=(1, 1, 0), ref="isothermal", T0=250.0)


def _imex_pin_errors(orc, mod, box_reference):
    from .test_oracle_imex import (SOLVE_BAR, THIN, THIN_BUBBLE, _column_perturbation, _linear_problem,
                                   _solve_residual, _thin_shell)

    def in_range(r, lo, hi):
        return max(lo / r, r / hi) if r > 0 else np.inf

    out = {}
    # the column derivative is exact on polynomials of degree <= N, on
    # elements of unequal height
    edges = np.array([0.0, 130.0, 400.0, 460.0, 1000.0])
    e = 0.0
    for N in (2, 4):
        xi, _ = orc.lgl(N)
        z = np.concatenate([a + 0.5 * (1 + xi[:-1]) * (b - a) for a, b in zip(edges[:-1], edges[1:])]
                           + [edges[-1:]])
        Dz = mod.cg_derivative_1d(z, N)
        for j in range(N + 1):
            exact = j * z ** (j - 1) if j else np.zeros_like(z)
            e = max(e, np.abs(Dz @ z**j - exact).max() / (1e-11 * max(1.0, np.abs(exact).max())))
        # at a kink on a shared node the one-sided derivatives are averaged by
        # the mass each element gives the node
        expect = np.sign(z - 400.0)
        expect[z == 400.0] = (60.0 - 270.0) / (60.0 + 270.0)
        e = max(e, np.abs(Dz @ np.abs(z - 400.0) - expect).max() / 1e-11)
    out["derivative"] = e
    # L is the central-difference linearisation of the full right-hand side
    # for height-only perturbations (isentropic and isothermal references),
    # with the W rows zero at the walls
    e = 0.0
    for cfg in (THIN, IMEX_ISOTHERMAL):
        m = orc.Mesh(cfg)
        cols = mod.VerticalColumns(m)
        dq = _column_perturbation(m)
        Lq = cols.apply(dq)
        fd = (m.rhs(1e-3 * dq) - m.rhs(-1e-3 * dq)) / 2e-3
        e = max([e] + [np.abs(fd[v] - Lq[v]).max() / (1e-9 * np.abs(Lq[v]).max()) for v in (0, 3, 4)])
        if np.abs(Lq[3][(m.wall() & 4) != 0]).max() != 0.0:
            e = np.inf
    out["L_box"] = e
    # the same on a thin shell, for radial perturbations W(r) r_hat
    cfg = _thin_shell(3)
    m = orc.Mesh(cfg)
    cols = mod.VerticalColumns(m)
    xyz = m.coords()
    h = (np.sqrt((xyz**2).sum(0)) - cfg["r_inner"]) / 12e3
    rho0, Th0, _ = m.ref()
    W = rho0 * np.sin(np.pi * h) * np.cos(1.3 * h)
    W[(m.wall() & 8) != 0] = 0.0
    dq = np.zeros((5, m.Ng))
    dq[0] = 1e-3 * rho0 * np.sin(2.1 * h + 0.3)
    dq[1:4] = cols.nhat * W
    dq[4] = 1e-3 * Th0 * np.cos(3.0 * h)
    Lq = cols.apply(dq)
    fd = (m.rhs(1e-3 * dq) - m.rhs(-1e-3 * dq)) / 2e-3
    out["L_shell"] = max(np.abs(a - b).max() / (1e-9 * np.abs(b).max())
                         for a, b in ((fd[0], Lq[0]), (cols.radial(fd), cols.radial(Lq)), (fd[4], Lq[4])))
    # the column solve inverts I - tau L
    out["solve"] = max(_solve_residual(orc, mod, THIN, 5.0), _solve_residual(orc, mod, _thin_shell(3), 20.0)) / SOLVE_BAR
    # R = L = B: the start step is the Cayley map of dt / 2 (forward Euler
    # and the trapezoidal rule over dt for q^0 -> q^1), a step the Cayley map
    # of dt from the filtered q^{n-1}
    _, B, q0 = _linear_problem()
    n = len(q0)
    R = Lop = lambda q: B @ q
    solve = lambda tau, b: np.linalg.solve(np.eye(n) - tau * B, b)
    cay = lambda hh: np.linalg.solve(np.eye(n) - hh * B, np.eye(n) + hh * B)
    dt = 0.37
    q1 = mod.lf_imex_start(R, Lop, solve, q0, dt)
    q2, _ = mod.lf_imex_step(R, Lop, solve, q0 + 0.1, q1, dt, 0.0)
    out["cayley"] = max(np.abs(q1 - cay(dt / 2) @ q0).max(), np.abs(q2 - cay(dt) @ (q0 + 0.1)).max()) / 1e-13
    # second order on a linear system with an explicit part
    from scipy.linalg import expm

    A, B, q0 = _linear_problem()
    R = lambda q: (A + B) @ q
    Lop = lambda q: B @ q
    ex = expm((A + B) * 2.0) @ q0
    errs = [np.abs(mod.lf_imex_run(R, Lop, solve, q0, dt, int(round(2.0 / dt)), 0.0)[0] - ex).max()
            for dt in (0.01, 0.005, 0.0025)]
    out["second_order"] = max(in_range(a / b, 3.6, 4.4) for a, b in zip(errs, errs[1:]))
    # Asselin's recurrence on the oscillation equation (nu = 0.2)
    nu, w, dt = 0.2, 1.0, 0.3
    z = 1j * w * dt
    mu = np.linalg.eigvals(np.array([[2 * z, 1.0], [1 - 2 * nu + 2 * nu * z, 2 * nu]]))
    phys = mu[np.argmax(np.abs(mu))]
    R = lambda q: 1j * w * q
    qa, _ = mod.lf_imex_run(R, lambda q: 0.0 * q, lambda tau, b: b, np.array([1.0 + 0.0j]), dt, 400, nu)
    qb, _ = mod.lf_imex_run(R, lambda q: 0.0 * q, lambda tau, b: b, np.array([1.0 + 0.0j]), dt, 401, nu)
    out["asselin"] = abs(qb[0] / qa[0] - phys) / 1e-9
    # past the explicit limit on the thin box the run stays near a fine
    # explicit run
    m = orc.Mesh(THIN)
    qi, _ = mod.run_imex(m, m.init_state("bubble", THIN_BUBBLE), 0.4, 20, 0.05)
    if not np.isfinite(qi).all():
        out["stable"] = np.inf
    else:
        out["stable"] = max(np.abs(qi[3] - box_reference[3]).max() / (0.1 * np.abs(box_reference[3]).max()),
                            np.abs(qi[0] - box_reference[0]).max() / (0.05 * np.abs(box_reference[0]).max()))
    return out


@pytest.fixture(scope="module")
def imex_box_reference(orc):
    """A fine explicit run of the bubble on the thin box to t = 8 s."""
    from .test_oracle_imex import THIN, THIN_BUBBLE

    m = orc.Mesh(THIN)
    return m.run(m.init_state("bubble", THIN_BUBBLE), 0.02, 400)


def test_correct_imex_meets_every_bar(orc, imex_box_reference):
    from oracle import imex

    errs = _imex_pin_errors(orc, imex, imex_box_reference)
    assert all(v <= 1.0 for v in errs.values()), errs


def test_imex_variant_without_edits_is_the_oracle(orc, imex_box_reference):
    errs = _imex_pin_errors(orc, _imex_variant([], "none"), imex_box_reference)
    assert all(v <= 1.0 for v in errs.values()), errs


@pytest.mark.parametrize("mistake", sorted(IMEX_PLANTED))
def test_planted_imex_mistake_breaks_a_pin(orc, imex_box_reference, mistake):
    errs = _imex_pin_errors(orc, _imex_variant(IMEX_PLANTED[mistake], mistake), imex_box_reference)
    assert [k for k, v in errs.items() if not v <= 1.0], (mistake, errs)
