"""Pins of the oracle's right-hand side (Eqs. 1, 4, 5): exact balances,
free-stream and linear-field exactness on curved meshes, discrete
conservation, closed forms, symmetries, and convergence to the analytic
divergence of a manufactured state."""
import math

import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I


def _gamma(cfg):
    return cfg["cp"] / cfg["cv"]


# ---------------------------------------------------------------- EOS ----

def test_eos_zero_and_naive_agreement(orc):
    cfg = I.box(1, 1)
    gam = _gamma(cfg)
    th0, p0 = 348.0, 1.0e5
    p_ref = cfg["P00"] * (cfg["Rd"] * th0 / cfg["P00"]) ** gam
    assert orc.pprime(0.0, th0, p_ref, gam) == 0.0
    for x in (1e-4, -3e-3, 2e-2, -0.1, 0.3):
        a = orc.pprime(x * th0, th0, p_ref, gam)
        b = orc.pprime_naive(x * th0, th0, p_ref, cfg)
        assert abs(a - b) <= 1e-10 * abs(a)
        # (1+x)^gamma - 1 by the binomial series, independent of libm
        s, term = 0.0, 1.0
        for k in range(1, 60):
            term *= (gam - k + 1) / k * x
            s += term
        assert abs(a - p_ref * s) <= 2e-15 * abs(a)
    # tiny perturbations keep full relative accuracy (first-order term)
    x = 1e-12
    a = orc.pprime(x * th0, th0, p0, gam)
    assert abs(a / (p0 * gam * x) - 1.0) < 1e-11


@pytest.mark.parametrize("ref", ["isentropic", "isothermal"])
def test_reference_state_is_hydrostatic(orc, ref):
    """dp0/dz = -rho0 g and p0 = p(rho theta_0) on a fine column."""
    cfg = I.box((1, 1, 16), 4, L=(100.0, 100.0, 10000.0), ref=ref, T0=250.0)
    m = orc.Mesh(cfg)
    xyz, (rho0, th0, p0) = m.coords(), m.ref()
    col = (np.abs(xyz[0]) < 1e-9) & (np.abs(xyz[1]) < 1e-9)
    z, p, r = xyz[2][col], p0[col], rho0[col]
    o = np.argsort(z)
    z, p, r = z[o], p[o], r[o]
    c = np.polynomial.polynomial.polyfit(z / 1e4, p / 1e5, 14)
    dpdz = np.polynomial.polynomial.polyval(z / 1e4, np.polynomial.polynomial.polyder(c)) * 1e5 / 1e4
    np.testing.assert_allclose(dpdz, -r * cfg["g"], rtol=1e-7)
    gam = _gamma(cfg)
    peos = cfg["P00"] * (cfg["Rd"] * th0 / cfg["P00"]) ** gam
    np.testing.assert_allclose(peos, p0, rtol=1e-13)


# ------------------------------------------------------- exact balances ----

@pytest.mark.parametrize(
    "cfg",
    [I.box(3, 4), I.box(2, 3, ref="isothermal", T0=250.0), I.box(2, 4, warp=0.05), I.shell(2, 2, 3)],
)
def test_rest_state_gives_zero_rhs_bitwise(orc, cfg):
    m = orc.Mesh(cfg)
    R = m.rhs(m.init_state("rest"))
    assert np.all(R == 0.0)


@pytest.mark.parametrize("warp", [0.0, 0.05])
def test_uniform_flow_without_gravity_is_preserved(orc, warp):
    cfg = I.box((3, 2, 2), 4, periodic=(1, 1, 1), warp=warp, g=0.0)
    m = orc.Mesh(cfg)
    q = m.init_state("uniform", (10.0, -4.0, 2.5))
    R = m.rhs(q)
    rho0 = m.ref()[0].max()
    scale = rho0 * 10.0 * 10.0 / (1000.0 / 12)  # rho |u|^2 / dx_min
    assert np.abs(R).max() < 1e-12 * scale


def test_linear_pressure_gradient_exact_on_curved_meshes(orc):
    """With U = 0 and p' linear in x, R_U = -grad p' exactly at non-wall
    nodes on any isoparametric mesh: the isoparametric metrics invert the
    coordinate derivatives exactly.  Transposing D or the metric fails this."""
    b = np.array([3.0e-3, -2.0e-3, 5.0e-3])
    for cfg in (I.box((2, 3, 2), 4, warp=0.06, g=0.0), I.shell(2, 2, 4, g=0.0, Omega=0.0)):
        m = orc.Mesh(cfg)
        xyz = m.coords()
        rho0, th0, p0 = m.ref()
        pp = (b @ (xyz - xyz.mean(axis=1, keepdims=True))) * (1.0 if cfg["kind"] == "shell" else 1e3)
        gam = _gamma(cfg)
        q = np.zeros((5, m.Ng))
        q[4] = th0 * ((1.0 + pp / p0) ** (1.0 / gam) - 1.0)
        R = m.rhs(q)
        bb = b * (1.0 if cfg["kind"] == "shell" else 1e3)
        wall = m.wall()
        inner = wall == 0
        for a in range(3):
            assert np.abs(R[1 + a][inner] + bb[a]).max() < 1e-9 * np.abs(bb).max(), a
        assert np.abs(R[0]).max() == 0.0 and np.abs(R[4]).max() == 0.0


def test_linear_momentum_divergence_exact(orc):
    G = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [-0.6, 0.9, 0.25]]) * 1e-2
    cfg = I.box((2, 2, 3), 4, warp=0.05, g=0.0)
    m = orc.Mesh(cfg)
    xyz = m.coords()
    q = np.zeros((5, m.Ng))
    q[1:4] = G @ xyz
    R = m.rhs(q)
    assert np.abs(R[0] + np.trace(G)).max() < 1e-12 * 1e3 * np.abs(G).max()


# --------------------------------------------------------- conservation ----

@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_discrete_conservation(orc, periodic):
    g = 9.81 if not any(periodic) else 0.0
    cfg = I.box((3, 2, 2), 4, periodic=periodic, g=g)
    m = orc.Mesh(cfg)
    q = I.random_perturbation(m.Ng, seed=3)
    wall = m.wall()
    for a in range(3):
        q[1 + a][(wall >> a) & 1 == 1] = 0.0
    R = m.rhs(q)
    M = m.mass()
    vars_ = [0, 4] if not any(periodic) else [0, 1, 2, 3, 4]
    for v in vars_:
        tot = M @ R[v]
        assert abs(tot) < 1e-13 * (M @ np.abs(R[v])), v


# ------------------------------------------------------------ closed form ----

def test_bubble_first_rhs_closed_form(orc):
    cfg = I.box(4, 4)
    m = orc.Mesh(cfg)
    q = m.init_state("bubble", I.BUBBLE_PARAMS)
    assert np.all(q[1:] == 0.0) and q[0].min() < 0.0
    R = m.rhs(q)
    assert np.all(R[[0, 1, 2, 4]] == 0.0)
    wall = m.wall()
    top_bottom = (wall & 4) != 0
    assert np.all(R[3][top_bottom] == 0.0)
    exact = -q[0] * cfg["g"]
    np.testing.assert_allclose(R[3][~top_bottom], exact[~top_bottom], rtol=1e-14, atol=0)


def test_bubble_initial_state(orc):
    cfg = I.box(4, 4)
    m = orc.Mesh(cfg)
    q = m.init_state("bubble", I.BUBBLE_PARAMS)
    xyz = m.coords()
    rho0, th0, _ = m.ref()
    r = np.sqrt(((xyz - np.array([[500.0], [500.0], [350.0]])) ** 2).sum(axis=0))
    thp = np.where(r <= 250.0, 0.25 * (1 + np.cos(np.pi * r / 250.0)), 0.0)
    theta = th0 / (rho0 + q[0])
    np.testing.assert_allclose(theta - 300.0, thp, atol=1e-11)


def _jetwave_error(orc):
    """The shell's stand-in state: rest perturbations rho' = Theta' = 0 and
    a purely zonal momentum (no radial or meridional part), 35 m/s at
    45 degrees of latitude away from the bump and none at the equator and
    the poles away from it, a bump of 1 m/s on top at (0 E, 45 N).  Returns
    a normalised error (at most 1 when every property holds)."""
    Uj, amp, rad, lc, pc = I.JETWAVE_PARAMS
    m = orc.Mesh(I.shell(3, 1, 4))
    q = m.init_state("jetwave", I.JETWAVE_PARAMS)
    if not (np.all(q[0] == 0.0) and np.all(q[4] == 0.0)):
        return np.inf
    xyz = m.coords()
    rho0 = m.ref()[0]
    r = np.sqrt((xyz**2).sum(axis=0))
    lam = np.arctan2(xyz[1], xyz[0])
    phi = np.arcsin(xyz[2] / r)
    U = q[1:4]
    east = np.array([-np.sin(lam), np.cos(lam), np.zeros_like(lam)])
    if np.any(U[2] != 0.0):
        return np.inf
    e = np.abs((U * xyz / r).sum(axis=0)).max() / (1e-12 * np.abs(U).max())
    u = (U * east).sum(axis=0) / rho0
    d = np.arccos(np.clip(np.sin(pc) * np.sin(phi) + np.cos(pc) * np.cos(phi) * np.cos(lam - lc), -1, 1))
    far = d > 5 * rad
    at45 = np.abs(np.abs(phi) - np.pi / 4) < 1e-9
    zero = (np.abs(phi) < 1e-9) | (np.abs(np.abs(phi) - np.pi / 2) < 1e-9)
    if not (at45 & far).any() or not (zero & far).any():
        return np.inf
    e = max(e, np.abs(u[at45 & far] - Uj).max() / (1e-12 * Uj), np.abs(u[zero & far]).max() / 1e-9)
    e = max(e, abs(u.max() - (Uj + amp)) / (0.05 * amp), max(0.0, u.max() - (Uj + amp)) / 1e-12)
    return e


def test_jetwave_initial_state(orc):
    assert _jetwave_error(orc) <= 1.0


# ------------------------------------------------------------- symmetry ----

def _box_grid(m, cfg):
    nx = [cfg["ne"][a] * cfg["N"] + 1 for a in range(3)]
    return nx


def test_mirror_and_swap_symmetry(orc):
    cfg = I.box((3, 3, 2), 4)
    m = orc.Mesh(cfg)
    nx, ny, nz = _box_grid(m, cfg)
    xyz = m.coords()
    q = I.smooth_perturbation(xyz, seed=11, length=700.0)

    def grid(a):
        return a.reshape(5, nz, ny, nx)

    Q = grid(q.copy())
    # x- and y-mirror symmetric state: U_x odd in x, U_y odd in y
    Qm = Q[:, :, :, ::-1].copy()
    Qm[1] *= -1
    Q = 0.5 * (Q + Qm)
    Qm = Q[:, :, ::-1, :].copy()
    Qm[2] *= -1
    Q = 0.5 * (Q + Qm)
    # x<->y swap symmetric state (keeps both mirror symmetries)
    Qs = Q.transpose(0, 1, 3, 2).copy()
    Qs[[1, 2]] = Qs[[2, 1]]
    Q = 0.5 * (Q + Qs)
    q = Q.reshape(5, -1)
    R = grid(m.rhs(q))
    scale = np.abs(R).max(axis=(1, 2, 3))
    Rm = R[:, :, :, ::-1].copy()
    Rm[1] *= -1
    for v in range(5):
        assert np.abs(R[v] - Rm[v]).max() <= 1e-12 * scale[v], v
    Rs = R.transpose(0, 1, 3, 2).copy()
    Rs[[1, 2]] = Rs[[2, 1]]
    for v in range(5):
        assert np.abs(R[v] - Rs[v]).max() <= 1e-12 * scale[v], v


# ------------------------------------------------------- manufactured ----

def _manufactured(cfg):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    Lx, Ly, Lz = cfg["L"]
    X, Y, Zs = x / Lx, y / Ly, z / Lz
    Rd, cp, cv, P00, g, th0 = (cfg[k] for k in ("Rd", "cp", "cv", "P00", "g", "theta0"))
    gam = sp.Rational(cp * 2, 1) / sp.Rational(cv * 2, 1)
    pi0 = 1 - g * z / (cp * th0)
    p0 = P00 * pi0 ** (cp / Rd)
    Th0 = p0 / (Rd * pi0)
    rho0 = Th0 / th0
    rp = 0.01 * sp.sin(2 * sp.pi * X + 0.3) * sp.cos(sp.pi * Y) * sp.cos(sp.pi * Zs + 0.2)
    U = [3.0 * sp.sin(sp.pi * X + 0.4) * sp.cos(2 * sp.pi * Y + 0.1) * sp.cos(sp.pi * Zs),
         2.0 * sp.cos(sp.pi * X + 0.2) * sp.sin(sp.pi * Y + 0.5) * sp.cos(sp.pi * Zs + 0.3),
         1.5 * sp.cos(sp.pi * X) * sp.cos(sp.pi * Y + 0.3) * sp.sin(sp.pi * Zs + 0.6)]
    Tp = 0.5 * sp.cos(sp.pi * X) * sp.cos(sp.pi * Y + 0.4) * sp.sin(2 * sp.pi * Zs + 0.5)
    rho = rho0 + rp
    theta = (Th0 + Tp) / rho
    pp = P00 * (Rd * (Th0 + Tp) / P00) ** gam - p0
    u = [Ui / rho for Ui in U]
    xs = (x, y, z)
    Rr = -sum(sp.diff(U[c], xs[c]) for c in range(3))
    RU = [-sum(sp.diff(U[a] * u[c] + (pp if a == c else 0), xs[c]) for c in range(3)) for a in range(3)]
    RU[2] += -rp * g
    RT = -sum(sp.diff(theta * U[c], xs[c]) for c in range(3))
    fields = [rp, U[0], U[1], U[2], Tp]
    rhs = [Rr, RU[0], RU[1], RU[2], RT]
    f_state = sp.lambdify((x, y, z), fields, "numpy")
    f_rhs = sp.lambdify((x, y, z), rhs, "numpy")
    return f_state, f_rhs


@pytest.mark.parametrize("N", [3, 4])
def test_manufactured_state_converges_to_analytic_rhs(orc, N):
    """On a warped box the discrete R converges to -div F + S of a smooth
    analytic state at the rate of the order-N interpolant (Eqs. 4-5)."""
    errs = []
    for ne in (4, 8):
        cfg = I.box(ne, N, L=(1000.0, 800.0, 600.0), warp=0.04)
        m = orc.Mesh(cfg)
        f_state, f_rhs = _manufactured(cfg)
        xyz = m.coords()
        q = np.array([np.broadcast_to(f, xyz[0].shape) for f in f_state(*xyz)])
        ex = np.array([np.broadcast_to(f, xyz[0].shape) for f in f_rhs(*xyz)])
        R = m.rhs(q)
        inner = m.wall() == 0
        e = [np.abs(R[v][inner] - ex[v][inner]).max() / np.abs(ex[v]).max() for v in range(5)]
        errs.append(e)
    errs = np.array(errs)
    assert np.all(errs[-1] < 3e-3), errs
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > N - 1.2), (errs, rates)


def test_isothermal_rest_about_isentropic_reference_converges(orc):
    """An isothermal atmosphere at rest written as a perturbation of the
    isentropic reference is in hydrostatic balance only up to the
    discretisation error, which must fall quickly with the order."""
    errs = []
    for N in (2, 4, 6):
        cfg = I.box((1, 1, 4), N, L=(1000.0, 1000.0, 8000.0))
        m = orc.Mesh(cfg)
        rho0, th0, p0 = m.ref()
        z = m.coords()[2]
        T0, Rd, P00, cp, cv, g = 260.0, cfg["Rd"], cfg["P00"], cfg["cp"], cfg["cv"], cfg["g"]
        piso = P00 * np.exp(-g * z / (Rd * T0))
        rho_iso = piso / (Rd * T0)
        th_iso = (P00 / Rd) * (piso / P00) ** (cv / cp)
        q = np.zeros((5, m.Ng))
        q[0] = rho_iso - rho0
        q[4] = th_iso - th0
        R = m.rhs(q)
        inner = m.wall() == 0
        errs.append(np.abs(R[3][inner]).max() / (g * np.abs(q[0]).max()))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


# ------------------------------------------ deep-atmosphere shell terms ----
# The source of Eq. 1 on the rotating sphere (Sec. 1: deep-atmosphere
# equations, no shallow-atmosphere approximation): Coriolis -2 Omega z x U and
# buoyancy along the radial gravity g(r) = g0 (a/r)^2, and the hydrostatic
# reference state in that gravity.  Each pin below also runs on copies of the
# oracle with a plausible mistake planted in its C source, and must fail
# there.

CORIOLIS = ("S[1] = -rp * gr * x / r + 2.0 * c->Omega * q[2 * Ng + g];\n"
            "            S[2] = -rp * gr * y / r - 2.0 * c->Omega * q[1 * Ng + g];")
GRAVITY = "double gr = c->g * (c->r_inner / r) * (c->r_inner / r);"
GEOPOTENTIAL = "return c->g * c->r_inner * h / (c->r_inner + h);"

PLANTED = {
    # +2 Omega z x U (both signs flipped)
    "coriolis_sign": [(CORIOLIS, "S[1] = -rp * gr * x / r - 2.0 * c->Omega * q[2 * Ng + g];\n"
                                 "            S[2] = -rp * gr * y / r + 2.0 * c->Omega * q[1 * Ng + g];")],
    # -Omega z x U (factor 2 dropped)
    "coriolis_factor": [(CORIOLIS, "S[1] = -rp * gr * x / r + c->Omega * q[2 * Ng + g];\n"
                                   "            S[2] = -rp * gr * y / r - c->Omega * q[1 * Ng + g];")],
    # each component taken from the wrong momentum component
    "coriolis_transposed": [(CORIOLIS, "S[1] = -rp * gr * x / r + 2.0 * c->Omega * q[1 * Ng + g];\n"
                                       "            S[2] = -rp * gr * y / r - 2.0 * c->Omega * q[2 * Ng + g];")],
    # shallow (constant) gravity in the buoyancy
    "gravity_constant": [(GRAVITY, "double gr = c->g;")],
    # g0 a / r instead of g0 (a/r)^2
    "gravity_power": [(GRAVITY, "double gr = c->g * (c->r_inner / r);")],
    # geopotential of constant gravity in the reference state
    "geopotential_flat": [(GEOPOTENTIAL, "return c->g * h;")],
}


@pytest.fixture(scope="module")
def planted(orc):
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = orc.build_variant(PLANTED[name], name)
        return cache[name]

    return get


def _rhat(m):
    xyz = m.coords()
    return xyz / np.linalg.norm(xyz, axis=0)


def _coriolis_error(orc):
    """max |R_U(Omega) - R_U(0) - P (2 Omega (U_y, -U_x, 0))| relative to
    max |2 Omega U| for rho' = Theta' = 0 and a smooth U; P removes the radial
    component at the bottom and lid nodes (the wall condition)."""
    cfg = I.shell(2, 2, 4)
    Om = cfg["Omega"]
    m1, m0 = orc.Mesh(cfg), orc.Mesh(dict(cfg, Omega=0.0))
    xyz = m1.coords()
    rho0 = m1.ref()[0]
    q = np.zeros((5, m1.Ng))
    q[1:4] = I.smooth_perturbation(xyz, seed=41, length=3.0e6, U=1.0)[1:4] * 10.0 * rho0
    d = m1.rhs(q)[1:4] - m0.rhs(q)[1:4]
    exact = 2.0 * Om * np.array([q[2], -q[1], np.zeros(m1.Ng)])
    walls = (m1.wall() & 8) != 0
    rh = _rhat(m1)
    exact[:, walls] -= (exact[:, walls] * rh[:, walls]).sum(0) * rh[:, walls]
    assert np.abs(exact).max() > 1e-4  # a Coriolis tendency of size
    return np.abs(d - exact).max() / np.abs(exact).max()


def test_coriolis_closed_form(orc):
    """The rotation enters R only through -2 Omega z x U: the difference of
    the tendencies with and without rotation is that term, at every node."""
    assert _coriolis_error(orc) < 1e-12


def _gravity_error(orc):
    """rho' != 0, U = 0, Theta' = 0: every flux vanishes exactly, so
    R_rho = R_Theta = 0 and R_U = -rho' g0 (a/r)^2 r_hat (Eq. 4: the DSS of a
    nodal source is the source), with the radial part removed at the bottom
    and lid.  Returns the largest relative deviation."""
    cfg = I.shell(2, 2, 4)
    m = orc.Mesh(cfg)
    rho0 = m.ref()[0]
    q = np.zeros((5, m.Ng))
    q[0] = 0.01 * rho0 * I.smooth_perturbation(m.coords(), seed=42, length=3.0e6, rho=1.0)[0]
    R = m.rhs(q)
    assert np.all(R[0] == 0.0) and np.all(R[4] == 0.0)
    r = np.linalg.norm(m.coords(), axis=0)
    g = cfg["g"] * (cfg["r_inner"] / r) ** 2
    exact = -q[0] * g * _rhat(m)
    walls = (m.wall() & 8) != 0
    scale = np.abs(exact).max()
    err_in = np.abs(R[1:4][:, ~walls] - exact[:, ~walls]).max() / scale
    err_wall = np.abs(R[1:4][:, walls]).max() / scale  # a purely radial tendency is removed
    return max(err_in, err_wall)


def test_deep_gravity_buoyancy_closed_form(orc):
    assert _gravity_error(orc) < 1e-13


def _column_balance_error(orc, cfg):
    """Along one radial column of the shell, the reference state satisfies
    dp0/dr = -rho0 g0 (a/r)^2 (hydrostatic balance in the deep-atmosphere
    gravity).  dp0/dr is taken from a Chebyshev fit of the oracle's p0 at the
    column's nodes; returns the largest relative deviation."""
    m = orc.Mesh(cfg)
    xyz = m.coords()
    r = np.linalg.norm(xyz, axis=0)
    rh = xyz / r
    k = int(np.argmax(rh[2]))  # the column through the node nearest the pole
    col = np.where(np.abs(rh - rh[:, [k]]).max(axis=0) < 1e-12)[0]
    assert len(col) == cfg["nlayer"] * cfg["N"] + 1
    o = col[np.argsort(r[col])]
    rho0, _, p0 = m.ref()
    h = r[o] - cfg["r_inner"]
    fit = np.polynomial.Chebyshev.fit(h, p0[o], 24)
    dpdr = fit.deriv()(h)
    exact = -rho0[o] * cfg["g"] * (cfg["r_inner"] / r[o]) ** 2
    return np.abs(dpdr - exact).max() / np.abs(exact).max()


SHELL_REFS = [
    I.shell(1, 12, 6),  # isothermal 250 K to 30 km (the shell workloads' reference)
    I.shell(1, 12, 6, ref="isentropic", theta0=300.0, r_outer=I.EARTH_RADIUS + 10.0e3),
]


@pytest.mark.parametrize("cfg", SHELL_REFS, ids=["isothermal", "isentropic"])
def test_shell_reference_is_hydrostatic(orc, cfg):
    assert _column_balance_error(orc, cfg) < 1e-9
    m = orc.Mesh(cfg)
    _, th0, p0 = m.ref()
    peos = cfg["P00"] * (cfg["Rd"] * th0 / cfg["P00"]) ** _gamma(cfg)
    np.testing.assert_allclose(peos, p0, rtol=1e-13)


@pytest.mark.parametrize("mistake", ["coriolis_sign", "coriolis_factor", "coriolis_transposed"])
def test_coriolis_pin_catches_planted_mistakes(orc, planted, mistake):
    with orc.using_library(planted(mistake)):
        assert _coriolis_error(orc) > 1e-3


@pytest.mark.parametrize("mistake", ["gravity_constant", "gravity_power"])
def test_gravity_pin_catches_planted_mistakes(orc, planted, mistake):
    with orc.using_library(planted(mistake)):
        assert _gravity_error(orc) > 1e-4


def test_reference_pin_catches_flat_geopotential(orc, planted):
    with orc.using_library(planted("geopotential_flat")):
        assert _column_balance_error(orc, SHELL_REFS[0]) > 1e-4
        assert _column_balance_error(orc, SHELL_REFS[1]) > 1e-4
