"""Pins of the 1D-IMEX oracle (Sec. 2.2: leapfrog with implicit corrections
along vertical columns) against facts that do not come from the oracle's own
formulas: exactness of the column derivative on polynomials, the vertical
operator as the linearisation of the full right-hand side of Eq. 1, closed
forms of the scheme on linear problems, the Robert-Asselin recurrence,
second-order convergence, and stability past the explicit limit."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

THIN = I.box((3, 2, 4), 3, L=(4000.0, 3000.0, 1000.0))
THIN_BUBBLE = (0.5, 900.0, 2000.0, 1500.0, 350.0)


@pytest.fixture(scope="module")
def imex(orc):
    from oracle import imex as mod
    return mod


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_column_derivative_exact_on_polynomials(imex, N):
    # unequal element heights: the assembly must weight each element by its Jacobian
    edges = np.array([0.0, 130.0, 400.0, 460.0, 1000.0])
    xi, _ = imex.O.lgl(N)
    z = np.concatenate([a + 0.5 * (1 + xi[:-1]) * (b - a) for a, b in zip(edges[:-1], edges[1:])] + [edges[-1:]])
    Dz = imex.cg_derivative_1d(z, N)
    for j in range(N + 1):
        exact = j * z ** (j - 1) if j else np.zeros_like(z)
        scale = max(1.0, np.abs(exact).max())
        assert np.abs(Dz @ z**j - exact).max() <= 1e-11 * scale
    # a kink at the node z = 400 shared by elements of heights 270 (below) and
    # 60 (above): the one-sided derivatives -1 and +1 meet at that node,
    # averaged by the mass each element gives it (w_N h_below / 2 and
    # w_0 h_above / 2, w_0 = w_N), i.e. (60 - 270) / (60 + 270); every other
    # node sees a linear function
    f = np.abs(z - 400.0)
    expect = np.sign(z - 400.0)
    expect[z == 400.0] = (60.0 - 270.0) / (60.0 + 270.0)
    assert np.abs(Dz @ f - expect).max() <= 1e-11


def _column_perturbation(m, zwall_W_zero=True):
    rho0, Th0, _ = m.ref()
    z = m.coords()[2] / 1000.0
    dq = np.zeros((5, m.Ng))
    dq[0] = 1e-3 * rho0 * np.sin(2.1 * z + 0.3)
    dq[3] = rho0 * np.sin(np.pi * z) * np.cos(1.3 * z)
    dq[4] = 1e-3 * Th0 * np.cos(3.0 * z)
    if zwall_W_zero:
        dq[3][(m.wall() & 4) != 0] = 0.0
    return dq


@pytest.mark.parametrize("cfg", [
    THIN,
    I.box((2, 2, 3), 4, L=(3000.0, 3000.0, 1500.0), periodic=(1, 1, 0), ref="isothermal", T0=250.0),
    I.box((2, 1, 2), 2, L=(800.0, 500.0, 2000.0)),
], ids=["thin_N3", "periodic_xy_isothermal_N4", "tall_N2"])
def test_L_is_the_linearised_rhs(orc, imex, cfg):
    """For perturbations that depend on z only, the full RHS about the rest
    state, differentiated by central differences, is L: the horizontal
    derivatives vanish and the EOS and advection terms linearise to c2 and
    theta0 (the difference quotient converges as eps^2)."""
    m = orc.Mesh(cfg)
    cols = imex.VerticalColumns(m)
    dq = _column_perturbation(m)
    Lq = cols.apply(dq)
    errs = []
    for eps in (1e-2, 1e-3):
        fd = (m.rhs(eps * dq) - m.rhs(-eps * dq)) / (2 * eps)
        errs.append([np.abs(fd[v] - Lq[v]).max() / np.abs(Lq[v]).max() for v in (0, 3, 4)])
        for v in (1, 2):  # no horizontal momentum tendency
            assert np.abs(fd[v]).max() <= 1e-12 * np.abs(Lq[3]).max()
    errs = np.array(errs)
    assert errs[1].max() <= 1e-9, errs
    assert np.all(errs[1] <= 0.02 * errs[0] + 1e-14), errs  # eps^2 convergence
    assert np.abs(Lq[3][(m.wall() & 4) != 0]).max() == 0.0


def _solve_residual(orc, imex, cfg, tau, seed=5):
    """x = solve(tau, b) for a random b of atmospheric scale; the largest
    residual |x - tau L x - b| over the five variables, relative to
    |b| + tau |L x|.  L is pinned above as the linearised right-hand side,
    so this holds the column solve (its dense blocks and the momentum
    correction along r_hat) to inverting I - tau L."""
    m = orc.Mesh(cfg)
    cols = imex.VerticalColumns(m)
    rho0, Th0, _ = m.ref()
    b = np.random.default_rng(seed).standard_normal((5, m.Ng))
    b[0] *= 1e-3 * rho0
    b[4] *= 1e-3 * Th0
    x = cols.solve(tau, b)
    Lx = cols.apply(x)
    res = x - tau * Lx - b
    return max(np.abs(res[v]).max() / (np.abs(b[v]).max() + tau * np.abs(Lx[v]).max()) for v in range(5))


SOLVE_BAR = 1e-12


@pytest.mark.parametrize("where,tau", [("box", 0.4), ("box", 5.0), ("shell", 10.0), ("shell", 20.0)])
def test_solve_inverts_I_minus_tau_L(orc, imex, where, tau):
    cfg = THIN if where == "box" else _thin_shell(3)
    assert _solve_residual(orc, imex, cfg, tau) <= SOLVE_BAR


def _linear_problem(n=4, seed=1, stiff=3.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = A - A.T
    B = rng.standard_normal((n, n))
    B = (B - B.T) * stiff
    return A, B, rng.standard_normal(n)


def test_scheme_on_a_linear_problem_is_the_cayley_map(imex):
    """With R = L = B (nothing explicit) the step maps the filtered q^{n-1}
    to q^{n+1} by the Cayley transform (I - dt B)^-1 (I + dt B), and the
    start step is the trapezoidal rule over dt."""
    _, B, q0 = _linear_problem()
    n = len(q0)
    R = Lop = lambda q: B @ q
    solve = lambda tau, b: np.linalg.solve(np.eye(n) - tau * B, b)
    dt = 0.37
    cay = lambda h: np.linalg.solve(np.eye(n) - h * B, np.eye(n) + h * B)
    q1 = imex.lf_imex_start(R, Lop, solve, q0, dt)
    assert np.allclose(q1, cay(dt / 2) @ q0, rtol=0, atol=1e-13)
    q_prev = q0 + 0.1
    q2, _ = imex.lf_imex_step(R, Lop, solve, q_prev, q1, dt, 0.0)
    assert np.allclose(q2, cay(dt) @ q_prev, rtol=0, atol=1e-13)
    # the Cayley map is orthogonal for skew B: the norm of each parity class is kept
    qs, _ = imex.lf_imex_run(R, Lop, solve, q0, dt, 41, 0.0)
    assert abs(np.linalg.norm(qs) - np.linalg.norm(q1)) <= 1e-12 * np.linalg.norm(q1)


def test_scheme_is_second_order(imex):
    from scipy.linalg import expm

    A, B, q0 = _linear_problem()
    n = len(q0)
    R = lambda q: (A + B) @ q
    Lop = lambda q: B @ q
    solve = lambda tau, b: np.linalg.solve(np.eye(n) - tau * B, b)
    T = 2.0
    ex = expm((A + B) * T) @ q0
    errs = [np.abs(imex.lf_imex_run(R, Lop, solve, q0, dt, int(round(T / dt)), 0.0)[0] - ex).max()
            for dt in (0.01, 0.005, 0.0025)]
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4, errs


@pytest.mark.parametrize("nu", [0.0, 0.05, 0.2])
def test_robert_asselin_recurrence(imex, nu):
    """Oscillation equation q' = i w q, L = 0: the filtered leapfrog state
    (q^n, qbar^{n-1}) evolves by the 2x2 matrix [[2z, 1], [1 - 2nu + 2nu z, 2nu]],
    z = i w dt (Asselin's filter written as a recurrence); after many steps
    q^{n+1}/q^n is its dominant eigenvalue, and with nu = 0 both modes keep
    modulus one."""
    w, dt = 1.0, 0.3
    z = 1j * w * dt
    mu = np.linalg.eigvals(np.array([[2 * z, 1.0], [1 - 2 * nu + 2 * nu * z, 2 * nu]]))
    phys = mu[np.argmax(np.abs(mu))]
    R = lambda q: 1j * w * q
    Lop = lambda q: 0.0 * q
    solve = lambda tau, b: b
    q0 = np.array([1.0 + 0.0j])
    qa, _ = imex.lf_imex_run(R, Lop, solve, q0, dt, 400, nu)
    qb, _ = imex.lf_imex_run(R, Lop, solve, q0, dt, 401, nu)
    if nu > 0:
        assert abs(qb[0] / qa[0] - phys) <= 1e-9
        assert np.abs(mu).min() < 1 - nu  # computational mode damped
        # the filter damps the physical mode at second order in w dt
        assert 0 < 1 - abs(phys) < nu * (w * dt) ** 2
    else:
        assert np.allclose(np.abs(mu), 1.0, atol=1e-14)
        assert abs(abs(qa[0]) - 1) < 0.05


def test_imex_run_second_order_on_the_mesh(orc, imex):
    m = orc.Mesh(THIN)
    cols = imex.VerticalColumns(m)
    q0 = m.init_state("bubble", THIN_BUBBLE)
    T = 2.0
    res = [imex.run_imex(m, q0, dt, int(round(T / dt)), 0.0, cols)[0] for dt in (0.05, 0.025, 0.0125)]
    d1, d2 = res[0] - res[1], res[1] - res[2]
    ratios = [np.abs(d1[v]).max() / np.abs(d2[v]).max() for v in (0, 3, 4)]
    assert all(3.0 < r < 6.0 for r in ratios), ratios


def test_imex_stable_past_the_explicit_limit(orc, imex):
    """dt = 0.4 s puts the vertical acoustic Courant number near 2 on the thin
    box: SSP-RK3 diverges, the 1D-IMEX run stays close to a fine explicit run."""
    m = orc.Mesh(THIN)
    q0 = m.init_state("bubble", THIN_BUBBLE)
    T, dt = 8.0, 0.4
    n = int(round(T / dt))
    qr = m.run(q0, dt, n)
    assert not (np.isfinite(qr).all() and np.abs(qr[3]).max() < 1.0)
    qi, _ = imex.run_imex(m, q0, dt, n, 0.05)
    ref = m.run(q0, 0.02, int(round(T / 0.02)))
    assert np.abs(qi[3] - ref[3]).max() <= 0.1 * np.abs(ref[3]).max()
    assert np.abs(qi[0] - ref[0]).max() <= 0.05 * np.abs(ref[0]).max()


def _thin_shell(N, lid=12e3, npanel=2, nlayer=3):
    cfg = I.shell(npanel, nlayer, N)
    cfg["r_outer"] = cfg["r_inner"] + lid
    return cfg


def test_L_is_the_linearised_rhs_on_the_shell(orc, imex):
    """Radial perturbations W(r) r_hat, rho'(r), Theta'(r) on the cubed-sphere
    shell: the rho', radial-momentum and Theta' tendencies of the linearised
    full RHS are L's, spherical divergence term 2 W / r included; the
    horizontal momentum tendency, which L leaves to the explicit part, is a
    discretisation error that falls with N."""
    horiz = []
    for N in (3, 5):
        cfg = _thin_shell(N)
        m = orc.Mesh(cfg)
        cols = imex.VerticalColumns(m)
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
        eps = 1e-3
        fd = (m.rhs(eps * dq) - m.rhs(-eps * dq)) / (2 * eps)
        fW, LW = cols.radial(fd), cols.radial(Lq)
        for a, b in ((fd[0], Lq[0]), (fW, LW), (fd[4], Lq[4])):
            assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
        # without the 2 W / r term the density tendency is off at the 1e-4 level
        G_only = -np.concatenate([Dz @ W[c] for c, Dz in zip(cols.cols, cols.Dz)])
        idx = np.concatenate(list(cols.cols))
        assert np.abs(G_only - fd[0][idx]).max() > 1e-5 * np.abs(Lq[0]).max()
        horiz.append(np.abs(fd[1:4] - fW * cols.nhat).max() / np.abs(LW).max())
    assert horiz[0] < 0.05 and horiz[1] < 0.7 * horiz[0], horiz


def test_imex_on_the_shell_second_order_and_stable(orc, imex):
    cfg = _thin_shell(4)
    m = orc.Mesh(cfg)
    cols = imex.VerticalColumns(m)
    q0 = m.init_state("jetwave", I.JETWAVE_PARAMS)
    T = 4.0
    res = [imex.run_imex(m, q0, dt, int(round(T / dt)), 0.0, cols)[0] for dt in (0.2, 0.1, 0.05)]
    d1, d2 = res[0] - res[1], res[1] - res[2]
    ratios = [np.abs(d1[v]).max() / np.abs(d2[v]).max() for v in range(5)]
    assert all(3.3 < r < 4.8 for r in ratios), ratios
    # dt = 20 s: vertical acoustic Courant number near 10; SSP-RK3 already fails at 3 s
    qr = m.run(q0, 3.0, 100)
    assert not (np.isfinite(qr).all() and np.abs(qr).max() < 1e6)
    ref = m.run(q0, 0.5, 600)
    qi, _ = imex.run_imex(m, q0, 20.0, 15, 0.05, cols)
    assert np.abs(qi[1:4] - ref[1:4]).max() <= 0.01 * np.abs(ref[1:4]).max()


def test_filtered_imex_run_composes(orc, imex):
    """The filtered run is the plain run when the filter never fires, and
    when it is the identity (mu = 0: DSS(Jw q) / M = q for a continuous q)
    it matches to rounding; a real filter changes the state."""
    m = orc.Mesh(THIN)
    q0 = m.init_state("bubble", THIN_BUBBLE)
    plain, plain_prev = imex.run_imex(m, q0, 0.4, 7, 0.1)
    never, never_prev = imex.run_imex_filtered(m, q0, 0.4, 7, 0.1, 0, 2, 12.0, 0.5)
    assert np.array_equal(plain, never) and np.array_equal(plain_prev, never_prev)
    ident, _ = imex.run_imex_filtered(m, q0, 0.4, 7, 0.1, 1, 2, 12.0, 0.0)
    assert np.abs(ident - plain).max() <= 1e-12 * np.abs(plain).max()
    filt, _ = imex.run_imex_filtered(m, q0, 0.4, 7, 0.1, 2, 2, 12.0, 0.5)
    assert np.abs(filt - plain).max() > 1e-6 * np.abs(plain).max()
