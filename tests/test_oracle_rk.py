"""Pins of the oracle's time integrators (Sec. 2.2 explicit stages).

SSP-RK3: the one-step amplification polynomial on a linear system and third-
order convergence on a nonlinear ODE.  The five-stage low-storage scheme: the
eight fourth-order conditions of its Butcher form, agreement with exp(Z)
through Z^4 on a linear system, and fourth-order convergence.  For both, the
NUMA run loop is the same stage code."""
import numpy as np

from paper_1511_01561_gb300 import inputs as I


def test_linear_system_amplification(orc):
    A = np.array([[-0.3, 1.2, 0.0], [-1.1, -0.2, 0.4], [0.1, 0.0, -0.9]])
    dt = 0.37
    q0 = np.array([1.0, -2.0, 0.5])
    q1 = orc.ssprk3_step(q0, dt, lambda q: A @ q)
    Z = A * dt
    amp = np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
    np.testing.assert_allclose(q1, amp @ q0, rtol=1e-14, atol=1e-15)


def test_third_order_convergence(orc):
    f = lambda q: -q * q  # q(t) = 1/(1+t)
    errs = []
    for n in (10, 20, 40):
        q = np.array([1.0])
        dt = 1.0 / n
        for _ in range(n):
            q = orc.ssprk3_step(q, dt, f)
        errs.append(abs(q[0] - 0.5))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 2.8 < r1 < 3.2 and 2.8 < r2 < 3.2, errs


def test_run_equals_stagewise_rk(orc):
    m = orc.Mesh(I.box(2, 3))
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS) + 1e-3 * I.random_perturbation(m.Ng, seed=5)
    dt = 0.02
    a = m.run(q0, dt, 2)
    b = q0.copy()
    for _ in range(2):
        b = orc.ssprk3_step(b.ravel(), dt, lambda q: m.rhs(q.reshape(5, -1)).ravel()).reshape(5, -1)
    assert np.array_equal(a, b)


# ---- five-stage low-storage RK (Carpenter-Kennedy 2N form, order four) ----

def _butcher_from_2n(A, B):
    """Butcher matrix and weights of the 2N scheme dq <- A_i dq + dt F(q),
    q <- q + B_i dq, by tracking each quantity's coefficients of F_1..F_5."""
    s = len(A)
    a = np.zeros((s, s))
    dq = np.zeros(s)
    q = np.zeros(s)
    for i in range(s):
        a[i] = q
        dq = A[i] * dq
        dq[i] += 1.0
        q = q + B[i] * dq
    return a, q


def test_lsrk54_order_conditions(orc):
    """The oracle's coefficients satisfy all eight fourth-order conditions."""
    A, B = orc.lsrk54_coefficients()
    assert A[0] == 0.0
    a, b = _butcher_from_2n(A, B)
    c = a.sum(axis=1)
    e = np.ones(5)
    conds = [
        (b @ e, 1.0), (b @ c, 1 / 2), (b @ c**2, 1 / 3), (b @ (a @ c), 1 / 6),
        (b @ c**3, 1 / 4), (b @ (c * (a @ c)), 1 / 8), (b @ (a @ c**2), 1 / 12), (b @ (a @ (a @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-15
    assert abs(b @ c**4 - 1 / 5) > 1e-6  # not fifth order


def test_lsrk54_linear_system(orc):
    A = np.array([[-0.3, 1.2, 0.0], [-1.1, -0.2, 0.4], [0.1, 0.0, -0.9]])
    q0 = np.array([1.0, -2.0, 0.5])
    res = []
    for dt in (0.2, 0.1):
        Z = A * dt
        taylor4 = np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
        res.append(np.abs(orc.lsrk54_step(q0, dt, lambda q: A @ q) - taylor4 @ q0).max())
    # the step agrees with exp(Z) through Z^4; the rest is O(dt^5)
    assert 28.0 < res[0] / res[1] < 36.0, res


def test_lsrk54_fourth_order_convergence(orc):
    f = lambda q: -q * q  # q(t) = 1/(1+t)
    errs = []
    for n in (8, 16, 32):
        q = np.array([1.0])
        for _ in range(n):
            q = orc.lsrk54_step(q, 1.0 / n, f)
        errs.append(abs(q[0] - 0.5))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 3.7 < r1 < 4.3 and 3.7 < r2 < 4.3, errs


def test_lsrk54_run_equals_stagewise(orc):
    m = orc.Mesh(I.box(2, 3))
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS) + 1e-3 * I.random_perturbation(m.Ng, seed=5)
    dt = 0.02
    a = m.run_lsrk54(q0, dt, 2)
    b = q0.copy()
    for _ in range(2):
        b = orc.lsrk54_step(b.ravel(), dt, lambda q: m.rhs(q.reshape(5, -1)).ravel()).reshape(5, -1)
    assert np.array_equal(a, b)
