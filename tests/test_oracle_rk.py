"""Pins of the oracle's SSP-RK3 stage code (Sec. 2.2 explicit stages):
the one-step amplification polynomial on a linear system and third-order
convergence on a nonlinear ODE; and the NUMA run loop is the same code."""
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
