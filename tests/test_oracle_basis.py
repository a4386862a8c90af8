"""Pins of the oracle's 1D basis: Lobatto nodes, weights and the
differentiation matrix (Sec. 2.1, Eqs. 2-5), checked against closed forms,
quadrature exactness and library polynomial routines."""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lgl_closed_forms.json")


def test_lgl_closed_forms(orc):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for N, c in cases.items():
        xi, w = orc.lgl(int(N))
        ex_x = np.array([eval(s, {"math": math}) for s in c["nodes"]])
        ex_w = np.array([eval(s, {"math": math}) for s in c["weights"]])
        np.testing.assert_allclose(xi, ex_x, rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, ex_w, rtol=0, atol=4e-16)


@pytest.mark.parametrize("N", range(1, 9))
def test_lgl_quadrature_exact_to_2N_minus_1(orc, N):
    xi, w = orc.lgl(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ xi**k - exact) < 1e-14, k
    # Lobatto quadrature is not exact at degree 2N (Gauss would be): this
    # separates Lobatto from Gauss points.
    k = 2 * N
    assert abs(w @ xi**k - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("N", range(2, 9))
def test_lgl_interior_nodes_are_roots_of_dPN(orc, N):
    xi, _ = orc.lgl(N)
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    roots = np.sort(np.real(dP.roots()))
    np.testing.assert_allclose(xi[1:-1], roots, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 9))
def test_dmatrix_exact_on_polynomials_up_to_N(orc, N):
    xi, _ = orc.lgl(N)
    D = orc.dmatrix(N)
    for k in range(0, N + 1):
        d = D @ xi**k
        exact = k * xi ** (k - 1) if k else np.zeros_like(xi)
        assert np.abs(d - exact).max() < 1e-12 * max(1, N * N), (N, k)
    # degree N+1 is beyond the interpolation space: not reproduced
    d = D @ xi ** (N + 1)
    assert np.abs(d - (N + 1) * xi**N).max() > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_dmatrix_structure(orc, N):
    D = orc.dmatrix(N)
    P = N + 1
    assert np.abs(D.sum(axis=1)).max() < 1e-13 * N * N
    for i in range(P):
        for j in range(P):
            assert abs(D[N - i, N - j] + D[i, j]) < 1e-12 * N * N
    # closed-form corner entries of the Lobatto differentiation matrix
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-12 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-12 * N * N


@pytest.mark.parametrize("N", range(1, 9))
def test_dmatrix_matches_library_lagrange_derivative(orc, N):
    xi, _ = orc.lgl(N)
    D = orc.dmatrix(N)
    V = np.vander(xi, N + 1, increasing=True)
    for j in range(N + 1):
        e = np.zeros(N + 1)
        e[j] = 1.0
        coef = np.linalg.solve(V, e)  # psi_j in the monomial basis
        dcoef = np.polynomial.polynomial.polyder(coef)
        dpsi = np.polynomial.polynomial.polyval(xi, dcoef)
        np.testing.assert_allclose(D[:, j], dpsi, rtol=0, atol=1e-10 * N * N)
