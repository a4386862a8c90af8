"""Pins of the oracle's Boyd-Vandeven filter (Sec. 2.3, applied with DSS and
the inverse mass matrix after each time step as in the time loop of Sec. 7).

The weights are checked against closed-form values, the symmetry of the
erfc-log form and Vandeven's original filter (a regularized incomplete beta
function); the 1D matrix against Legendre polynomials evaluated by numpy (its
eigenvectors); the 3D application with DSS against polynomial invariance,
conservation, and a Kronecker-product computation on single elements."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

P_ORDER = 12.0


def test_weights_closed_forms(orc):
    s = orc.filter_weights(4, 2, P_ORDER)
    assert np.array_equal(s[:2], [1.0, 1.0])
    assert s[2] == 1.0 and s[4] == 0.0  # theta = 0 and theta = 1
    assert s[3] == 0.5  # theta = 1/2: erfc(0) / 2
    s6 = orc.filter_weights(6, 2, P_ORDER)
    # erfc-log form: sigma(theta) + sigma(1 - theta) = 1
    assert abs(s6[3] + s6[5] - 1.0) < 1e-15
    assert s6[4] == 0.5
    assert np.all(np.diff(s6) <= 0.0)
    # strength mu blends with the identity
    for mu in (0.0, 0.3, 1.0):
        sm = orc.filter_weights(6, 2, P_ORDER, mu)
        assert np.allclose(sm, 1.0 - mu * (1.0 - s6), atol=1e-15, rtol=0)
    # s = N damps only the top mode, completely
    assert np.array_equal(orc.filter_weights(5, 5, P_ORDER), [1, 1, 1, 1, 1, 0])
    # s > N keeps everything
    assert np.array_equal(orc.filter_weights(4, 5, P_ORDER), np.ones(5))


def test_weights_approximate_vandeven(orc):
    """Boyd's erfc-log form approximates Vandeven's filter of order p,
    1 - I_theta(p, p) (regularized incomplete beta), uniformly in theta."""
    betainc = pytest.importorskip("scipy.special").betainc
    N, s = 8, 0
    for p in (4.0, 8.0, 12.0):
        sig = orc.filter_weights(N, s, p)
        theta = np.arange(N + 1) / N
        vand = 1.0 - betainc(p, p, theta)
        assert np.abs(sig - vand).max() < 0.02, (p, sig, vand)


@pytest.mark.parametrize("N,s", [(2, 1), (4, 2), (4, 4), (6, 3), (8, 5)])
def test_matrix_eigenvectors_are_legendre(orc, N, s):
    """F P_k(xi) = sigma_k P_k(xi) at the Lobatto points, with P_k from numpy."""
    from numpy.polynomial import legendre as L

    xi, _ = orc.lgl(N)
    F = orc.filter_matrix(N, s, P_ORDER)
    sig = orc.filter_weights(N, s, P_ORDER)
    for k in range(N + 1):
        c = np.zeros(k + 1)
        c[k] = 1.0
        pk = L.legval(xi, c)
        assert np.abs(F @ pk - sig[k] * pk).max() < 5e-14, k
    assert np.abs(F.sum(axis=1) - 1.0).max() < 5e-15  # constants are kept
    assert np.abs(orc.filter_matrix(N, s, P_ORDER, 0.0) - np.eye(N + 1)).max() < 5e-15


MESHES = [
    ("box_walls", I.box((3, 2, 2), 4, L=(900.0, 600.0, 700.0))),
    ("box_periodic", I.box(2, 4, periodic=(1, 1, 1))),
    ("box_warped", I.box(2, 3, warp=0.05)),
    ("shell", I.shell(2, 1, 3)),
]


def _random_state(m, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((5, m.Ng))


@pytest.mark.parametrize("name,cfg", MESHES, ids=[c[0] for c in MESHES])
def test_zero_strength_is_identity(orc, name, cfg):
    m = orc.Mesh(cfg)
    q = _random_state(m, 1)
    out = m.filter(q, 2, P_ORDER, 0.0)
    assert np.abs(out - q).max() < 1e-13 * np.abs(q).max()


def test_low_degree_polynomials_are_kept(orc):
    """A field of degree < s in each coordinate is a sum of kept modes on an
    affine element; continuous, so DSS returns it."""
    cfg = I.box((3, 2, 2), 5, L=(900.0, 600.0, 700.0))
    m = orc.Mesh(cfg)
    x, y, z = m.coords() / 1000.0
    f = 1.0 + x - 2 * y * y + 0.5 * x * z + x * x * y * z * z
    q = np.stack([f, 2 * f, -f, 0.5 * f, 3 * f])
    out = m.filter(q, 3, P_ORDER)  # modes 0, 1, 2 kept; degree <= 2 per coordinate
    assert np.abs(out - q).max() < 1e-13 * np.abs(q).max()


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_conservation_on_affine_boxes(orc, periodic):
    m = orc.Mesh(I.box((3, 2, 2), 4, periodic=periodic))
    q = _random_state(m, 2)
    M = m.mass()
    out = m.filter(q, 2, P_ORDER)
    vars_ = range(5) if periodic[0] else (0, 4)  # walls keep the normal momentum
    for v in vars_:
        assert abs(M @ out[v] - M @ q[v]) < 1e-12 * (M @ np.abs(q[v])), v
    assert np.abs(out - q).max() > 1e-3  # it did damp something


def test_single_element_is_the_tensor_product(orc):
    """One walled element: every node is its own global node, so the filter is
    exactly (F x F x F) q on each variable (node l = i + P (j + P k))."""
    N = 4
    m = orc.Mesh(I.box(1, N, L=(800.0, 900.0, 1000.0)))
    F = orc.filter_matrix(N, 2, P_ORDER)
    q = _random_state(m, 3)
    out = m.filter(q, 2, P_ORDER)
    xyz = m.coords()
    K = np.kron(F, np.kron(F, F))  # acts on index k*P^2 + j*P + i
    # global node numbering of the single box element is lexicographic in x, y, z
    order = np.lexsort((xyz[0], xyz[1], xyz[2]))
    for v in (0, 4):
        ref = np.empty(m.Ng)
        ref[order] = K @ q[v][order]
        assert np.abs(out[v] - ref).max() < 1e-13 * np.abs(q[v]).max()
    # the top Legendre mode in x is removed (sigma_N = 0)
    from numpy.polynomial import legendre as L

    X = 2.0 * xyz[0] / 800.0 - 1.0
    top = L.legval(X, np.eye(N + 1)[N])
    qt = np.zeros((5, m.Ng))
    qt[0] = top
    assert np.abs(m.filter(qt, 2, P_ORDER)[0]).max() < 1e-13


def test_two_elements_brute_force(orc):
    """Two elements along x: the shared face's nodes get the Jw-weighted mean
    of the two element results (coordinate matching, no oracle maps)."""
    N = 3
    P = N + 1
    cfg = I.box((2, 1, 1), N, L=(600.0, 500.0, 400.0))
    m = orc.Mesh(cfg)
    F = orc.filter_matrix(N, 1, P_ORDER)
    K = np.kron(F, np.kron(F, F))
    q = _random_state(m, 4)
    xyz = m.coords()
    exyz = m.elem_coords()
    jw = m.jw()
    acc = np.zeros((5, m.Ng))
    wsum = np.zeros(m.Ng)
    for e in range(2):
        sl = slice(e * P**3, (e + 1) * P**3)
        pts = exyz[:, sl]
        gi = np.array([np.argmin(np.sum((xyz.T - p) ** 2, axis=1)) for p in pts.T])
        for v in range(5):
            acc[v, gi] += jw[sl] * (K @ q[v, gi])
        wsum[gi] += jw[sl]
    ref = acc / wsum
    out = m.filter(q, 1, P_ORDER)
    walls = m.wall()
    for v in (0, 4):
        assert np.abs(out[v] - ref[v]).max() < 1e-13 * np.abs(q[v]).max()
    # walled momentum components keep their pre-filter values
    for a in range(3):
        w = (walls & (1 << a)) != 0
        assert np.array_equal(out[1 + a][w], q[1 + a][w])
        assert np.abs(out[1 + a][~w] - ref[1 + a][~w]).max() < 1e-13 * np.abs(q).max()


def test_filtered_run(orc):
    cfg = I.box(2, 3)
    m = orc.Mesh(cfg)
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS)
    a = m.run(q0, 0.01, 4)
    assert np.array_equal(m.run_filtered(q0, 0.01, 4, 0, 2, P_ORDER), a)
    b = m.run_filtered(q0, 0.01, 4, 2, 2, P_ORDER)
    # by hand: two steps, filter, two steps, filter
    h = m.filter(m.run(m.filter(m.run(q0, 0.01, 2), 2, P_ORDER), 0.01, 2), 2, P_ORDER)
    assert np.array_equal(b, h)
