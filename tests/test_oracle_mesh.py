"""Pins of the oracle's mesh, metric terms (Eq. 5), mass matrix (Eq. 4) and
element-to-global maps: closed forms on the affine box, volumes, node counts,
and brute-force per-node assembly by coordinate search on tiny meshes."""
import math

import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I


def test_box_metrics_closed_form(orc):
    ne, L = (2, 3, 4), (1000.0, 600.0, 800.0)
    m = orc.Mesh(I.box(ne, 3, L=L))
    met = m.metrics()
    h = [L[a] / ne[a] for a in range(3)]
    for d in range(3):
        for c in range(3):
            exact = 2.0 / h[c] if c == d else 0.0
            assert np.abs(met[3 * d + c] - exact).max() < 1e-13 * 2.0 / min(h)
    np.testing.assert_allclose(met[9], h[0] * h[1] * h[2] / 8.0, rtol=1e-13)
    assert abs(m.jw().sum() - L[0] * L[1] * L[2]) < 1e-12 * L[0] * L[1] * L[2]
    assert abs(m.mass().sum() - L[0] * L[1] * L[2]) < 1e-12 * L[0] * L[1] * L[2]


def test_box_sizes_walls_and_periodic(orc):
    m = orc.Mesh(I.box((2, 3, 4), 3))
    assert (m.Ne, m.Nl, m.Ng) == (24, 24 * 64, 7 * 10 * 13)
    wall = m.wall().reshape(13, 10, 7)
    assert np.all(wall[:, :, 0] & 1) and np.all(wall[:, :, -1] & 1)
    assert not np.any(wall[:, :, 1:-1] & 1)
    assert np.all(wall[0] & 4) and np.all(wall[-1] & 4)
    mp = orc.Mesh(I.box((2, 3, 4), 3, periodic=(1, 1, 0)))
    assert mp.Ng == 6 * 9 * 13
    assert not np.any(mp.wall() & 3)


def test_warped_box_volume_is_exact(orc):
    """The warp moves no boundary node, so the image is still the box; the
    Lobatto quadrature of the isoparametric Jacobian reproduces its volume
    to roundoff (summation-by-parts property of D with the Lobatto weights)."""
    for N in (2, 3, 4, 5):
        for warp in (0.03, 0.15):
            m = orc.Mesh(I.box(2, N, warp=warp))
            assert abs(m.jw().sum() / 1e9 - 1.0) < 1e-13
            assert np.all(m.metrics()[9] > 0)


def test_shell_counts_radii_and_volume(orc):
    a, top = I.PHYS_SHELL["r_inner"], I.PHYS_SHELL["r_outer"]
    exact = 4.0 * math.pi / 3.0 * (top**3 - a**3)
    errs = []
    for N in (2, 3, 4, 5):
        m = orc.Mesh(I.shell(2, 1, N))
        assert m.Ng == (6 * (2 * N) ** 2 + 2) * (N + 1)
        xyz = m.coords()
        r = np.sqrt((xyz**2).sum(axis=0))
        assert r.min() > a - 1e-6 and r.max() < top + 1e-6
        errs.append(abs(m.jw().sum() / exact - 1.0))
    assert errs[-1] < 1e-6
    assert errs[-1] < errs[0] * 1e-2
    m = orc.Mesh(I.shell(3, 2, 3))
    assert m.Ng == (6 * 9 * 9 + 2) * (2 * 3 + 1)
    w = m.wall()
    assert np.count_nonzero(w & 8) == 2 * (6 * 9 * 9 + 2)


def _brute_force_ids(exyz, gxyz, period=None):
    """Global id of each element node by nearest coordinate search."""
    ids = np.empty(exyz.shape[1], dtype=np.int64)
    for n in range(exyz.shape[1]):
        d = gxyz - exyz[:, n : n + 1]
        if period is not None:
            for a in range(3):
                if period[a]:
                    d[a] -= period[a] * np.round(d[a] / period[a])
        ids[n] = np.argmin((d**2).sum(axis=0))
        assert (d[:, ids[n]] ** 2).sum() < 1e-12
    return ids


@pytest.mark.parametrize(
    "cfg",
    [
        I.box(2, 2),
        I.box((2, 1, 3), 3, L=(700.0, 300.0, 900.0)),
        I.box(2, 2, periodic=(1, 0, 1)),
        I.box(2, 3, warp=0.05),
        I.shell(1, 1, 2),
        I.shell(2, 2, 2),
    ],
)
def test_assembly_equals_brute_force(orc, cfg):
    """Direct stiffness summation (Eq. 4, DSS) of the element residuals equals
    a per-node sum found by coordinate search, followed by the mass and wall
    conditions."""
    m = orc.Mesh(cfg)
    period = None
    if cfg["kind"] == "box" and any(cfg["periodic"]):
        period = [cfg["L"][a] if cfg["periodic"][a] else 0.0 for a in range(3)]
    ids = _brute_force_ids(m.elem_coords(), m.coords(), period)
    np.testing.assert_array_equal(ids, m.l2g())
    q = I.random_perturbation(m.Ng, seed=7)
    rho0 = m.ref()[0]
    q[0] *= rho0 / rho0.max()
    re = m.rhs_elem(q)
    jw = m.jw()
    R = np.zeros((5, m.Ng))
    M = np.zeros(m.Ng)
    for n in range(m.Nl):
        R[:, ids[n]] += re[:, n]
        M[ids[n]] += jw[n]
    np.testing.assert_allclose(M, m.mass(), rtol=1e-14)
    R /= M
    wall = m.wall()
    xyz = m.coords()
    for g in range(m.Ng):
        for a in range(3):
            if wall[g] & (1 << a):
                R[1 + a, g] = 0.0
        if wall[g] & 8:
            rh = xyz[:, g] / np.linalg.norm(xyz[:, g])
            R[1:4, g] -= (R[1:4, g] @ rh) * rh
    Ro = m.rhs(q)
    scale = np.abs(Ro).max(axis=1, keepdims=True)
    assert np.abs(R - Ro).max() <= 1e-13 * scale.max()
    for v in range(5):
        assert np.abs(R[v] - Ro[v]).max() <= 1e-13 * scale[v, 0]


def _equator_longitudes(orc, npanel, N):
    """Distinct longitudes of the nodes on the equator (z = 0) of a shell
    with an even number of columns per panel edge, sorted, in [-pi, pi)."""
    m = orc.Mesh(I.shell(npanel, 1, N))
    xyz = m.coords()
    r = np.sqrt((xyz**2).sum(axis=0))
    eq = np.abs(xyz[2]) < 1e-9 * r
    lon = np.unique(np.round(np.arctan2(xyz[1][eq], xyz[0][eq]), 12))
    return lon


@pytest.mark.parametrize("npanel,N", [(2, 4), (4, 3)])
def test_shell_is_equiangular(orc, npanel, N):
    """Equiangular cubed sphere (Sec. 4): along a panel's central great
    circle the element boundaries are equally spaced in angle, 90 degrees
    per panel split into npanel elements, and inside each element the nodes
    sit at the Lobatto points of the angle (not of the tangent)."""
    lon = _equator_longitudes(orc, npanel, N)
    assert lon.size == 4 * npanel * N  # every equator node, once
    d = 0.5 * np.pi / npanel
    xi, _ = orc.lgl(N)
    pos = (lon + np.pi) / d  # element widths from longitude -180
    frac = np.unique(np.round(pos % 1.0, 9) % 1.0)
    np.testing.assert_allclose(frac, np.sort((xi[:-1] + 1.0) / 2.0), atol=1e-9)
    corners = np.sort(lon[np.abs(pos - np.round(pos)) < 1e-9])
    assert corners.size == 4 * npanel
    np.testing.assert_allclose(np.diff(corners), d, atol=1e-11)

