"""GPU parity of the CUDA hot path against the FP64 oracle, through the C ABI.

Bars, relative error per variable in L2 and in Linf over global nodes (with
the floors of tests/helpers.py):
- FP64: 1e-12 for one right-hand side and 1e-10 after 100 steps; bitwise
  determinism.
- FP64-pairs (48-bit significands, 2^-48 against FP64's 2^-53): the FP64 bars
  on affine elements.  On curved elements (warped boxes, shells) the metric
  terms and the chain-rule products are rounded at 2^-48 of terms that cancel
  in the divergence, so its bars there are 2^5 = 32 times the FP64 bars:
  3.2e-11 and 3.2e-9.  It is FP64-equivalent on affine meshes only.
- FP32-mixed: 2e-5 in L2 and 1e-4 in Linf for one right-hand side; 1e-4 in
  L2 and 5e-4 in Linf after 100 steps.  FP32 rounds at 2^-24 = 6e-8; a
  derivative sums about 2(N+1) products of fluxes and D entries whose row
  sums reach 10 at N=4, and the chain rule adds three directions of such
  terms, which puts the per-node error near 1e-5 of the flux-divergence
  scale; the Linf bar is 5 times the L2 bar, the usual spread between a mean
  and the largest node of such errors."""
import zlib

import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .helpers import match_nodes, rel_errors, rhs_floors, scaled_random_state, state_floors

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-12
TOL_100 = 1e-10
PAIRS_CURVED = 32.0  # 2^(53-48): the pairs mode's bars on curved elements, relative to FP64's


def _curved(cfg) -> bool:
    return cfg["kind"] == "shell" or float(cfg.get("warp", 0.0)) != 0.0


def _bar(precision, cfg, tol):
    """FP64 bar `tol`, scaled for the pairs mode on curved elements."""
    return tol * PAIRS_CURVED if precision == "fp64_pairs" and _curved(cfg) else tol


@pytest.fixture(scope="module")
def numa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_01561_gb300 import build
    build.build()
    from paper_1511_01561_gb300 import numa as mod
    return mod


def _dx_min(cfg, orc_mesh):
    xyz = orc_mesh.coords()
    if cfg["kind"] == "box":
        return min(cfg["L"][a] / cfg["ne"][a] for a in range(3)) * 0.5 * (1 - np.cos(np.pi / cfg["N"]))
    return (cfg["r_outer"] - cfg["r_inner"]) / cfg["nlayer"] * 0.1


def _gpu_rhs(numa, cfg, q, precision="fp64"):
    """RHS through the C ABI, twice (the two results must agree bit for bit)."""
    s = numa.Solver(cfg, precision)
    try:
        R = s.rhs(q).cpu().numpy()
        R2 = s.rhs(q).cpu().numpy()
        assert np.array_equal(R, R2), "RHS not bitwise deterministic"
        return R, s.coords()
    finally:
        s.close()


BOX_CASES = [
    ("bubble_4x4x4_N4+pert", I.box(4, 4), "bubble+smooth"),
    ("walls_ragged_3x2x5_N3", I.box((3, 2, 5), 3, L=(900.0, 500.0, 1200.0)), "random"),
    ("periodic_2x2x2_N6", I.box(2, 6, periodic=(1, 1, 1)), "smooth"),
    ("warped_2x3x2_N4", I.box((2, 3, 2), 4, warp=0.05), "random"),
    ("warped_smooth_3x3x3_N5", I.box(3, 5, warp=0.04, periodic=(0, 1, 0)), "smooth"),
    ("N1_3x2x2", I.box((3, 2, 2), 1), "random"),
    ("N2_2x2x3", I.box((2, 2, 3), 2), "smooth"),
    ("N7_1x2x1", I.box((1, 2, 1), 7), "random"),
    ("N8_2x1x1", I.box((2, 1, 1), 8), "smooth"),
    ("single_element_N4", I.box(1, 4), "random"),
    ("single_element_periodic_N3", I.box(1, 3, periodic=(1, 1, 1)), "random"),
    ("isothermal_2x2x2_N4", I.box(2, 4, ref="isothermal", T0=250.0), "smooth"),
]


def _state(m, cfg, kind, seed):
    rho0, th0, _ = m.ref()
    xyz = m.coords()
    if kind == "random":
        return scaled_random_state(m.Ng, rho0, th0, seed)
    L = 700.0 if cfg["kind"] == "box" else 2.0e6
    q = I.smooth_perturbation(xyz, seed, L, rho=1.0, U=1.0, Theta=1.0)
    q[0] *= 0.01 * rho0
    q[1:4] *= 5.0 * rho0
    q[4] *= 0.01 * th0
    if kind == "bubble+smooth":
        q = 0.1 * q + m.init_state("bubble", I.BUBBLE_PARAMS)
    return q


FP64_MODES = ["fp64", "fp64_pairs"]  # the FP64 bars (pairs: 32x on curved elements, see _bar)


@pytest.mark.parametrize("precision", FP64_MODES)
@pytest.mark.parametrize("name,cfg,kind", BOX_CASES, ids=[c[0] for c in BOX_CASES])
def test_rhs_parity_box(numa, orc, name, cfg, kind, precision):
    m = orc.Mesh(cfg)
    q = _state(m, cfg, kind, seed=zlib.crc32(name.encode()) % 1000)
    Ro = m.rhs(q)
    Rg, xyz = _gpu_rhs(numa, cfg, q, precision)
    assert np.abs(xyz - m.coords()).max() < 1e-9
    err = rel_errors(Rg, Ro, rhs_floors(Ro, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    assert err.max() <= _bar(precision, cfg, TOL_RHS), err


# Boxes without warp take the affine-element (contravariant flux) kernel by
# default; the per-node form of Eq. 5 is held to the same bars on them.
NODAL_CASES = [c for c in BOX_CASES if c[1].get("warp", 0.0) == 0.0]


@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs", "fp32_mixed"])
@pytest.mark.parametrize("name,cfg,kind", NODAL_CASES, ids=[c[0] for c in NODAL_CASES])
def test_rhs_parity_box_nodal_form(numa, orc, name, cfg, kind, precision):
    m = orc.Mesh(cfg)
    q = _state(m, cfg, kind, seed=zlib.crc32(name.encode()) % 1000)
    Ro = m.rhs(q)
    Rg, _ = _gpu_rhs(numa, dict(cfg, metric_form="nodal"), q, precision)
    err = rel_errors(Rg, Ro, rhs_floors(Ro, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    if precision in FP64_MODES:
        assert err.max() <= TOL_RHS, err
    else:
        _fp32_rhs_ok(err)


@pytest.mark.parametrize("precision", FP64_MODES)
@pytest.mark.parametrize("cfg", [I.shell(2, 2, 4), I.shell(3, 1, 3), I.shell(1, 2, 6, Omega=0.0)])
def test_rhs_parity_shell(numa, orc, cfg, precision):
    m = orc.Mesh(cfg)
    q = _state(m, cfg, "smooth", seed=5) + 0.1 * _state(m, cfg, "random", seed=6)
    Ro = m.rhs(q)
    s = numa.Solver(cfg, precision)
    try:
        perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
        Rg = s.rhs(np.ascontiguousarray(q[:, perm])).cpu().numpy()
    finally:
        s.close()
    Rref = Ro[:, perm]
    err = rel_errors(Rg, Rref, rhs_floors(Rref, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    assert err.max() <= _bar(precision, cfg, TOL_RHS), err


def test_init_state_parity(numa, orc):
    cfg = I.box(4, 4)
    m = orc.Mesh(cfg)
    s = numa.Solver(cfg)
    try:
        s.init_state("bubble", I.BUBBLE_PARAMS)
        qg = s.get_state().numpy()
        s.init_state("uniform", (3.0, -1.0, 0.5))
        qu = s.get_state().numpy()
    finally:
        s.close()
    qo = m.init_state("bubble", I.BUBBLE_PARAMS)
    assert np.abs(qg - qo).max() <= 1e-15 + 1e-13 * np.abs(qo).max()
    qo = m.init_state("uniform", (3.0, -1.0, 0.5))
    assert np.abs(qu - qo).max() <= 1e-13 * np.abs(qo).max()
    cfg = I.shell(2, 2, 3)
    m = orc.Mesh(cfg)
    s = numa.Solver(cfg)
    try:
        s.init_state("jetwave", I.JETWAVE_PARAMS)
        qg = s.get_state().numpy()
        perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
    finally:
        s.close()
    qo = m.init_state("jetwave", I.JETWAVE_PARAMS)[:, perm]
    assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()


@pytest.mark.parametrize("precision,form", [("fp64", "auto"), ("fp64_pairs", "auto"), ("fp64", "nodal"),
                                            ("fp64_pairs", "nodal")])
def test_rk3_100_steps_bubble(numa, orc, precision, form):
    """Workload bubble_4x4x4_N4: 100 SSP-RK3 steps at dt = 0.01 s."""
    w = I.WORKLOADS["bubble_4x4x4_N4"]
    cfg = dict(w["cfg"], metric_form=form)
    m = orc.Mesh(w["cfg"])
    q0 = m.init_state(*w["ic"])
    qo = m.run(q0, w["dt"], w["steps"])
    s = numa.Solver(cfg, precision)
    try:
        s.set_state(q0)
        s.run(w["dt"], w["steps"])
        qg = s.get_state().numpy()
        # the graph-replayed loop equals plain stage launches bit for bit
        s.set_state(q0)
        for _ in range(w["steps"]):
            s.rk_step(w["dt"])
        qg2 = s.get_state().numpy()
    finally:
        s.close()
    assert np.array_equal(qg, qg2)
    err = rel_errors(qg, qo, state_floors(qo, m.ref()[0].max()))
    assert err.max() <= TOL_100, err
    assert np.abs(qo[3]).max() > 1e-4  # the bubble has started to rise


@pytest.mark.parametrize("precision", FP64_MODES)
def test_rk3_steps_shell_and_warped(numa, orc, precision):
    for cfg, dt, steps in ((I.shell(2, 2, 3), 2.0, 20), (I.box(2, 4, warp=0.05), 0.01, 30)):
        m = orc.Mesh(cfg)
        q0 = 0.3 * _state(m, cfg, "smooth", seed=9)
        if cfg["kind"] == "shell":
            q0 = q0 + m.init_state("jetwave", I.JETWAVE_PARAMS)
            rhat = m.coords() / np.linalg.norm(m.coords(), axis=0)
            walls = (m.wall() & 8) != 0
            q0[1:4, walls] -= (q0[1:4, walls] * rhat[:, walls]).sum(0) * rhat[:, walls]
        qo = m.run(q0, dt, steps)
        s = numa.Solver(cfg, precision)
        try:
            perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
            s.set_state(np.ascontiguousarray(q0[:, perm]))
            s.run(dt, steps)
            qg = s.get_state().numpy()
        finally:
            s.close()
        qr = qo[:, perm]
        err = rel_errors(qg, qr, state_floors(qr, m.ref()[0].max()))
        assert err.max() <= _bar(precision, cfg, TOL_100), (cfg["kind"], err)


def test_full_size_bubble_rhs(numa, orc):
    """Workload bubble_32x32x32_N4 at full size: all 2.15M global nodes."""
    cfg = I.WORKLOADS["bubble_32x32x32_N4"]["cfg"]
    m = orc.Mesh(cfg)
    q = m.init_state("bubble", I.BUBBLE_PARAMS) + 0.1 * _state(m, cfg, "smooth", seed=21)
    Ro = m.rhs(q)
    floors = rhs_floors(Ro, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max())
    for precision, form in (("fp64", "auto"), ("fp64_pairs", "auto"), ("fp64", "nodal"), ("fp64_pairs", "nodal")):
        Rg, _ = _gpu_rhs(numa, dict(cfg, metric_form=form), q, precision)
        err = rel_errors(Rg, Ro, floors)
        print(f"full-size RHS {precision} {form}: max rel L2 {err[:, 0].max():.3e}, Linf {err[:, 1].max():.3e}")
        assert err.max() <= TOL_RHS, (precision, form, err)


def test_nonfinite_flag_and_errors(numa):
    cfg = I.box(2, 3)
    s = numa.Solver(cfg)
    try:
        s.init_state("bubble", I.BUBBLE_PARAMS)
        q0 = s.get_state().numpy().copy()
        s.run(0.01, 0)
        assert np.array_equal(s.get_state().numpy(), q0)
        bad = q0.copy()
        bad[0, 7] = np.nan
        s.set_state(bad)
        with pytest.raises(numa.NumaError) as e:
            s.run(0.01, 1)
        assert e.value.code == -4
        assert s.check_finite() == 0  # flag was reset
        s.set_state(q0)
        s.run(0.01, 2)
        assert np.isfinite(s.get_state().numpy()).all()
        with pytest.raises(numa.NumaError) as e:
            s.run(0.01, -1)
        assert e.value.code == -1
    finally:
        s.close()


# ----------------------------------------------------- FP32 mixed form ----

TOL_FP32_RHS = 2e-5
TOL_FP32_RHS_INF = 1e-4
TOL_FP32_100 = 1e-4
TOL_FP32_100_INF = 5e-4


def _fp32_rhs_ok(err):
    assert err[:, 0].max() <= TOL_FP32_RHS and err[:, 1].max() <= TOL_FP32_RHS_INF, err


def _fp32_100_ok(err):
    assert err[:, 0].max() <= TOL_FP32_100 and err[:, 1].max() <= TOL_FP32_100_INF, err


@pytest.mark.parametrize("name,cfg,kind", BOX_CASES, ids=[c[0] for c in BOX_CASES])
def test_fp32_mixed_rhs_error(numa, orc, name, cfg, kind):
    m = orc.Mesh(cfg)
    q = _state(m, cfg, kind, seed=31)
    Ro = m.rhs(q)
    Rg, _ = _gpu_rhs(numa, cfg, q, "fp32_mixed")
    err = rel_errors(Rg, Ro, rhs_floors(Ro, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    _fp32_rhs_ok(err)


@pytest.mark.parametrize("cfg", [I.shell(2, 2, 4), I.shell(1, 2, 6, Omega=0.0)])
def test_fp32_mixed_rhs_error_shell(numa, orc, cfg):
    m = orc.Mesh(cfg)
    q = _state(m, cfg, "smooth", seed=5) + 0.1 * _state(m, cfg, "random", seed=6)
    Ro = m.rhs(q)
    s = numa.Solver(cfg, "fp32_mixed")
    try:
        perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
        Rg = s.rhs(np.ascontiguousarray(q[:, perm])).cpu().numpy()
    finally:
        s.close()
    Rref = Ro[:, perm]
    err = rel_errors(Rg, Rref, rhs_floors(Rref, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    _fp32_rhs_ok(err)


def test_fp32_mixed_100_steps(numa, orc):
    w = I.WORKLOADS["bubble_4x4x4_N4"]
    m = orc.Mesh(w["cfg"])
    q0 = m.init_state(*w["ic"])
    qo = m.run(q0, w["dt"], w["steps"])
    s = numa.Solver(w["cfg"], "fp32_mixed")
    try:
        s.set_state(q0)
        s.run(w["dt"], w["steps"])
        qg = s.get_state().numpy()
    finally:
        s.close()
    err = rel_errors(qg, qo, state_floors(qo, m.ref()[0].max()))
    _fp32_100_ok(err)


# ------------------------------------ five-stage low-storage integrator ----

@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs", "fp32_mixed"])
def test_lsrk54_100_steps_bubble(numa, orc, precision):
    """100 steps of the five-stage low-storage RK on bubble_4x4x4_N4."""
    w = I.WORKLOADS["bubble_4x4x4_N4"]
    m = orc.Mesh(w["cfg"])
    q0 = m.init_state(*w["ic"])
    qo = m.run_lsrk54(q0, w["dt"], w["steps"])
    s = numa.Solver(w["cfg"], precision)
    try:
        s.set_time_scheme("ls54")
        s.set_state(q0)
        s.run(w["dt"], w["steps"])
        qg = s.get_state().numpy().copy()
        s.set_state(q0)
        for _ in range(w["steps"]):
            s.rk_step(w["dt"])
        qg2 = s.get_state().numpy()
    finally:
        s.close()
    assert np.array_equal(qg, qg2)
    err = rel_errors(qg, qo, state_floors(qo, m.ref()[0].max()))
    if precision in FP64_MODES:
        assert err.max() <= TOL_100, err
    else:
        _fp32_100_ok(err)
    # a different integrator: the SSP-RK3 result differs by more than the bar
    assert np.abs(qo - m.run(q0, w["dt"], w["steps"])).max() > 0.0


def test_lsrk54_shell(numa, orc):
    cfg, dt, steps = I.shell(2, 2, 3), 2.0, 12
    m = orc.Mesh(cfg)
    q0 = 0.3 * _state(m, cfg, "smooth", seed=9) + m.init_state("jetwave", I.JETWAVE_PARAMS)
    rhat = m.coords() / np.linalg.norm(m.coords(), axis=0)
    walls = (m.wall() & 8) != 0
    q0[1:4, walls] -= (q0[1:4, walls] * rhat[:, walls]).sum(0) * rhat[:, walls]
    qo = m.run_lsrk54(q0, dt, steps)
    s = numa.Solver(cfg, "fp64")
    try:
        perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
        s.set_time_scheme("ls54")
        s.set_state(np.ascontiguousarray(q0[:, perm]))
        s.run(dt, steps)
        qg = s.get_state().numpy()
    finally:
        s.close()
    qr = qo[:, perm]
    err = rel_errors(qg, qr, state_floors(qr, m.ref()[0].max()))
    assert err.max() <= TOL_100, err


def test_full_size_shell_rhs(numa, orc):
    """Workload shell_6x30x30x8_N4 at full size: 43,200 curved elements,
    2.85M global nodes, every output compared."""
    w = I.WORKLOADS["shell_6x30x30x8_N4"]
    cfg = w["cfg"]
    m = orc.Mesh(cfg)
    q = m.init_state(*w["ic"]) + 0.05 * _state(m, cfg, "smooth", seed=23)
    rhat = m.coords() / np.linalg.norm(m.coords(), axis=0)
    walls = (m.wall() & 8) != 0
    q[1:4, walls] -= (q[1:4, walls] * rhat[:, walls]).sum(0) * rhat[:, walls]
    Ro = m.rhs(q)
    perm = None
    for precision in ("fp64", "fp64_pairs", "fp32_mixed"):
        s = numa.Solver(cfg, precision)
        try:
            if perm is None:
                perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
            Rg = s.rhs(np.ascontiguousarray(q[:, perm])).cpu().numpy()
        finally:
            s.close()
        Rref = Ro[:, perm]
        err = rel_errors(Rg, Rref, rhs_floors(Rref, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
        print(f"full-size shell RHS {precision}: max rel L2 {err[:, 0].max():.3e}, Linf {err[:, 1].max():.3e}")
        if precision == "fp32_mixed":
            _fp32_rhs_ok(err)
        else:
            assert err.max() <= _bar(precision, cfg, TOL_RHS), (precision, err)


@pytest.mark.slow
def test_largest_serving_member_rhs(numa, orc):
    """The largest request of the serving workload, a 48^3-element box at N=6
    (24.1M global nodes, 37.9M element nodes): the full FP64 RHS against the
    oracle, which exercises the index arithmetic at the largest size served."""
    cfg = I.box(48, 6)
    m = orc.Mesh(cfg)
    assert m.Ng == 289**3
    q = m.init_state("bubble", (1.5, 200.0, 450.0, 550.0, 400.0))
    q += 0.05 * scaled_random_state(m.Ng, *m.ref()[:2], seed=48)
    Ro = m.rhs(q)
    Rg, _ = _gpu_rhs(numa, cfg, q, "fp64")
    err = rel_errors(Rg, Ro, rhs_floors(Ro, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    print(f"48^3 N=6 RHS fp64: max rel L2 {err[:, 0].max():.3e}, Linf {err[:, 1].max():.3e}")
    assert err.max() <= TOL_RHS, err


@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs", "fp32_mixed"])
def test_rhs_parity_large_theta_perturbation(numa, orc, precision):
    """Theta' up to 5% of (rho theta)_0: the equation of state leaves the
    binomial series (|x| > 2^-5) for expm1(gamma log1p(x)) at many nodes."""
    cfg = I.box((3, 2, 2), 4)
    m = orc.Mesh(cfg)
    rho0, th0, _ = m.ref()
    q = scaled_random_state(m.Ng, rho0, th0, seed=55, rel=0.05)
    assert (np.abs(q[4] / th0) > 2.0**-5).mean() > 0.2
    Ro = m.rhs(q)
    Rg, _ = _gpu_rhs(numa, cfg, q, precision)
    err = rel_errors(Rg, Ro, rhs_floors(Ro, m.ref()[0].max(), _dx_min(cfg, m), np.abs(q[1:4]).max()))
    if precision == "fp32_mixed":
        _fp32_rhs_ok(err)
    else:
        assert err.max() <= TOL_RHS, err
