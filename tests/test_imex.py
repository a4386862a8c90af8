"""The 1D-IMEX leapfrog (Sec. 2.2: an explicit leapfrog step, then implicit
corrections along the vertical columns) through the C ABI.

CPU: which configurations the scheme accepts, and its parameter checks.
GPU: parity with the oracle (oracle/imex.py) for the start step and
filtered leapfrog runs past the explicit limit, single steps against graph
replay, and the restart after a new state."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .helpers import rel_errors, state_floors

THIN = I.box((3, 2, 4), 3, L=(4000.0, 3000.0, 1000.0))
THIN_BUBBLE = (0.5, 900.0, 2000.0, 1500.0, 350.0)


@pytest.fixture(scope="module")
def lib():
    from paper_1511_01561_gb300 import numa as mod
    return mod


def _scheme_rc(lib, cfg, precision="fp64"):
    ctx = lib.numa_create(cfg, precision)
    try:
        rc = lib.lib.numa_set_time_scheme(ctx, 2)
        return rc, lib.numa_last_error(ctx)
    finally:
        lib.numa_destroy(ctx)


def _thin_shell(N, lid=12e3, npanel=2, nlayer=3):
    cfg = I.shell(npanel, nlayer, N)
    cfg["r_outer"] = cfg["r_inner"] + lid
    return cfg


def test_imex_accepts_walled_unwarped_fp64_boxes_and_shells(lib):
    for cfg in (THIN, I.box((2, 2, 3), 4, periodic=(1, 1, 0)), I.box(1, 1), I.shell(2, 1, 3), _thin_shell(4)):
        assert _scheme_rc(lib, cfg)[0] == 0
        assert _scheme_rc(lib, cfg, "fp64_pairs")[0] == 0


@pytest.mark.parametrize("cfg,precision,word", [
    (I.box(2, 3, periodic=(0, 0, 1)), "fp64", "bottom and top"),
    (I.box(2, 3, warp=0.05), "fp64", "warp"),
    (I.box(2, 3), "fp32_mixed", "FP64"),
    (dict(I.box(2, 3), storage="dg"), "fp64", "CG storage"),
], ids=["periodic_z", "warped", "fp32", "dg"])
def test_imex_refuses(lib, cfg, precision, word):
    rc, msg = _scheme_rc(lib, cfg, precision)
    assert rc == -1 and word in msg


def test_robert_asselin_range(lib):
    ctx = lib.numa_create(THIN)
    try:
        lib.numa_set_robert_asselin(ctx, 0.0)
        lib.numa_set_robert_asselin(ctx, 0.2)
        for bad in (-0.01, 0.5, float("nan")):
            with pytest.raises(lib.NumaError) as e:
                lib.numa_set_robert_asselin(ctx, bad)
            assert e.value.code == -1
    finally:
        lib.numa_destroy(ctx)


def test_imex_tables_in_the_workspace(lib):
    """Walled boxes reserve the column tables; the same node count periodic in z does not."""
    a = lib.numa_create(I.box((2, 2, 4), 2))
    b = lib.numa_create(I.box((2, 2, 4), 2, periodic=(0, 0, 1)))
    try:
        ia, ib = lib.numa_get_mesh_info(a), lib.numa_get_mesh_info(b)
        nz = 4 * 2 + 1
        tables = 8 * (nz * 5 + 2 * nz + 2 * (nz * 4 + nz * 9)) + 4 * 2 * nz
        assert ia["Ng"] > ib["Ng"]
        assert ia["workspace_bytes"] >= tables
    finally:
        lib.numa_destroy(a)
        lib.numa_destroy(b)


# ---- GPU ---------------------------------------------------------------------

@pytest.fixture(scope="module")
def numa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_01561_gb300 import build
    build.build()
    from paper_1511_01561_gb300 import numa as mod
    return mod


CASES = [
    ("thin_N3", THIN, ("bubble", THIN_BUBBLE), 0.4),
    ("periodic_xy_isothermal_N4",
     I.box((2, 2, 3), 4, L=(3000.0, 3000.0, 1500.0), periodic=(1, 1, 0), ref="isothermal", T0=250.0),
     ("bubble", (0.5, 800.0, 1500.0, 1500.0, 600.0)), 0.3),
    ("tall_N2", I.box((2, 1, 5), 2, L=(2000.0, 1000.0, 1000.0)), ("bubble", (0.5, 500.0, 1000.0, 500.0, 400.0)), 0.2),
    ("N1", I.box((3, 3, 6), 1, L=(3000.0, 3000.0, 600.0)), ("bubble", (0.5, 900.0, 1500.0, 1500.0, 300.0)), 0.2),
    ("N8", I.box((1, 1, 2), 8, L=(2000.0, 2000.0, 1000.0)), ("bubble", (0.5, 700.0, 1000.0, 1000.0, 400.0)), 0.05),
]


SHELL_CASES = [
    ("thin_shell_N4", _thin_shell(4), 20.0),
    ("thin_shell_N3_4layers", _thin_shell(3, lid=16e3, nlayer=4), 10.0),
    ("shell_N2_isentropic_deep", dict(I.shell(3, 2, 2), ref="isentropic", theta0=300.0, r_outer=6371e3 + 20e3), 5.0),
]


def _gpu_run(numa, cfg, ic, dt, nsteps, nu, single=False, precision="fp64"):
    sv = numa.Solver(cfg, precision)
    try:
        sv.set_time_scheme("imex")
        sv.set_robert_asselin(nu)
        sv.init_state(*ic)
        if single:
            for _ in range(nsteps):
                sv.rk_step(dt)
        else:
            sv.run(dt, nsteps)
        return sv.get_state().numpy().copy()
    finally:
        sv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("nsteps,nu", [(1, 0.1), (2, 0.1), (12, 0.1), (12, 0.0)])
@pytest.mark.parametrize("name,cfg,ic,dt", CASES, ids=[c[0] for c in CASES])
def test_imex_parity(numa, orc, name, cfg, ic, dt, nsteps, nu):
    from oracle import imex

    m = orc.Mesh(cfg)
    q0 = m.init_state(*ic)
    ref, _ = imex.run_imex(m, q0, dt, nsteps, nu)
    got = _gpu_run(numa, cfg, ic, dt, nsteps, nu)
    err = rel_errors(got, ref, state_floors(ref, m.ref()[0].max()))
    assert err.max() <= 1e-10, err
    assert np.abs(ref[3]).max() > 0  # the bubble moved


@pytest.mark.gpu
@pytest.mark.parametrize("name,cfg,ic,dt", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_imex_parity_pairs(numa, orc, name, cfg, ic, dt):
    """The pairs mode's element kernel (FP64-level error) under the same scheme."""
    from oracle import imex

    m = orc.Mesh(cfg)
    q0 = m.init_state(*ic)
    ref, _ = imex.run_imex(m, q0, dt, 12, 0.1)
    got = _gpu_run(numa, cfg, ic, dt, 12, 0.1, precision="fp64_pairs")
    err = rel_errors(got, ref, state_floors(ref, m.ref()[0].max()))
    assert err.max() <= 1e-10, err


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs"])
@pytest.mark.parametrize("nsteps,nu", [(1, 0.1), (2, 0.1), (10, 0.1), (10, 0.0)])
@pytest.mark.parametrize("name,cfg,dt", SHELL_CASES, ids=[c[0] for c in SHELL_CASES])
def test_imex_parity_shell(numa, orc, name, cfg, dt, nsteps, nu, precision):
    """Radial columns of the cubed-sphere shell, past the explicit limit; the
    oracle's node order differs, so states are matched by coordinates."""
    from oracle import imex

    from .helpers import match_nodes

    m = orc.Mesh(cfg)
    ic = ("jetwave", I.JETWAVE_PARAMS)
    q0 = m.init_state(*ic)
    ref, _ = imex.run_imex(m, q0, dt, nsteps, nu)
    sv = numa.Solver(cfg, precision)
    try:
        perm = match_nodes(sv.coords(), m.coords(), tol=1e-3)
        sv.set_time_scheme("imex")
        sv.set_robert_asselin(nu)
        sv.set_state(np.ascontiguousarray(q0[:, perm]))
        sv.run(dt, nsteps)
        got = sv.get_state().numpy().copy()
    finally:
        sv.close()
    ref = ref[:, perm]
    err = rel_errors(got, ref, state_floors(ref, m.ref()[0].max()))
    # the pairs mode's stated bar on curved elements: 2^(53-48) = 32 times
    # the FP64 bar (48-bit pair arithmetic; tests/test_gpu_parity.py)
    tol = 1e-10 * (32.0 if precision == "fp64_pairs" else 1.0)
    assert err.max() <= tol, err


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs"])
def test_imex_with_the_filter(numa, orc, precision):
    """The Boyd-Vandeven filter after every second step, after the IMEX
    correction as in the time loop of Sec. 7."""
    from oracle import imex

    cfg, ic, dt = THIN, ("bubble", THIN_BUBBLE), 0.4
    m = orc.Mesh(cfg)
    q0 = m.init_state(*ic)
    ref, _ = imex.run_imex_filtered(m, q0, dt, 9, 0.1, 2, 2, 12.0, 0.5)
    assert not np.allclose(ref, imex.run_imex(m, q0, dt, 9, 0.1)[0], rtol=0, atol=1e-9)
    sv = numa.Solver(cfg, precision)
    try:
        sv.set_time_scheme("imex")
        sv.set_robert_asselin(0.1)
        sv.set_filter(2, 2, 12.0, 0.5)
        sv.init_state(*ic)
        sv.run(dt, 9)
        got = sv.get_state().numpy().copy()
    finally:
        sv.close()
    err = rel_errors(got, ref, state_floors(ref, m.ref()[0].max()))
    assert err.max() <= 1e-10, err


@pytest.mark.gpu
def test_imex_graph_equals_single_steps_and_restarts(numa):
    cfg, ic, dt = THIN, ("bubble", THIN_BUBBLE), 0.4
    a = _gpu_run(numa, cfg, ic, dt, 9, 0.1)
    b = _gpu_run(numa, cfg, ic, dt, 9, 0.1, single=True)
    assert np.array_equal(a, b)
    sv = numa.Solver(cfg, "fp64")
    try:
        sv.set_time_scheme("imex")
        sv.set_robert_asselin(0.1)
        sv.init_state(*ic)
        sv.run(dt, 4)
        sv.init_state(*ic)  # a new state: the next step is a start step again
        sv.run(dt, 5)
        sv.run(dt, 4)  # continuing needs no restart
        c = sv.get_state().numpy().copy()
    finally:
        sv.close()
    assert np.array_equal(a, c)


@pytest.mark.gpu
def test_imex_time_kernels(numa):
    sv = numa.Solver(THIN, "fp64")
    try:
        sv.set_time_scheme("imex")
        sv.init_state("bubble", THIN_BUBBLE)
        vol, upd = sv.time_kernels(0.4, 3)
        assert vol > 0 and upd > 0
        assert sv.check_finite() == 0
    finally:
        sv.close()


@pytest.mark.gpu
def test_imex_tall_columns(numa, orc):
    """145 levels per column: fewer columns per CTA (16), so half a warp runs
    the banded sweeps; still the oracle's result."""
    from oracle import imex

    cfg = I.box((2, 2, 36), 4, L=(2000.0, 2000.0, 3600.0))
    ic = ("bubble", (0.5, 900.0, 1000.0, 1000.0, 1500.0))
    m = orc.Mesh(cfg)
    ref, _ = imex.run_imex(m, m.init_state(*ic), 0.05, 3, 0.1)
    got = _gpu_run(numa, cfg, ic, 0.05, 3, 0.1)
    err = rel_errors(got, ref, state_floors(ref, m.ref()[0].max()))
    assert err.max() <= 1e-10, err


@pytest.mark.gpu
def test_imex_reports_a_non_finite_state(numa):
    sv = numa.Solver(THIN, "fp64")
    try:
        sv.set_time_scheme("imex")
        sv.init_state("bubble", THIN_BUBBLE)
        q = sv.get_state().numpy().copy()
        q[4, 17] = np.nan
        sv.set_state(q)
        with pytest.raises(numa.NumaError) as e:
            sv.run(0.4, 2)
        assert e.value.code == -4
    finally:
        sv.close()
