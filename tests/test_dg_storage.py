"""DG storage of the node data (Sec. 6 compares CG, DG and CG/DG storage).

CPU part: the expanded mesh that numa_create builds for DG storage, checked
against the CG mesh through the host coordinates: one storage node per
element node, each a copy of a CG global node, every global node copied once
per element node at its point (the DSS multiplicity of Eq. 4's assembly).

GPU part: a run with DG storage equals the CG run at every copy, bit for bit
(the DSS sums the same element residuals in the same order), in every
precision, time scheme and with the filter, and the serving calls reject DG
storage."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

MESHES = [
    ("box_walls_N4", I.box((3, 2, 2), 4, L=(900.0, 600.0, 700.0))),
    ("box_periodic_N3", I.box(2, 3, periodic=(1, 1, 1))),
    ("box_warped_N5", I.box(2, 5, warp=0.05)),
    ("box_N1", I.box((3, 2, 2), 1)),
    ("shell_N4", I.shell(2, 1, 4)),
]


def _with(cfg, **kw):
    c = dict(cfg)
    c.update(kw)
    return c


@pytest.fixture(scope="module")
def lib():
    from paper_1511_01561_gb300 import numa as mod
    return mod


def copy_map(xyz_cg: np.ndarray, xyz_dg: np.ndarray) -> np.ndarray:
    """g[n]: the CG global node whose coordinates storage node n copies
    (exact equality: DG storage copies them)."""
    where = {tuple(p): g for g, p in enumerate(xyz_cg.T)}
    assert len(where) == xyz_cg.shape[1]  # distinct CG points
    return np.array([where[tuple(p)] for p in xyz_dg.T], dtype=np.int64)


def _coords(lib, cfg):
    h = lib.numa_create(cfg)
    try:
        return lib.numa_get_mesh_info(h), lib.numa_get_coords(h)
    finally:
        lib.numa_destroy(h)


@pytest.mark.parametrize("name,cfg", MESHES, ids=[m[0] for m in MESHES])
def test_dg_mesh_copies_cg_nodes(lib, orc, name, cfg):
    info_cg, x_cg = _coords(lib, cfg)
    info_dg, x_dg = _coords(lib, _with(cfg, storage="dg"))
    assert info_dg["Ng"] == info_dg["Nl"] == info_cg["Nl"]
    assert info_dg["Ne"] == info_cg["Ne"]
    assert info_dg["workspace_bytes"] > info_cg["workspace_bytes"]
    g = copy_map(x_cg, x_dg)
    # every global node is copied once per element node at its point: the
    # oracle's assembly multiplicity (element nodes per global node)
    m = orc.Mesh(cfg)
    l2g = m.l2g()
    mult = np.bincount(l2g, minlength=m.Ng)
    perm = np.arange(m.Ng) if cfg["kind"] == "box" else None
    if perm is None:
        from .helpers import match_nodes
        perm = match_nodes(x_cg, m.coords(), tol=1e-3)
    copies = np.bincount(g, minlength=info_cg["Ng"])
    assert np.array_equal(copies, mult[perm])
    assert info_cg["dss_entries"] == info_cg["Nl"]
    assert info_dg["dss_entries"] == int((mult.astype(np.int64) ** 2).sum())
    assert x_dg.shape[1] == info_dg["Ne"] * (cfg["N"] + 1) ** 3
    if cfg["kind"] == "box":
        # element order: storage node e*Np + k copies the global node of the
        # oracle's element node (e, k) (box elements are numbered alike; the
        # two compute coordinates with different rounding)
        assert np.abs(x_dg - m.coords()[:, l2g]).max() <= 1e-12 * np.abs(x_dg).max()


def test_storage_value_checked(lib):
    with pytest.raises(KeyError):
        lib.make_config(_with(I.box(2, 3), storage="cgdg"))
    c = lib.make_config(I.box(2, 3))
    c.storage = 2
    import ctypes

    h = ctypes.c_void_p()
    assert lib.lib.numa_create(ctypes.byref(c), ctypes.byref(h)) == -1


# ---- GPU: DG storage runs equal CG storage runs at every copy --------------

@pytest.fixture(scope="module")
def numa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_01561_gb300 import build
    build.build()
    from paper_1511_01561_gb300 import numa as mod
    return mod


def _start_state(orc, cfg, x_cg, seed):
    """A scaled random state in the library's CG node order."""
    from .helpers import match_nodes, scaled_random_state

    m = orc.Mesh(cfg)
    rho0, th0, _ = m.ref()
    q = scaled_random_state(m.Ng, rho0, th0, seed=seed, u=5.0)
    if cfg["kind"] == "shell":
        q = np.ascontiguousarray(q[:, match_nodes(x_cg, m.coords(), tol=1e-3)])
    return q


def _pair(numa, cfg, precision):
    cg = numa.Solver(cfg, precision)
    dg = numa.Solver(_with(cfg, storage="dg"), precision)
    return cg, dg, copy_map(cg.coords(), dg.coords())


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs", "fp32_mixed"])
@pytest.mark.parametrize("name,cfg", MESHES, ids=[m[0] for m in MESHES])
def test_dg_equals_cg(numa, orc, name, cfg, precision):
    cg, dg, g = _pair(numa, cfg, precision)
    try:
        q0 = _start_state(orc, cfg, cg.coords(), seed=len(name))
        Rc = cg.rhs(q0).cpu().numpy()
        Rd = dg.rhs(q0[:, g]).cpu().numpy()
        assert np.array_equal(Rd, Rc[:, g])
        cg.set_state(q0)
        dg.set_state(q0[:, g])
        cg.run(0.01, 5)
        dg.run(0.01, 5)
        qc = cg.get_state().numpy()
        qd = dg.get_state().numpy()
        assert np.array_equal(qd, qc[:, g])
        assert not np.array_equal(qc, q0)
    finally:
        cg.close()
        dg.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_dg_equals_cg_ls54_filtered(numa, precision):
    """Initial state from numa_init_state, five-stage RK and the filter."""
    cfg = I.box((3, 2, 2), 4, L=(900.0, 600.0, 700.0))
    cg, dg, g = _pair(numa, cfg, precision)
    try:
        for s in (cg, dg):
            s.init_state("bubble", I.BUBBLE_PARAMS)
        assert np.array_equal(dg.get_state().numpy(), cg.get_state().numpy()[:, g])
        for s in (cg, dg):
            s.set_time_scheme("ls54")
            s.set_filter(2, 3, 12.0, 0.5)
            s.run(0.01, 6)
        assert np.array_equal(dg.get_state().numpy(), cg.get_state().numpy()[:, g])
    finally:
        cg.close()
        dg.close()


@pytest.mark.gpu
def test_dg_against_oracle(numa, orc):
    """20 SSP-RK3 steps of the bubble with DG storage against the oracle's
    CG run, read at every copy."""
    from .helpers import rel_errors, state_floors

    cfg = I.box(4, 4)
    m = orc.Mesh(cfg)
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS)
    qo = m.run(q0, 0.01, 20)
    sv = numa.Solver(_with(cfg, storage="dg"), "fp64")
    try:
        l2g = m.l2g()  # box: the library's storage node n copies the oracle's global node l2g[n]
        sv.set_state(q0[:, l2g])
        sv.run(0.01, 20)
        qd = sv.get_state().numpy()
    finally:
        sv.close()
    err = rel_errors(qd, qo[:, l2g], state_floors(qo, m.ref()[0].max()))
    assert err.max() <= 1e-10, err


@pytest.mark.gpu
def test_serving_rejects_dg(numa):
    torch = pytest.importorskip("torch")
    sch = numa.Scheduler(64 << 20)
    try:
        with pytest.raises(numa.NumaError) as e:
            sch.submit(_with(I.box(2, 3), storage="dg"), "bubble", I.BUBBLE_PARAMS, nsteps=1)
        assert e.value.code == -1
    finally:
        sch.close()
        torch.cuda.synchronize()
