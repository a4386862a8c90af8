"""GPU parity of the Boyd-Vandeven filter (Sec. 2.3, applied with DSS and the
inverse mass matrix as in the time loop of Sec. 7) against the oracle,
through the C ABI: one application on walled, periodic, warped and shell
meshes in every precision, and a filtered SSP-RK3 run."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .helpers import match_nodes, rel_errors, scaled_random_state, state_floors

pytestmark = pytest.mark.gpu

P_ORDER = 12.0


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
    ("box_walls_N4", I.box((3, 2, 2), 4, L=(900.0, 600.0, 700.0)), 2),
    ("box_periodic_N3", I.box(2, 3, periodic=(1, 1, 1)), 1),
    ("box_warped_N5", I.box(2, 5, warp=0.05), 3),
    ("box_N1", I.box((3, 2, 2), 1), 1),
    ("box_N2_top_only", I.box((2, 2, 3), 2), 2),
    ("box_N8", I.box((2, 1, 1), 8), 5),
    ("shell_N4", I.shell(2, 1, 4), 2),
]

TOL = {"fp64": 1e-13, "fp64_pairs": 1e-13, "fp32_mixed": 2e-6}


def _filtered(numa, cfg, xyz_ref, q, s, precision, mu):
    """The GPU filter of q (in the oracle's node order) and the permutation
    from the oracle's to the library's global nodes (None for boxes)."""
    sv = numa.Solver(cfg, precision)
    try:
        perm = match_nodes(sv.coords(), xyz_ref, tol=1e-3) if cfg["kind"] == "shell" else None
        sv.set_state(q if perm is None else np.ascontiguousarray(q[:, perm]))
        sv.set_filter(0, s, P_ORDER, mu)
        sv.filter()
        a = sv.get_state().numpy().copy()
        sv.set_state(q if perm is None else np.ascontiguousarray(q[:, perm]))
        sv.filter()
        b = sv.get_state().numpy().copy()
        assert np.array_equal(a, b), "filter not bitwise deterministic"
        return a, perm
    finally:
        sv.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs", "fp32_mixed"])
@pytest.mark.parametrize("name,cfg,s", CASES, ids=[c[0] for c in CASES])
def test_filter_parity(numa, orc, name, cfg, s, precision):
    m = orc.Mesh(cfg)
    rho0, th0, _ = m.ref()
    q = scaled_random_state(m.Ng, rho0, th0, seed=len(name), u=5.0)
    mu = 0.7
    ref = m.filter(q, s, P_ORDER, mu)
    got, perm = _filtered(numa, cfg, m.coords(), q, s, precision, mu)
    if perm is not None:
        ref = ref[:, perm]
        q = q[:, perm]
    scale = np.abs(q).max(axis=1)
    err = np.abs(got - ref).max(axis=1) / scale
    assert err.max() <= TOL[precision], err
    assert np.abs(ref - q).max() > 1e-6 * scale.max()  # the filter changed the state


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp64_pairs", 1e-10), ("fp32_mixed", 1e-4)])
def test_filtered_run(numa, orc, precision, tol):
    """20 SSP-RK3 steps of the bubble with the filter after every 2nd step."""
    cfg = I.box(4, 4)
    m = orc.Mesh(cfg)
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS)
    s, every, mu, dt, n = 3, 2, 0.5, 0.01, 20
    qo = m.run_filtered(q0, dt, n, every, s, P_ORDER, mu)
    assert not np.array_equal(qo, m.run(q0, dt, n))
    sv = numa.Solver(cfg, precision)
    try:
        sv.set_filter(every, s, P_ORDER, mu)
        sv.set_state(q0)
        sv.run(dt, n)
        qg = sv.get_state().numpy().copy()
        # the same through single steps (counting carries over between calls)
        sv.set_state(q0)
        for _ in range(n):
            sv.rk_step(dt)
        qs = sv.get_state().numpy()
    finally:
        sv.close()
    assert np.array_equal(qg, qs)
    err = rel_errors(qg, qo, state_floors(qo, m.ref()[0].max()))
    assert (err if precision != "fp32_mixed" else err[:, 0]).max() <= tol, err


def test_filter_errors(numa):
    sv = numa.Solver(I.box(2, 3), "fp64")
    try:
        with pytest.raises(numa.NumaError) as e:
            sv.filter()  # no filter set
        assert e.value.code == -7
        for bad in ((-1, 2, 12.0, 1.0), (1, 5, 12.0, 1.0), (1, 2, 0.0, 1.0), (1, 2, 12.0, 1.5)):
            with pytest.raises(numa.NumaError) as e:
                sv.set_filter(*bad)
            assert e.value.code == -1
    finally:
        sv.close()


def test_filter_set_before_bind(numa, orc):
    """A filter configured before numa_bind is uploaded by the bind."""
    torch = pytest.importorskip("torch")
    cfg = I.box(2, 3)
    m = orc.Mesh(cfg)
    rho0, th0, _ = m.ref()
    q = scaled_random_state(m.Ng, rho0, th0, seed=17)
    ref = m.filter(q, 2, P_ORDER, 0.6)
    ctx = numa.numa_create(cfg)
    try:
        numa.numa_set_filter(ctx, 0, 2, P_ORDER, 0.6)
        info = numa.numa_get_mesh_info(ctx)
        ws = torch.empty(info["workspace_bytes"] + 256, dtype=torch.uint8, device="cuda")
        base = (ws.data_ptr() + 255) // 256 * 256
        stream = torch.cuda.current_stream()
        numa.numa_bind(ctx, base, info["workspace_bytes"], stream.cuda_stream)
        qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        numa.numa_set_state(ctx, qd.data_ptr(), True)
        numa.numa_filter(ctx)
        out = torch.empty_like(qd)
        numa.numa_get_state(ctx, out.data_ptr(), True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    finally:
        numa.numa_destroy(ctx)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(q).max()
