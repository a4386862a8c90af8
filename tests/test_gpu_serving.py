"""GPU tests of the continuous-batching ensemble server (numa_sched_*):
members of different sizes, orders, precisions and step counts, arriving
while others run, give bit for bit the same result in the mix as alone, and
each served result matches the oracle's own run of that request (the stage
loop of Sec. 2.2 over Eq. 4) within the parity bars; admission waits for
room in the arena; over-budget, poisoned and cancelled requests neither
disturb the others nor trap the GPU."""
import time

import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .helpers import match_nodes, rel_errors, state_floors

pytestmark = pytest.mark.gpu

# parity bars of a trajectory against the oracle (tests/test_gpu_parity.py):
# FP64 1e-10, pairs 1e-10 on affine and 3.2e-9 on curved elements, FP32-mixed
# 1e-4 (L2) and 5e-4 (Linf)


@pytest.fixture(scope="module")
def numa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_01561_gb300 import build
    build.build()
    from paper_1511_01561_gb300 import numa as mod
    return mod


REQUESTS = [
    # cfg, initial condition, params, dt, steps, precision
    (I.box(3, 4), "bubble", I.BUBBLE_PARAMS, 0.01, 7, "fp64"),
    (I.box((2, 3, 2), 3), "bubble", (1.5, 200.0, 400.0, 600.0, 300.0), 0.01, 12, "fp32_mixed"),
    (I.box(2, 6), "bubble", (2.0, 300.0, 500.0, 500.0, 400.0), 0.01, 5, "fp64"),
    (I.box(4, 4), "bubble", (0.3, 250.0, 450.0, 520.0, 350.0), 0.01, 9, "fp64"),
    (I.shell(2, 1, 3), "jetwave", I.JETWAVE_PARAMS, 1.0, 4, "fp64"),
    (I.box((3, 2, 2), 4), "bubble", (0.8, 250.0, 500.0, 300.0, 300.0), 0.01, 0, "fp32_mixed"),
    (I.box((2, 2, 3), 4), "bubble", (1.2, 220.0, 480.0, 520.0, 380.0), 0.01, 6, "fp64_pairs"),
    (I.box(2, 3, warp=0.04), "bubble", I.BUBBLE_PARAMS, 0.01, 5, "fp64_pairs"),
    (I.box(3, 3, warp=0.03), "bubble", I.BUBBLE_PARAMS, 0.01, 4, "fp64"),
]


def _alone(numa, cfg, ic, params, dt, steps, precision):
    s = numa.Solver(cfg, precision)
    try:
        s.init_state(ic, params)
        s.run(dt, steps)
        return s.get_state().numpy().copy()
    finally:
        s.close()


def _drain(sched, ids, seconds=120.0):
    """Step until every request has finished (meshes build in the background,
    so idle steps wait a little instead of spinning)."""
    deadline = time.time() + seconds
    max_active = 0
    while time.time() < deadline:
        active, _ = sched.step()
        max_active = max(max_active, active)
        if all(sched.poll(i)[0] in ("done", "failed", "cancelled") for i in ids):
            return max_active
        if active == 0:
            time.sleep(0.005)
    raise AssertionError("scheduler did not finish")


def _oracle_check(numa, orc, cfg, ic, params, dt, steps, precision, got):
    """The served result against the oracle's run of the same request."""
    m = orc.Mesh(cfg)
    qo = m.run(m.init_state(ic, params), dt, steps)
    if cfg["kind"] == "shell":  # shell nodes are numbered differently: match them by coordinates
        s = numa.Solver(cfg)
        try:
            perm = match_nodes(s.coords(), m.coords(), tol=1e-3)
        finally:
            s.close()
        qo = qo[:, perm]
    err = rel_errors(got, qo, state_floors(qo, m.ref()[0].max()))
    if precision == "fp32_mixed":
        assert err[:, 0].max() <= 1e-4 and err[:, 1].max() <= 5e-4, (cfg, precision, err)
    else:
        curved = cfg["kind"] == "shell" or float(cfg.get("warp", 0.0)) != 0.0
        tol = 1e-10 * (32.0 if precision == "fp64_pairs" and curved else 1.0)
        assert err.max() <= tol, (cfg, precision, err)


def _close(a, b):
    scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-300)
    return np.all(np.abs(a - b) <= 1e-12 * scale)


def test_mix_equals_alone_with_arrivals(numa, orc):
    sched = numa.Scheduler(512 << 20, build_threads=3)
    try:
        ids = [sched.submit(*r[:2], params=r[2], dt=r[3], nsteps=r[4], precision=r[5]) for r in REQUESTS[:3]]
        steps = 0
        deadline = time.time() + 60
        while steps < 3 and time.time() < deadline:  # later arrivals join a running batch
            active, _ = sched.step()
            steps += active > 0
            if active == 0:
                time.sleep(0.005)
        ids += [sched.submit(*r[:2], params=r[2], dt=r[3], nsteps=r[4], precision=r[5]) for r in REQUESTS[3:]]
        _drain(sched, ids)
        for rid, r in zip(ids, REQUESTS):
            status, done, _ = sched.poll(rid)
            assert status == "done" and done == r[4], (r, status, done)
            got = sched.result(rid)
            ref = _alone(numa, *r)
            assert np.array_equal(got, ref), (r, np.abs(got - ref).max())  # alone == in the mix, bitwise
            _oracle_check(numa, orc, *r, got)
    finally:
        sched.close()


def test_admission_waits_for_room(numa):
    cfg = I.box(6, 4)
    ctx = numa.numa_create(cfg)
    need = numa.numa_get_mesh_info(ctx)["workspace_bytes"]
    numa.numa_destroy(ctx)
    # room for one member at a time (the scheduler's own tables take < 1 MiB)
    sched = numa.Scheduler(int(1.5 * need) + (1 << 20), build_threads=2)
    try:
        ids = [sched.submit(cfg, "bubble", I.BUBBLE_PARAMS, dt=0.01, nsteps=n) for n in (3, 4, 2)]
        assert _drain(sched, ids) == 1
        for rid, n in zip(ids, (3, 4, 2)):
            assert _close(sched.result(rid), _alone(numa, cfg, "bubble", I.BUBBLE_PARAMS, 0.01, n, "fp64"))
        with pytest.raises(numa.NumaError) as e:
            sched.submit(I.box(9, 4), "bubble", I.BUBBLE_PARAMS, dt=0.01, nsteps=1)
        assert e.value.code == -6  # NUMA_EBUDGET
    finally:
        sched.close()


def test_poisoned_and_cancelled_requests_do_not_disturb_others(numa):
    sched = numa.Scheduler(256 << 20, build_threads=2)
    try:
        good = sched.submit(I.box(3, 3), "bubble", I.BUBBLE_PARAMS, dt=0.01, nsteps=6)
        bad = sched.submit(I.box(2, 3), "bubble", (float("nan"), 250.0, 500.0, 500.0, 350.0), dt=0.01, nsteps=4)
        gone = sched.submit(I.box(5, 4), "bubble", I.BUBBLE_PARAMS, dt=0.01, nsteps=50)
        sched.cancel(gone)
        _drain(sched, [good, bad, gone])
        assert sched.poll(gone)[0] == "cancelled"
        assert sched.poll(bad)[0] == "failed"
        with pytest.raises(numa.NumaError) as e:
            sched.result(bad)
        assert e.value.code == -4  # NUMA_ENONFINITE
        assert sched.poll(good)[0] == "done"
        assert _close(sched.result(good), _alone(numa, I.box(3, 3), "bubble", I.BUBBLE_PARAMS, 0.01, 6, "fp64"))
    finally:
        sched.close()
