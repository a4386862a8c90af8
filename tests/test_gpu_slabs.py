"""The slab-pipelined RK step (numa_set_slabs): element and node slabs of a
box along z on two streams, ordered by events.  Every node is computed as
without slabs, so the states must be identical bit for bit, in every
precision and integrator, through numa_run (graph) and numa_rk_step, and
after 100 steps still match the oracle within the parity bar."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .helpers import rel_errors, state_floors

pytestmark = pytest.mark.gpu


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
    ("walled_4x4x8_N4", I.box((4, 4, 8), 4), 0.01),
    ("periodic_xy_5x4x6_N4", I.box((5, 4, 6), 4, periodic=(1, 1, 0)), 0.01),
    ("N3_5x5x9", I.box((5, 5, 9), 3), 0.01),
]


def _run(numa, cfg, precision, scheme, slabs, q0, dt, steps, graph):
    s = numa.Solver(cfg, precision)
    try:
        used = s.set_slabs(slabs)
        s.set_time_scheme(scheme)
        s.set_state(q0)
        if graph:
            s.run(dt, steps)
        else:
            for _ in range(steps):
                s.rk_step(dt)
        return s.get_state().numpy().copy(), used
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp64_pairs"])
@pytest.mark.parametrize("name,cfg,dt", CASES, ids=[c[0] for c in CASES])
def test_slabs_are_bitwise_equal_to_one_slab(numa, orc, name, cfg, dt, precision):
    m = orc.Mesh(cfg)
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS)
    q0 += I.random_perturbation(m.Ng, seed=9, rho=1e-4, U=0.3, Theta=0.02)
    ref, used = _run(numa, cfg, precision, "ssp3", 1, q0, dt, 6, True)
    assert used == 1
    for slabs in (2, 3, 4):
        got, used = _run(numa, cfg, precision, "ssp3", slabs, q0, dt, 6, slabs != 3)
        assert used == slabs
        assert np.array_equal(got, ref), (slabs, np.abs(got - ref).max())
    got, _ = _run(numa, cfg, precision, "ls54", 4, q0, dt, 4, True)
    ref_ls, _ = _run(numa, cfg, precision, "ls54", 1, q0, dt, 4, True)
    assert np.array_equal(got, ref_ls)


def test_slabs_100_steps_match_the_oracle(numa, orc):
    cfg = I.box((4, 4, 8), 4)
    m = orc.Mesh(cfg)
    q0 = m.init_state("bubble", I.BUBBLE_PARAMS)
    qo = m.run(q0, 0.01, 100)
    got, used = _run(numa, cfg, "fp64", "ssp3", 4, q0, 0.01, 100, True)
    assert used == 4
    err = rel_errors(got, qo, state_floors(qo, m.ref()[0].max()))
    assert err.max() <= 1e-10, err
