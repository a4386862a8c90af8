"""numa.HostStepper: host-to-host steps with the copies of consecutive
submits overlapping each other's steps.  Each result must equal, bit for
bit, the same state advanced by numa_set_state / numa_rk_step /
numa_get_state one after the other, for several different inputs submitted
back to back (so that the double-buffered staging is exercised)."""
import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

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


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_host_stepper_equals_plain_steps(numa, precision):
    import torch

    cfg = I.box((3, 4, 5), 4)
    s = numa.Solver(cfg, precision)
    try:
        s.init_state("bubble", I.BUBBLE_PARAMS)
        q0 = s.get_state().numpy().copy()
        inputs = [q0 + I.random_perturbation(s.Ng, seed=k, rho=1e-4, U=0.2, Theta=0.01) for k in range(5)]
        expect = []
        for q in inputs:
            s.set_state(q)
            s.rk_step(0.01)
            s.rk_step(0.01)
            expect.append(s.get_state().numpy().copy())
        hs = numa.HostStepper(s)
        pin_in = [torch.from_numpy(q).pin_memory() for q in inputs]
        pin_out = [torch.empty((5, s.Ng), dtype=torch.float64).pin_memory() for _ in inputs]
        for a, b in zip(pin_in, pin_out):
            hs.submit(a, b, 0.01, nsteps=2)
        hs.synchronize()
        for k, (got, want) in enumerate(zip(pin_out, expect)):
            assert np.array_equal(got.numpy(), want), k
    finally:
        s.close()
