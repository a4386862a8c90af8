"""numa_rhs_static_scratch: the right-hand side for callers that cannot
allocate device memory (allocation-free real-time loops, plug-ins that are
handed only input and output buffers).  Its scratch (primitive fields and
element residuals) is a fixed 16 MiB array inside the library; it runs the
same kernels on the same input as numa_rhs, so its result must equal
numa_rhs's bit for bit, call after call, in every precision (the three lay
out their primitive fields differently: 40, 32 and 64 bytes per node), and
it must refuse meshes that do not fit.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

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


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp64_pairs"])
def test_static_scratch_matches_numa_rhs_twice(numa, precision):
    import torch

    cfg = I.box((4, 3, 5), 4, warp=0.03)
    s = numa.Solver(cfg, precision)
    try:
        q = I.random_perturbation(s.Ng, seed=77, rho=0.01, U=3.0, Theta=0.5)
        qd = torch.from_numpy(q).cuda().contiguous()
        r_ref = torch.empty_like(qd)
        numa.numa_rhs(s.ctx, qd.data_ptr(), r_ref.data_ptr())
        ref = r_ref.cpu().numpy()
        assert np.isfinite(ref).all() and np.abs(ref).max() > 0.0
        for call in range(2):
            out = torch.full_like(qd, float("nan"))
            # through the C ABI directly
            rc = numa.lib.numa_rhs_static_scratch(s.ctx, ctypes.c_void_p(qd.data_ptr()),
                                                  ctypes.c_void_p(out.data_ptr()))
            assert rc == 0, numa.numa_last_error(s.ctx)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.array_equal(got, ref), (call, np.abs(got - ref).max())
    finally:
        s.close()


def test_static_scratch_rejects_meshes_that_do_not_fit(numa):
    import torch

    cfg = I.box(16, 4)  # 512,000 element nodes need 20.5 MB of residual scratch
    s = numa.Solver(cfg)
    try:
        qd = torch.zeros((5, s.Ng), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(qd)
        rc = numa.lib.numa_rhs_static_scratch(s.ctx, ctypes.c_void_p(qd.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()))
        assert rc == -1
        assert "static array" in numa.numa_last_error(s.ctx)
    finally:
        s.close()


# The largest cubic N=4 box that fits the 16 MiB array in each precision, and
# the next size up (scratch per global node / per element node: FP64 72 / 40
# bytes, FP32-mixed 32 / 20, pairs 64 / 40).
LIMITS = [("fp64", 11), ("fp32_mixed", 15), ("fp64_pairs", 12)]


@pytest.mark.parametrize("precision,n", LIMITS)
def test_static_scratch_size_limit(numa, precision, n):
    import torch

    s = numa.Solver(I.box(n, 4), precision)
    try:
        q = I.random_perturbation(s.Ng, seed=5, rho=0.01, U=3.0, Theta=0.5)
        qd = torch.from_numpy(q).cuda().contiguous()
        ref, out = torch.empty_like(qd), torch.full_like(qd, float("nan"))
        numa.numa_rhs(s.ctx, qd.data_ptr(), ref.data_ptr())
        rc = numa.lib.numa_rhs_static_scratch(s.ctx, ctypes.c_void_p(qd.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, numa.numa_last_error(s.ctx)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        s.close()
    s = numa.Solver(I.box(n + 1, 4), precision)
    try:
        qd = torch.zeros((5, s.Ng), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(qd)
        rc = numa.lib.numa_rhs_static_scratch(s.ctx, ctypes.c_void_p(qd.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == -1 and "static array" in numa.numa_last_error(s.ctx)
    finally:
        s.close()
