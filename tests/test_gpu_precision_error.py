"""Error of each precision form against the FP64 oracle after 100 and 500
steps, on the full-size workloads: the rising-bubble box (32^3 elements,
N=4, dt 0.01 s) and the deep-atmosphere shell (6x30x30 columns, 8 layers,
N=4, dt 1 s), both from their initial states, SSP-RK3.

The oracle runs 500 steps on all host cores (a few minutes); the GPU runs
the same trajectory in FP64, FP64-pairs and FP32-mixed.  Every variable's
relative L2 and Linf error (floored as in the parity tests) is printed and
held to a stated bar:
- FP64: 1e-10 after 100 steps (the parity bar), 5e-10 after 500 (rounding
  errors of a stable run grow at most linearly with the step count);
- FP64-pairs: the same on the affine box; 32 times that on the curved shell
  (48-bit pair arithmetic, see tests/test_gpu_parity.py);
- FP32-mixed: 1e-4 (L2) and 5e-4 (Linf) after 100 steps, 5e-4 and 2.5e-3
  after 500."""
import json
import time

import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

from .helpers import match_nodes, rel_errors, state_floors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

VARS = ["rho'", "U_x", "U_y", "U_z", "Theta'"]
STEPS = (100, 500)


def _bars(precision, curved, T):
    grow = T / 100.0
    if precision == "fp32_mixed":
        return 1e-4 * grow, 5e-4 * grow
    tol = 1e-10 * grow * (32.0 if precision == "fp64_pairs" and curved else 1.0)
    return tol, tol


def _plain(a, b):
    """Per variable ||a-b|| / ||b|| in L2 and Linf (None where b is zero)."""
    out = []
    for v in range(a.shape[0]):
        d, n2, ni = a[v] - b[v], np.linalg.norm(b[v]), np.abs(b[v]).max()
        out.append((float(np.linalg.norm(d) / n2) if n2 > 0 else None, float(np.abs(d).max() / ni) if ni > 0 else None))
    return out


@pytest.fixture(scope="module")
def numa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_01561_gb300 import build
    build.build()
    from paper_1511_01561_gb300 import numa as mod
    return mod


@pytest.mark.parametrize("workload", ["bubble_32x32x32_N4", "shell_6x30x30x8_N4"])
def test_precision_forms_against_the_oracle(numa, orc, workload):
    w = I.WORKLOADS[workload]
    cfg, dt = w["cfg"], w["dt"]
    curved = cfg["kind"] == "shell"
    m = orc.Mesh(cfg)
    q0 = m.init_state(*w["ic"])
    rho_max = m.ref()[0].max()
    t0 = time.perf_counter()
    ref, q, done = {}, q0, 0
    for T in STEPS:
        q = m.run(q, dt, T - done)
        done = T
        ref[T] = q
    print(json.dumps({"workload": workload, "impl": "oracle", "steps": done,
                      "seconds": round(time.perf_counter() - t0, 1), "global_nodes": m.Ng}))
    failures = []
    for precision in ("fp64", "fp64_pairs", "fp32_mixed"):
        s = numa.Solver(cfg, precision)
        try:
            perm = match_nodes(s.coords(), m.coords(), tol=1e-3) if curved else None
            s.set_state(q0 if perm is None else np.ascontiguousarray(q0[:, perm]))
            done = 0
            for T in STEPS:
                s.run(dt, T - done)
                done = T
                got = s.get_state().numpy()
                want = ref[T] if perm is None else ref[T][:, perm]
                err = rel_errors(got, want, state_floors(want, rho_max))
                plain = _plain(got, want)
                print(json.dumps({"workload": workload, "precision": precision, "steps": T,
                                  "rel_l2": {VARS[v]: plain[v][0] for v in range(5)},
                                  "rel_linf": {VARS[v]: plain[v][1] for v in range(5)},
                                  "floored_l2_max": float(err[:, 0].max()),
                                  "floored_linf_max": float(err[:, 1].max())}))
                b2, binf = _bars(precision, curved, T)
                if not (err[:, 0].max() <= b2 and err[:, 1].max() <= binf):
                    failures.append((precision, T, err.tolist()))
        finally:
            s.close()
    assert not failures, failures
