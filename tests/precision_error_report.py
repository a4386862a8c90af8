"""Error of each GPU precision form against the FP64 oracle after T steps.

Runs the full-size rising-bubble box (32^3 elements, N=4, dt 0.01 s) and the
deep-atmosphere shell (6x30x30 columns, 8 layers, N=4, dt 1 s) from their
initial states, in the oracle (FP64, all host cores) and on the GPU in FP64,
FP32-mixed and FP64-pairs form.  After 100 and 500 SSP-RK3 steps it prints one
JSON line per (workload, precision, T) with the relative L2 and Linf error of
every prognostic variable (rho', U_x, U_y, U_z, Theta'), ||a - b|| / ||b|| over
global nodes, and the floored form the parity tests use.  The oracle's wall
time is printed as well.

Usage (needs a GPU and the compiled library):
    python -m tests.precision_error_report [--steps 100 500] [--workload NAME ...]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1511_01561_gb300 import inputs as I  # noqa: E402

from tests.helpers import match_nodes, state_floors  # noqa: E402

VARS = ["rho'", "U_x", "U_y", "U_z", "Theta'"]
PRECISIONS = ["fp64", "fp32_mixed", "fp64_pairs"]


def plain_rel(a: np.ndarray, b: np.ndarray):
    """Per variable: (||a-b||_2 / ||b||_2, ||a-b||_inf / ||b||_inf)."""
    out = []
    for v in range(a.shape[0]):
        d = a[v] - b[v]
        n2 = np.sqrt(np.sum(b[v] ** 2))
        ni = np.abs(b[v]).max()
        out.append((float(np.sqrt(np.sum(d**2)) / n2) if n2 > 0 else None,
                    float(np.abs(d).max() / ni) if ni > 0 else None))
    return out


def floored_rel(a: np.ndarray, b: np.ndarray, rho_max: float):
    fl = state_floors(b, rho_max)
    out = []
    for v in range(a.shape[0]):
        d = a[v] - b[v]
        n2 = max(np.sqrt(np.mean(b[v] ** 2)), fl[v])
        ni = max(np.abs(b[v]).max(), fl[v])
        out.append((float(np.sqrt(np.mean(d**2)) / n2), float(np.abs(d).max() / ni)))
    return out


def run(workload: str, steps: list, emit):
    from oracle import oracle
    from paper_1511_01561_gb300 import numa

    oracle.build()
    w = I.WORKLOADS[workload]
    cfg, dt = w["cfg"], w["dt"]
    m = oracle.Mesh(cfg)
    q0 = m.init_state(*w["ic"])
    rho_max = m.ref()[0].max()

    # oracle trajectory, kept at every reporting step
    ref = {}
    q = q0
    done = 0
    t0 = time.perf_counter()
    for T in sorted(steps):
        q = m.run(q, dt, T - done)
        done = T
        ref[T] = q.copy()
    t_orc = time.perf_counter() - t0
    emit({"workload": workload, "impl": "oracle", "steps": done, "seconds": t_orc,
          "threads": os.cpu_count(), "global_nodes": m.Ng})

    for prec in PRECISIONS:
        s = numa.Solver(cfg, prec)
        try:
            perm = match_nodes(s.coords(), m.coords(), tol=1e-3) if cfg["kind"] == "shell" else None
            s.set_state(q0 if perm is None else np.ascontiguousarray(q0[:, perm]))
            done = 0
            for T in sorted(steps):
                s.run(dt, T - done)
                done = T
                got = s.get_state().numpy()
                want = ref[T] if perm is None else ref[T][:, perm]
                emit({"workload": workload, "precision": prec, "steps": T,
                      "rel_l2": {VARS[v]: e[0] for v, e in enumerate(plain_rel(got, want))},
                      "rel_linf": {VARS[v]: e[1] for v, e in enumerate(plain_rel(got, want))},
                      "floored_max": max(max(e) for e in floored_rel(got, want, rho_max)),
                      "finite": bool(np.isfinite(got).all())})
        finally:
            s.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, nargs="+", default=[100, 500])
    ap.add_argument("--workload", nargs="+", default=["bubble_32x32x32_N4", "shell_6x30x30x8_N4"])
    a = ap.parse_args(argv)

    def emit(d):
        print(json.dumps(d), flush=True)

    for wl in a.workload:
        run(wl, a.steps, emit)


if __name__ == "__main__":
    main()
