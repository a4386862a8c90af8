#!/usr/bin/env python3
"""Benchmark of the CG spectral-element RHS / SSP-RK3 hot path (NUMA, Sec. 2).

Workload (default): the rising thermal bubble in a 1000 m box with 32^3
elements of order N=4 (129^3 = 2,146,689 global nodes), FP64, dt = 0.01 s.
One benchmark step is one SSP-RK3 time step = three RK stages, each
create_rhs (element volume kernel) + DSS / inverse mass / update kernel.
Metric: node-updates per second per RK stage = Ng * 3 * steps / time.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (each step: one full SSP-RK3 step of the same
workload).  With torchrun (N > 1) every rank advances its own replica of the
workload on its own GPU (no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "node-updates/s per RK stage"
UNIT = "node-updates/s"
STAGES = 3


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="mine", choices=["mine", "reference"])
    p.add_argument("--workload", default="bubble_32x32x32_N4")
    p.add_argument("--no-fp32", action="store_true", help="skip the FP32 mixed-precision line")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-dg", action="store_true", help="skip the DG-storage comparison")
    p.add_argument("--no-imex", action="store_true", help="skip the 1D-IMEX comparison")
    p.add_argument("--imex-only", action="store_true", help="run only the 1D-IMEX comparison (profiling)")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline sample length")
    p.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--filter-reps", type=int, default=20, help="filter applications timed (0 skips)")
    p.add_argument("--serve", action="store_true", help="ensemble-serving workload instead of the RK3 steps")
    p.add_argument("--serve-requests", type=int, default=64)
    p.add_argument("--serve-steps-scale", type=float, default=1.0, help="scale every request's step count")
    p.add_argument("--serve-budget-frac", type=float, default=0.5, help="arena = this fraction of free HBM")
    p.add_argument("--serve-load", type=float, default=0.8, help="Poisson rate / saturated request rate")
    p.add_argument("--serve-overload", type=float, default=2.0,
                   help="rate of a second Poisson stream / saturated request rate (0 skips it)")
    p.add_argument("--no-shell", action="store_true", help="skip the cubed-sphere shell block")
    p.add_argument("--no-serve-block", action="store_true", help="skip the reduced serving block")
    p.add_argument("--no-precision", action="store_true",
                   help="skip the FP32-mixed / FP64-pairs difference from the FP64 state")
    p.add_argument("--serve-block-requests", type=int, default=16)
    p.add_argument("--serve-block-steps-scale", type=float, default=0.1)
    p.add_argument("--peaks", action="store_true",
                   help="measure the FP64/FP32 FMA and FP64/TF32 mma.sync throughput of the GPU instead")
    return p.parse_args(argv)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 peak of the GB300 (dense, non-tensor): the nominal 1.25 TFLOP/s (152
# SMs x 2 FP64 FMA per clock x 2070 MHz); `bench.py --peaks` measured 1.258
# with register-only FMA chains and 1.10 with FP64 mma.sync
# (profiles/p0_arithmetic_peaks_gb300.md).
FP64_PEAK_TFLOPS = 1.25
FP64_PEAK_SOURCE = "nominal FP64 FMA rate; measured 1.258 TFLOP/s (profiles/p0_arithmetic_peaks_gb300.md)"

# DRAM bytes (read + write) per launch from one ncu capture of each kernel on
# this workload (profiles/*_bubble_32x32x32_N4.md), valid only for the kernel
# sources they were taken on (first 16 hex digits of the sha256 of the kernel
# sources, see kernel_source_hash).
NCU_TRAFFIC = {"kernels_sha256_16": "c162b3edd950e364", "workload": "bubble_32x32x32_N4",
               "volume_fp64_affine": 223.360000e6 + 130.280448e6,
               "volume_pairs_affine": 154.657536e6 + 122.701056e6,
               "volume_fp32_affine": 139.263232e6 + 49.111808e6}

# the sources the element kernels with committed traffic figures are built from
KERNEL_SOURCES = ["kernels_common.cuh", "volume_fp64.cu", "volume_fp32.cu", "volume_pairs.cu"]


def code_lines(text: str) -> list:
    """The lines of a C/CUDA source with comments and blank lines removed
    (a `//` inside a string literal stays), stripped of surrounding spaces."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    out = []
    for ln in text.splitlines():
        cut = len(ln)
        start = 0
        while True:
            k = ln.find("//", start)
            if k < 0:
                break
            if ln.count('"', 0, k) % 2 == 0:
                cut = k
                break
            start = k + 2
        ln = ln[:cut].strip()
        if ln:
            out.append(ln)
    return out


def kernel_source_hash() -> str:
    """Hash of the kernel sources' code (comments and blank lines left out, so
    that a comment edit does not invalidate a capture)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1511_01561_gb300", "csrc", name), encoding="utf-8") as f:
            h.update("\n".join(code_lines(f.read())).encode())
    return h.hexdigest()[:16]


def ncu_traffic(key: str, workload: str):
    """DRAM bytes per launch of a kernel from the committed capture: only for
    the workload it was captured on, and only while the kernel sources hash
    to the value they had then."""
    if workload != NCU_TRAFFIC["workload"] or kernel_source_hash() != NCU_TRAFFIC["kernels_sha256_16"]:
        return None
    return NCU_TRAFFIC.get(key)


def volume_fp64_cost(N: int, form: str) -> tuple:
    """(flops, FP64 operations) per element node of the FP64 element kernel
    of `form`.  A flop count takes an FMA as 2; an operation count takes an
    FMA, a product and a sum as 1 each (each takes one slot of the FP64 pipe).
    The 12 flux fields (U, the symmetric U (x) u + p' I, theta U) come
    gathered: the update forms them once per global node.
    - "nodal", the per-node form of Eq. 5 (any element): each field
      differentiated along xi, eta and zeta (3 (N+1) operations, 6 (N+1) - 3
      flops), and 15 uses of a derivative triple folded into their equations
      with the -Jw-weighted metric (3 operations; 6 flops, 5 for the first
      use in each of the 5 equations): 36 (N+1) + 45 operations,
      72 (N+1) + 49 flops.
    - "rect", rectilinear affine elements: per equation three contractions
      of length N+1 with K_d D (3 (N+1) operations, the first a product:
      6 (N+1) - 1 flops); the weight w_i w_j w_k goes with the inverse mass
      into the update; the element's K_d D, 3 (N+1)^2 products shared by its
      (N+1)^3 nodes: 15 (N+1) + 3 / (N+1) operations, 5 (6 (N+1) - 1) +
      3 / (N+1) flops.
    Affine meshes whose elements are not rectilinear take the per-node
    form in FP64."""
    P = N + 1
    if form == "rect":
        return 5.0 * (6 * P - 1) + 3.0 / P, 15.0 * P + 3.0 / P
    return 72.0 * P + 49.0, 36.0 * P + 45.0


def volume_flops_per_elem_node(N: int, affine: bool = False) -> float:
    """Flops per element node of the FP64 element kernel that a box
    (rectilinear elements, affine=True) or a curved mesh takes."""
    return volume_fp64_cost(N, "rect" if affine else "nodal")[0]


def filter_flops_per_elem_node(N: int) -> float:
    """Algorithmic flops per element node of the filter's element part: three
    contractions of length N+1 on five variables, the subtraction of q and
    the Jw weight."""
    return 30.0 * (N + 1) + 10.0


def volume_bytes(Nl: int, Ng: int, fp: int, N: int = 4, affine: bool = False, gathered: int = 8) -> float:
    """Algorithmic DRAM bytes of one volume-kernel launch (fp = 8 for FP64 and
    the pairs mode, 4 for the FP32-mixed form): metric terms and Jw (10
    values per element node; affine elements: Jw per node and 9 metric terms
    per element), l2g (4 B), the residual write (5 values), and one read per
    global node of the `gathered` values (FP64: U and the nine flux
    components, 12; pairs: U and u, theta, p' as pairs, 8; FP32: 8 floats)."""
    if affine:
        return Nl * (fp + 4 + 5 * fp) + Nl // (N + 1) ** 3 * 9 * fp + Ng * gathered * fp
    return Nl * (10 * fp + 4 + 5 * fp) + Ng * gathered * fp


def update_bytes(Nl: int, Ng: int, fp: int, stage_reads_qn: float, entries: int = None, prim: int = None) -> float:
    """Algorithmic DRAM bytes of one DSS/update launch: CSR (4 B per entry +
    4 B per node; `entries` = Nl unless given), residual read (5 values per
    element node, once), M^-1, wall flag, q^k read, q^{k+1} write, q^n on the
    stages that use it, the reference state (4 doubles) and the
    primitive-field write (`prim` bytes: 72 in FP64, 32 in FP32-mixed)."""
    entries = Nl if entries is None else entries
    prim = (72 if fp == 8 else 32) if prim is None else prim
    return (entries * 4 + Nl * 5 * fp
            + Ng * (4 + 8 + 1 + 40 + 40 + 40 * stage_reads_qn + 32 + prim))


def stage_bytes_model(Nl: int, Ng: int, fp: int) -> float:
    """Algorithmic DRAM bytes of one whole RK stage, counted the way the
    paper's performance model counts (Sec. 6): per element node the metric
    terms and Jw (10 values of fp bytes) and l2g (4 B); per global node q^k,
    q^n and q^{k+1} (40 B each), the reference state (24 B), M^-1 (8 B) and
    the residual round trip of the global DSS (80 B)."""
    return Nl * (10 * fp + 4) + Ng * 232


def max_over_ranks(dist, x: float, device=None) -> float:
    """The largest x over all ranks of the default process group (x itself
    when there is none); every rank gets the result."""
    if dist is None or not dist.is_initialized():
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, Ng: int, steps: int, ms: float) -> float:
    """Node-updates/s per RK stage of `world` replicas that each advanced Ng
    global nodes by `steps` SSP-RK3 steps, the slowest in `ms` milliseconds."""
    return world * Ng * STAGES * steps / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 200 ms) of one GPU
    while the timed region runs, into a temporary CSV read back by stop()."""

    def __init__(self, index: int):
        import tempfile

        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="numa_clocks_", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_worker(args):
    """Time the FP64 CPU oracle on the host cores (child process)."""
    from oracle import oracle
    from paper_1511_01561_gb300 import inputs as I

    w = I.WORKLOADS[args.workload]
    m = oracle.Mesh(w["cfg"])
    q = m.init_state(*w["ic"])
    t0 = time.perf_counter()
    q = m.run(q, w["dt"], 1)
    t1 = time.perf_counter() - t0
    n = max(1, int(round(args.cpu_seconds / max(t1, 1e-3))) - 1)
    t0 = time.perf_counter()
    m.run(q, w["dt"], n)
    t = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({"value": m.Ng * STAGES * n / t, "steps": n, "seconds": t, "cores": cores,
                      "Ng": m.Ng}))


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (empty if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return ""
    for ln in out.splitlines():
        if ln.strip().lower().startswith("model name"):
            return ln.split(":", 1)[1].strip()
    return ""


def cpu_baseline(args):
    """The oracle on all host cores (OpenMP), and a short sample on one core."""
    def run(threads, seconds):
        env = dict(os.environ)
        env["OMP_NUM_THREADS"] = str(threads)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", args.workload,
                            "--cpu-seconds", str(seconds)], capture_output=True, text=True, env=env)
        if r.returncode != 0:
            return None, r.stderr.strip().splitlines()[-1] if r.stderr else "failed"
        return json.loads(r.stdout.strip().splitlines()[-1]), None

    d, err = run(int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), args.cpu_seconds)
    if d is None:
        return {"error": err}
    out = {"value": d["value"], "unit": UNIT, "cores": d["cores"], "kind": "oracle",
           "sample": f"{d['steps']} SSP-RK3 steps ({STAGES * d['steps']} stages) of {args.workload} "
                     f"on all {d['Ng']} global nodes, {d['seconds']:.1f} s, FP64 C oracle (-O2, OpenMP)",
           "cpu_model": cpu_model()}
    one, _ = run(1, 0.0)  # one warm-up step, then one timed step
    if one is not None:
        out["one_core"] = {"value": one["value"], "unit": UNIT,
                           "sample": f"{one['steps']} SSP-RK3 step(s), {one['seconds']:.1f} s, one thread"}
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, each step one SSP-RK3 step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle
    from paper_1511_01561_gb300 import inputs as I

    w = I.WORKLOADS[args.workload]
    m = oracle.Mesh(w["cfg"])
    q = m.init_state(*w["ic"])
    if args.warmup:
        q = m.run(q, w["dt"], args.warmup)
    t0 = time.perf_counter()
    m.run(q, w["dt"], args.steps)
    t = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = m.Ng * STAGES * args.steps / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "global_nodes": m.Ng, "elements": m.Ne, "N": w["cfg"]["N"],
                   "dt": w["dt"], "rk": "ssp-rk3"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} SSP-RK3 steps of {args.workload}, all global nodes"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_mine(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)  # child process, before heavy GPU work

    from paper_1511_01561_gb300 import inputs as I
    from paper_1511_01561_gb300 import numa

    w = I.WORKLOADS[args.workload]
    cfg, dt = w["cfg"], w["dt"]
    hbm_gbs, peak_src = load_peaks()
    # a box without warp has affine elements: the kernels take the
    # contravariant-flux form unless the per-node form is asked for
    affine = cfg["kind"] == "box" and float(cfg.get("warp", 0.0)) == 0.0

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_ranks(x: float) -> float:
        return max_over_ranks(dist, x, dev)

    if args.imex_only:
        # the 1D-IMEX comparison alone (for profiling its kernels)
        out = imex_block(args, numa, torch, dev, barrier, max_ranks)
        if rank == 0:
            print(json.dumps({"imex": out}))
        if dist is not None:
            dist.destroy_process_group()
        return

    snaps = {} if not args.no_precision else None

    def measure(precision, form="auto", scheme="ssp3", storage="cg", wl=None):
        wl = w if wl is None else wl
        s = numa.Solver(dict(wl["cfg"], metric_form=form, storage=storage), precision, device=str(dev))
        s.set_time_scheme(scheme)
        s.init_state(*wl["ic"])
        s.run(wl["dt"], args.warmup)
        stream = s.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        headline = (precision, form, scheme) == ("fp64", "auto", "ssp3") and wl is w
        clocks = ClockSampler(local) if headline else None
        e0.record(stream)
        s.run(wl["dt"], args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = max_ranks(e0.elapsed_time(e1))
        ck = clocks.stop() if clocks else None
        if snaps is not None and storage == "cg" and scheme == "ssp3" and form == "auto":
            # the state after warm-up + timed steps, for the precision-form comparison
            snaps[(precision, wl["cfg"]["kind"])] = s.get_state(
                torch.empty((5, s.Ng), dtype=torch.float64, device=dev))
        # per-kernel device times over the same number of steps (event-bracketed launches)
        ms_vol, ms_upd = s.time_kernels(wl["dt"], args.steps)
        info = s.info
        e2e = None
        if not args.no_e2e and headline:
            # every step: the state from pinned host memory to the device, one
            # RK step, the new state back to pinned host memory; the public
            # HostStepper overlaps each step's copies with its neighbours' steps
            q_host = torch.empty((5, s.Ng), dtype=torch.float64, pin_memory=True)
            out_host = [torch.empty((5, s.Ng), dtype=torch.float64, pin_memory=True) for _ in range(2)]
            s.get_state(q_host)
            nb = 5 * s.Ng * 8
            hs = numa.HostStepper(s)
            hs.submit(q_host, out_host[0], dt)  # warm-up (stream and event set-up)
            hs.synchronize()
            barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for k in range(args.steps):
                hs.submit(q_host, out_host[k % 2], dt)
            hs.synchronize()
            torch.cuda.synchronize(dev)
            te = max_ranks(time.perf_counter() - t0)
            e2e = {"value": world * s.Ng * STAGES * args.steps / te, "unit": UNIT,
                   "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
                   "how": "numa.HostStepper: per step a pinned host->device copy of the state, one SSP-RK3 step "
                          "and a device->host copy of the result, copies on two copy streams overlapping the "
                          "neighbouring steps"}
        filt = None
        if headline and args.filter_reps > 0:
            # Boyd-Vandeven filter (element kernel + DSS update), applied on its own
            s.set_filter(0, max(0, w["cfg"]["N"] - 1), 12.0, 1.0)
            s.filter()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            f0.record(stream)
            for _ in range(args.filter_reps):
                s.filter()
            f1.record(stream)
            torch.cuda.synchronize(dev)
            filt = f0.elapsed_time(f1) / args.filter_reps
        finite = s.check_finite() == 0
        s.close()
        return ms, ms_vol, ms_upd, info, e2e, ck, finite, filt

    ms, ms_vol, ms_upd, info, e2e, ck, finite, filt_ms = measure("fp64")
    Ng, Nl, N = info["Ng"], info["Nl"], info["N"]
    value = whole_job_rate(world, Ng, args.steps, ms)
    nlaunch = STAGES * args.steps
    vol_avg_s = ms_vol * 1e-3 / nlaunch
    fl_el, ops_el = volume_fp64_cost(N, "rect" if affine else "nodal")
    flops = fl_el * Nl
    achieved_tf = flops / vol_avg_s / 1e12
    # FP64 pipe slots: 2 per SM per clock, i.e. half the FMA flop peak
    pipe_frac = ops_el * Nl / vol_avg_s / (FP64_PEAK_TFLOPS * 1e12 / 2)
    form_name = "affine" if affine else "nodal"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "global_nodes": Ng, "elements": info["Ne"], "N": N, "dt": dt,
                   "rk": "ssp-rk3", "stages_per_step": STAGES,
                   "l2": f"working set {info['workspace_bytes'] / 1e6:.0f} MB > 129 MB L2, no flush",
                   "parallelism": f"replica x{world}" if world > 1 else "single GPU"},
        "e2e": e2e,
        "gpu_launches": 2 * nlaunch,
        "roofline": {"kernel": f"volume_kernel<{N},double,{form_name}>",
                     "form": "rectilinear (K_d D, w_i w_j w_k)" if affine else "per-node (Eq. 5)",
                     "bound": "alu", "achieved": achieved_tf,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_TFLOPS,
                     "traffic": ncu_traffic(f"volume_fp64_{form_name}", args.workload),
                     "algorithmic_flops": flops, "fp64_ops_per_element_node": ops_el,
                     "fp64_pipe_frac": pipe_frac,
                     "algorithmic_bytes": volume_bytes(Nl, Ng, 8, N, affine, gathered=12),
                     "peak_source": FP64_PEAK_SOURCE,
                     "avg_launch_ms": 1e3 * vol_avg_s,
                     "share_of_step": ms_vol / (ms_vol + ms_upd)},
        "kernels": {"volume_ms_avg": 1e3 * vol_avg_s, "update_ms_avg": ms_upd / nlaunch,
                    "update_hbm_frac": update_bytes(Nl, Ng, 8, 2 / 3) / (ms_upd * 1e-3 / nlaunch) / 1e9 / hbm_gbs,
                    "stage_hbm_frac": stage_bytes_model(Nl, Ng, 8) / (ms * 1e-3 / nlaunch) / 1e9 / hbm_gbs,
                    "stage_hbm_model": "84 B per element node + 232 B per global node"},
        "clocks": ck,
        "finite": finite,
    }
    if filt_ms is not None:
        ff = filter_flops_per_elem_node(N) * Nl
        line["filter"] = {
            "what": "one Boyd-Vandeven filter application (element kernel + DSS), FP64, s = N-1, p = 12",
            "ms_per_application": filt_ms, "reps": args.filter_reps,
            "element_fp64_tflops_lower_bound": ff / (filt_ms * 1e-3) / 1e12,
            "frac_of_fp64_peak_lower_bound": ff / (filt_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
        }
    # the five-stage low-storage integrator (the paper's stage count), FP64
    msl, voll, updl, _, _, _, finl, _ = measure("fp64", "auto", "ls54")
    line["fp64_ls54"] = {
        "what": "five-stage low-storage RK (order four) instead of SSP-RK3, same workload and dt",
        "value": whole_job_rate(world, Ng, args.steps, msl) * 5 / STAGES, "unit": UNIT,
        "ms_per_step": msl / args.steps, "stages_per_step": 5, "finite": finl,
        "volume_ms_avg": voll / (5 * args.steps), "update_ms_avg": updl / (5 * args.steps)}
    if affine:
        # the same workload through the per-node form of Eq. 5 (metric terms
        # read and applied at every node), for comparison
        msn, voln, updn, _, _, _, finn, _ = measure("fp64", "nodal")
        voln_s = voln * 1e-3 / nlaunch
        fl_n = volume_flops_per_elem_node(N, False) * Nl
        op_n = volume_fp64_cost(N, "nodal")[1] * Nl
        line["fp64_nodal_form"] = {
            "value": world * Ng * STAGES * args.steps / (msn * 1e-3), "unit": UNIT, "ms_per_step": msn / args.steps,
            "finite": finn, "volume_ms_avg": 1e3 * voln_s, "update_ms_avg": updn / nlaunch,
            "roofline": {"kernel": f"volume_kernel<{N},double,nodal>", "bound": "alu",
                         "achieved": fl_n / voln_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": fl_n / voln_s / 1e12 / FP64_PEAK_TFLOPS,
                         "fp64_pipe_frac": op_n / voln_s / (FP64_PEAK_TFLOPS * 1e12 / 2),
                         "traffic": ncu_traffic("volume_fp64_nodal", args.workload)},
        }
    if not args.no_fp32:
        ms32, vol32, upd32, _, _, _, fin32, _ = measure("fp32_mixed")
        v32 = world * Ng * STAGES * args.steps / (ms32 * 1e-3)
        vol32_s = vol32 * 1e-3 / nlaunch
        b = volume_bytes(Nl, Ng, 4, N, affine)
        line["fp32_mixed"] = {
            "value": v32, "unit": UNIT, "ms_per_step": ms32 / args.steps, "speedup_vs_fp64": v32 / value,
            "finite": fin32,
            "roofline": {"kernel": f"volume_kernel<{N},float,{form_name}>", "bound": "hbm",
                         "achieved": b / vol32_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                         "frac": b / vol32_s / 1e9 / hbm_gbs,
                         "traffic": ncu_traffic(f"volume_fp32_{form_name}", args.workload), "algorithmic_bytes": b,
                         "peak_source": peak_src, "avg_launch_ms": 1e3 * vol32_s},
            "update_ms_avg": upd32 / nlaunch,
            "update_hbm_frac": update_bytes(Nl, Ng, 4, 2 / 3) / (upd32 * 1e-3 / nlaunch) / 1e9 / hbm_gbs,
            "stage_hbm_frac": stage_bytes_model(Nl, Ng, 4) / (ms32 * 1e-3 / nlaunch) / 1e9 / hbm_gbs,
            "stage_hbm_model": "44 B per element node + 232 B per global node",
        }
        if affine:
            ms32n, vol32n, _, _, _, _, fin32n, _ = measure("fp32_mixed", "nodal")
            vol32n_s = vol32n * 1e-3 / nlaunch
            bn = volume_bytes(Nl, Ng, 4)
            line["fp32_mixed"]["nodal_form"] = {
                "value": world * Ng * STAGES * args.steps / (ms32n * 1e-3), "ms_per_step": ms32n / args.steps,
                "finite": fin32n, "volume_ms_avg": 1e3 * vol32n_s, "volume_hbm_frac": bn / vol32n_s / 1e9 / hbm_gbs,
                "traffic": ncu_traffic("volume_fp32_nodal", args.workload)}
    if not args.no_fp32:
        # FP64-accurate element kernel on the FP32 units ((hi, lo) float pairs)
        msp, volp, updp, _, _, _, finp, _ = measure("fp64_pairs")
        vp = world * Ng * STAGES * args.steps / (msp * 1e-3)
        volp_s = volp * 1e-3 / nlaunch
        bp = volume_bytes(Nl, Ng, 8, N, affine)
        line["fp64_pairs"] = {
            "value": vp, "unit": UNIT, "ms_per_step": msp / args.steps, "speedup_vs_fp64": vp / value,
            "form": form_name, "finite": finp, "volume_ms_avg": 1e3 * volp_s, "update_ms_avg": updp / nlaunch,
            "volume_fp64_equiv_tflops": volume_flops_per_elem_node(N, affine) * Nl / volp_s / 1e12,
            "volume_traffic": ncu_traffic(f"volume_pairs_{form_name}", args.workload),
            "volume_hbm_gbs": bp / volp_s / 1e9, "volume_hbm_frac": bp / volp_s / 1e9 / hbm_gbs,
        }
        if affine:
            mspn, volpn, _, _, _, _, finpn, _ = measure("fp64_pairs", "nodal")
            line["fp64_pairs"]["nodal_form"] = {
                "value": world * Ng * STAGES * args.steps / (mspn * 1e-3), "ms_per_step": mspn / args.steps,
                "finite": finpn, "volume_ms_avg": volpn / nlaunch}
    if not args.no_dg:
        # DG storage of the node data (one copy per element node) against CG
        # storage, same workload; rates count the CG global nodes advanced
        line["storage_dg"] = {"what": "DG storage (one value per element node) instead of CG storage, "
                                      "same workload and dt; value counts CG global nodes", "unit": UNIT}
        for prec, fp, ref_v in (("fp64", 8, value), ("fp32_mixed", 4, line.get("fp32_mixed", {}).get("value"))):
            if prec == "fp32_mixed" and args.no_fp32:
                continue
            msd, vold, updd, infod, _, _, find, _ = measure(prec, "auto", "ssp3", "dg")
            vd = whole_job_rate(world, Ng, args.steps, msd)
            upd_s = updd * 1e-3 / nlaunch
            line["storage_dg"][prec] = {
                "value": vd, "ms_per_step": msd / args.steps, "vs_cg_storage": vd / ref_v if ref_v else None,
                "storage_nodes": infod["Ng"], "dss_entries": infod["dss_entries"], "finite": find,
                "volume_ms_avg": vold / nlaunch, "update_ms_avg": 1e3 * upd_s,
                "update_hbm_frac": update_bytes(Nl, infod["Ng"], fp, 2 / 3, infod["dss_entries"])
                / upd_s / 1e9 / hbm_gbs}
    if not args.no_imex:
        line["imex"] = imex_block(args, numa, torch, dev, barrier, max_ranks)
    if not args.no_shell and args.workload != "shell_6x30x30x8_N4":
        # the deep-atmosphere shell (curved elements, per-node form of Eq. 5)
        ws = I.WORKLOADS["shell_6x30x30x8_N4"]
        sh = {"workload": "shell_6x30x30x8_N4", "unit": UNIT, "steps": args.steps, "dt": ws["dt"],
              "form": "per-node (curved elements)"}
        for prec in ("fp64", "fp32_mixed", "fp64_pairs"):
            if prec != "fp64" and args.no_fp32:
                continue
            mss, vols, upds, infos, _, _, fins, _ = measure(prec, wl=ws)
            nl = STAGES * args.steps
            sh[prec] = {"value": whole_job_rate(world, infos["Ng"], args.steps, mss), "ms_per_step": mss / args.steps,
                        "volume_ms_avg": vols / nl, "update_ms_avg": upds / nl, "finite": fins}
            if prec == "fp64":
                fl_e, op_e = volume_fp64_cost(infos["N"], "nodal")
                t_s = vols * 1e-3 / nl
                sh[prec]["roofline"] = {"kernel": f"volume_kernel<{infos['N']},double,nodal>", "bound": "alu",
                                        "achieved": fl_e * infos["Nl"] / t_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                                        "unit": "TFLOP/s",
                                        "frac": fl_e * infos["Nl"] / t_s / 1e12 / FP64_PEAK_TFLOPS,
                                        "fp64_pipe_frac": op_e * infos["Nl"] / t_s / (FP64_PEAK_TFLOPS * 1e12 / 2)}
            if prec == "fp32_mixed":
                b32 = volume_bytes(infos["Nl"], infos["Ng"], 4)
                sh[prec]["speedup_vs_fp64"] = sh[prec]["value"] / sh["fp64"]["value"]
                sh[prec]["volume_hbm_frac"] = b32 / (vols * 1e-3 / nl) / 1e9 / hbm_gbs
        line["shell"] = sh
    if snaps:
        line["precision_forms"] = precision_block(snaps, args)
        snaps.clear()
    if not args.no_serve_block and world == 1:
        line["serving"] = serving_block(args, numa, torch)
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def precision_block(snaps, args):
    """Difference of the FP32-mixed and FP64-pairs states from the FP64 state
    after the same warm-up + timed SSP-RK3 steps from the same initial state:
    per variable, relative L2 and Linf (||a - b|| / ||b||, b the FP64 state).
    The FP64 path itself is held to the oracle by the parity tests; this is
    the precision forms' drift from it on the bench workloads."""
    vars_ = ["rho'", "U_x", "U_y", "U_z", "Theta'"]
    out = {"what": "relative L2 / Linf difference from the FP64 state after the same steps, per variable",
           "steps": args.warmup + args.steps}
    for kind in ("box", "shell"):
        ref = snaps.get(("fp64", kind))
        if ref is None:
            continue
        blk = {}
        for prec in ("fp32_mixed", "fp64_pairs"):
            a = snaps.get((prec, kind))
            if a is None:
                continue
            d = (a - ref)
            res = {}
            for v, name in enumerate(vars_):
                n2, ni = float(ref[v].norm()), float(ref[v].abs().max())
                res[name] = [float(d[v].norm()) / n2 if n2 > 0 else None,
                             float(d[v].abs().max()) / ni if ni > 0 else None]
            blk[prec] = res
        out[kind] = blk
    return out


def imex_block(args, numa, torch, dev, barrier, max_ranks):
    """The 1D-IMEX leapfrog against SSP-RK3 on the thin box (z-columns) and
    the cubed-sphere shell (radial columns), each scheme at a time step it is
    stable at: device time per step, node-updates/s (one element kernel per
    step against three) and model seconds per wall second."""
    from paper_1511_01561_gb300 import inputs as I

    out = {"unit": UNIT, "workloads": {}}
    for name in ("thin_64x64x8_N4", "shell_6x30x30x8_N4"):
        w = I.WORKLOADS[name]

        def timed(scheme, dt, precision="fp64"):
            s = numa.Solver(w["cfg"], precision, device=str(dev))
            s.set_time_scheme(scheme)
            s.init_state(*w["ic"])
            s.run(dt, max(3, args.warmup))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize(dev)
            e0.record(s.stream)
            s.run(dt, args.steps)
            e1.record(s.stream)
            torch.cuda.synchronize(dev)
            barrier()
            ms = max_ranks(e0.elapsed_time(e1))
            vol, upd = s.time_kernels(dt, args.steps)
            finite = s.check_finite() == 0
            ng = s.Ng
            s.close()
            return ms / args.steps, vol / args.steps, upd / args.steps, finite, ng

        dt_i, dt_e = w["dt_imex"], w["dt_explicit"]
        ms_i, vol_i, upd_i, fin_i, ng = timed("imex", dt_i)
        ms_e, vol_e, upd_e, fin_e, _ = timed("ssp3", dt_e)
        ms_p, vol_p, upd_p, fin_p, _ = timed("imex", dt_i, "fp64_pairs")
        r = {
            "global_nodes": ng,
            "leapfrog_imex": {"dt": dt_i, "ms_per_step": ms_i, "finite": fin_i, "volume_ms": vol_i,
                              "dss_plus_column_ms": upd_i, "node_updates_per_s": ng / (ms_i * 1e-3),
                              "model_s_per_s": dt_i / (ms_i * 1e-3)},
            "ssp_rk3": {"dt": dt_e, "ms_per_step": ms_e, "finite": fin_e, "volume_ms_per_stage": vol_e / STAGES,
                        "update_ms_per_stage": upd_e / STAGES,
                        "node_updates_per_s": ng * STAGES / (ms_e * 1e-3), "model_s_per_s": dt_e / (ms_e * 1e-3)},
        }
        r["leapfrog_imex_pairs"] = {"dt": dt_i, "ms_per_step": ms_p, "finite": fin_p, "volume_ms": vol_p,
                                    "dss_plus_column_ms": upd_p, "model_s_per_s": dt_i / (ms_p * 1e-3)}
        r["model_time_speedup"] = r["leapfrog_imex"]["model_s_per_s"] / r["ssp_rk3"]["model_s_per_s"]
        r["model_time_speedup_pairs"] = r["leapfrog_imex_pairs"]["model_s_per_s"] / r["ssp_rk3"]["model_s_per_s"]
        out["workloads"][name] = r
    return out


def serve_streams(numa, reqs, budget, load, overload=0.0, build_threads=8):
    """Serve `reqs` (inputs.serving_stream) with continuous batching: first
    all at once (the saturated request rate), then a Poisson stream at `load`
    times that rate, then (overload > 0) the same arrival gaps at `overload`
    times it.  Per stream: makespan, p50/p99 time-to-forecast (arrival to
    result on the host), aggregate node-updates/s, most members at once."""
    import numpy as np

    def node_count(cfg):
        return (cfg["ne"][0] * cfg["N"] + 1) * (cfg["ne"][1] * cfg["N"] + 1) * (cfg["ne"][2] * cfg["N"] + 1)

    work = sum(node_count(r["cfg"]) * STAGES * r["nsteps"] for r in reqs)

    def serve(arrivals):
        sched = numa.Scheduler(budget, build_threads=build_threads)
        t0 = time.perf_counter()
        pending = sorted(range(len(reqs)), key=lambda i: arrivals[i])
        ids, done_at, max_active = {}, {}, 0
        while len(done_at) < len(reqs):
            now = time.perf_counter() - t0
            while pending and arrivals[pending[0]] <= now:
                i = pending.pop(0)
                r = reqs[i]
                ids[i] = sched.submit(r["cfg"], r["ic"], r["params"], r["dt"], r["nsteps"], r["precision"])
            active, waiting = sched.step()
            max_active = max(max_active, active)
            now = time.perf_counter() - t0
            for i, rid in ids.items():
                if i not in done_at and sched.poll(rid)[0] in ("done", "failed"):
                    done_at[i] = now
            if active == 0 and waiting == 0 and pending:
                time.sleep(max(0.0, min(0.05, arrivals[pending[0]] - now)))
        makespan = max(done_at.values()) - min(arrivals)
        ttf = sorted(done_at[i] - arrivals[i] for i in range(len(reqs)))
        statuses = [sched.poll(ids[i])[0] for i in range(len(reqs))]
        sched.close()
        return dict(makespan_s=makespan, p50_s=float(np.percentile(ttf, 50)), p99_s=float(np.percentile(ttf, 99)),
                    node_updates_per_s=work / makespan, max_active=max_active,
                    failed=sum(st == "failed" for st in statuses))

    sat = serve([0.0] * len(reqs))
    rate = load * len(reqs) / sat["makespan_s"]
    gaps = np.array([r["gap"] for r in reqs]) / rate
    arr = list(np.cumsum(gaps) - gaps[0])
    poi = serve(arr)
    over = None
    if overload > 0:
        over = serve([t * load / overload for t in arr])
        over["load"] = overload
    return dict(saturated=sat, poisson=poi, overload=over, rate=rate, work=work)


def serving_budget(torch, frac: float) -> int:
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    return int(frac * free) // 256 * 256


def serving_block(args, numa, torch):
    """A reduced copy of the serving workload inside the default line: the
    first serve_block_requests requests of the seeded stream, step counts
    scaled by serve_block_steps_scale, saturated then Poisson at serve_load
    times the saturated request rate."""
    from paper_1511_01561_gb300 import inputs as I

    reqs = I.serving_stream(n=args.serve_block_requests)
    for r in reqs:
        r["nsteps"] = max(1, int(round(r["nsteps"] * args.serve_block_steps_scale)))
    budget = serving_budget(torch, args.serve_budget_frac)
    out = serve_streams(numa, reqs, budget, args.serve_load, 0.0, min(8, os.cpu_count() or 1))
    poi = out["poisson"]
    return {"metric": "time-to-forecast p50/p99 (s) and aggregate node-updates/s", "p50_s": poi["p50_s"],
            "p99_s": poi["p99_s"], "node_updates_per_s": poi["node_updates_per_s"], "unit": UNIT,
            "config": {"workload": "bubble ensemble stream", "requests": len(reqs), "seed": 1511,
                       "steps_scale": args.serve_block_steps_scale, "arena_bytes": budget,
                       "poisson_rate_per_s": out["rate"], "load": args.serve_load,
                       "fp32_mixed_requests": sum(r["precision"] == "fp32_mixed" for r in reqs),
                       "total_node_updates": out["work"]},
            "saturated": out["saturated"], "poisson": poi}


def run_serve(args):
    """Ensemble serving: a seeded stream of rising-bubble forecast requests
    (edge 8..48 elements, N in {3, 4, 6}, 100..1000 steps, FP64 or FP32-mixed)
    served with continuous batching.  First all requests at once (saturated
    request rate), then a Poisson stream at serve_load times that rate, then
    one at serve_overload times it (the same arrival gaps, rescaled);
    reports p50/p99 time-to-forecast and aggregate node-updates/s."""
    import torch

    from paper_1511_01561_gb300 import inputs as I
    from paper_1511_01561_gb300 import numa

    torch.cuda.set_device(0)
    budget = serving_budget(torch, args.serve_budget_frac)
    reqs = I.serving_stream(n=args.serve_requests)
    for r in reqs:
        r["nsteps"] = max(1, int(round(r["nsteps"] * args.serve_steps_scale)))
    out = serve_streams(numa, reqs, budget, args.serve_load, args.serve_overload, min(8, os.cpu_count() or 1))
    poi = out["poisson"]
    print(json.dumps({
        "metric": "ensemble time-to-forecast p50/p99 and aggregate node-updates/s", "unit": "s",
        "p50": poi["p50_s"], "p99": poi["p99_s"], "value": poi["node_updates_per_s"],
        "value_unit": UNIT, "higher_is_better": False, "data": "synthetic",
        "config": {"workload": "bubble ensemble stream", "requests": len(reqs), "seed": 1511,
                   "edge": [8, 48], "N": [3, 4, 6], "steps_scale": args.serve_steps_scale,
                   "arena_bytes": budget, "arena_frac_of_free": args.serve_budget_frac,
                   "poisson_rate_per_s": out["rate"], "load": args.serve_load,
                   "fp32_mixed_requests": sum(r["precision"] == "fp32_mixed" for r in reqs),
                   "total_node_updates": out["work"]},
        "saturated": out["saturated"], "poisson": poi, "overload": out["overload"],
    }))


def run_peaks(args):
    """Throughput of the units an element kernel could run on: FP64 and FP32
    FMA chains and FP64 / TF32 mma.sync, each a register-only kernel timed
    with CUDA events (best of three runs of about half a second), with the
    SM clock sampled by nvidia-smi during the runs."""
    import torch

    from paper_1511_01561_gb300 import numa

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nbytes = sms * 8 * 256 * 8
    buf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = {"metric": "arithmetic throughput per unit", "unit": "TFLOP/s", "sms": sms, "units": {}}
    for kind in numa.PEAK_KINDS:
        numa.numa_probe_peak(kind, 16, buf.data_ptr(), nbytes, stream)  # warm-up
        ms, _ = numa.numa_probe_peak(kind, 1000, buf.data_ptr(), nbytes, stream)
        iters = max(1000, int(1000 * 500.0 / max(ms, 1e-3)))
        clocks = ClockSampler(0)
        runs = [numa.numa_probe_peak(kind, iters, buf.data_ptr(), nbytes, stream) for _ in range(3)]
        ck = clocks.stop()
        best = max(r[1] for r in runs)
        d = {"tflops": best, "runs_tflops": [r[1] for r in runs], "ms": [r[0] for r in runs], "iters": iters,
             "clocks": ck}
        if ck and ck.get("sm_mhz"):
            # flops per SM per clock at the median sampled clock
            d["flops_per_sm_per_clock"] = best * 1e12 / (sms * ck["sm_mhz"] * 1e6)
        out["units"][kind] = d
    print(json.dumps(out))


def main():
    args = parse_args()
    if args.cpu_worker:
        cpu_worker(args)
    elif args.peaks:
        run_peaks(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
