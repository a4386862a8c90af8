"""Thin ctypes binding of the C ABI in ``include/numa.h``.

Argument marshalling only: every step of the hot path runs in the CUDA
library ``libnuma_gb300.so``.  Importing this module loads the library and
raises ``ImportError`` if it has not been built -- there is no CPU fallback.
PyTorch is used for device memory (the workspace) and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnuma_gb300.so")

NUMA_OK = 0
ERRORS = {-1: "NUMA_EINVAL", -2: "NUMA_ENOMEM", -3: "NUMA_ECUDA", -4: "NUMA_ENONFINITE",
          -5: "NUMA_ETIMEOUT", -6: "NUMA_EBUDGET", -7: "NUMA_ESTATE"}
MESH = {"box": 0, "shell": 1}
REF = {"isentropic": 0, "isothermal": 1}
METRIC_FORM = {"auto": 0, "nodal": 1}
STORAGE = {"cg": 0, "dg": 1}
PRECISION = {"fp64": 0, "fp32_mixed": 1, "fp64_pairs": 2}
IC = {"rest": 0, "bubble": 1, "uniform": 2, "jetwave": 3}


class NumaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class numa_config(ctypes.Structure):
    _fields_ = [
        ("mesh_kind", ctypes.c_int), ("N", ctypes.c_int),
        ("nex", ctypes.c_int), ("ney", ctypes.c_int), ("nez", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("periodic", ctypes.c_int * 3), ("warp", ctypes.c_double),
        ("npanel", ctypes.c_int), ("nlayer", ctypes.c_int),
        ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double),
        ("Rd", ctypes.c_double), ("cp", ctypes.c_double), ("cv", ctypes.c_double),
        ("P00", ctypes.c_double), ("g", ctypes.c_double), ("Omega", ctypes.c_double),
        ("ref_kind", ctypes.c_int), ("theta0", ctypes.c_double), ("T0", ctypes.c_double),
        ("precision", ctypes.c_int), ("metric_form", ctypes.c_int), ("storage", ctypes.c_int),
    ]


class numa_mesh_info(ctypes.Structure):
    _fields_ = [("Ne", ctypes.c_longlong), ("Nl", ctypes.c_longlong), ("Ng", ctypes.c_longlong),
                ("workspace_bytes", ctypes.c_size_t), ("N", ctypes.c_int), ("dss_entries", ctypes.c_longlong)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1511_01561_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    sig = {
        "numa_create": [ctypes.POINTER(numa_config), ctypes.POINTER(vp)],
        "numa_get_mesh_info": [vp, ctypes.POINTER(numa_mesh_info)],
        "numa_bind": [vp, vp, ctypes.c_size_t, vp],
        "numa_init_state": [vp, i, dp, i],
        "numa_set_state": [vp, vp, i],
        "numa_get_state": [vp, vp, i],
        "numa_rhs": [vp, vp, vp],
        "numa_rhs_static_scratch": [vp, vp, vp],
        "numa_rk_step": [vp, d],
        "numa_run": [vp, d, i],
        "numa_set_filter": [vp, i, i, d, d],
        "numa_set_time_scheme": [vp, i],
        "numa_set_robert_asselin": [vp, d],
        "numa_set_slabs": [vp, i, ctypes.POINTER(i)],
        "numa_filter": [vp],
        "numa_check_finite": [vp, ctypes.POINTER(i)],
        "numa_time_kernels": [vp, d, i, dp, dp],
        "numa_get_coords": [vp, dp],
        "numa_destroy": [vp],
        "numa_sched_create": [vp, ctypes.c_size_t, vp, i, ctypes.POINTER(vp)],
        "numa_sched_submit": [vp, ctypes.POINTER(numa_config), i, dp, i, d, i, ctypes.POINTER(ctypes.c_longlong)],
        "numa_sched_step": [vp, ctypes.POINTER(i), ctypes.POINTER(i)],
        "numa_sched_poll": [vp, ctypes.c_longlong, ctypes.POINTER(i), ctypes.POINTER(i),
                            ctypes.POINTER(ctypes.c_longlong)],
        "numa_sched_result": [vp, ctypes.c_longlong, dp, ctypes.c_longlong],
        "numa_sched_cancel": [vp, ctypes.c_longlong],
        "numa_sched_destroy": [vp],
        "numa_probe_peak": [i, i, vp, ctypes.c_size_t, vp, dp, dp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.numa_last_error.argtypes = [vp]
    L.numa_last_error.restype = ctypes.c_char_p
    L.numa_sched_last_error.argtypes = [vp]
    L.numa_sched_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(ctx, rc: int):
    if rc != NUMA_OK:
        msg = lib.numa_last_error(ctx).decode() if ctx else ""
        raise NumaError(rc, msg)


def make_config(cfg: dict, precision: str = "fp64") -> numa_config:
    c = numa_config()
    c.mesh_kind = MESH[cfg["kind"]]
    c.N = int(cfg["N"])
    c.nex, c.ney, c.nez = (int(v) for v in cfg.get("ne", (1, 1, 1)))
    c.Lx, c.Ly, c.Lz = (float(v) for v in cfg.get("L", (1.0, 1.0, 1.0)))
    for a, p in enumerate(cfg.get("periodic", (0, 0, 0))):
        c.periodic[a] = int(bool(p))
    c.warp = float(cfg.get("warp", 0.0))
    c.npanel = int(cfg.get("npanel", 0))
    c.nlayer = int(cfg.get("nlayer", 0))
    c.r_inner = float(cfg.get("r_inner", 0.0))
    c.r_outer = float(cfg.get("r_outer", 0.0))
    c.Rd, c.cp, c.cv, c.P00 = (float(cfg[k]) for k in ("Rd", "cp", "cv", "P00"))
    c.g = float(cfg["g"])
    c.Omega = float(cfg.get("Omega", 0.0))
    c.ref_kind = REF[cfg.get("ref", "isentropic")]
    c.theta0 = float(cfg.get("theta0", 300.0))
    c.T0 = float(cfg.get("T0", 300.0))
    c.precision = PRECISION[cfg.get("precision", precision)]
    c.metric_form = METRIC_FORM[cfg.get("metric_form", "auto")]
    c.storage = STORAGE[cfg.get("storage", "cg")]
    return c


# ---- C-ABI calls, same names as include/numa.h ---------------------------

def numa_create(cfg: dict, precision: str = "fp64") -> ctypes.c_void_p:
    c = make_config(cfg, precision)
    h = ctypes.c_void_p()
    rc = lib.numa_create(ctypes.byref(c), ctypes.byref(h))
    if rc != NUMA_OK:
        raise NumaError(rc, "numa_create")
    return h


def numa_get_mesh_info(ctx) -> dict:
    info = numa_mesh_info()
    _check(ctx, lib.numa_get_mesh_info(ctx, ctypes.byref(info)))
    return dict(Ne=info.Ne, Nl=info.Nl, Ng=info.Ng, workspace_bytes=info.workspace_bytes, N=info.N,
                dss_entries=info.dss_entries)


def numa_bind(ctx, workspace_ptr: int, nbytes: int, stream_ptr: int) -> None:
    _check(ctx, lib.numa_bind(ctx, ctypes.c_void_p(workspace_ptr), nbytes, ctypes.c_void_p(stream_ptr)))


def numa_init_state(ctx, kind: str, params=()) -> None:
    p = (ctypes.c_double * max(1, len(params)))(*params)
    _check(ctx, lib.numa_init_state(ctx, IC[kind], p, len(params)))


def numa_set_state(ctx, ptr: int, on_device: bool) -> None:
    _check(ctx, lib.numa_set_state(ctx, ctypes.c_void_p(ptr), int(on_device)))


def numa_get_state(ctx, ptr: int, on_device: bool) -> None:
    _check(ctx, lib.numa_get_state(ctx, ctypes.c_void_p(ptr), int(on_device)))


def numa_rhs(ctx, q_ptr: int, r_ptr: int) -> None:
    _check(ctx, lib.numa_rhs(ctx, ctypes.c_void_p(q_ptr), ctypes.c_void_p(r_ptr)))


def numa_rhs_static_scratch(ctx, q_ptr: int, r_ptr: int) -> None:
    """numa_rhs with its residual scratch in the library's fixed device array
    (for callers that cannot allocate device memory)."""
    _check(ctx, lib.numa_rhs_static_scratch(ctx, ctypes.c_void_p(q_ptr), ctypes.c_void_p(r_ptr)))


def numa_rk_step(ctx, dt: float) -> None:
    _check(ctx, lib.numa_rk_step(ctx, dt))


def numa_run(ctx, dt: float, nsteps: int) -> None:
    _check(ctx, lib.numa_run(ctx, dt, nsteps))


RK_SCHEME = {"ssp3": 0, "ls54": 1, "imex": 2}


def numa_set_time_scheme(ctx, scheme: str) -> None:
    _check(ctx, lib.numa_set_time_scheme(ctx, RK_SCHEME[scheme]))


def numa_set_robert_asselin(ctx, nu: float) -> None:
    _check(ctx, lib.numa_set_robert_asselin(ctx, nu))


def numa_set_slabs(ctx, nslabs: int) -> int:
    """Slabs of the pipelined RK step (0: automatic, 1: off); returns the
    slabs in effect."""
    used = ctypes.c_int()
    _check(ctx, lib.numa_set_slabs(ctx, int(nslabs), ctypes.byref(used)))
    return used.value


def numa_set_filter(ctx, every: int, s: int, p: float, mu: float = 1.0) -> None:
    _check(ctx, lib.numa_set_filter(ctx, int(every), int(s), float(p), float(mu)))


def numa_filter(ctx) -> None:
    _check(ctx, lib.numa_filter(ctx))


def numa_time_kernels(ctx, dt: float, nsteps: int):
    """(ms of volume kernels, ms of DSS/update kernels) over nsteps RK3 steps."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib.numa_time_kernels(ctx, dt, nsteps, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def numa_check_finite(ctx) -> int:
    f = ctypes.c_int()
    _check(ctx, lib.numa_check_finite(ctx, ctypes.byref(f)))
    return f.value


PEAK_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp64_mma_m8n8k4": 2, "tf32_mma_m16n8k8": 3,
              "fp64_fma_with_mma": 4}


def numa_probe_peak(kind: str, iters: int, out_ptr: int, out_bytes: int, stream_ptr: int):
    """(ms, TFLOP/s) of one register-only throughput kernel of the given unit."""
    ms, tf = ctypes.c_double(), ctypes.c_double()
    _check(None, lib.numa_probe_peak(PEAK_KINDS[kind], int(iters), ctypes.c_void_p(out_ptr), int(out_bytes),
                                     ctypes.c_void_p(stream_ptr), ctypes.byref(ms), ctypes.byref(tf)))
    return ms.value, tf.value


def numa_get_coords(ctx) -> np.ndarray:
    ng = numa_get_mesh_info(ctx)["Ng"]
    a = np.zeros((3, ng))
    _check(ctx, lib.numa_get_coords(ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return a


def numa_last_error(ctx) -> str:
    return lib.numa_last_error(ctx).decode()


def numa_destroy(ctx) -> None:
    _check(None, lib.numa_destroy(ctx))


# ---- convenience wrapper: torch owns the workspace and the stream ----------

class Solver:
    """One bound context: a device workspace allocated by torch on `device`
    and the current torch stream of that device."""

    def __init__(self, cfg: dict, precision: str = "fp64", device: str = "cuda:0", stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.ctx = numa_create(cfg, precision)
        self.info = numa_get_mesh_info(self.ctx)
        self.Ng = int(self.info["Ng"])
        self.precision = precision
        self.workspace = torch.empty(self.info["workspace_bytes"] + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        numa_bind(self.ctx, self._ws_ptr, self.info["workspace_bytes"], self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            numa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coords(self) -> np.ndarray:
        return numa_get_coords(self.ctx)

    def init_state(self, kind: str, params=()):
        numa_init_state(self.ctx, kind, params)

    def set_state(self, q):
        t = self.torch
        if isinstance(q, np.ndarray):
            q = t.from_numpy(np.ascontiguousarray(q, dtype=np.float64))
        q = q.contiguous()
        assert q.dtype == t.float64 and q.numel() == 5 * self.Ng
        numa_set_state(self.ctx, q.data_ptr(), q.is_cuda)

    def get_state(self, out=None):
        t = self.torch
        if out is None:
            out = t.empty((5, self.Ng), dtype=t.float64)
        numa_get_state(self.ctx, out.data_ptr(), out.is_cuda)
        return out

    def rhs(self, q, out=None):
        t = self.torch
        if isinstance(q, np.ndarray):
            q = t.from_numpy(np.ascontiguousarray(q, dtype=np.float64))
        q = q.to(self.device, dtype=t.float64).contiguous()
        if q.numel() != 5 * self.Ng:
            raise ValueError(f"state must hold 5*Ng = {5 * self.Ng} values")
        if out is None:
            out = t.empty((5, self.Ng), dtype=t.float64, device=self.device)
        if out.numel() != 5 * self.Ng or not out.is_cuda or out.dtype != t.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 CUDA tensor of 5*Ng values")
        numa_rhs(self.ctx, q.data_ptr(), out.data_ptr())
        return out

    def rk_step(self, dt: float):
        numa_rk_step(self.ctx, dt)

    def run(self, dt: float, nsteps: int):
        numa_run(self.ctx, dt, nsteps)

    def set_time_scheme(self, scheme: str):
        """"ssp3" (three-stage SSP-RK3, the default), "ls54" (five-stage
        low-storage RK of order four) or "imex" (leapfrog with implicit
        vertical-column corrections, walled unwarped boxes in FP64)."""
        numa_set_time_scheme(self.ctx, scheme)

    def set_robert_asselin(self, nu: float):
        """Robert-Asselin filter strength of the "imex" scheme (default 0.05)."""
        numa_set_robert_asselin(self.ctx, nu)

    def set_slabs(self, nslabs: int) -> int:
        """Slabs of the pipelined RK step on boxes (0: automatic, 1: off)."""
        return numa_set_slabs(self.ctx, nslabs)

    def set_filter(self, every: int, s: int, p: float, mu: float = 1.0):
        """Boyd-Vandeven filter after every `every`-th step (0: off)."""
        numa_set_filter(self.ctx, every, s, p, mu)

    def filter(self):
        """Apply the filter once to the state now."""
        numa_filter(self.ctx)

    def time_kernels(self, dt: float, nsteps: int):
        return numa_time_kernels(self.ctx, dt, nsteps)

    def check_finite(self) -> int:
        return numa_check_finite(self.ctx)


class HostStepper:
    """Steps from host memory to host memory, pipelined: each submit() copies
    a state from pinned host memory to the device, advances it by nsteps
    steps of the solver's integrator, and copies the result back to pinned
    host memory.  The host-to-device copy of the next state and the
    device-to-host copy of the previous result run on two copy streams of
    their own while the solver's stream computes, so that consecutive
    submits overlap their copies with each other's steps.  Two device
    staging buffers per direction alternate between submits.  synchronize()
    waits until every result has landed; an output buffer may be read only
    after it.  The states go through numa_set_state / numa_get_state
    (device to device) and the steps through numa_rk_step."""

    def __init__(self, solver: "Solver"):
        t = solver.torch
        self.s = solver
        self.t = t
        dev = solver.device
        self.h2d = t.cuda.Stream(dev)
        self.d2h = t.cuda.Stream(dev)
        shape = (5, solver.Ng)
        self.din = [t.empty(shape, dtype=t.float64, device=dev) for _ in range(2)]
        self.dout = [t.empty(shape, dtype=t.float64, device=dev) for _ in range(2)]
        ev = lambda: t.cuda.Event()  # noqa: E731
        self.in_ready, self.in_used = [ev(), ev()], [ev(), ev()]
        self.out_ready, self.out_done = [ev(), ev()], [ev(), ev()]
        for e in self.in_used + self.out_done:
            e.record(solver.stream)
        self.k = 0

    def submit(self, q_host, out_host, dt: float, nsteps: int = 1):
        t, main, i = self.t, self.s.stream, self.k % 2
        ctx = self.s.ctx
        # host -> device staging i, once the step that read it last has copied it in
        self.h2d.wait_event(self.in_used[i])
        with t.cuda.stream(self.h2d):
            self.din[i].copy_(q_host, non_blocking=True)
        self.in_ready[i].record(self.h2d)
        main.wait_event(self.in_ready[i])
        numa_set_state(ctx, self.din[i].data_ptr(), True)
        self.in_used[i].record(main)
        for _ in range(nsteps):
            numa_rk_step(ctx, dt)
        # result -> device staging i (free once its previous copy out is done) -> host
        main.wait_event(self.out_done[i])
        numa_get_state(ctx, self.dout[i].data_ptr(), True)
        self.out_ready[i].record(main)
        self.d2h.wait_event(self.out_ready[i])
        with t.cuda.stream(self.d2h):
            out_host.copy_(self.dout[i], non_blocking=True)
        self.out_done[i].record(self.d2h)
        self.k += 1

    def synchronize(self):
        self.s.stream.synchronize()
        self.h2d.synchronize()
        self.d2h.synchronize()


# ---- serving: continuous batching over one device arena --------------------

REQ_STATUS = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


def _sched_check(s, rc: int):
    if rc != NUMA_OK:
        raise NumaError(rc, lib.numa_sched_last_error(s).decode() if s else "")


def numa_sched_create(arena_ptr: int, arena_bytes: int, stream_ptr: int, build_threads: int = 4):
    h = ctypes.c_void_p()
    rc = lib.numa_sched_create(ctypes.c_void_p(arena_ptr), arena_bytes, ctypes.c_void_p(stream_ptr),
                               build_threads, ctypes.byref(h))
    if rc != NUMA_OK:
        raise NumaError(rc, "numa_sched_create")
    return h


def numa_sched_submit(s, cfg: dict, ic: str, params=(), dt: float = 0.01, nsteps: int = 1,
                      precision: str = "fp64") -> int:
    c = make_config(cfg, precision)
    p = (ctypes.c_double * max(1, len(params)))(*params)
    rid = ctypes.c_longlong()
    _sched_check(s, lib.numa_sched_submit(s, ctypes.byref(c), IC[ic], p, len(params), dt, nsteps, ctypes.byref(rid)))
    return rid.value


def numa_sched_step(s):
    a, w = ctypes.c_int(), ctypes.c_int()
    _sched_check(s, lib.numa_sched_step(s, ctypes.byref(a), ctypes.byref(w)))
    return a.value, w.value


def numa_sched_poll(s, rid: int):
    """(status name, steps done, global-node count) of a request."""
    st, done, ng = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _sched_check(s, lib.numa_sched_poll(s, rid, ctypes.byref(st), ctypes.byref(done), ctypes.byref(ng)))
    return REQ_STATUS.get(st.value, st.value), done.value, ng.value


def numa_sched_result(s, rid: int, Ng: int) -> np.ndarray:
    q = np.zeros((5, Ng))
    _sched_check(s, lib.numa_sched_result(s, rid, q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 5 * Ng))
    return q


def numa_sched_cancel(s, rid: int) -> None:
    _sched_check(s, lib.numa_sched_cancel(s, rid))


def numa_sched_destroy(s) -> None:
    _sched_check(None, lib.numa_sched_destroy(s))


class Scheduler:
    """Continuous-batching ensemble server on one GPU: a torch-owned device
    arena of `arena_bytes` holds every admitted member's workspace."""

    def __init__(self, arena_bytes: int, device: str = "cuda:0", build_threads: int = 4, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device=self.device)
        base = (self.arena.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = numa_sched_create(base, int(arena_bytes), self.stream.cuda_stream, build_threads)

    def submit(self, cfg: dict, ic: str, params=(), dt: float = 0.01, nsteps: int = 1, precision: str = "fp64"):
        return numa_sched_submit(self.h, cfg, ic, params, dt, nsteps, precision)

    def step(self):
        """(active members, waiting requests) after one scheduler step."""
        return numa_sched_step(self.h)

    def poll(self, rid: int):
        """(status, steps done, Ng)."""
        return numa_sched_poll(self.h, rid)

    def result(self, rid: int) -> np.ndarray:
        return numa_sched_result(self.h, rid, self.poll(rid)[2])

    def cancel(self, rid: int):
        numa_sched_cancel(self.h, rid)

    def close(self):
        if getattr(self, "h", None):
            numa_sched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
