"""ctypes wrapper of the plain FP64 CPU oracle (``numa_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the independent reference of the
CG spectral-element right-hand side, DSS, inverse mass matrix and SSP-RK3
stage (Mueller et al., Sec. 2, Eqs. 1-5).  Only the test suite, the smoke
check and the CPU-baseline leg of the benchmark may import this module.  It
shares no code with the GPU library and never imports it.

Configs are plain dicts (see ``paper_1511_01561_gb300.inputs``); arrays are
numpy float64 in the layouts documented in ``numa_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "numa_oracle.c")
_SO = os.path.join(_HERE, "liborc.so")

BOX, SHELL = 0, 1
IC = {"rest": 0, "bubble": 1, "uniform": 2, "jetwave": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
               "-o", _SO, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
    return _SO


class _Config(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("N", ctypes.c_int),
        ("nex", ctypes.c_int), ("ney", ctypes.c_int), ("nez", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("periodic", ctypes.c_int * 3), ("warp", ctypes.c_double),
        ("npanel", ctypes.c_int), ("nlayer", ctypes.c_int),
        ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double),
        ("Rd", ctypes.c_double), ("cp", ctypes.c_double), ("cv", ctypes.c_double),
        ("P00", ctypes.c_double), ("g", ctypes.c_double), ("Omega", ctypes.c_double),
        ("ref_kind", ctypes.c_int), ("theta0", ctypes.c_double), ("T0", ctypes.c_double),
    ]


RHS_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double))

_lib_handle = None


def _load_lib(path: str):
    """Load an oracle shared library and declare its signatures."""
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_lgl.argtypes = [ctypes.c_int, dp, dp]
    L.orc_dmatrix.argtypes = [ctypes.c_int, dp, dp]
    L.orc_build.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_void_p)]
    L.orc_build.restype = ctypes.c_int
    L.orc_free.argtypes = [ctypes.c_void_p]
    L.orc_sizes.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_long)] * 3
    for name in ("orc_get_coords", "orc_get_elem_coords", "orc_get_metrics", "orc_get_jw",
                 "orc_get_mass", "orc_get_ref"):
        getattr(L, name).argtypes = [ctypes.c_void_p, dp]
    L.orc_get_l2g.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_long)]
    L.orc_get_wall.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ubyte)]
    L.orc_pprime.argtypes = [ctypes.c_double] * 4
    L.orc_pprime.restype = ctypes.c_double
    L.orc_pprime_naive.argtypes = [ctypes.c_double] * 3 + [ctypes.POINTER(_Config)]
    L.orc_pprime_naive.restype = ctypes.c_double
    L.orc_init_state.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp]
    L.orc_init_state.restype = ctypes.c_int
    L.orc_rhs_elem.argtypes = [ctypes.c_void_p, dp, dp]
    L.orc_rhs.argtypes = [ctypes.c_void_p, dp, dp]
    L.orc_ssprk3_step.argtypes = [ctypes.c_long, dp, ctypes.c_double, RHS_FN, ctypes.c_void_p, dp]
    L.orc_run.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_int]
    L.orc_run.restype = ctypes.c_int
    L.orc_lsrk54_coefficients.argtypes = [dp, dp]
    L.orc_lsrk54_step.argtypes = [ctypes.c_long, dp, ctypes.c_double, RHS_FN, ctypes.c_void_p, dp]
    L.orc_run_lsrk54.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_int]
    L.orc_run_lsrk54.restype = ctypes.c_int
    L.orc_filter_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
    L.orc_filter_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
    L.orc_filter_matrix.restype = ctypes.c_int
    L.orc_filter.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.orc_filter.restype = ctypes.c_int
    L.orc_run_filtered.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.orc_run_filtered.restype = ctypes.c_int
    return L


def lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        _lib_handle = _load_lib(_SO)
    return _lib_handle


def build_variant(edits, tag: str) -> str:
    """Compile a copy of the oracle with textual edits [(old, new), ...]
    applied, each old snippet occurring exactly once.  The tests plant
    mistakes this way, to show that a pin catches them; the variant goes to
    a temporary directory, never next to the real oracle."""
    import tempfile

    with open(_SRC) as f:
        src = f.read()
    for old, new in edits:
        n = src.count(old)
        if n != 1:
            raise ValueError(f"edit target occurs {n} times: {old!r}")
        src = src.replace(old, new)
    d = tempfile.mkdtemp(prefix=f"orc_{tag}_")
    c_path = os.path.join(d, "numa_oracle.c")
    with open(c_path, "w") as f:
        f.write(src)
    with open(os.path.join(_HERE, "numa_oracle.h")) as f:
        hdr = f.read()
    with open(os.path.join(d, "numa_oracle.h"), "w") as f:
        f.write(hdr)
    so = os.path.join(d, "liborc_variant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", so,
                    c_path, "-lm"], check=True, cwd=d)
    return so


class using_library:
    """Context manager: every oracle call made inside it (Mesh objects built
    inside it included) goes to the library at `path`."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib_handle
        self._saved = lib()
        _lib_handle = _load_lib(self.path)
        return _lib_handle

    def __exit__(self, *exc):
        global _lib_handle
        _lib_handle = self._saved
        return False


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_config(cfg: dict) -> _Config:
    c = _Config()
    c.kind = BOX if cfg["kind"] == "box" else SHELL
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
    c.ref_kind = 0 if cfg.get("ref", "isentropic") == "isentropic" else 1
    c.theta0 = float(cfg.get("theta0", 300.0))
    c.T0 = float(cfg.get("T0", 300.0))
    return c


def lgl(N: int):
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    lib().orc_lgl(N, _dp(xi), _dp(w))
    return xi, w


def dmatrix(N: int) -> np.ndarray:
    xi, _ = lgl(N)
    D = np.zeros((N + 1) * (N + 1))
    lib().orc_dmatrix(N, _dp(xi), _dp(D))
    return D.reshape(N + 1, N + 1)


def filter_weights(N: int, s: int, p: float, mu: float = 1.0) -> np.ndarray:
    """Boyd-Vandeven weights of the Legendre modes 0..N (Sec. 2.3)."""
    sigma = np.zeros(N + 1)
    lib().orc_filter_weights(N, s, p, mu, _dp(sigma))
    return sigma


def filter_matrix(N: int, s: int, p: float, mu: float = 1.0) -> np.ndarray:
    """1D filter matrix F = V diag(sigma) V^-1 on the Lobatto points."""
    F = np.zeros((N + 1) * (N + 1))
    if lib().orc_filter_matrix(N, s, p, mu, _dp(F)) != 0:
        raise ValueError("bad filter")
    return F.reshape(N + 1, N + 1)


def pprime(Th_pert: float, Th0: float, p0: float, gamma: float) -> float:
    return lib().orc_pprime(Th_pert, Th0, p0, gamma)


def pprime_naive(Th_pert: float, Th0: float, p0: float, cfg: dict) -> float:
    c = make_config(cfg)
    return lib().orc_pprime_naive(Th_pert, Th0, p0, ctypes.byref(c))


def ssprk3_step(q: np.ndarray, dt: float, f) -> np.ndarray:
    """One SSP-RK3 step of dq/dt = f(q) using the oracle's stage code."""
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    n = q.size

    def cb(_ctx, qp, rp):
        qa = np.ctypeslib.as_array(qp, shape=(n,))
        ra = np.ctypeslib.as_array(rp, shape=(n,))
        ra[:] = f(qa.copy())

    fn = RHS_FN(cb)
    work = np.zeros(3 * n)
    lib().orc_ssprk3_step(n, _dp(q), dt, fn, None, _dp(work))
    return q


def lsrk54_step(q: np.ndarray, dt: float, f) -> np.ndarray:
    """One step of the five-stage low-storage RK of dq/dt = f(q)."""
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    n = q.size

    def cb(_ctx, qp, rp):
        qa = np.ctypeslib.as_array(qp, shape=(n,))
        ra = np.ctypeslib.as_array(rp, shape=(n,))
        ra[:] = f(qa.copy())

    fn = RHS_FN(cb)
    work = np.zeros(2 * n)
    lib().orc_lsrk54_step(n, _dp(q), dt, fn, None, _dp(work))
    return q


def lsrk54_coefficients():
    A = np.zeros(5)
    B = np.zeros(5)
    lib().orc_lsrk54_coefficients(_dp(A), _dp(B))
    return A, B


class Mesh:
    """An oracle mesh with its geometry, maps, mass matrix and reference state."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self._L = lib()  # the library this mesh was built with serves all its calls
        h = ctypes.c_void_p()
        rc = self._L.orc_build(ctypes.byref(self._c), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle mesh build failed (rc={rc})")
        self._h = h
        ne, nl, ng = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        self._L.orc_sizes(h, ctypes.byref(ne), ctypes.byref(nl), ctypes.byref(ng))
        self.Ne, self.Nl, self.Ng = ne.value, nl.value, ng.value
        self.N = int(cfg["N"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_free(h)
            self._h = None

    def _get(self, name, shape):
        a = np.zeros(shape)
        getattr(self._L, name)(self._h, _dp(a))
        return a

    def coords(self):
        return self._get("orc_get_coords", (3, self.Ng))

    def elem_coords(self):
        return self._get("orc_get_elem_coords", (3, self.Nl))

    def metrics(self):
        """[10][Nl]: dxi_d/dx_c at row 3*d+c, then J."""
        return self._get("orc_get_metrics", (10, self.Nl))

    def jw(self):
        return self._get("orc_get_jw", (self.Nl,))

    def mass(self):
        return self._get("orc_get_mass", (self.Ng,))

    def ref(self):
        """[3][Ng]: rho0, (rho theta)_0, p0."""
        return self._get("orc_get_ref", (3, self.Ng))

    def l2g(self):
        a = np.zeros(self.Nl, dtype=np.int64)
        self._L.orc_get_l2g(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
        return a

    def wall(self):
        a = np.zeros(self.Ng, dtype=np.uint8)
        self._L.orc_get_wall(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return a

    def init_state(self, kind: str, params=()) -> np.ndarray:
        q = np.zeros((5, self.Ng))
        p = np.zeros(8)
        p[: len(params)] = params
        rc = self._L.orc_init_state(self._h, IC[kind], _dp(p), _dp(q))
        if rc != 0:
            raise ValueError(f"oracle init_state failed (rc={rc})")
        return q

    def rhs_elem(self, q: np.ndarray) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        re = np.zeros((5, self.Nl))
        self._L.orc_rhs_elem(self._h, _dp(q), _dp(re))
        return re

    def rhs(self, q: np.ndarray) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        R = np.zeros((5, self.Ng))
        self._L.orc_rhs(self._h, _dp(q), _dp(R))
        return R

    def run(self, q: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        rc = self._L.orc_run(self._h, _dp(q), dt, nsteps)
        if rc != 0:
            raise MemoryError("oracle run failed")
        return q

    def run_lsrk54(self, q: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
        """nsteps steps of the five-stage low-storage RK."""
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        if self._L.orc_run_lsrk54(self._h, _dp(q), dt, nsteps) != 0:
            raise MemoryError("oracle run failed")
        return q

    def filter(self, q: np.ndarray, s: int, p: float, mu: float = 1.0) -> np.ndarray:
        """One application of the Boyd-Vandeven filter with DSS (Sec. 7 loop)."""
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        if self._L.orc_filter(self._h, _dp(q), s, p, mu) != 0:
            raise ValueError("oracle filter failed")
        return q

    def run_filtered(self, q: np.ndarray, dt: float, nsteps: int, every: int, s: int, p: float,
                     mu: float = 1.0) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64).copy()
        if self._L.orc_run_filtered(self._h, _dp(q), dt, nsteps, every, s, p, mu) != 0:
            raise ValueError("oracle filtered run failed")
        return q
