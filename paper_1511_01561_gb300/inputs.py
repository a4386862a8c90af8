"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
harness.

This module holds workload descriptions (mesh sizes, physical constants,
initial-condition parameters, time steps) and seeded random numbers only.  It
contains none of the method's arithmetic: no geometry, no reference state, no
equation of state, no fluxes.  Both the GPU library and the oracle build
everything else from these descriptions independently.

Physical constants (the paper gives none): dry air R = 287, cp = 1004.5,
cv = cp - R = 717.5, P00 = 1e5 Pa; g = 9.81 in the box; Earth radius
6.37122e6 m, surface gravity 9.80616, rotation 7.292e-5 /s on the shell, whose
reference atmosphere is isothermal at 250 K (an isentropic 300 K atmosphere
would reach zero Exner pressure near 30.7 km, just above the 30 km lid).
"""
from __future__ import annotations

import math

import numpy as np

PHYS_BOX = dict(Rd=287.0, cp=1004.5, cv=717.5, P00=1.0e5, g=9.81, Omega=0.0,
                ref="isentropic", theta0=300.0, T0=300.0)

EARTH_RADIUS = 6.37122e6
PHYS_SHELL = dict(Rd=287.0, cp=1004.5, cv=717.5, P00=1.0e5, g=9.80616, Omega=7.292e-5,
                  ref="isothermal", theta0=300.0, T0=250.0,
                  r_inner=EARTH_RADIUS, r_outer=EARTH_RADIUS + 30.0e3)

# rising thermal bubble: amplitude 0.5 K, radius 250 m, centre (500, 500, 350) m
BUBBLE_PARAMS = (0.5, 250.0, 500.0, 500.0, 350.0)
# zonal jet 35 m/s with a 1 m/s Gaussian bump of radius a/10 at (0 E, 45 N)
JETWAVE_PARAMS = (35.0, 1.0, 0.1, 0.0, math.pi / 4.0)


def box(ne, N, L=1000.0, periodic=(0, 0, 0), warp=0.0, **over) -> dict:
    """A box mesh description: ne elements per axis (int or 3-tuple)."""
    if isinstance(ne, int):
        ne = (ne, ne, ne)
    if isinstance(L, (int, float)):
        L = (float(L),) * 3
    cfg = dict(kind="box", N=int(N), ne=tuple(int(v) for v in ne), L=tuple(L),
               periodic=tuple(int(bool(p)) for p in periodic), warp=float(warp), **PHYS_BOX)
    cfg.update(over)
    return cfg


def shell(npanel, nlayer, N, **over) -> dict:
    """A cubed-sphere shell: npanel x npanel columns per cube face, nlayer layers."""
    cfg = dict(kind="shell", N=int(N), npanel=int(npanel), nlayer=int(nlayer), **PHYS_SHELL)
    cfg.update(over)
    return cfg


WORKLOADS = {
    # 3D rising thermal bubble, 1000 m box, 4^3 elements, N=4, 100 steps
    "bubble_4x4x4_N4": dict(cfg=box(4, 4), ic=("bubble", BUBBLE_PARAMS), dt=0.01, steps=100),
    # same bubble at 32^3 elements (129^3 global nodes), 200 steps
    "bubble_32x32x32_N4": dict(cfg=box(32, 4), ic=("bubble", BUBBLE_PARAMS), dt=0.01, steps=200),
    # deep-atmosphere shell, 6 x 30 x 30 columns, 8 layers to 30 km, N=4, 500 steps
    # (1D-IMEX: dt_imex = 12 s puts the vertical acoustic Courant number near
    # 6.4, as in the paper's baroclinic runs; SSP-RK3 is stable to about 2 s)
    "shell_6x30x30x8_N4": dict(cfg=shell(30, 8, 4), ic=("jetwave", JETWAVE_PARAMS), dt=1.0, steps=500,
                               dt_imex=12.0, dt_explicit=2.0),
    # thin box for the 1D-IMEX leapfrog: 16 km x 16 km x 1 km elements (the
    # aspect of the paper's baroclinic-wave runs), 257 x 257 x 33 global nodes,
    # a 0.5 K bubble of radius 30 km; dt = 2 s puts the vertical acoustic
    # Courant number near 4, SSP-RK3 needs dt <= 0.6 s on these elements
    "thin_64x64x8_N4": dict(cfg=box((64, 64, 8), 4, L=(1024e3, 1024e3, 8e3)),
                            ic=("bubble", (0.5, 30e3, 512e3, 512e3, 4e3)), dt=2.0, steps=100,
                            dt_imex=2.0, dt_explicit=0.5),
}


def serving_stream(n: int = 64, seed: int = 1511, edge=(8, 48), orders=(3, 4, 6), amp=(0.1, 2.0),
                   steps=(100, 1000), p_fp32: float = 0.5, L: float = 1000.0, r_c: float = 250.0) -> list:
    """Forecast requests of the ensemble-serving workload: rising-bubble boxes
    with edge ~ U{edge} elements per axis, order from `orders`, amplitude
    ~ U(amp) K, centre uniform in the box at least r_c from every wall, step
    count ~ U{steps}, FP32-mixed with probability p_fp32.  `gap` is the
    request's exponential inter-arrival gap in units of the mean gap (a
    Poisson stream once scaled by a rate).  The time step keeps an acoustic
    Courant number of 0.5 on the closest node pair, taken as
    (L/edge)(1 - cos(pi/N))/2 at 350 m/s (at most 0.01 s)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ne = int(rng.integers(edge[0], edge[1] + 1))
        N = int(rng.choice(orders))
        A = float(rng.uniform(*amp))
        c = rng.uniform(r_c, L - r_c, 3)
        nsteps = int(rng.integers(steps[0], steps[1] + 1))
        prec = "fp32_mixed" if rng.random() < p_fp32 else "fp64"
        gap = float(rng.exponential(1.0))
        dx_min = (L / ne) * 0.5 * (1.0 - math.cos(math.pi / N))
        dt = min(0.01, 0.5 * dx_min / 350.0)
        out.append(dict(cfg=box(ne, N), ic="bubble", params=(A, r_c, float(c[0]), float(c[1]), float(c[2])),
                        dt=dt, nsteps=nsteps, precision=prec, gap=gap))
    return out


def random_perturbation(Ng: int, seed: int, rho=0.01, U=5.0, Theta=1.0) -> np.ndarray:
    """Uniform random nodal perturbations [5][Ng] of (rho', U_x, U_y, U_z, Theta')."""
    rng = np.random.default_rng(seed)
    q = np.empty((5, Ng))
    q[0] = rng.uniform(-rho, rho, Ng)
    q[1:4] = rng.uniform(-U, U, (3, Ng))
    q[4] = rng.uniform(-Theta, Theta, Ng)
    return q


def smooth_perturbation(xyz: np.ndarray, seed: int, length: float, rho=0.01, U=5.0, Theta=1.0,
                        modes: int = 3) -> np.ndarray:
    """Smooth random field [5][Ng]: a few random Fourier modes of wavelength
    about `length`, evaluated at the given node coordinates [3][Ng]."""
    rng = np.random.default_rng(seed)
    amps = (rho, U, U, U, Theta)
    q = np.zeros((5, xyz.shape[1]))
    for v in range(5):
        for _ in range(modes):
            k = rng.normal(size=3) * (2.0 * math.pi / length)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            q[v] += amps[v] / modes * np.sin(k @ xyz + ph)
    return q
