"""CPU checks of the C-ABI library: it loads, exports every function that
include/numa.h declares, validates arguments without a GPU, and its host mesh
setup agrees with the oracle's node coordinates."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1511_01561_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def numa():
    from paper_1511_01561_gb300 import build
    build.build()
    from paper_1511_01561_gb300 import numa as mod
    return mod


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(numa_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(numa):
    names = _declared("numa.h")
    assert "numa_rhs" in names and "numa_run" in names
    for n in names:
        assert hasattr(numa.lib, n), n
    for h in os.listdir(os.path.join(ROOT, "include")):
        for n in _declared(h):
            assert hasattr(numa.lib, n), (h, n)


def test_config_struct_matches_header(numa):
    src = open(os.path.join(ROOT, "include", "numa.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} numa_config;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]
        for nm in names.split(","):
            fields.append(re.sub(r"\[.*\]", "", nm).strip())
    assert fields == [f[0] for f in numa.numa_config._fields_]


@pytest.mark.parametrize("cfg", [I.box((3, 2, 4), 4), I.box((2, 3, 2), 3, periodic=(1, 0, 1), warp=0.05)])
def test_host_mesh_matches_oracle_coordinates(numa, orc, cfg):
    ctx = numa.numa_create(cfg)
    try:
        info = numa.numa_get_mesh_info(ctx)
        m = orc.Mesh(cfg)
        assert (info["Ne"], info["Nl"], info["Ng"]) == (m.Ne, m.Nl, m.Ng)
        assert np.abs(numa.numa_get_coords(ctx) - m.coords()).max() < 1e-9
    finally:
        numa.numa_destroy(ctx)


def test_shell_sizes_match_oracle(numa, orc):
    cfg = I.shell(3, 2, 3)
    ctx = numa.numa_create(cfg)
    try:
        info = numa.numa_get_mesh_info(ctx)
        m = orc.Mesh(cfg)
        assert (info["Ne"], info["Nl"], info["Ng"]) == (m.Ne, m.Nl, m.Ng)
        a = numa.numa_get_coords(ctx)
        b = m.coords()
        ka = np.lexsort(np.round(a / 1e-3))
        kb = np.lexsort(np.round(b / 1e-3))
        assert np.abs(a[:, ka] - b[:, kb]).max() < 1e-6
    finally:
        numa.numa_destroy(ctx)


def test_argument_errors_without_gpu(numa):
    with pytest.raises(numa.NumaError) as e:
        numa.numa_create(I.box(2, 9))
    assert e.value.code == -1
    with pytest.raises(numa.NumaError):
        numa.numa_create(I.box(0, 4))
    ctx = numa.numa_create(I.box(2, 2))
    try:
        with pytest.raises(numa.NumaError) as e:
            numa.numa_rhs(ctx, 256, 512)
        assert e.value.code == -7  # NUMA_ESTATE: not bound
        with pytest.raises(numa.NumaError) as e:
            numa.numa_bind(ctx, 0, 1 << 20, 0)
        assert e.value.code == -1
        with pytest.raises(numa.NumaError) as e:
            numa.numa_bind(ctx, 256, 16, 0)
        assert e.value.code == -2  # workspace too small
        assert "workspace" in numa.numa_last_error(ctx)
        # the filter can be configured before binding; bad parameters are refused
        numa.numa_set_filter(ctx, 1, 2, 12.0, 0.5)
        for bad in ((-1, 2, 12.0, 1.0), (1, 4, 12.0, 1.0), (1, 2, -3.0, 1.0), (1, 2, 12.0, -0.1)):
            with pytest.raises(numa.NumaError) as e:
                numa.numa_set_filter(ctx, *bad)
            assert e.value.code == -1
        with pytest.raises(numa.NumaError) as e:
            numa.numa_filter(ctx)
        assert e.value.code == -7  # not bound
        numa.numa_set_time_scheme(ctx, "ls54")
        numa.numa_set_time_scheme(ctx, "ssp3")
        assert numa.lib.numa_set_time_scheme(ctx, 7) == -1
    finally:
        numa.numa_destroy(ctx)
    assert numa.lib.numa_destroy(None) == -1
    assert numa.lib.numa_rhs(None, None, None) == -1


def test_meshes_beyond_32_bit_indices_are_refused(numa):
    """Node indices are 32-bit: a mesh with 2^31 or more element nodes is
    refused (NUMA_EINVAL) from its configuration, before any of its arrays is
    built (so at once, without the tens of GB its host arrays would take).
    At N=4 (125 element nodes per element) the largest cubic box below the
    limit has 258^3 elements."""
    import time
    assert 258 ** 3 * 125 < 2 ** 31 <= 259 ** 3 * 125
    for cfg in (I.box(259, 4), I.box((1024, 1024, 17), 4), I.shell(200, 100, 4)):
        ne = (6 * cfg["npanel"] ** 2 * cfg["nlayer"] if cfg["kind"] == "shell"
              else cfg["ne"][0] * cfg["ne"][1] * cfg["ne"][2])
        assert ne * (cfg["N"] + 1) ** 3 >= 2 ** 31  # never build a mesh of that size here
        t0 = time.perf_counter()
        with pytest.raises(numa.NumaError) as e:
            numa.numa_create(cfg)
        assert e.value.code == -1
        assert time.perf_counter() - t0 < 1.0


@pytest.mark.parametrize("cfg,want,expect", [
    (dict(I.box(32, 4), precision="fp32_mixed"), 0, 3),  # FP32-mixed, 2.1M nodes: three by default
    (I.box(32, 4), 0, 1),                       # FP64: none by default
    (I.box((4, 4, 8), 4), 0, 1),                # small mesh: none by default
    (I.box((4, 4, 8), 4), 4, 4),
    (I.box((4, 4, 8), 4), 16, 8),               # at most one slab per element layer
    (I.box((4, 4, 8), 1), 4, 1),                # slabs thinner than two node planes
    (I.box((4, 4, 8), 4, periodic=(0, 0, 1)), 4, 1),  # periodic seam in z
    (I.box((2, 2, 8), 4), 4, 1),                # planes of fewer than 128 nodes
    (I.shell(2, 2, 3), 4, 1),
    (dict(I.box((4, 4, 8), 4), storage="dg"), 4, 1),
])
def test_slab_plan(numa, cfg, want, expect):
    """numa_set_slabs before numa_bind reports the slabs the bind will use
    (host logic only: no GPU call)."""
    ctx = numa.numa_create(cfg)
    try:
        assert numa.numa_set_slabs(ctx, want) == expect
        with pytest.raises(numa.NumaError):
            numa.numa_set_slabs(ctx, 17)
    finally:
        numa.numa_destroy(ctx)
