"""Host logic of bench.py that needs no GPU: the algorithmic byte and flop
models behind the roofline, the whole-job rate, the command line, and the
rule that a committed ncu traffic figure is reported only for the workload
and kernel sources it was captured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_flop_models():
    # the 12 flux fields come gathered (formed once per global node by the
    # update).  Per-node form at N=4: 12 fields x 3 directions x 5 terms (the
    # first a product) and 15 chain-rule triples (the first of each of the 5
    # equations a product and two FMAs)
    fl, ops = bench.volume_fp64_cost(4, "nodal")
    assert ops == 12 * 3 * 5 + 15 * 3
    assert fl == 12 * 3 * (1 + 4 * 2) + 5 * (1 + 2 * 2) + 10 * 3 * 2
    # rectilinear form at N=4: 5 equations x 15 terms (the first a product);
    # K_d D: 75 products per 125 nodes (the weight w_i w_j w_k is applied in
    # the update)
    fl, ops = bench.volume_fp64_cost(4, "rect")
    assert ops == 5 * 15 + 75 / 125
    assert fl == 5 * (1 + 14 * 2) + 75 / 125
    assert bench.volume_flops_per_elem_node(4, affine=True) == bench.volume_fp64_cost(4, "rect")[0]
    for N in range(1, 9):
        assert bench.volume_fp64_cost(N, "rect")[1] < bench.volume_fp64_cost(N, "nodal")[1]


def test_byte_models():
    Nl, Ng, N = 4_096_000, 2_146_689, 4
    # FP64 affine: Jw 8 + l2g 4 + residual 40 per element node, 72 per element, 64 per global node
    assert bench.volume_bytes(Nl, Ng, 8, N, True) == Nl * 52 + Nl // 125 * 72 + Ng * 64
    # per-node form reads all ten metric values at every element node
    assert bench.volume_bytes(Nl, Ng, 8) - bench.volume_bytes(Nl, Ng, 8, N, True) == Nl * 72 - Nl // 125 * 72
    # FP64 gathers U and the nine flux components (12 doubles per global node)
    assert bench.volume_bytes(Nl, Ng, 8, N, True, gathered=12) - bench.volume_bytes(Nl, Ng, 8, N, True) == Ng * 32
    # the FP64 update writes 72 B of flux components per node, FP32-mixed 32 B
    assert bench.update_bytes(Nl, Ng, 8, 0) - bench.update_bytes(Nl, Ng, 8, 0, prim=32) == Ng * 40
    # the DSS map of CG storage has one entry per element node; DG storage more
    cg = bench.update_bytes(Nl, Ng, 8, 2 / 3)
    assert bench.update_bytes(Nl, Ng, 8, 2 / 3, entries=Nl) == cg
    assert bench.update_bytes(Nl, Nl, 8, 2 / 3, entries=10_941_048) > cg


def test_stage_byte_model():
    # the stage byte model on the 32^3 bubble: 842 MB per FP64 stage,
    # 678 MB with FP32 metric terms
    Nl, Ng = 4_096_000, 2_146_689
    assert round(bench.stage_bytes_model(Nl, Ng, 8) / 1e6) == 842
    assert round(bench.stage_bytes_model(Nl, Ng, 4) / 1e6) == 678


def test_reading_of_the_papers_performance_model():
    """Tables 1 and 2 (Sec. 6) read as totals per BG/Q node over the whole
    bubble run: their intensity and optimal-runtime rows follow from the flop
    and traffic rows under that reading, and per grid point and right-hand
    side the CG column is 905 flops and 641 + 199 B (1305 B with scattered
    access).  The stage byte model of this library is less than half of
    that at the paper's p = 3."""
    import json

    with open(os.path.join(ROOT, "tests", "golden", "paper_performance_model.json")) as f:
        g = json.load(f)
    w = g["workload"]
    assert w["rhs_evaluations"] == 5 * w["time_steps"]
    per_point_rhs = w["grid_points"] / w["nodes"] * w["rhs_evaluations"]
    for table in ("table1", "table2"):
        for col in g[table].values():
            traffic = col["read_gb"] + col["write_gb"]
            assert abs(col["gflops"] / traffic - col["intensity"]) <= 0.005
            assert abs(traffic / w["stream_gbs"] - col["runtime_s"]) <= 0.005
    cg, cg_scattered = g["table1"]["CG"], g["table2"]["CG"]
    assert round(cg["gflops"] * 1e9 / per_point_rhs) == 905
    assert [round(cg[k] * 1e9 / per_point_rhs) for k in ("read_gb", "write_gb")] == [641, 199]
    assert round((cg_scattered["read_gb"] + cg_scattered["write_gb"]) * 1e9 / per_point_rhs) == 1305
    # 32^3 elements at N = 3: 425 B per global node and stage in FP64
    N, ne = 3, 32
    Nl, Ng = ne**3 * (N + 1) ** 3, (ne * N + 1) ** 3
    ours = bench.stage_bytes_model(Nl, Ng, 8) / Ng
    assert round(ours) == 425
    assert ours < 0.55 * (cg["read_gb"] + cg["write_gb"]) * 1e9 / per_point_rhs


def test_whole_job_rate():
    # node-updates per RK stage of all replicas: world * Ng * 3 stages * steps / seconds
    assert bench.whole_job_rate(1, 1000, 10, 1000.0) == pytest.approx(30_000.0)
    assert bench.whole_job_rate(4, 1000, 10, 1000.0) == pytest.approx(120_000.0)


def test_command_line():
    a = bench.parse_args([])
    assert (a.gpus, a.impl, a.workload) == (1, "mine", "bubble_32x32x32_N4")
    assert a.warmup >= 3 and not a.imex_only and not a.no_dg and not a.no_imex
    b = bench.parse_args(["--imex-only", "--no-dg", "--no-imex", "--steps", "7", "--warmup", "4"])
    assert b.imex_only and b.no_dg and b.no_imex and (b.steps, b.warmup) == (7, 4)
    with pytest.raises(SystemExit):
        bench.parse_args(["--impl", "other"])


def test_traffic_only_for_its_workload_and_sources(monkeypatch):
    wl = bench.NCU_TRAFFIC["workload"]
    key = "volume_fp64_affine"
    if bench.kernel_source_hash() == bench.NCU_TRAFFIC["kernels_sha256_16"]:
        assert bench.ncu_traffic(key, wl) == bench.NCU_TRAFFIC[key]
    assert bench.ncu_traffic(key, "shell_6x30x30x8_N4") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic(key, wl) is None


def test_kernel_source_hash_ignores_comments_only():
    src = 'int a = 1; // one\n/* two\n lines */ const char* s = "x//y";\n\n  // only\nb();\n'
    assert bench.code_lines(src) == ["int a = 1;", 'const char* s = "x//y";', "b();"]
    assert bench.code_lines(src.replace("b()", "c()")) != bench.code_lines(src)


def test_kernel_source_hash_covers_the_kernel_files():
    csrc = os.path.join(ROOT, "paper_1511_01561_gb300", "csrc")
    for name in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
