"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun would start
them.  The workload is replicated per GPU (no data-path collective), so the
multi-rank logic is the barrier, the max over ranks of the timed region, the
whole-job rate, and the reference arm staying silent on ranks other than 0."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        dist.barrier()
        ms = bench.max_over_ranks(dist, local_ms)
        rate = bench.whole_job_rate(world, 1000, 7, ms)
        # the reference arm prints only on rank 0
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"]))
        out[rank] = (ms, rate, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        ms, rate, printed = res[rank]
        assert ms == 15.0  # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1000 * 3 * 7 / 0.015)
    assert res[1][2] == ""


def test_single_process_has_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.whole_job_rate(1, 10, 2, 1000.0) == pytest.approx(60.0)
