"""The N > 1 host path of the benchmark on CPU: world_size 2 over gloo.

Multi-GPU is replicas only (the path has no exchange step): each rank runs the
whole workload on its own GPU, and the only collectives are the barrier and the
maximum of the timed region over the ranks.  These tests run that reduction,
the whole-job throughput and the reference arm's rank-0-only output in two
spawned processes on 127.0.0.1.
"""
import io
import json
import os
import socket
import sys
import tempfile
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(10.0 + 3.0 * rank, "cpu")       # rank 1 is the slower one
        rate = bench.job_rate(1000, world, 5, ms)
        dist.barrier()
        printed = ""
        if rank != 0:                                               # the reference arm: rank 0 alone runs
            args = type("A", (), {"steps": 1, "warmup": 0})()
            buf = io.StringIO()
            with redirect_stdout(buf):
                ret = bench.run_reference(args, rank, world)
            printed = buf.getvalue()
            assert ret is None
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "rate": rate, "printed": printed}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_the_whole_job_rate():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, start_method="spawn")
        res = [json.load(open(os.path.join(d, f"r{r}.json"))) for r in range(world)]
    for r in res:
        assert r["ms"] == 13.0                                       # max over ranks, on every rank
        assert r["rate"] == pytest.approx(2 * 1000 * 5 / 13.0e-3)    # units of all ranks / slowest time
    assert res[1]["printed"] == ""                                   # no line from rank 1
