"""Host-side logic of bench.py's multi-rank mode, exercised with two gloo
ranks on the CPU: every rank advances its own replica, the slowest rank's
time sets the whole-job throughput, and only rank 0 reports."""
import io
import json
import os
import socket
import sys
import contextlib

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")
    value = bench.throughput(262144, 20, world, slowest * 1e-3)
    buf = io.StringIO()

    class Args:
        steps, warmup, workload = 1, 1, "c2"
    bench._ARGS = Args
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args, rank, world)
    out[rank] = (slowest, value, buf.getvalue())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_rank0_reports():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, value, text = res[rank]
        assert slowest == 15.0                              # max over ranks, on every rank
        assert value == pytest.approx(262144 * 20 * 2 / 15e-3 / 1e6)
    assert res[1][2] == ""                                  # only rank 0 prints
    line = json.loads(res[0][2].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.throughput(1000, 10, 4, 2.0) == pytest.approx(0.02)
