"""bench.py's multi-replica logic on CPU: two gloo ranks (127.0.0.1)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 40, world)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_slowest_rank_and_sums_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 150.0                       # max over the ranks
        assert abs(value - 2 * 40 / 0.150) < 1e-9  # frames of both ranks in that time


def test_single_rank_is_local_time():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_ranks(80.0, 10, 1)
    assert ms == 80.0 and abs(value - 125.0) < 1e-9


def test_reference_arm_other_ranks_exit_without_output(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        n_gauss = 1000
        steps = 1
        warmup = 0
    bench.run_reference(A(), 1, 2)
    assert capsys.readouterr().out == ""
