"""The N > 1 path of bench.py (independent replicas, max-over-ranks timing),
exercised with the gloo backend on CPU, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends its timed region took 100 + 50 r ms for 10 steps of 4 units
    ms_per_step, value = bench.aggregate_timing(100.0 + 50.0 * rank, 10, 4, world, dist, "cpu")
    q.put((rank, ms_per_step, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert abs(ms - 15.0) < 1e-12          # max over ranks (150 ms) / 10 steps
        assert abs(value - 2 * 4 * 10 / 0.150) < 1e-9  # units of both ranks / max time


def test_single_rank_timing():
    import bench
    ms, value = bench.aggregate_timing(200.0, 20, 1, 1)
    assert ms == 10.0 and abs(value - 100.0) < 1e-12
