"""Multi-rank host logic of bench.py on CPU: two gloo ranks (replicas) agree on the slowest
rank's time and on the whole-job throughput, as the N-GPU launch does over NCCL."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        my_ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
        ms = bench.max_over_ranks(my_ms, world, device="cpu")
        units = 128 ** 3 * 5 * 60   # point-stages per rank
        out[rank] = (ms, bench.whole_job_rate(units, world, ms * 1e-3))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    ms, rate = res[0]
    assert ms == 15.0
    assert rate == pytest.approx(128 ** 3 * 5 * 60 * 2 / 15e-3 / 1e6)


def test_single_rank_is_the_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1e6, 1, 0.5) == pytest.approx(2.0)

