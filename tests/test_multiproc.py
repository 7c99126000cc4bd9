"""The multi-process path of bench.py (replicas, one rank per GPU) on CPU with
two gloo ranks: the job time is the slowest rank's, rank 0 alone reports, and
the reference arm returns without work on the other ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 * (rank + 1), "cpu", world)
    dist.barrier()
    ran = bench.run_reference(None, rank, world) if rank != 0 else "skipped"
    q.put((rank, ms, bench.job_ms_per_step(ms, 5, world), ran))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]          # max over ranks
    assert res[0][2] == pytest.approx(2.0)               # 20 ms for 2 x 5 steps
    assert res[1][3] is None                             # reference arm: rank 1 does no work
