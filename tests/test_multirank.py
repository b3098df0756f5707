"""Multi-process (world size 2, gloo, CPU) coverage of bench.py's replica timing logic.

Replicas run the same per-GPU workload; the job's rate is the units of all ranks divided by the
slowest rank's time.
"""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units, rate = bench.job_throughput(100.0 * (rank + 1), 512, world, "cpu")
    mx = bench.rank_reduce(rank + 0.5, "max", world, "cpu")
    dist.barrier()
    q.put((rank, ms, units, rate, mx))
    dist.destroy_process_group()


def test_two_rank_throughput_is_sum_over_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, rate, mx in res:
        assert ms == 200.0 and units == 1024 and abs(rate - 5120.0) < 1e-9 and mx == 1.5


def test_single_process_is_identity():
    import bench
    assert bench.job_throughput(250.0, 512, 1) == (250.0, 512.0, 2048.0)
