"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size
2): every rank runs its own flame (replicas); the job's rate is all ranks'
updates over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    m = bench.reduce_max(local_ms, device="cpu")
    rate = bench.whole_job_rate(4096 * 8192, 20, world, m)
    q.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_and_rate_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, m, rate in out:
        assert m == 15.0
        assert rate == pytest.approx(4096 * 8192 * 20 * 2 / 15e-3)


def test_single_process_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_rate(100, 10, 1, 1.0) == pytest.approx(1e6)
