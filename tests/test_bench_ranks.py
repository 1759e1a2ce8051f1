"""The multi-rank host logic of bench.py on CPU: two processes over gloo.

Every rank solves its own seeded batch (weak scaling, no collective on the data path); the
job's throughput is the sweeps of all ranks over the slowest rank's time, and every rank
must agree on it.
"""
import os
import socket
import sys

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    params, b = bench.make_batch(rank, 15, 3)
    sweeps = 100.0 * (rank + 1)  # ranks do different amounts of work
    ms = 20.0 if rank == 0 else 5.0  # and rank 0 is the slowest
    value, tmax = bench.job_throughput(sweeps, ms, dist)
    launches = bench.reduce_over_ranks(7 + rank, dist, "sum")
    q.put((rank, [tuple(map(float, p)) for p in params], float(b.sum()), value, tmax, launches))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_the_batch_and_agree_on_the_job_throughput():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, params, bsum, value, tmax, launches = q.get(timeout=180)
            out[rank] = (params, bsum, value, tmax, launches)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert out[0][0] != out[1][0] and out[0][1] != out[1][1]  # each rank its own seeded batch
    for r in (0, 1):
        assert out[r][3] == pytest.approx(20.0)  # the slowest rank's time
        assert out[r][2] == pytest.approx((100.0 + 200.0) / 0.020)  # all ranks' sweeps over it
        assert out[r][4] == pytest.approx(15.0)


def test_one_process_needs_no_collective():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    assert bench.job_throughput(50.0, 10.0, None) == pytest.approx((5000.0, 10.0))
    assert bench.reduce_over_ranks(3.0, None, "sum") == 3.0
