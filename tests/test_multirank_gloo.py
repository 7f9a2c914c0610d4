"""The N > 1 path of bench.py (independent replicas, one per rank) with world
size 2 on the gloo backend, on CPU: distinct per-rank inputs, the slowest
rank's time shared by all ranks, and the whole-job rate."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.replica_seed(rank)
        A, _ = bench.inputs(3, 2, 1, seed)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        rate = bench.whole_job_rate(4, world, ms)
        q.put((rank, seed, float(A[0, 1, 0, 0].real), ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    (r0, s0, a0, ms0, rate0), (r1, s1, a1, ms1, rate1) = res
    assert s0 != s1 and a0 != a1            # each rank multiplies its own batch
    assert ms0 == ms1 == 15.0               # max over ranks
    assert rate0 == rate1 == pytest.approx(2 * 4 / 15e-3)
