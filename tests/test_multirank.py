"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
replica (replicas only, no data-path collective), reduce the timed region to
the slowest rank and report the whole job's rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1310_0998_gb300 import synth
    t_local = 1.0 + 0.5 * rank                       # rank 1 is the slow one
    t = bench.max_over_ranks(t_local, world)
    rate = bench.job_throughput(world, 1000, 10, t)
    # each rank draws its own replica from its rank-seeded generator
    x, _ = synth.dimers(50, 16.0, 0.5, seed=rank)
    out.put((rank, t, rate, float(x[:, 0].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_sum_work():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, s0), (r1, t1, v1, s1) = res
    assert t0 == t1 == 1.5
    assert v0 == v1 == 2 * 1000 * 10 / 1.5
    assert s0 != s1                                  # independent replicas


def test_single_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_throughput(1, 100, 4, 2.0) == 200.0
