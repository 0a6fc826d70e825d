"""The multi-rank host logic of bench.py on CPU: two gloo ranks, as torchrun
launches them (replicas of the workload, no data-path collective).  The barrier
and the max-over-ranks timing are the only collectives."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # rank r "took" 1 + r seconds: the job time is the slowest rank's
        slowest = bench.max_over_ranks(world, 1.0 + rank)
        rate = bench.whole_job_rate(1_000_000, 10, world, slowest)
        bench.barrier(world)
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, slowest, rate in res:
        assert slowest == 2.0
        assert rate == pytest.approx(1_000_000 * 10 * 2 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    bench.barrier(1)
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.whole_job_rate(100, 4, 1, 2.0) == 200.0
