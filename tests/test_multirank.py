"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): ranks run
independent images, the job value uses the slowest rank's time, and the only
collectives are the barrier and that max."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      CANNY_BENCH_BACKEND="gloo")
    import bench
    r, w = bench.dist_init(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    mine = 10.0 + 5.0 * rank            # rank 1 is the slower one
    slowest = bench.max_over_ranks(mine, w)
    q.put((rank, slowest, bench.job_value(w, 4, 1000, slowest)))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in got:
        assert slowest == 15.0
        assert value == pytest.approx(2 * 4 * 1000 / 0.015 / 1e6)


def test_job_value_single_rank():
    import bench
    assert bench.job_value(1, 10, 268435456, 9.62) == pytest.approx(10 * 268435456 / 0.00962 / 1e6)
