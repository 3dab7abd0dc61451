"""The multi-process path of bench.py (replicas only: every rank processes its
own copy of the workload, no data-path collective): the slowest rank's time
is taken with a max all-reduce and the whole-job value counts every rank's
units.  Two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slower one
    worst = bench.max_over_ranks(ms)
    value = bench.replica_value(1000.0, worst, world)
    r, w, lr = bench.dist_env()
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, worst, value, r, w, lr))


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, value, r, w, lr in res:
        assert worst == 15.0
        assert value == pytest.approx(2 * 1000.0 / 0.015)
        assert (r, w, lr) == (rank, 2, rank)


def test_single_process_is_its_own_max():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(10.0, 1000.0, 1) == 10.0
