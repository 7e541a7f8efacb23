"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank gets its own field, and the timed region is reduced with a max over
ranks -- the only collective (fields are independent, weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2007_09625_gb300 import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    x = workloads.random_walk_1d(4096, seed=bench.rank_seed(r))
    t = bench.reduce_max(10.0 * (r + 1), "cpu")
    dist.barrier()
    q.put((r, ws, float(x[100]), t))
    dist.destroy_process_group()


def test_two_ranks_independent_fields_and_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert res[0][2] != res[1][2]            # different fields per rank
    assert all(r[3] == 20.0 for r in res)    # max over ranks on every rank
