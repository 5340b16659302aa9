"""The multi-GPU path is replicas only: each rank solves its own instance and the ranks exchange
nothing but the timing. Its host logic runs here as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2203_05027_b300 import instances as I
from paper_2203_05027_b300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.env()
    ms = replicas.max_over_ranks(10.0 + 5.0 * r, dist)  # rank 1 is the slower one
    prob = I.small_lp(r)  # each replica its own seeded instance
    out[r] = (r, w, lr, ms, replicas.job_throughput(1000, w, ms), float(prob["b"].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time_and_solve_different_instances():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rank, w, lr, ms, thr, bsum = res[r]
        assert (rank, w, lr) == (r, 2, r)
        assert ms == 15.0  # the maximum over ranks, on every rank
        assert np.isclose(thr, 2 * 1000 / 15e-3)
    assert res[0][5] != res[1][5]


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10, 1, 1000.0) == 10.0
