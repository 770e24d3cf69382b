"""The multi-GPU path of bench.py on CPU: two gloo ranks (no GPU).

Instances are independent, so N GPUs run N replicas, each on its own seeded batch, with no
collective on the data path; after the timed region one gather of four numbers gives the whole-
job figures: the slowest rank's step time and the summed counts (weak scaling).
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2601_14414_gb300 import workloads as W


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 12.5][rank]
    res = bench.combine_ranks(torch, dist, torch.device("cpu"), ms, 100 + rank, 1000.0 * (rank + 1),
                              5e5 * (rank + 1))
    dims = W.batched_dims(seed=bench.rank_seed(3, rank), batch=64)
    out[rank] = (res, [d.tolist() for d in dims])
    dist.destroy_process_group()


def test_two_ranks_combine_and_solve_distinct_batches():
    world = 2
    port = free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(worker, args=(world, port, out), nprocs=world, join=True)
        res = {k: out[k] for k in range(world)}
    for rank in range(world):
        ms, ok, it, st = res[rank][0]
        assert ms == 12.5                       # the slowest rank sets the job time
        assert ok == 201 and it == 3000.0 and st == 1.5e6
    assert res[0][1] != res[1][1]               # each rank draws its own instances


def test_single_process_combination_is_the_identity():
    assert bench.combine_ranks(torch, None, None, 3.0, 7, 11.0, 13.0) == (3.0, 7.0, 11.0, 13.0)
