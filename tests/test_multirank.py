"""Replica path of bench.py on the CPU: two gloo ranks on 127.0.0.1. Rays are
independent, so N GPUs run N replicas with no data-path collective; the only
collective is the max-over-ranks reduction of the timings."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2404_16221_b300 import synthetic as sy

        res = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank])
        w = sy.workload("grid8", n_rays=4096)
        o, d = bench.rank_rays(w, rank)
        # every rank sees the other ranks' first ray through a gather (test only)
        first = torch.tensor(np.concatenate([o[0], d[0]]), dtype=torch.float64)
        gathered = [torch.zeros(6, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, first)
        out[rank] = (res, len(o), [g.tolist() for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_timing_and_distinct_rays():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res0, n0, g0 = out[0]
        res1, n1, _ = out[1]
    assert res0 == res1 == [2.0, 10.0, 0.5]
    assert n0 == n1 == 4096
    assert g0[0] != g0[1]  # each replica renders its own rays
