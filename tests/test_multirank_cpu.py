"""The bench's multi-rank host logic on CPU: two gloo ranks (world_size 2, 127.0.0.1).

Each rank advances its own seeded ensemble (no data-path collective); the job time is the slowest
rank's time and the throughput counts the cells of every rank.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1508_02899_gb300 import inputs as I


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed_tab, seed_flow = bench.rank_seeds(rank)
    tab = I.ensemble_table(64, seed_tab, nv=65)
    ms_local = 10.0 + 5.0 * rank
    ms_max = bench.max_over_ranks(ms_local, world, dist, torch, "cpu")
    cells = int(tab.nx.sum()) * 65
    total = torch.tensor([cells], dtype=torch.int64)
    dist.all_reduce(total)
    value = bench.job_throughput(cells, 100, world, ms_max)
    dist.barrier()
    out[rank] = (ms_max, cells, int(total.item()), value, int(tab.nx[:16].sum()), seed_flow)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0              # slowest rank's time on every rank
    assert res[0][5] != res[1][5]                       # independent flow seeds per rank
    assert res[0][4] != res[1][4]                       # independent ensembles per rank
    # weak scaling: every rank counts the same per-rank work, world x cells per step
    for r in range(world):
        assert np.isclose(res[r][3], world * res[r][1] * 100 / (15.0e-3) / 1e9)
