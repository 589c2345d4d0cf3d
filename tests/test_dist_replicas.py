"""Replica sharding of the benchmark on several ranks (gloo, CPU): each rank
runs an independent replica of the workload with no data-path collective;
only the timing is reduced (max over ranks) to the whole-job rate."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2310_04676_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_setup()
    seconds = 1.0 + 0.5 * r                  # ranks finish at different times
    rate = bench.aggregate_rate(100.0, seconds, w)
    wl = W.config("C1", num_envs=8)
    d = bench.replica_desc(wl, r)
    out[r] = (rate, float(d["link_len"].sum()))
    dist.destroy_process_group()


def test_two_rank_replicas_reduce_time_not_data():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    rates = [out[r][0] for r in range(world)]
    # whole-job rate = all ranks' units over the slowest rank's time
    assert np.allclose(rates, world * 100.0 / 1.5)
    # each rank simulates its own replica (different seeded parameters)
    assert out[0][1] != out[1][1]


def test_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate_rate(10.0, 2.0, 1) == 5.0
