"""The multi-GPU bench path on CPU: two gloo ranks, each with its own vertex
shard, no data-path collective, timing reduced by max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    pos, nrm = bench.shard_vertices(1, rank, 64)
    t = bench.max_over_ranks(10.0 + rank, torch.device("cpu"))
    out[rank] = (float(pos.sum()), t, bench.whole_job_value(1000, t, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    s0, t0, v0 = out[0]
    s1, t1, v1 = out[1]
    assert s0 != s1                      # each rank shades its own vertex shard
    assert t0 == t1 == 11.0              # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(2 * 1000 / 11.0e-3 / 1e6)
