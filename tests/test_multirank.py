"""The multi-GPU path of the benchmark is independent replicas (no data
exchange); its host logic -- per-rank Philox keys and the whole-job figures
(max time over ranks, summed events) -- runs here on 2 gloo ranks on CPU."""
import os
import socket

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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    events = [1000, 3000][rank]
    sweeps = [10, 10][rank]
    res = bench.combine_over_ranks(ms, events, sweeps)
    keys = [bench.replica_key(rank, r) for r in range(96)]
    out[rank] = (res, keys)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_benchmark():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (r0, k0), (r1, k1) = out[0], out[1]
    assert r0 == r1 == (20.0, 4000.0, 20.0)
    assert not set(k0) & set(k1)  # ranks never share a Philox stream
