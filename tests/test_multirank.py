"""The N>1 path of bench.py on CPU: world_size-2 gloo ranks each time their
own graph; the whole-job time is the slowest rank's and the units add up.
Ranks draw different graphs (weak scaling over independent graphs)."""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 100.0 + 50.0 * rank          # rank 1 is the slow one
    res = bench.aggregate(t, 2 * t, 1000 + rank, 10 + rank, world)
    src, _, _ = bench.generate(dict(kind="rmat", scale=8, edge_factor=4, seed=7), rank)
    q.put((rank, res, int(src[:64].astype(np.int64).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    for _, res, _ in out:
        assert res == (150.0, 300.0, 2001, 21)
    assert out[0][2] != out[1][2]        # per-rank graphs differ


def test_single_rank_identity():
    assert bench.aggregate(3.0, 4.0, 5, 6, 1) == (3.0, 4.0, 5, 6)
