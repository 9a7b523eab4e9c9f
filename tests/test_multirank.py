"""The N>1 paths of bench.py on CPU with world_size-2 gloo ranks: replicas
(each rank times its own graph; the whole-job time is the slowest rank's
and the units add up) and the exchange step of one graph sharded across
the ranks (partial counts summed, flags OR-ed: equal to the unsharded
oracle result)."""
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


def _triangles(src, dst, n):
    """All triangles a < b < c of the simple graph on the pairs (small n)."""
    A = np.zeros((n, n), dtype=bool)
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            A[a, b] = A[b, a] = True
    out = []
    for a in range(n):
        for b in np.nonzero(A[a, a + 1:])[0] + a + 1:
            for c in np.nonzero(A[b, b + 1:] & A[a, b + 1:])[0] + b + 1:
                out.append((a, int(b), int(c)))
    return out


def _exchange_worker(rank, world, port, q):
    import torch

    import graphgen as gg
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, d, n = gg.gnp(40, 0.25, 61)
    ref = oracle.run(s, d, n)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ref["ptr"]))
    keep = ref["adj"] > rows
    eu, ev = rows[keep], ref["adj"][keep]
    index = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(eu, ev))}
    tri = np.zeros(n, np.uint64)
    flags = np.zeros(len(eu), np.uint8)
    for i, (a, b, c) in enumerate(_triangles(s, d, n)):
        if i % world != rank:            # this rank's share of the triangles
            continue
        for x in (a, b, c):
            tri[x] += 1
        for e in ((a, b), (a, c), (b, c)):
            flags[index[e]] = 1
    t = torch.from_numpy(tri.view(np.int64)).view(torch.uint64)
    f = torch.from_numpy(flags)
    bench.shard_exchange(t, f)          # the bench's exchange step of a sharded count
    ok = (np.array_equal(t.view(torch.int64).numpy().view(np.uint64), ref["tri"]) and
          np.array_equal(f.numpy(), ref["flag"][keep]))
    q.put((rank, ok, int(ref["total"])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_count_exchange():
    # the exchange step of a sharded count: partial counts sum, flags OR
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in out)
    assert out[0][2] > 10                # the graph has triangles to split
