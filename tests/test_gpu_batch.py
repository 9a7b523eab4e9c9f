"""Batches: every graph of a batch gets exactly the results of the oracle on
that graph alone (and of the single-graph path), in one build and one set
of persistent launches; a CUDA-graph replay and the autotuner change no
result."""
from __future__ import annotations

import os
import random

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2105_00110_gb300 as tcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    tcg.build()
    torch.cuda.init()


def mixed_graphs(seed, count):
    rnd = random.Random(seed)
    graphs = []
    for i in range(count):
        kind = rnd.choice(["ba", "hier", "gnp", "rmat"])
        if kind == "ba":
            graphs.append(gg.barabasi_albert(rnd.randint(10, 3000), rnd.randint(2, 8), seed=seed * 1000 + i))
        elif kind == "hier":
            c, k = rnd.randint(4, 12), rnd.randint(3, 8)
            graphs.append(gg.planted_hierarchy(1 + c * k + rnd.randint(0, 500), c, k, 0.01, seed=seed * 1000 + i))
        elif kind == "gnp":
            graphs.append(gg.gnp(rnd.randint(5, 60), rnd.choice([0.1, 0.3]), seed * 1000 + i))
        else:
            graphs.append(gg.rmat(rnd.randint(6, 11), seed=seed * 1000 + i))
    # degenerate members: empty, no edges, a tree (no triangles), a clique
    graphs.insert(3, (np.zeros(0, np.int32), np.zeros(0, np.int32), 0))
    graphs.insert(7, (np.zeros(0, np.int32), np.zeros(0, np.int32), 5))
    graphs.insert(9, (np.arange(1, 30, dtype=np.int32), (np.arange(1, 30) // 2).astype(np.int32), 30))
    graphs.append(gg.complete_graph(12))
    return graphs


def check_batch(graphs, out, b):
    tri = out["tri"].cpu().numpy()
    flag = out["flag"].cpu().numpy()
    numer = out["numer"].cpu().numpy()
    tcv = out["tc"].cpu().numpy()
    totals = out["totals"].cpu().numpy()
    eu, ev = (x.cpu().numpy() for x in b.edges())
    for k, (s, d, n) in enumerate(graphs):
        ref = oracle.run(s, d, n)
        v0, v1 = b.voff[k], b.voff[k + 1]
        e0, e1 = b.eoff[k], b.eoff[k + 1]
        assert v1 - v0 == n
        assert int(totals[k]) == ref["total"]
        np.testing.assert_array_equal(tri[v0:v1], ref["tri"])
        np.testing.assert_array_equal(numer[v0:v1], ref["numer"])
        np.testing.assert_array_equal(tcv[v0:v1].view(np.uint64), ref["tc"].view(np.uint64))
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ref["ptr"]))
        keep = ref["adj"] > rows
        np.testing.assert_array_equal(eu[e0:e1] - v0, rows[keep])
        np.testing.assert_array_equal(ev[e0:e1] - v0, ref["adj"][keep])
        np.testing.assert_array_equal(flag[e0:e1], ref["flag"][keep])


@pytest.mark.parametrize("on_device", [True, False])
def test_batch_matches_oracle_per_graph(on_device):
    graphs = mixed_graphs(1, 40)
    src, dst, off, nv = tcg.pack_graphs(graphs)
    s, d = torch.from_numpy(src), torch.from_numpy(dst)
    if on_device:
        s, d = s.cuda(), d.cuda()
    b = tcg.Batch(s, d, off, nv)
    out = b.run()
    torch.cuda.synchronize()
    check_batch(graphs, out, b)
    b.close()


def test_batch_equals_single_graph_path():
    graphs = mixed_graphs(2, 12)
    src, dst, off, nv = tcg.pack_graphs(graphs)
    b = tcg.Batch(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), off, nv)
    out = {k: v.cpu().numpy() for k, v in b.run().items()}
    for k, (s, d, n) in enumerate(graphs):
        if n == 0:
            continue
        one = tcg.triangle_centrality(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
        v0, v1 = b.voff[k], b.voff[k + 1]
        np.testing.assert_array_equal(out["tri"][v0:v1], one["tri"].cpu().numpy())
        np.testing.assert_array_equal(out["numer"][v0:v1], one["numer"].cpu().numpy())
        np.testing.assert_array_equal(out["tc"][v0:v1].view(np.uint64), one["tc"].cpu().numpy().view(np.uint64))
    b.close()


def test_cuda_graph_replay_and_autotune():
    graphs = mixed_graphs(3, 30)
    src, dst, off, nv = tcg.pack_graphs(graphs)
    b = tcg.Batch(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), off, nv)
    ref = {k: v.clone() for k, v in b.run().items()}
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.run(stream)                       # settles launch attributes on this stream
    stream.synchronize()
    for v in b.out.values():
        v.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.run(stream)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    bits = lambda t: t.view(torch.int64) if t.dtype == torch.float64 else t   # NaN-safe equality
    for k in ref:
        assert torch.equal(bits(ref[k]), bits(b.out[k])), k
    params = b.autotune(reps=1)
    assert set(params) == {"cta_min_work", "cta_chunk", "warp_chunk"}
    out = b.run()
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(bits(ref[k]), bits(out[k])), k
    b.close()


def test_batch_rejects_out_of_graph_ids():
    src = np.array([0, 1, 0, 7], np.int32)
    dst = np.array([1, 2, 1, 1], np.int32)
    with pytest.raises(tcg.TCError) as ei:
        tcg.Batch(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
                  np.array([0, 2, 4]), np.array([3, 3]))
    assert ei.value.status == tcg.TC_ERR_INVALID_ARG


def test_full_batched_workload_sampled():
    # the bench's batched workload at full size (8192 graphs): per-graph
    # totals add up, and sampled members equal the oracle and the single path
    graphs = gg.batch_config3(8192, 0x5EED0003)
    src, dst, off, nv = tcg.pack_graphs(graphs)
    b = tcg.Batch(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), off, nv)
    out = b.run()
    torch.cuda.synchronize()
    tri = out["tri"].view(torch.int64)
    totals = out["totals"].view(torch.int64).cpu().numpy()
    voff = torch.from_numpy(np.asarray(b.voff, np.int64)).cuda()
    per = torch.zeros(len(graphs), dtype=torch.int64, device="cuda")
    owner = torch.searchsorted(voff[1:], torch.arange(int(voff[-1]), device="cuda"), right=True)
    per.index_add_(0, owner, tri)
    np.testing.assert_array_equal(per.cpu().numpy(), 3 * totals)
    rnd = random.Random(9)
    pick = rnd.sample(range(len(graphs)), 24)
    pick.append(max(range(len(graphs)), key=lambda k: len(graphs[k][0])))   # the largest member too
    tri_h = tri.cpu().numpy()
    tc_h = out["tc"].view(torch.int64).cpu().numpy()
    threads = os.cpu_count() or 1
    for k in pick:
        s, d, n = graphs[k]
        v0, v1 = b.voff[k], b.voff[k + 1]
        # every sampled member against the oracle (its degree-ordered listing,
        # pinned against the definition, on the host's threads for the large ones)
        ref = oracle.run(s, d, n) if n <= 3000 else oracle.run(s, d, n, "fast", threads=threads, algebraic=False)
        np.testing.assert_array_equal(tri_h[v0:v1], ref["tri"].astype(np.int64))
        np.testing.assert_array_equal(tc_h[v0:v1], ref["tc"].view(np.int64))
        one = tcg.triangle_centrality(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
        np.testing.assert_array_equal(tri_h[v0:v1], one["tri"].view(torch.int64).cpu().numpy())
        np.testing.assert_array_equal(tc_h[v0:v1], one["tc"].view(torch.int64).cpu().numpy())
        assert int(totals[k]) == one["total"]
    b.close()
