"""The dense core of the count step: with a forced core size (the top C
ranks take their mutual triangles from one matrix product, the sparse
kernels skip them), every output against the oracle — △(v), △(G), flags,
per-edge counts t(u, v), numerators, TC — for every strategy, both count
modes and sharded counts; the automatic choice leaves small graphs alone."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2105_00110_gb300 as tcg

pytestmark = pytest.mark.gpu

STRATS = ["auto", "bsearch", "merge", "bitmap", "global"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    tcg.build()
    torch.cuda.init()


@pytest.fixture(autouse=True)
def _auto_core_after():
    yield
    tcg.tc_set_dense_core(-1)


def run(src, dst, n, strategy, core, shards=0):
    tcg.tc_set_dense_core(core)
    g = tcg.Graph(torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                  torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda(), n)
    tcg.tc_set_dense_core(-1)
    try:
        g.set_strategy(strategy)
        out = {"core": g.stats()["core_vertices"], "m": g.m}
        tri, flags, total, _ = g.count()
        numer, tcv, den, _ = g.centrality()
        eu, ev = g.edges()
        out.update(tri=tri.cpu().numpy(), flag=flags.cpu().numpy(), total=total, numer=numer.cpu().numpy(),
                   tc=tcv.cpu().numpy(), eu=eu.cpu().numpy(), ev=ev.cpu().numpy())
        tri2, et, total2, _ = g.edge_triangles()
        out.update(tri2=tri2.cpu().numpy(), et=et.cpu().numpy().view(np.int32).astype(np.int64), total2=total2)
        if shards:
            tsum = torch.zeros(n, dtype=torch.int64, device="cuda")
            fmax = torch.zeros(max(g.m, 1), dtype=torch.uint8, device="cuda")
            for k in range(shards):
                t = torch.empty(n, dtype=torch.uint64, device="cuda")
                f = torch.empty(max(g.m, 1), dtype=torch.uint8, device="cuda")
                tcg.tc_count_shard(g.h, k, shards, t, f[:g.m])
                tsum += t.view(torch.int64)
                fmax = torch.maximum(fmax, f)
            tcg.tc_load_counts(g.h, tsum.view(torch.uint64), fmax[:g.m])
            numer_s, tc_s, _, _ = g.centrality()
            out.update(tri_s=tsum.cpu().numpy(), flag_s=fmax[:g.m].cpu().numpy(), tc_s=tc_s.cpu().numpy())
        torch.cuda.synchronize()
        return out
    finally:
        g.close()


def check(src, dst, n, strategy, core, shards=0):
    ref = oracle.run(src, dst, n)
    res = run(src, dst, n, strategy, core, shards)
    assert res["core"] == (min(core, n) if core >= 3 and res["m"] > 0 else 0)
    ptr, adj = ref["ptr"], ref["adj"]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ptr))
    keep = adj > rows
    np.testing.assert_array_equal(res["eu"], rows[keep])
    np.testing.assert_array_equal(res["ev"], adj[keep])
    assert res["total"] == res["total2"] == ref["total"]
    for k in ("tri", "tri2"):
        np.testing.assert_array_equal(res[k].view(np.int64), ref["tri"].astype(np.int64))
    np.testing.assert_array_equal(res["flag"], ref["flag"][keep])
    np.testing.assert_array_equal(res["et"], ref["t"][keep].astype(np.int64))
    np.testing.assert_array_equal(res["numer"].view(np.int64), ref["numer"].astype(np.int64))
    if ref["total"] > 0:
        np.testing.assert_array_equal(res["tc"].view(np.int64), ref["tc"].view(np.int64))
    if shards:
        np.testing.assert_array_equal(res["tri_s"], ref["tri"].astype(np.int64))
        np.testing.assert_array_equal(res["flag_s"], ref["flag"][keep])
        np.testing.assert_array_equal(res["tc_s"].view(np.int64), res["tc"].view(np.int64))
    return res


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("core", [3, 64, 700])
def test_forced_core_rmat(strategy, core):
    check(*gg.rmat(12, seed=0x5EED0500), strategy, core)


@pytest.mark.parametrize("core", [40, 120])
def test_forced_core_shapes(core):
    check(*gg.complete_graph(120), "auto", core)                 # the whole graph or part of it dense
    check(*gg.planted_hierarchy(800, 16, 8, 0.01, seed=53), "auto", core)
    check(*gg.barabasi_albert(2000, 6, seed=54), "auto", core)
    check(*gg.gnp(150, 0.2, 55), "bitmap", core)
    check(*gg.grid_chung_lu(side=48, seed=56), "auto", core)


def test_forced_core_sharded():
    check(*gg.rmat(13, seed=0x5EED0501), "auto", 512, shards=3)
    check(*gg.rmat(11, seed=0x5EED0502), "merge", 2048, shards=2)   # every vertex in the core


def test_core_without_triangles_and_tiny():
    tree = (np.arange(1, 300, dtype=np.int32), (np.arange(1, 300) // 2).astype(np.int32), 300)
    res = run(*tree, "auto", 64)
    assert res["core"] == 64 and res["total"] == 0 and not res["tri"].any()
    check(np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), 3, "auto", 3)   # one triangle, all core
    assert run(np.array([0], np.int32), np.array([1], np.int32), 2, "auto", 64)["core"] == 0


def test_auto_leaves_small_graphs_alone():
    res = run(*gg.rmat(12, seed=0x5EED0503), "auto", -1)
    assert res["core"] == 0
    with pytest.raises(tcg.TCError):
        tcg.tc_set_dense_core(-2)
