"""Per-edge triangle counts t(u, v) = (A² ∘ A)(u, v) through
tc_edge_triangles, against the oracle's edge triangle matrix, entry by
entry, under every count strategy; and the centrality that follows them is
the same as after tc_count."""
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


def edge_run(src, dst, n, strategy):
    g = tcg.Graph(torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                  torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda(), n)
    try:
        g.set_strategy(strategy)
        tri, et, total, st = g.edge_triangles()
        numer, tcv, den, _ = g.centrality()
        eu, ev = g.edges()
        torch.cuda.synchronize()
        return dict(tri=tri.cpu().numpy(), et=et.cpu().numpy().view(np.int32).astype(np.int64),
                    total=total, status=st, numer=numer.cpu().numpy(), tc=tcv.cpu().numpy(),
                    eu=eu.cpu().numpy(), ev=ev.cpu().numpy(), m=g.m)
    finally:
        g.close()


def check(src, dst, n, strategy, mode="definition"):
    ref = oracle.run(src, dst, n, mode)
    res = edge_run(src, dst, n, strategy)
    ptr, adj = ref["ptr"], ref["adj"]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ptr))
    keep = adj > rows
    np.testing.assert_array_equal(res["eu"], rows[keep])
    np.testing.assert_array_equal(res["ev"], adj[keep])
    np.testing.assert_array_equal(res["et"], ref["t"][keep].astype(np.int64))
    assert int(res["et"].sum()) == 3 * ref["total"]
    assert res["total"] == ref["total"]
    np.testing.assert_array_equal(res["tri"], ref["tri"])
    np.testing.assert_array_equal(res["numer"], ref["numer"])
    np.testing.assert_array_equal(res["tc"].view(np.int64), ref["tc"].view(np.int64))
    return res


@pytest.mark.parametrize("strategy", STRATS)
def test_complete_graph(strategy):
    k = 40
    res = check(*gg.complete_graph(k), strategy)
    assert np.all(res["et"] == k - 2)                 # every edge of K_k is in k - 2 triangles


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("scale", [8, 10, 12])
def test_rmat(scale, strategy):
    check(*gg.rmat(scale, seed=0x5EED0100 + scale), strategy)


@pytest.mark.parametrize("strategy", STRATS)
def test_mixed_shapes(strategy):
    check(*gg.barabasi_albert(3000, 5, seed=41), strategy)
    check(*gg.planted_hierarchy(600, 12, 8, 0.01, seed=42), strategy)
    check(*gg.grid_chung_lu(side=64, seed=43), strategy)
    check(*gg.gnp(50, 0.3, 44), strategy)


def test_triangle_free_and_empty():
    tree = (np.arange(1, 200, dtype=np.int32), (np.arange(1, 200) // 2).astype(np.int32), 200)
    res = check(*tree, "auto")
    assert res["status"] == tcg.TC_NO_TRIANGLES and not res["et"].any()
    res = edge_run(np.zeros(0, np.int32), np.zeros(0, np.int32), 5, "auto")
    assert res["m"] == 0 and res["total"] == 0


@pytest.mark.parametrize("strategy", STRATS)
def test_rmat16_many_tiles(strategy):
    check(*gg.rmat(16, seed=0x5EED0010), strategy, mode="fast")


def test_counts_then_edges_then_counts_agree():
    # the two modes share the graph's plan and flags: alternate them
    s, d, n = gg.rmat(14, seed=0x5EED0114)
    g = tcg.Graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    try:
        tri0, flags0, total0, _ = g.count()
        _, tc0, _, _ = g.centrality()
        tri1, et, total1, _ = g.edge_triangles()
        _, tc1, _, _ = g.centrality()
        tri2, flags2, total2, _ = g.count()
        torch.cuda.synchronize()
        assert total0 == total1 == total2
        assert torch.equal(tri0.view(torch.int64), tri1.view(torch.int64))
        assert torch.equal(tri0.view(torch.int64), tri2.view(torch.int64))
        assert torch.equal(flags0, flags2)
        assert torch.equal(flags0.to(torch.int64), (et.view(torch.int32) > 0).to(torch.int64))
        assert torch.equal(tc0.view(torch.int64), tc1.view(torch.int64))
    finally:
        g.close()
