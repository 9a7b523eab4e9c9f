"""Sharded count as K virtual shards on one GPU: each shard counts its share
of the work items (tc_count_shard); summing the partial △(v) and OR-ing the
flags over the shards, loading the result (tc_load_counts) and running the
centrality gives bit for bit what the unsharded tc_count + tc_centrality
give, for every strategy and shard count."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import graphgen as gg
import paper_2105_00110_gb300 as tcg

pytestmark = pytest.mark.gpu

STRATS = ["auto", "bsearch", "merge", "bitmap", "global"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    tcg.build()
    torch.cuda.init()


def unsharded(g):
    tri, flags, total, _ = g.count()
    numer, tcv, den, _ = g.centrality()
    torch.cuda.synchronize()
    return tri.clone(), flags.clone(), total, numer.clone(), tcv.clone()


def sharded(g, k):
    tri_sum = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    flag_or = torch.zeros(g.m, dtype=torch.uint8, device="cuda")
    parts = []
    for shard in range(k):
        tri = torch.empty(g.n, dtype=torch.uint64, device="cuda")
        flags = torch.empty(max(g.m, 1), dtype=torch.uint8, device="cuda")
        parts.append(tcg.tc_count_shard(g.h, shard, k, tri, flags[:g.m] if g.m else None))
        tri_sum += tri.view(torch.int64)
        if g.m:
            flag_or = torch.maximum(flag_or, flags[:g.m])
    tri_sum = tri_sum.view(torch.uint64)
    st, total = tcg.tc_load_counts(g.h, tri_sum, flag_or)
    numer, tcv, den, _ = g.centrality()
    torch.cuda.synchronize()
    return tri_sum, flag_or, total, numer, tcv, parts


def same(a, b):
    return torch.equal(a.view(torch.int64) if a.dtype in (torch.uint64, torch.float64) else a,
                       b.view(torch.int64) if b.dtype in (torch.uint64, torch.float64) else b)


def check(src, dst, n, strategy, shards):
    g = tcg.Graph(torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                  torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda(), n)
    try:
        g.set_strategy(strategy)
        ref = unsharded(g)
        for k in shards:
            got = sharded(g, k)
            assert got[2] == ref[2]
            assert sum(got[5]) == ref[2]                # each triangle in exactly one shard
            assert same(got[0], ref[0]) and same(got[1], ref[1])
            assert same(got[3], ref[3]) and same(got[4], ref[4])
            if k > 1 and ref[2] > 100:
                assert max(got[5]) < ref[2]             # the work is really split
    finally:
        g.close()


@pytest.mark.parametrize("strategy", STRATS)
def test_rmat_shards(strategy):
    check(*gg.rmat(12, seed=0x5EED0200), strategy, [1, 2, 3, 7])


@pytest.mark.parametrize("strategy", ["auto", "bitmap"])
def test_rmat16_shards(strategy):
    check(*gg.rmat(16, seed=0x5EED0210), strategy, [2, 5])


def test_mixed_and_degenerate_shards():
    check(*gg.planted_hierarchy(800, 16, 8, 0.01, seed=51), "auto", [2, 4])
    check(*gg.grid_chung_lu(side=64, seed=52), "auto", [3])
    check(*gg.complete_graph(30), "auto", [2, 64])      # more shards than items of some classes
    tree = (np.arange(1, 100, dtype=np.int32), (np.arange(1, 100) // 2).astype(np.int32), 100)
    g = tcg.Graph(torch.from_numpy(tree[0]).cuda(), torch.from_numpy(tree[1]).cuda(), 100)
    try:
        got = sharded(g, 3)
        assert got[2] == 0 and not got[0].view(torch.int64).any()
    finally:
        g.close()


def test_bad_arguments_and_incomplete_counts():
    s, d, n = gg.complete_graph(6)
    g = tcg.Graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    try:
        for shard, k in ((2, 2), (-1, 2), (0, 0)):
            with pytest.raises(tcg.TCError) as e:
                tcg.tc_count_shard(g.h, shard, k)
            assert e.value.status == tcg.TC_ERR_INVALID_ARG
        tri = torch.ones(n, dtype=torch.int64, device="cuda").view(torch.uint64)   # Σ = 6: fine
        flags = torch.ones(g.m, dtype=torch.uint8, device="cuda")
        tcg.tc_load_counts(g.h, tri, flags)
        tri = torch.zeros(n, dtype=torch.int64, device="cuda")
        tri[0] = 1                                      # Σ = 1: not a multiple of 3
        with pytest.raises(tcg.TCError) as e:
            tcg.tc_load_counts(g.h, tri.view(torch.uint64), flags)
        assert e.value.status == tcg.TC_ERR_INVALID_ARG
        # partial counts leave no valid centrality input
        tcg.tc_count_shard(g.h, 0, 2)
        with pytest.raises(tcg.TCError) as e:
            g.centrality()
        assert e.value.status == tcg.TC_ERR_STATE
    finally:
        g.close()
