"""Serving: every request gets exactly the results of its graph run alone
(and of the oracle), whatever batch it lands in; requests over the memory
budget are refused at submission; a bad request fails alone."""
from __future__ import annotations

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


def request_mix(seed, count):
    rnd = random.Random(seed)
    out = []
    for i in range(count):
        kind = rnd.choice(["ba", "hier", "gnp", "rmat", "rmat"])
        if kind == "ba":
            out.append(gg.barabasi_albert(rnd.randint(10, 4000), rnd.randint(2, 8), seed=seed * 100 + i))
        elif kind == "hier":
            c, k = rnd.randint(4, 12), rnd.randint(3, 8)
            out.append(gg.planted_hierarchy(1 + c * k + rnd.randint(0, 400), c, k, 0.01, seed=seed * 100 + i))
        elif kind == "gnp":
            out.append(gg.gnp(rnd.randint(5, 60), 0.2, seed * 100 + i))
        else:
            out.append(gg.rmat(rnd.randint(6, 13), seed=seed * 100 + i))
    out.insert(2, (np.zeros(0, np.int32), np.zeros(0, np.int32), 0))
    out.insert(5, (np.zeros(0, np.int32), np.zeros(0, np.int32), 9))
    out.insert(8, gg.complete_graph(30))
    out.append(gg.rmat(18, seed=seed))       # large enough to travel directly, not staged
    return out


def alone(s, d, n):
    if n == 0:
        return np.zeros(0, np.uint64), np.zeros(0, np.float64)
    r = tcg.triangle_centrality(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    return r["tri"].cpu().numpy(), r["tc"].cpu().numpy()


def bits(x):
    return np.asarray(x).view(np.int64)


def test_each_request_matches_its_graph_alone_and_the_oracle():
    reqs = request_mix(3, 48)
    srv = tcg.Server(memory_budget_bytes=8 << 30, max_batch_pairs=1 << 20, workers=2)
    ids = [srv.submit(s, d, n) for s, d, n in reqs]
    done = {r["id"]: r for r in srv.wait_all(300)}
    stats = srv.stats()
    srv.close()
    assert sorted(done) == sorted(ids)
    assert max(r["batch_size"] for r in done.values()) > 1      # requests were batched
    assert stats["batches"] < len(reqs)
    for rid, (s, d, n) in zip(ids, reqs):
        r = done[rid]
        tri, tcv = alone(s, d, n)
        assert r["status"] in (tcg.TC_OK, tcg.TC_NO_TRIANGLES)
        np.testing.assert_array_equal(r["tri"], tri)
        np.testing.assert_array_equal(bits(r["tc"]), bits(tcv))
        assert r["triangles"] == int(tri.sum()) // 3
        if n <= 5000:
            ref = oracle.run(s, d, n)
            np.testing.assert_array_equal(r["tri"], ref["tri"])
            np.testing.assert_array_equal(bits(r["tc"]), bits(ref["tc"]))
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]


def test_alone_and_in_the_mix_are_identical():
    s, d, n = gg.rmat(12, seed=77)
    srv = tcg.Server(memory_budget_bytes=4 << 30, workers=1)
    srv.submit(s, d, n)
    (first,) = srv.wait_all(60)
    assert first["batch_size"] == 1
    mix = request_mix(4, 24)
    ids = [srv.submit(*g) for g in mix[:10]]
    rid = srv.submit(s, d, n)
    ids += [srv.submit(*g) for g in mix[10:]]
    done = {r["id"]: r for r in srv.wait_all(300)}
    srv.close()
    again = done[rid]
    np.testing.assert_array_equal(again["tri"], first["tri"])
    np.testing.assert_array_equal(bits(again["tc"]), bits(first["tc"]))
    assert again["triangles"] == first["triangles"]


def test_over_budget_request_is_refused_without_device_work():
    srv = tcg.Server(memory_budget_bytes=64 << 20, workers=1)
    big = np.zeros(1 << 20, np.int32)           # estimate > 64 MB
    with pytest.raises(tcg.TCError) as e:
        srv.submit(big, big, 10)
    assert e.value.status == tcg.TC_ERR_OUT_OF_MEMORY
    st = srv.stats()
    assert st["batches"] == 0 and st["waiting"] == 0 and st["memory_in_use"] == 0
    s, d, n = gg.complete_graph(8)                # a small one still runs
    srv.submit(s, d, n)
    (r,) = srv.wait_all(60)
    assert r["triangles"] == 56
    srv.close()


def test_bad_request_fails_alone():
    good = [gg.complete_graph(k) for k in (4, 5, 6)]
    bad = (np.array([0, 1, 2], np.int32), np.array([1, 2, 99], np.int32), 3)   # id 99 outside [0, 3)
    srv = tcg.Server(memory_budget_bytes=1 << 30, workers=1)
    # hold the single worker on a first request so the rest queue up into one batch
    first = srv.submit(*gg.rmat(16, seed=5))
    ids = [srv.submit(*good[0]), srv.submit(*bad), srv.submit(*good[1]), srv.submit(*good[2])]
    done = {r["id"]: r for r in srv.wait_all(120)}
    srv.close()
    assert done[first]["status"] == tcg.TC_OK
    assert done[ids[1]]["status"] == tcg.TC_ERR_INVALID_ARG
    for rid, k in zip((ids[0], ids[2], ids[3]), (4, 5, 6)):
        assert done[rid]["status"] == tcg.TC_OK
        assert done[rid]["triangles"] == k * (k - 1) * (k - 2) // 6


def test_free_with_waiting_requests_drops_them():
    srv = tcg.Server(memory_budget_bytes=1 << 30, workers=1)
    for i in range(30):
        srv.submit(*gg.rmat(10, seed=i))
    srv.close()                                   # must return; running batch finishes


def test_served_pool_requests_against_the_oracle():
    # entries of the served workload's own request pool (its seed, both
    # generator kinds, every decade of size up to 3·10^7 pairs), through a
    # server set up as in the served workload, each against the whole oracle
    # run on the host's threads
    import os
    specs = gg.served_pool_specs(256, 0x5EED0004, 1e3, 1e8)
    pick = []
    for lo, hi in ((1e3, 1e4), (1e4, 1e5), (1e5, 1e6), (1e6, 1e7), (1e7, 3e7)):
        for kind in ("rmat", "grid"):
            pick += [sp for sp in specs if sp["kind"] == kind and lo <= sp["pairs"] < hi][:2]
    assert {sp["kind"] for sp in pick} == {"rmat", "grid"} and max(sp["pairs"] for sp in pick) >= 1e7
    reqs = [gg.served_graph(sp) for sp in pick]
    srv = tcg.Server(memory_budget_bytes=32 << 30, max_batch_pairs=1 << 25, workers=2)
    try:
        ids = [srv.submit(s, d, n) for s, d, n in reqs]
        done = {r["id"]: r for r in srv.wait_all(600)}
    finally:
        srv.close()
    assert sorted(done) == sorted(ids)
    threads = os.cpu_count() or 1
    for rid, (s, d, n) in zip(ids, reqs):
        r = done[rid]
        ref = oracle.run(s, d, n, "fast", threads=threads, algebraic=False)
        assert r["status"] in (tcg.TC_OK, tcg.TC_NO_TRIANGLES)
        assert r["triangles"] == ref["total"]
        np.testing.assert_array_equal(bits(r["tri"]), bits(ref["tri"].astype(np.int64)))
        np.testing.assert_array_equal(bits(r["tc"]), bits(ref["tc"]))
