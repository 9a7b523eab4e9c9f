"""Failure handling, with no GPU fault: a device allocation made to fail (the
library's own injector, on the host) at every allocation an entry point
makes.  Each such call returns TC_ERR_OUT_OF_MEMORY, gives back every
allocation it had taken, and leaves the library usable: the next call
succeeds and matches the oracle.  The request loop absorbs injected
failures: a request either gets its exact results or, if the failure hit
it alone, an out-of-memory status, and the server keeps serving."""
from __future__ import annotations

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


@pytest.fixture(autouse=True)
def _disarm():
    yield
    tcg.tc_debug_fail_allocation(-1)
    tcg.tc_set_dense_core(-1)


def live():
    torch.cuda.synchronize()
    return tcg.tc_debug_live_allocations()


def allocations_of(fn):
    a0 = tcg.tc_debug_allocations()
    fn()
    torch.cuda.synchronize()
    return tcg.tc_debug_allocations() - a0


def expect_oom(fn):
    with pytest.raises(tcg.TCError) as e:
        fn()
    assert e.value.status == tcg.TC_ERR_OUT_OF_MEMORY


def check_full(src, dst, n, res):
    ref = oracle.run(src, dst, n)
    assert res["total"] == ref["total"]
    np.testing.assert_array_equal(res["tri"].cpu().numpy().view(np.int64), ref["tri"].astype(np.int64))
    np.testing.assert_array_equal(res["numer"].cpu().numpy().view(np.int64), ref["numer"].astype(np.int64))
    np.testing.assert_array_equal(res["tc"].cpu().numpy().view(np.int64), ref["tc"].view(np.int64))
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ref["ptr"]))
    keep = ref["adj"] > rows
    np.testing.assert_array_equal(res["flag"].cpu().numpy(), ref["flag"][keep])


@pytest.mark.parametrize("on_device", [True, False])
def test_build_fails_cleanly_at_every_allocation(on_device):
    src, dst, n = gg.rmat(10, seed=0x5EED0700)
    s = torch.from_numpy(src).cuda() if on_device else torch.from_numpy(src)
    d = torch.from_numpy(dst).cuda() if on_device else torch.from_numpy(dst)
    A = allocations_of(lambda: tcg.tc_graph_free(tcg.tc_build_csr(s, d, n)))
    assert A >= 10
    base = live()
    for k in range(A):
        tcg.tc_debug_fail_allocation(k)
        expect_oom(lambda: tcg.tc_build_csr(s, d, n))
        assert live() == base, k
    tcg.tc_debug_fail_allocation(-1)
    check_full(src, dst, n, tcg.triangle_centrality(s, d, n))
    assert live() == base


@pytest.mark.parametrize("core", [0, 200])
@pytest.mark.parametrize("call", ["count", "edge_triangles", "shard", "replan"])
def test_count_fails_cleanly_at_every_allocation(call, core):
    src, dst, n = gg.rmat(11, seed=0x5EED0701)
    tcg.tc_set_dense_core(core)
    g = tcg.Graph(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    tcg.tc_set_dense_core(-1)
    assert g.stats()["core_vertices"] == core
    tri = torch.empty(n, dtype=torch.uint64, device="cuda")
    flags = torch.empty(g.m, dtype=torch.uint8, device="cuda")
    et = torch.empty(g.m, dtype=torch.int32, device="cuda").view(torch.uint32)

    def run():
        if call == "replan":   # a strategy change re-plans inside the count
            g.set_strategy("bitmap" if g.__dict__.setdefault("_flip", 0) % 2 == 0 else "auto")
            g._flip += 1
        if call == "edge_triangles":
            tcg.tc_edge_triangles(g.h, tri, et)
        elif call == "shard":
            tcg.tc_count_shard(g.h, 0, 1, tri, flags)
        else:
            tcg.tc_count(g.h, tri, flags)

    try:
        run()                  # first call: buffers the graph keeps (edge counts) are made once
        A = allocations_of(run)
        if call == "replan" or core:
            assert A > 0
        base = live()
        for k in range(A):
            tcg.tc_debug_fail_allocation(k)
            expect_oom(run)
            assert live() <= base, k
            with pytest.raises(tcg.TCError) as e:   # no valid counts after a failed count
                tcg.tc_centrality(g.h)
            assert e.value.status == tcg.TC_ERR_STATE
        tcg.tc_debug_fail_allocation(-1)
        run()
        if call == "shard":
            tcg.tc_load_counts(g.h, tri, flags)
        numer, tcv, den, _ = g.centrality()
        eu, ev = g.edges()
        check_full(src, dst, n, dict(total=den // 3, tri=tri, numer=numer, tc=tcv,
                                     flag=(et.view(torch.int32) > 0).to(torch.uint8) if call == "edge_triangles" else flags))
    finally:
        g.close()


def test_centrality_and_batch_run_allocate_nothing():
    src, dst, n = gg.rmat(10, seed=0x5EED0702)
    g = tcg.Graph(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    try:
        g.count()
        assert allocations_of(lambda: g.centrality()) == 0
    finally:
        g.close()
    graphs = [gg.barabasi_albert(300 + 40 * i, 3, seed=i) for i in range(12)]
    b = tcg.Batch(*tcg.pack_graphs(graphs))
    try:
        assert allocations_of(lambda: b.run()) == 0
    finally:
        b.close()


def test_batch_build_fails_cleanly_at_every_allocation():
    graphs = [gg.barabasi_albert(200 + 50 * i, 4, seed=10 + i) for i in range(6)]
    graphs += [gg.planted_hierarchy(300, 8, 5, 0.01, seed=20 + i) for i in range(4)]
    src, dst, off, nv = tcg.pack_graphs(graphs)
    A = allocations_of(lambda: tcg.Batch(src, dst, off, nv).close())
    assert A >= 10
    base = live()
    for k in range(A):
        tcg.tc_debug_fail_allocation(k)
        expect_oom(lambda: tcg.Batch(src, dst, off, nv))
        assert live() == base, k
    tcg.tc_debug_fail_allocation(-1)
    b = tcg.Batch(src, dst, off, nv)
    try:
        out = b.run()
        torch.cuda.synchronize()
        for i, (s, d, n) in enumerate(graphs):
            ref = oracle.run(s, d, n)
            lo, hi = b.voff[i], b.voff[i + 1]
            np.testing.assert_array_equal(out["tri"][lo:hi].cpu().numpy().view(np.int64),
                                          ref["tri"].astype(np.int64))
            np.testing.assert_array_equal(out["tc"][lo:hi].cpu().numpy().view(np.int64), ref["tc"].view(np.int64))
    finally:
        b.close()
    assert live() == base


def test_server_keeps_serving_through_injected_failures():
    reqs = [gg.rmat(9 + (i % 4), seed=0x5EED0710 + i) for i in range(24)]
    refs = [oracle.run(s, d, n) for s, d, n in reqs]
    srv = tcg.Server(memory_budget_bytes=4 << 30, max_batch_pairs=1 << 18, workers=2)
    try:
        for k in (0, 5, 17, 40):
            tcg.tc_debug_fail_allocation(k)
            ids = {srv.submit(s, d, n): i for i, (s, d, n) in enumerate(reqs)}
            done = srv.wait_all(300)
            assert len(done) == len(reqs)
            failed = [r for r in done if r["status"] < 0]
            assert len(failed) <= 1
            for r in failed:
                assert r["status"] == tcg.TC_ERR_OUT_OF_MEMORY
            for r in done:
                if r["status"] >= 0:
                    ref = refs[ids[r["id"]]]
                    assert r["triangles"] == ref["total"]
                    np.testing.assert_array_equal(r["tri"].view(np.int64), ref["tri"].astype(np.int64))
                    np.testing.assert_array_equal(r["tc"].view(np.int64), ref["tc"].view(np.int64))
        tcg.tc_debug_fail_allocation(-1)
        ids = {srv.submit(s, d, n): i for i, (s, d, n) in enumerate(reqs)}
        done = srv.wait_all(300)
        assert len(done) == len(reqs) and all(r["status"] >= 0 for r in done)
    finally:
        srv.close()
