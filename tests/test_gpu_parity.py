"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element.  Counts, flags and numerators must be bit-exact and TC
must be the same binary64 value (both sides round the same exact rational
once, to nearest-even), i.e. 0 ulp where north of the 1-ulp bound."""
from __future__ import annotations

import random

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2105_00110_gb300 as tcg
from golden_io import fixtures, load

pytestmark = pytest.mark.gpu

STRATS = ["auto", "bsearch", "merge", "bitmap", "global"]


@pytest.fixture(scope="session", autouse=True)
def _built():
    tcg.build()
    torch.cuda.init()


def gpu_run(src, dst, n, strategy=None, ids=np.int32, on_device=True):
    s = torch.from_numpy(np.ascontiguousarray(src).astype(ids))
    d = torch.from_numpy(np.ascontiguousarray(dst).astype(ids))
    if on_device:
        s, d = s.cuda(), d.cuda()
    res = tcg.triangle_centrality(s, d, n, strategy=strategy)
    torch.cuda.synchronize()
    out = {}
    for k, v in res.items():
        out[k] = v.cpu().numpy() if isinstance(v, torch.Tensor) else v
    return out


def assert_parity(res, ref, n):
    assert res["n"] == n
    assert res["total"] == ref["total"]
    assert res["den"] == ref["den"]
    ptr, adj = ref["ptr"], ref["adj"]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ptr))
    keep = adj > rows
    assert res["m"] == int(keep.sum())
    np.testing.assert_array_equal(res["edge_u"], rows[keep])
    np.testing.assert_array_equal(res["edge_v"], adj[keep])
    np.testing.assert_array_equal(res["tri"], ref["tri"])
    np.testing.assert_array_equal(res["flag"], ref["flag"][keep])
    np.testing.assert_array_equal(res["numer"], ref["numer"])
    if ref["total"] == 0:
        assert res["status"] == tcg.TC_NO_TRIANGLES
        assert np.all(np.isnan(res["tc"]))
    else:
        assert res["status"] == tcg.TC_OK
        # identical binary64 values (0 ulp)
        np.testing.assert_array_equal(res["tc"].view(np.uint64), ref["tc"].view(np.uint64))


def check(src, dst, n, strategy=None, mode="definition", **kw):
    ref = oracle.run(src, dst, n, mode)
    res = gpu_run(src, dst, n, strategy, **kw)
    assert_parity(res, ref, n)
    return res, ref


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("name", fixtures())
def test_golden(name, strategy):
    src, dst, n, _, _ = load(name)
    check(src, dst, n, strategy)


@pytest.mark.parametrize("strategy", STRATS)
def test_closed_forms(strategy):
    for k in (3, 4, 40, 300, 600):
        check(*gg.complete_graph(k), strategy=strategy)
    check(*gg.bridge_to_cliques(5, 6), strategy=strategy)
    check(*gg.disjoint_cliques(4, 7), strategy=strategy)
    s, d, n, _, _ = gg.clique_chain(6, 5)
    check(s, d, n, strategy)
    s, d, n, _, _ = gg.clique_chain(5, 4, ring=True)
    check(s, d, n, strategy)
    check(*gg.single_triangle_with_pendants(3), strategy=strategy)


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("seed", range(4))
def test_gnp(seed, strategy):
    rnd = random.Random(100 + seed)
    n = rnd.randint(20, 160)
    p = rnd.choice([0.02, 0.1, 0.3, 0.7])
    check(*gg.gnp(n, p, seed), strategy=strategy)


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("scale", [8, 10, 12])
def test_rmat(scale, strategy):
    seed = 0x5EED0000 if scale == 12 else 0x5EED0000 + scale
    check(*gg.rmat(scale, seed=seed), strategy=strategy)


@pytest.mark.parametrize("ids,on_device", [(np.int64, False), (np.int64, True), (np.int32, False)])
def test_input_forms(ids, on_device):
    s, d, n = gg.rmat(9, seed=0x5EED0009)
    check(s, d, n, ids=ids, on_device=on_device)


@pytest.mark.parametrize("strategy", STRATS)
def test_rmat16_many_tiles(strategy):
    # hubs become CTA items; several items per hub; oracle in degree-ordered mode
    s, d, n = gg.rmat(16, seed=0x5EED0010)
    res, _ = check(s, d, n, strategy, mode="fast")
    items = res["stats"]["items"]
    assert sum(items) > 0
    if strategy == "auto":
        assert items[2] > 0 and items[4] > 0     # warp items (bitmap or list) and tiny thread items
    if strategy == "bitmap":
        assert items[0] > 0 and items[2] > 0     # CTA bitmaps beyond the per-warp window
    if strategy in ("bsearch", "merge"):
        assert items[0] == items[1] == items[4] == 0 and items[2] > 0
    if strategy == "global":
        assert items[3] == sum(items)


def test_both_bitmap_classes_repeatedly():
    # the bitmap kernel runs with two dynamic shared sizes (small and large
    # windows); alternating them across calls must keep every launch valid
    s, d, n = gg.rmat(21, seed=0x5EED0015)
    g = tcg.Graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    g.set_strategy("bitmap")                   # every window that fits 100 KB is a bitmap
    runs = []
    for it in range(3):
        tri, flags, total, _ = g.count()
        numer, tcv, den, _ = g.centrality()
        torch.cuda.synchronize()
        runs.append((tri.cpu().numpy(), flags.cpu().numpy(), total, tcv.cpu().numpy().view(np.int64)))
        if it == 0:
            items = g.stats()["items"]
            assert items[0] > 0 and items[1] > 0
    g.close()
    ref = gpu_run(s, d, n, strategy="merge")    # no bitmap at all
    for tri, flags, total, tcb in runs:
        assert total == ref["total"]
        np.testing.assert_array_equal(tri, ref["tri"])
        np.testing.assert_array_equal(flags, ref["flag"])
        np.testing.assert_array_equal(tcb, ref["tc"].view(np.int64))


def test_grid_chung_lu_small():
    for strategy in STRATS:
        check(*gg.grid_chung_lu(side=96, seed=0x5EED0002), strategy=strategy)


def test_batched_shapes():
    check(*gg.barabasi_albert(3000, 5, seed=31))
    check(*gg.planted_hierarchy(2000, 20, 8, 0.01, seed=32))


def test_edge_cases():
    e = np.zeros(0, np.int32)
    r = gpu_run(e, e, 0)
    assert r["n"] == 0 and r["m"] == 0 and r["total"] == 0
    r = gpu_run(e, e, 7)
    assert r["m"] == 0 and np.all(r["tri"] == 0) and np.all(np.isnan(r["tc"]))
    # self-loops and duplicates only
    check(np.array([1, 1, 2, 2, 2], np.int32), np.array([1, 2, 1, 2, 1], np.int32), 4)
    # a tree: triangle-free, explicit status
    src = np.arange(1, 50, dtype=np.int32)
    dst = (np.arange(1, 50) // 2).astype(np.int32)
    res, _ = check(src, dst, 50)
    assert res["status"] == tcg.TC_NO_TRIANGLES
    # one triangle plus isolated vertices
    check(np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), 10)


def test_invalid_ids_rejected():
    for bad in ([0, 5], [-1, 2]):
        with pytest.raises(tcg.TCError) as ei:
            gpu_run(np.array(bad, np.int32), np.array([1, 1], np.int32), 5)
        assert ei.value.status == tcg.TC_ERR_INVALID_ARG


def test_call_order():
    g = tcg.Graph(torch.tensor([0, 1], dtype=torch.int32, device="cuda"),
                  torch.tensor([1, 2], dtype=torch.int32, device="cuda"), 3)
    with pytest.raises(tcg.TCError) as ei:
        g.centrality()
    assert ei.value.status == tcg.TC_ERR_STATE
    g.close()


def test_divide_exact():
    rnd = random.Random(9)
    num, dens = [], []
    for _ in range(4000):
        b = rnd.choice([rnd.randint(1, 2**53 - 1), rnd.randint(2**53, 2**64 - 1), rnd.randint(1, 2**64 - 1)])
        a = rnd.randint(0, b)
        num.append(a)
        dens.append(b)
    for den in sorted(set(dens))[:40] + [2**64 - 1, 3, 2**53 + 1, 0]:
        a = np.array([x % (den + 1) if den else x for x in num[:512]] + [0, den], dtype=np.uint64)
        t = torch.from_numpy(a).cuda()
        out = torch.empty(len(a), dtype=torch.float64, device="cuda")
        tcg.tc_divide(t, den, out)
        got = out.cpu().numpy()
        want = np.array([oracle.div_rn(int(x), den) for x in a])
        np.testing.assert_array_equal(got.view(np.uint64), want.view(np.uint64))


def test_repeatable_and_relabel_invariant():
    s, d, n = gg.rmat(11, seed=0x5EED000B)
    a = gpu_run(s, d, n)
    b = gpu_run(s, d, n)
    for k in ("tri", "numer", "tc", "flag"):
        np.testing.assert_array_equal(a[k], b[k])
    ps, pd, perm = gg.permute_labels(s, d, n, seed=5)
    c = gpu_run(ps, pd, n)
    np.testing.assert_array_equal(c["tri"][perm], a["tri"])
    np.testing.assert_array_equal(c["numer"][perm], a["numer"])


def test_planner_settings_change_no_result():
    # chunk sizes and the CTA threshold move work between kernels and items;
    # counts, flags and TC stay the same
    s, d, n = gg.rmat(15, seed=0x5EED0300)
    g = tcg.Graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    try:
        # the default CTA chunk follows the graph's wedges: wedges / (64 SMs), within [2^16, 2^22]
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        chunk = int(min(4194304.0, max(65536.0, g.stats()["wedges"] / (64.0 * sms))))
        assert tcg.tc_get_plan_params(g.h) == dict(cta_min_work=4096, cta_chunk=chunk, warp_chunk=32768)
        runs = []
        for params in ((4096, 4194304, 32768), (256, 1024, 512), (1 << 40, 1 << 40, 1 << 40), (0, 1, 1)):
            tcg.tc_set_plan_params(g.h, *params)
            tri, flags, total, _ = g.count()
            _, tcv, _, _ = g.centrality()
            torch.cuda.synchronize()
            runs.append((total, tri.view(torch.int64).cpu(), flags.cpu(), tcv.view(torch.int64).cpu(),
                         g.stats()["items"]))
        for r in runs[1:]:
            assert r[0] == runs[0][0]
            assert torch.equal(r[1], runs[0][1]) and torch.equal(r[2], runs[0][2]) and torch.equal(r[3], runs[0][3])
        assert runs[1][4] != runs[0][4]          # the plan did change
        with pytest.raises(tcg.TCError):
            tcg.tc_set_plan_params(g.h, 4096, 0, 1)
    finally:
        g.close()


def test_upload_timed_not_counted():
    # host pairs: the profile times their upload as "copy_h2d_pairs"; the
    # launch count is the same as for the same pairs already on the device
    s, d, n = gg.rmat(12, seed=0x5EED0400)
    hs, hd = torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory()
    counts, profs = [], []
    for src, dst in ((hs, hd), (hs.cuda(), hd.cuda())):
        torch.cuda.synchronize()
        tcg.tc_profile_reset()
        tcg.tc_profile_enable(True)
        l0 = tcg.tc_launch_count()
        g = tcg.tc_build_csr(src, dst, n)
        torch.cuda.synchronize()
        counts.append(tcg.tc_launch_count() - l0)
        tcg.tc_profile_enable(False)
        profs.append(tcg.tc_profile_read())
        tcg.tc_graph_free(g)
    assert counts[0] == counts[1] > 0
    launches, ms = profs[0]["copy_h2d_pairs"]
    assert launches == 1 and ms > 0
    assert "copy_h2d_pairs" not in profs[1]
    assert {k: v[0] for k, v in profs[0].items() if k != "copy_h2d_pairs"} == {k: v[0] for k, v in profs[1].items()}


@pytest.mark.parametrize("strategy", ["auto", "bitmap", "global"])
def test_runs_of_every_length_closed_form(strategy):
    # K_k in rank space has a run of every length 0 .. k-1, so the build
    # sorts runs on both sides of each tier boundary (32, 256, 1024, and the
    # in-place sort above 4096); closed forms check every output
    k = 4200
    s, d, n = gg.complete_graph(k)
    g = tcg.Graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    try:
        g.set_strategy(strategy)
        tri, flags, total, _ = g.count()
        numer, tcv, den, _ = g.centrality()
        eu, ev = g.edges()
        tri2, et, total2, _ = g.edge_triangles()
        torch.cuda.synchronize()
        c2 = (k - 1) * (k - 2) // 2
        assert total == total2 == k * c2 // 3 and den == 3 * total
        assert torch.all(tri.view(torch.int64) == c2) and torch.equal(tri2.view(torch.int64), tri.view(torch.int64))
        assert torch.all(flags == 1) and torch.all(et.view(torch.int32) == k - 2)
        assert torch.all(numer.view(torch.int64) == k * c2)
        assert torch.all(tcv == 1.0)
        iu = np.triu_indices(k, 1)
        assert np.array_equal(eu.cpu().numpy(), iu[0]) and np.array_equal(ev.cpu().numpy(), iu[1])
    finally:
        g.close()
