"""The allocation-free entry point tc_csr_centrality_noalloc: on the same
graphs it returns exactly what tc_count followed by tc_centrality return
(counts, numerators, TC bit for bit), on two calls in a row and across
graphs, works from its fixed working array alone, and refuses sizes beyond
its limits before touching the device.

The file is named to be collected last, so it also runs after every other
GPU test has used (and released) the library's device pool."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import graphgen as gg
import paper_2105_00110_gb300 as tcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    tcg.build()
    torch.cuda.init()


def csr_of(src, dst, n):
    """Sorted, symmetric, loop-free CSR of the simple graph on the pairs."""
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    lo, hi = np.minimum(s[keep], d[keep]), np.maximum(s[keep], d[keep])
    key = np.unique(lo * n + hi) if lo.size else np.zeros(0, np.int64)
    lo, hi = key // max(n, 1), key % max(n, 1)
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32)


def graphs():
    tree = (np.arange(1, 300, dtype=np.int32), (np.arange(1, 300) // 3).astype(np.int32), 300)
    return {
        "rmat12": gg.rmat(12, seed=91),
        "ba3000": gg.barabasi_albert(3000, 6, seed=92),
        "k40": gg.complete_graph(40),
        "tree": tree,
        "isolated": (np.zeros(0, np.int32), np.zeros(0, np.int32), 7),
        "rmat16": gg.rmat(16, 14, seed=93),   # near both size limits
    }


def existing_path(src, dst, n):
    out = tcg.triangle_centrality(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    return out["tri"], out["numer"], out["tc"]


def noalloc(row_ptr, col, n):
    tri = torch.full((n,), 7, dtype=torch.int64, device="cuda").view(torch.uint64)
    numer = torch.full((n,), 7, dtype=torch.int64, device="cuda").view(torch.uint64)
    tc = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    tcg.tc_csr_centrality_noalloc(row_ptr, col, n, tri, numer, tc)
    return tri, numer, tc


def same(a, b):
    assert a.dtype == b.dtype and a.shape == b.shape
    return np.array_equal(a.cpu().numpy().view(np.int64), b.cpu().numpy().view(np.int64))


def test_limits_hold_for_the_large_case():
    s, d, n = graphs()["rmat16"]
    row_ptr, col = csr_of(s, d, n)
    assert n <= tcg.TC_NOALLOC_MAX_VERTICES and col.size <= tcg.TC_NOALLOC_MAX_ENTRIES
    assert col.size > tcg.TC_NOALLOC_MAX_ENTRIES // 2


@pytest.mark.parametrize("name", list(graphs()))
def test_matches_existing_entry_points_twice_in_a_row(name):
    s, d, n = graphs()[name]
    tri_ref, numer_ref, tc_ref = existing_path(s, d, n)
    row_ptr, col = csr_of(s, d, n)
    rp, cl = torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda()
    before = tcg.tc_launch_count()
    first = noalloc(rp, cl, n)
    second = noalloc(rp, cl, n)          # no synchronisation in between
    torch.cuda.synchronize()
    assert tcg.tc_launch_count() - before == (8 if n else 0)
    for got in (first, second):
        assert same(got[0], tri_ref)
        assert same(got[1], numer_ref)
        assert same(got[2], tc_ref)


def test_consecutive_graphs_share_the_array_cleanly():
    cases = list(graphs().values())
    inputs = []
    for s, d, n in cases:
        row_ptr, col = csr_of(s, d, n)
        inputs.append((torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda(), n))
    outs = [noalloc(*x) for x in inputs]   # back to back on one stream
    torch.cuda.synchronize()
    for (s, d, n), got in zip(cases, outs):
        tri_ref, numer_ref, tc_ref = existing_path(s, d, n)
        assert same(got[0], tri_ref) and same(got[1], numer_ref) and same(got[2], tc_ref)


def test_empty_graph_is_a_no_op():
    rp = torch.zeros(1, dtype=torch.int64, device="cuda")
    cl = torch.zeros(0, dtype=torch.int32, device="cuda")
    tcg.tc_csr_centrality_noalloc(rp, cl, 0)


def test_sizes_beyond_the_limits_are_refused():
    big = tcg.TC_NOALLOC_MAX_VERTICES + 1
    rp = torch.zeros(big + 1, dtype=torch.int64, device="cuda")
    cl = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(tcg.TCError) as e:
        tcg.tc_csr_centrality_noalloc(rp, cl, big)
    assert e.value.status == tcg.TC_ERR_INVALID_ARG
    rp = torch.zeros(101, dtype=torch.int64, device="cuda")
    cl = torch.zeros(tcg.TC_NOALLOC_MAX_ENTRIES + 2, dtype=torch.int32, device="cuda")
    with pytest.raises(tcg.TCError) as e:
        tcg.tc_csr_centrality_noalloc(rp, cl, 100)
    assert e.value.status == tcg.TC_ERR_INVALID_ARG
    cl = torch.zeros(3, dtype=torch.int32, device="cuda")      # odd: not symmetric
    with pytest.raises(tcg.TCError) as e:
        tcg.tc_csr_centrality_noalloc(rp, cl, 100)
    assert e.value.status == tcg.TC_ERR_INVALID_ARG


def test_unsorted_row_is_reported_in_the_outputs():
    s, d, n = gg.complete_graph(6)
    row_ptr, col = csr_of(s, d, n)
    col[[0, 1]] = col[[1, 0]]             # row 0 out of order; ids stay in range
    tri, numer, tc = noalloc(torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda(), n)
    torch.cuda.synchronize()
    assert (tri.cpu().numpy().view(np.int64) == -1).all()
    assert (numer.cpu().numpy().view(np.int64) == -1).all()
    assert np.isnan(tc.cpu().numpy()).all()
    # the next call on a valid graph is unaffected
    row_ptr, col = csr_of(s, d, n)
    got = noalloc(torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda(), n)
    ref = existing_path(s, d, n)
    assert all(same(a, b) for a, b in zip(got, ref))


def test_one_sided_upper_entry_is_reported_in_the_outputs():
    # rows {1, 2, 3}, {2}, {}, {}: entries above their row whose reverse
    # entry is missing (row 1 lacks 0, row 2 lacks 0 and 1, row 3 lacks 0)
    row_ptr = torch.tensor([0, 3, 4, 4, 4], dtype=torch.int64, device="cuda")
    col = torch.tensor([1, 2, 3, 2], dtype=torch.int32, device="cuda")
    tri, numer, tc = noalloc(row_ptr, col, 4)
    torch.cuda.synchronize()
    assert (tri.cpu().numpy().view(np.int64) == -1).all()
    assert (numer.cpu().numpy().view(np.int64) == -1).all()
    assert np.isnan(tc.cpu().numpy()).all()
    # one missing reverse entry in an otherwise valid graph: K_5 with row 4
    # lacking 3 (its rows stay sorted and nnz stays even by dropping 0 from row 3 too)
    s, d, n = gg.complete_graph(5)
    rp, cl = csr_of(s, d, n)
    rows = [list(cl[rp[i]:rp[i + 1]]) for i in range(n)]
    rows[4].remove(3)
    rows[3].remove(0)
    rp2 = np.zeros(n + 1, np.int64)
    np.cumsum([len(r) for r in rows], out=rp2[1:])
    cl2 = np.concatenate([np.asarray(r, np.int32) for r in rows])
    tri, numer, tc = noalloc(torch.from_numpy(rp2).cuda(), torch.from_numpy(cl2).cuda(), n)
    torch.cuda.synchronize()
    assert (tri.cpu().numpy().view(np.int64) == -1).all()
    assert np.isnan(tc.cpu().numpy()).all()


def test_triangle_free_graph_is_told_apart_from_a_rejected_one():
    tree = (np.arange(1, 50, dtype=np.int32), (np.arange(1, 50) // 2).astype(np.int32), 50)
    row_ptr, col = csr_of(*tree)
    tri, numer, tc = noalloc(torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda(), 50)
    torch.cuda.synchronize()
    assert (tri.cpu().numpy() == 0).all() and np.isnan(tc.cpu().numpy()).all()


def test_wrapper_rejects_bad_outputs_before_the_call():
    s, d, n = gg.complete_graph(6)
    row_ptr, col = csr_of(s, d, n)
    rp, cl = torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col).cuda()
    u64 = lambda k: torch.zeros(k, dtype=torch.int64, device="cuda").view(torch.uint64)
    bad = [
        dict(row_ptr=rp[:-1], col=cl, n=n),                                        # row_ptr too short
        dict(row_ptr=rp, col=cl.view(1, -1), n=n),                                 # col not 1-D
        dict(row_ptr=rp, col=cl, n=n, tri=u64(n - 1)),                             # tri too short
        dict(row_ptr=rp, col=cl, n=n, numer=torch.zeros(n, dtype=torch.int64, device="cuda")),  # not uint64
        dict(row_ptr=rp, col=cl, n=n, tc=torch.zeros(n, dtype=torch.float32, device="cuda")),   # float32
        dict(row_ptr=rp, col=cl, n=n, tc=torch.zeros(n, dtype=torch.float64)),     # host memory
        dict(row_ptr=rp.cpu(), col=cl, n=n),                                       # host memory
    ]
    before = tcg.tc_launch_count()
    for kw in bad:
        with pytest.raises(ValueError):
            tcg.tc_csr_centrality_noalloc(**kw)
    assert tcg.tc_launch_count() == before
