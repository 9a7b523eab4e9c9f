"""Pins for the CPU oracle (no GPU): brute force, closed forms, the paper's
worked examples, invariants and exact rounding."""
from __future__ import annotations

import random
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle
from brute import brute
from golden_io import fixtures, load


def _flag_of(res, v, u):
    ptr, adj = res["ptr"], res["adj"]
    row = adj[ptr[v]:ptr[v + 1]]
    k = int(np.searchsorted(row, u))
    assert row[k] == u
    return int(res["flag"][ptr[v] + k])


def _check_against_brute(src, dst, n, mode):
    b = brute(src, dst, n)
    r = oracle.run(src, dst, n, mode)
    assert r["total"] == b["total"]
    assert r["tri"].tolist() == b["tri"]
    for v in range(n):
        row = r["adj"][r["ptr"][v]:r["ptr"][v + 1]].tolist()
        assert row == np.flatnonzero(b["A"][v]).tolist()
        flagged = [u for u in row if _flag_of(r, v, u)]
        assert flagged == b["tnb"][v]
    assert r["core"].tolist() == b["core"]
    assert r["noncore"].tolist() == b["noncore"]
    if b["total"]:
        for v in range(n):
            assert Fraction(int(r["numer"][v]), r["den"]) == b["tc"][v]
            assert r["tc"][v] == float(b["tc"][v])          # correctly rounded
    else:
        assert np.all(np.isnan(r["tc"]))
        assert np.all(r["numer"] == 0)
    assert np.array_equal(r["numer"], r["numer_alg"])
    assert r["den_alg"] == r["den"]
    return r


@pytest.mark.parametrize("mode", ["definition", "fast"])
@pytest.mark.parametrize("seed", range(6))
def test_brute_force_gnp(seed, mode):
    rnd = random.Random(seed)
    n = rnd.randint(4, 36)
    p = rnd.choice([0.08, 0.2, 0.35, 0.6])
    src, dst, n = gg.gnp(n, p, seed)
    _check_against_brute(src, dst, n, mode)


@pytest.mark.parametrize("mode", ["definition", "fast"])
def test_brute_force_messy_input(mode):
    # duplicates, both directions, self-loops and isolated vertices
    src = np.array([0, 1, 1, 2, 2, 3, 0, 4, 4, 5, 7, 7], dtype=np.int32)
    dst = np.array([1, 0, 2, 0, 2, 0, 2, 5, 6, 6, 7, 4], dtype=np.int32)
    _check_against_brute(src, dst, 9, mode)


def test_empty_and_triangle_free():
    r = oracle.run(np.zeros(0, np.int32), np.zeros(0, np.int32), 5)
    assert r["total"] == 0 and np.all(np.isnan(r["tc"]))
    s, d, n = gg.gnp(30, 0.0, 1)
    r = oracle.run(s, d, n)
    assert r["total"] == 0
    # a tree: no triangles, counts and numerators all zero
    src = np.arange(1, 20, dtype=np.int32)
    dst = (np.arange(1, 20) // 2).astype(np.int32)
    r = oracle.run(src, dst, 20)
    assert r["total"] == 0 and not r["flag"].any() and not r["numer"].any()


def test_out_of_range_id_rejected():
    with pytest.raises(ValueError):
        oracle.OracleGraph(np.array([0], np.int32), np.array([5], np.int32), 5)


# ---------------- closed forms (section "Observations") ----------------

@pytest.mark.parametrize("k", [3, 4, 5, 9, 17])
def test_obs1_clique(k):
    r = oracle.run(*gg.complete_graph(k))
    assert r["total"] == k * (k - 1) * (k - 2) // 6
    assert np.all(r["tc"] == 1.0)


@pytest.mark.parametrize("d,k", [(1, 3), (4, 6), (3, 5), (7, 4)])
def test_obs2_bridge(d, k):
    r = oracle.run(*gg.bridge_to_cliques(d, k))
    assert Fraction(int(r["numer"][0]), r["den"]) == Fraction(3, k)


@pytest.mark.parametrize("p,k", [(1, 3), (2, 4), (4, 6), (5, 3)])
def test_obs3_disjoint(p, k):
    r = oracle.run(*gg.disjoint_cliques(p, k))
    for v in range(p * k):
        assert Fraction(int(r["numer"][v]), r["den"]) == Fraction(1, p)


@pytest.mark.parametrize("p,k", [(4, 3), (5, 4), (6, 5), (7, 3)])
def test_obs4_chain(p, k):
    src, dst, n, joiners, heads = gg.clique_chain(p, k)
    r = oracle.run(src, dst, n)
    # joiners of the first and last copy join a head/tail copy (case 2)
    end_joiners = {joiners[0], joiners[-1]}
    for v in range(n):
        got = Fraction(int(r["numer"][v]), r["den"])
        if v in joiners:
            want = Fraction(2 * k + 1, p * k) if v in end_joiners else Fraction(2 * k + 2, p * k)
        else:
            want = Fraction(k + 1, p * k) if v in heads else Fraction(k + 2, p * k)
        assert got == want, (v, got, want)


@pytest.mark.parametrize("p,k", [(4, 3), (5, 4), (6, 6)])
def test_obs5_ring(p, k):
    src, dst, n, joiners, _ = gg.clique_chain(p, k, ring=True)
    r = oracle.run(src, dst, n)
    for v in range(n):
        got = Fraction(int(r["numer"][v]), r["den"])
        want = Fraction(2 * k + 2, p * k) if v in joiners else Fraction(k + 2, p * k)
        assert got == want


def test_obs5_ring_of_three_is_not_covered():
    # Reading adopted: with p = 3 the three joiners form one extra triangle,
    # so the ring formula does not apply (checked here by brute force).
    src, dst, n, joiners, _ = gg.clique_chain(3, 3, ring=True)
    b = brute(src, dst, n)
    assert b["total"] == 4
    assert b["tc"][joiners[0]] != Fraction(2 * 3 + 2, 9)
    _check_against_brute(src, dst, n, "definition")


@pytest.mark.parametrize("pendants", [0, 1, 3])
def test_obs6_single_triangle(pendants):
    src, dst, n = gg.single_triangle_with_pendants(pendants)
    r = oracle.run(src, dst, n)
    assert r["total"] == 1
    for v in range(n):
        assert r["tc"][v] == 1.0        # triangle vertices and their leaves


# ---------------- worked examples printed in the paper ----------------

@pytest.mark.parametrize("name", fixtures())
def test_golden_fixture(name):
    src, dst, n, names, expect = load(name)
    for mode in ("definition", "fast"):
        r = oracle.run(src, dst, n, mode)
        tcf = [Fraction(int(r["numer"][v]), r["den"]) for v in range(n)]
        for kind, v, val in expect:
            if kind == "total":
                assert r["total"] == val
            elif kind == "n":
                assert r["ptr"].shape[0] - 1 == val
            elif kind == "m":
                assert len(r["adj"]) // 2 == val
            elif kind == "core":
                assert int(r["core"][v]) == val
            elif kind == "noncore":
                assert int(r["noncore"][v]) == val
            elif kind == "tc":
                assert tcf[v] == val
                assert r["tc"][v] == float(val)
            elif kind == "top":
                assert all(tcf[v] > tcf[u] for u in range(n) if u != v), names[v]
        # every fixture also agrees with brute force
        _check_against_brute(src, dst, n, mode)


# ---------------- invariants on R-MAT graphs ----------------

@pytest.fixture(scope="module")
def rmat10():
    s, d, n = gg.rmat(10, seed=0x5EED000A)
    return s, d, n, oracle.run(s, d, n, "definition")


def test_modes_agree(rmat10):
    s, d, n, r = rmat10
    f = oracle.run(s, d, n, "fast")
    for key in ("t", "tri", "numer", "tc"):
        assert np.array_equal(r[key], f[key], equal_nan=True), key
    assert r["total"] == f["total"]


def test_invariants(rmat10):
    s, d, n, r = rmat10
    assert int(r["tri"].sum()) == 3 * r["total"]
    assert int(r["t"].sum()) == 6 * r["total"]
    assert np.all(r["numer"] <= r["den"])                  # Proposition 1
    assert np.all((r["tc"] >= 0) & (r["tc"] <= 1))
    assert np.array_equal(r["numer"], r["numer_alg"])      # Proposition 2
    # each triangle puts at most 3 into a numerator and the flag is symmetric
    ptr, adj, fl = r["ptr"], r["adj"], r["flag"]
    rows = np.repeat(np.arange(n), np.diff(ptr))
    key = rows.astype(np.int64) * n + adj
    rkey = adj.astype(np.int64) * n + rows
    order = np.argsort(key)
    pos = np.searchsorted(key[order], rkey)
    assert np.array_equal(fl, fl[order][pos])


def test_relabel_invariance(rmat10):
    s, d, n, r = rmat10
    ps, pd, perm = gg.permute_labels(s, d, n, seed=77)
    q = oracle.run(ps, pd, n)
    assert np.array_equal(q["tri"][perm], r["tri"])
    assert np.array_equal(q["numer"][perm], r["numer"])
    assert np.array_equal(q["tc"][perm], r["tc"], equal_nan=True)


def test_disjoint_union(rmat10):
    s, d, n, r = rmat10
    s2, d2, n2 = gg.rmat(8, seed=0x5EED0008)
    r2 = oracle.run(s2, d2, n2)
    u = oracle.run(np.concatenate([s, s2 + n]), np.concatenate([d, d2 + n]), n + n2)
    assert np.array_equal(u["tri"], np.concatenate([r["tri"], r2["tri"]]))
    assert np.array_equal(u["numer"], np.concatenate([r["numer"], r2["numer"]]))
    assert u["total"] == r["total"] + r2["total"]


def test_sample_matches_full(rmat10):
    s, d, n, r = rmat10
    g = oracle.OracleGraph(s, d, n)
    vs = np.array([0, 5, 17, 1000, n - 1] + list(np.argsort(-np.diff(r["ptr"]))[:5]), np.int64)
    tri, num, rows = g.sample(vs, with_rows=True)
    assert np.array_equal(tri, r["tri"][vs])
    assert np.array_equal(num, r["numer"][vs])
    want = np.concatenate([r["t"][r["ptr"][v]:r["ptr"][v + 1]] for v in vs])
    assert np.array_equal(rows, want)


def test_sample_tri_matches_full_and_brute(rmat10):
    # the cheap sampler (△ and rows of T only) against the full routines and,
    # on a tiny graph, against the O(n^3) brute force
    s, d, n, r = rmat10
    g = oracle.OracleGraph(s, d, n)
    vs = np.array([0, 5, 17, 1000, n - 1] + list(np.argsort(-np.diff(r["ptr"]))[:5]), np.int64)
    tri, rows = g.sample_tri(vs)
    assert np.array_equal(tri, r["tri"][vs])
    want = np.concatenate([r["t"][r["ptr"][v]:r["ptr"][v + 1]] for v in vs])
    assert np.array_equal(rows, want)
    s2, d2, n2 = gg.gnp(30, 0.3, 77)
    b = brute(s2, d2, n2)
    tri2, _ = oracle.OracleGraph(s2, d2, n2).sample_tri(np.arange(n2))
    assert [int(x) for x in tri2] == list(b["tri"])


def test_plausible_mistakes_are_caught():
    """Mistakes a restatement could make, applied to the oracle's outputs on
    the fixtures, are each rejected by a pin."""
    src, dst, n, _, expect = load("fig2_worked_example.txt")
    r = oracle.run(src, dst, n)
    tcv = {v: val for kind, v, val in expect if kind == "tc"}
    v = next(iter(tcv))
    good = Fraction(int(r["numer"][v]), r["den"])
    assert good == tcv[v]
    # dropped △(v) from the core sum
    assert Fraction(int(r["numer"][v] - r["tri"][v]), r["den"]) != tcv[v]
    # non-core weighted 1 instead of 3
    assert Fraction(int(r["core"][v] + r["noncore"][v]), r["den"]) != tcv[v]
    # △(v) = ||T_v||_1 without the ½ (the printed "T_v^T 1"): the total
    # printed with the figure (3) rejects the doubled counts
    assert int((2 * r["tri"]).sum()) // 3 != 3 and r["total"] == 3
    # Observation 2 rejects the 1-weight non-core too
    s2, d2, n2 = gg.bridge_to_cliques(4, 6)
    r2 = oracle.run(s2, d2, n2)
    assert Fraction(int(r2["core"][0] + r2["noncore"][0]), r2["den"]) != Fraction(1, 2)


# ---------------- exact rounding ----------------

def test_division_small_is_ieee():
    rnd = random.Random(5)
    for _ in range(2000):
        b = rnd.randint(1, 2**53 - 1)
        a = rnd.randint(0, b)
        assert oracle.div_rn(a, b) == a / b
        assert oracle.div_rn_long(a, b) == float(Fraction(a, b))


def test_division_large_matches_fraction():
    rnd = random.Random(6)
    cases = [(2**64 - 1, 2**64 - 1), (1, 2**64 - 1), (2**63, 2**64 - 3), (3, 2**53 + 1),
             (2**53 + 1, 2**54 + 3), (2**62 + 12345, 3 * 2**61 + 7)]
    for _ in range(3000):
        b = rnd.randint(2**53, 2**64 - 1)
        a = rnd.randint(0, b)
        cases.append((a, b))
    # ties: a/b exactly halfway between two doubles
    for _ in range(200):
        m = rnd.randint(2**52, 2**53 - 1)
        a, b = 2 * m + 1, 2**55
        cases.append((a, b))
    for a, b in cases:
        assert oracle.div_rn(a, b) == float(Fraction(a, b)), (a, b)
    assert np.isnan(oracle.div_rn(0, 0))


@pytest.mark.parametrize("threads", [2, 7])
@pytest.mark.parametrize("mode", ["definition", "fast"])
def test_threaded_oracle_equals_single_thread(mode, threads):
    # the threaded routines time the oracle on all host cores; they must
    # return exactly what the pinned single-threaded routines return
    cases = [gg.rmat(12, seed=31), gg.barabasi_albert(3000, 5, seed=32),
             gg.planted_hierarchy(900, 12, 6, 0.01, seed=33), gg.grid_chung_lu(side=40, seed=34),
             gg.gnp(60, 0.3, 35), (np.zeros(0, np.int32), np.zeros(0, np.int32), 5),
             (np.array([0, 1, 1, 3], np.int32), np.array([1, 0, 2, 3], np.int32), 6)]
    for src, dst, n in cases:
        a = oracle.run(src, dst, n, mode)
        b = oracle.run(src, dst, n, mode, threads=threads, algebraic=False)
        for k in ("ptr", "adj", "t", "flag", "tri", "numer", "core", "noncore"):
            assert np.array_equal(a[k], b[k]), k
        assert a["total"] == b["total"] and a["den"] == b["den"]
        assert np.array_equal(a["tc"].view(np.int64), b["tc"].view(np.int64))
