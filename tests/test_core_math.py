"""The arithmetic the dense core of the count step relies on, checked by
brute force on small graphs (CPU only, numpy):

- in degree order, a triangle whose lowest vertex is among the top C ranks
  has all three vertices there, so the triangles split exactly into those
  inside the core and those whose lowest vertex lies outside it;
- on the core, T = A_c² ∘ A_c counts, on each edge, the triangles through it
  (the matrix form T = A² ∘ A of the section "Notation"), so half of the row
  sums of T are the core triangles at each vertex, ΣT / 3 is their number,
  and T > 0 marks the core edges that lie in a core triangle."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import graphgen as gg


def simple_graph(src, dst, n):
    A = np.zeros((n, n), dtype=np.int64)
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            A[a, b] = A[b, a] = 1
    return A


def degree_ranks(A):
    deg = A.sum(1)
    order = np.lexsort((np.arange(len(deg)), deg))   # ascending degree, ties by label
    rank = np.empty(len(deg), dtype=np.int64)
    rank[order] = np.arange(len(deg))
    return rank


def triangles(A):
    n = len(A)
    return [t for t in itertools.combinations(range(n), 3) if A[t[0], t[1]] and A[t[0], t[2]] and A[t[1], t[2]]]


@pytest.mark.parametrize("graph", ["gnp", "rmat", "hierarchy", "clique"])
def test_core_split_and_masked_product(graph):
    if graph == "gnp":
        src, dst, n = gg.gnp(60, 0.3, 71)
    elif graph == "rmat":
        src, dst, n = gg.rmat(6, seed=72)
    elif graph == "hierarchy":
        src, dst, n = gg.planted_hierarchy(70, 6, 4, 0.05, seed=73)
    else:
        src, dst, n = gg.complete_graph(12)
    A = simple_graph(src, dst, n)
    rank = degree_ranks(A)
    tris = triangles(A)
    assert tris
    for C in (1, 3, n // 4, n // 2, n):
        t = n - C                                    # the core: ranks t .. n-1
        core = rank >= t
        inside = [x for x in tris if core[list(x)].all()]
        low_in_core = [x for x in tris if rank[list(x)].min() >= t]
        assert sorted(inside) == sorted(low_in_core)                 # the split is exact
        idx = np.nonzero(core)[0]
        Ac = A[np.ix_(idx, idx)]
        T = (Ac @ Ac) * Ac
        per_vertex = np.zeros(n, dtype=np.int64)
        for x in inside:
            per_vertex[list(x)] += 1
        assert np.array_equal(T.sum(1) // 2, per_vertex[idx])        # half the row sums
        assert np.all(T.sum(1) % 2 == 0)
        assert np.triu(T, 1).sum() == 3 * len(inside)                # ΣT / 3, each core edge once
        in_core_triangle = np.zeros_like(Ac)
        pos = {v: i for i, v in enumerate(idx.tolist())}
        for x in inside:
            for a, b in itertools.combinations(x, 2):
                in_core_triangle[pos[a], pos[b]] = in_core_triangle[pos[b], pos[a]] = 1
        assert np.array_equal(T > 0, in_core_triangle > 0)           # the flags
