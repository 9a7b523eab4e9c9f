"""O(n^3) brute-force triangle centrality for tiny graphs (test pin only).

Written straight from the paper's Notation section and Definition 1, with no
shared code: the adjacency matrix, every vertex triple, exact fractions.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np


def brute(src, dst, n):
    A = np.zeros((n, n), dtype=bool)
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            A[a, b] = A[b, a] = True
    tri = [0] * n
    total = 0
    for i, j, k in combinations(range(n), 3):
        if A[i, j] and A[j, k] and A[i, k]:
            tri[i] += 1; tri[j] += 1; tri[k] += 1
            total += 1
    nbrs = [np.flatnonzero(A[v]).tolist() for v in range(n)]
    # u ∈ N△(v) iff N(u) ∩ N(v) is non-empty
    tnb = [[u for u in nbrs[v] if bool(np.any(A[u] & A[v]))] for v in range(n)]
    core = [tri[v] + sum(tri[u] for u in tnb[v]) for v in range(n)]
    noncore = [sum(tri[w] for w in nbrs[v] if w not in tnb[v]) for v in range(n)]
    tc = []
    for v in range(n):
        if total == 0:
            tc.append(None)
        else:
            tc.append((Fraction(core[v], 3) + noncore[v]) / total)
    return dict(A=A, tri=tri, total=total, tnb=tnb, core=core, noncore=noncore, tc=tc)
