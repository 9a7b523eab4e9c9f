"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module draws edge lists only; it holds none of the triangle-centrality
arithmetic.  The heavy generators (R-MAT, grid + Chung-Lu, Barabasi-Albert,
planted hierarchy) are plain C in ``graphgen.c``, compiled on first use
into ``graphgen/_build``; the closed-form families of the paper's
observations (section "Observations") are small pure-Python constructions.

Every generator returns ``(src, dst, n)`` with ``src``/``dst`` int32 numpy
arrays of equal length (loops and duplicates possibly present) and ``n`` the
vertex count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_SRC = os.path.join(_HERE, "graphgen.c")
_lock = threading.Lock()
_lib = None

# Quadrant probabilities of the R-MAT workloads (a, b, c); d = 1 - a - b - c.
RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (gcc, no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, u64, i32p, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double
            lib.gg_hash.restype = u64
            lib.gg_hash.argtypes = [u64, u64, u64]
            lib.gg_permutation.restype = ctypes.c_int
            lib.gg_permutation.argtypes = [u64, u64, i64, i32p]
            lib.gg_rmat.restype = ctypes.c_int
            lib.gg_rmat.argtypes = [u64, ctypes.c_int, i64, dbl, dbl, dbl, ctypes.c_int,
                                    ctypes.c_int, i32p, i32p]
            lib.gg_grid_cl.restype = i64
            lib.gg_grid_cl.argtypes = [u64, i64, dbl, dbl, dbl, ctypes.c_int, i64, i32p, i32p]
            lib.gg_ba_count.restype = i64
            lib.gg_ba_count.argtypes = [i64, i64]
            lib.gg_ba.restype = i64
            lib.gg_ba.argtypes = [u64, i64, i64, i32p, i32p]
            lib.gg_hierarchy.restype = i64
            lib.gg_hierarchy.argtypes = [u64, i64, i64, i64, dbl, i32p, i32p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def gen_hash(seed: int, stream: int, ctr: int) -> int:
    """The counter-based 64-bit draw every generator is built on."""
    return int(_load().gg_hash(seed & (2**64 - 1), stream, ctr))


def rmat(scale: int, edge_factor: int = 16, seed: int = 0x5EED0000, abc=RMAT_ABC,
         permute: bool = True, threads: int | None = None, samples: int | None = None):
    """R-MAT pairs: ``edge_factor * 2**scale`` samples over ``2**scale`` vertices."""
    n = 1 << scale
    s = int(samples) if samples is not None else edge_factor * n
    src = np.empty(s, dtype=np.int32)
    dst = np.empty(s, dtype=np.int32)
    rc = _load().gg_rmat(seed, scale, s, abc[0], abc[1], abc[2], 1 if permute else 0,
                         _threads(threads), _ptr(src), _ptr(dst))
    if rc != 0:
        raise RuntimeError("gg_rmat failed (%d)" % rc)
    return src, dst, n


def grid_chung_lu(side: int = 4096, pdiag: float = 0.05, gamma: float = 2.1,
                  mean_deg: float = 4.0, seed: int = 0x5EED0002, threads: int | None = None):
    """side x side grid + per-cell diagonal with prob. pdiag + Chung-Lu overlay."""
    lib = _load()
    total = lib.gg_grid_cl(seed, side, pdiag, gamma, mean_deg, 1, 0, None, None)
    if total < 0:
        raise RuntimeError("gg_grid_cl failed (%d)" % total)
    src = np.empty(total, dtype=np.int32)
    dst = np.empty(total, dtype=np.int32)
    got = lib.gg_grid_cl(seed, side, pdiag, gamma, mean_deg, _threads(threads), total,
                         _ptr(src), _ptr(dst))
    if got != total:
        raise RuntimeError("gg_grid_cl failed (%d)" % got)
    return src, dst, side * side


def barabasi_albert(n: int, mm: int, seed: int):
    lib = _load()
    total = lib.gg_ba_count(n, mm)
    if total < 0:
        raise ValueError("need n >= mm + 1")
    src = np.empty(total, dtype=np.int32)
    dst = np.empty(total, dtype=np.int32)
    got = lib.gg_ba(seed, n, mm, _ptr(src), _ptr(dst))
    if got != total:
        raise RuntimeError("gg_ba failed (%d)" % got)
    return src, dst, n


def planted_hierarchy(n: int, cliques: int, k: int, pnoise: float, seed: int):
    lib = _load()
    bound = lib.gg_hierarchy(seed, n, cliques, k, pnoise, None, None)
    if bound < 0:
        raise ValueError("need n >= 1 + cliques*k")
    src = np.empty(bound, dtype=np.int32)
    dst = np.empty(bound, dtype=np.int32)
    got = lib.gg_hierarchy(seed, n, cliques, k, pnoise, _ptr(src), _ptr(dst))
    if got < 0:
        raise RuntimeError("gg_hierarchy failed (%d)" % got)
    return src[:got].copy(), dst[:got].copy(), n


def gnp(n: int, p: float, seed: int):
    """G(n, p) on all unordered pairs (small n only)."""
    iu, ju = np.triu_indices(n, 1)
    draws = np.array([gen_hash(seed, 9, int(k)) for k in range(len(iu))], dtype=np.uint64)
    keep = (draws >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) < p
    return iu[keep].astype(np.int32), ju[keep].astype(np.int32), n


def permute_labels(src, dst, n, seed: int):
    """Relabel vertices through a seeded random permutation."""
    perm = np.empty(n, dtype=np.int32)
    _load().gg_permutation(seed, 11, n, _ptr(perm))
    return perm[src], perm[dst], perm


# ---------------------------------------------------------------------------
# Closed-form families (section "Observations") — small pure-Python builders.
# ---------------------------------------------------------------------------

def _pairs(edges, n):
    a = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return a[:, 0].copy(), a[:, 1].copy(), n


def clique(k: int, offset: int = 0):
    return [(offset + a, offset + b) for a in range(k) for b in range(a + 1, k)]


def complete_graph(k: int):
    return _pairs(clique(k), k)


def disjoint_cliques(p: int, k: int):
    edges = []
    for c in range(p):
        edges += clique(k, c * k)
    return _pairs(edges, p * k)


def bridge_to_cliques(d: int, k: int):
    """Vertex 0 adjacent to one member of each of d disjoint copies of K_k."""
    edges = []
    for c in range(d):
        base = 1 + c * k
        edges += clique(k, base)
        edges.append((0, base))
    return _pairs(edges, 1 + d * k)


def clique_chain(p: int, k: int, ring: bool = False):
    """p copies of K_k, consecutive copies sharing one vertex (a ring closes the
    last copy onto the first).  Returns (src, dst, n, joiners, heads) where
    joiners are the shared vertices and heads the members of the two end
    copies (empty for a ring)."""
    members = []
    nxt = 0
    first = None
    joiners = []
    for c in range(p):
        cur = []
        if c == 0:
            cur.append(nxt); first = nxt; nxt += 1
        else:
            cur.append(members[-1][-1])
        need = k - len(cur)
        if ring and c == p - 1:
            need -= 1
        for _ in range(need):
            cur.append(nxt); nxt += 1
        if ring and c == p - 1:
            cur.append(first)
        members.append(cur)
    for c in range(p - 1):
        joiners.append(members[c][-1])
    if ring:
        joiners.append(first)
    edges = []
    for cur in members:
        for a in range(len(cur)):
            for b in range(a + 1, len(cur)):
                edges.append((cur[a], cur[b]))
    heads = [] if ring else sorted(set(members[0]) | set(members[-1]))
    s, d, n = _pairs(edges, nxt)
    return s, d, n, sorted(set(joiners)), heads


def single_triangle_with_pendants(pendants: int = 2):
    """One triangle {0,1,2}; each triangle vertex gets `pendants` leaves."""
    edges = [(0, 1), (1, 2), (0, 2)]
    nxt = 3
    for v in range(3):
        for _ in range(pendants):
            edges.append((v, nxt)); nxt += 1
    return _pairs(edges, nxt)


def batch_config3(count: int = 8192, seed: int = 0x5EED0003, n_min: int = 32, n_max: int = 65536):
    """The batched workload: `count` graphs, n log-uniform in [n_min, n_max];
    half Barabasi-Albert with m uniform in 2..8, half planted hierarchies
    (root joined to c in 4..32 cliques of size k in 3..12, leaves on clique
    members, one noise edge per vertex with probability 0.01).  Graph i
    draws from seed + i.  Returns a list of (src, dst, n)."""
    graphs = []
    for i in range(count):
        s = seed + i
        u = (gen_hash(s, 20, 0) >> 11) * (1.0 / 9007199254740992.0)
        n = int(round(n_min * (n_max / n_min) ** u))
        if gen_hash(s, 20, 1) & 1:
            mm = 2 + int(gen_hash(s, 20, 2) % 7)
            graphs.append(barabasi_albert(max(n, mm + 1), mm, s))
        else:
            c = 4 + int(gen_hash(s, 20, 3) % 29)
            k = 3 + int(gen_hash(s, 20, 4) % 10)
            graphs.append(planted_hierarchy(max(n, 1 + c * k), c, k, 0.01, s))
    return graphs


def _unit(seed: int, stream: int, ctr: int) -> float:
    return (gen_hash(seed, stream, ctr) >> 11) * (1.0 / 9007199254740992.0)


def served_pool_specs(count: int = 256, seed: int = 0x5EED0004, e_min: float = 1e3, e_max: float = 1e8,
                      cl_share: float = 0.25):
    """The served workload's request pool: `count` graph specs whose pair
    counts E are stratified over the log-uniform law on [e_min, e_max]
    (pool entry i draws its quantile from stratum i, then the entries are
    shuffled).  Each is R-MAT with scale ceil(log2(E/16)), E samples and
    (a, b, c, d) each jittered uniformly by +-0.05 around RMAT_ABC (d kept
    >= 0.01, renormalised), or with probability cl_share the grid +
    diagonals + Chung-Lu overlay sized to about E pairs."""
    import math
    strata = list(range(count))
    for i in range(count - 1, 0, -1):            # Fisher-Yates on the strata
        j = int(gen_hash(seed, 30, i) % (i + 1))
        strata[i], strata[j] = strata[j], strata[i]
    specs = []
    for i in range(count):
        u = (strata[i] + _unit(seed, 31, i)) / count
        e = int(round(e_min * (e_max / e_min) ** u))
        if _unit(seed, 32, i) < cl_share:
            side = max(4, int(round(math.sqrt(e / 4.05))))
            specs.append(dict(kind="grid", side=side, pdiag=0.05, gamma=2.1, mean_deg=4.0,
                              seed=seed + 1 + i, pairs=e))
        else:
            a, b, c = RMAT_ABC
            w = [a, b, c, 1.0 - a - b - c]
            w = [x + 0.1 * (_unit(seed, 33 + k, i) - 0.5) for k, x in enumerate(w)]
            w[3] = max(w[3], 0.01)
            tot = sum(w)
            w = [x / tot for x in w]
            scale = max(4, math.ceil(math.log2(e / 16)))
            specs.append(dict(kind="rmat", scale=scale, samples=e, abc=(w[0], w[1], w[2]),
                              seed=seed + 1 + i, pairs=e))
    return specs


def served_graph(spec: dict, threads: int | None = None):
    """(src, dst, n) of one pool entry of served_pool_specs."""
    if spec["kind"] == "rmat":
        return rmat(spec["scale"], seed=spec["seed"], abc=spec["abc"], samples=spec["samples"],
                    threads=threads)
    return grid_chung_lu(spec["side"], spec["pdiag"], spec["gamma"], spec["mean_deg"], seed=spec["seed"],
                         threads=threads)
