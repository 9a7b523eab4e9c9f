"""Triangle-centrality oracle — TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of triangle centrality (P. Burkhardt, "Triangle
Centrality"): Definition 1 evaluated with exact integers, Proposition 2 as a
second, independent form of the same numerator, and one correctly rounded
binary64 quotient.  The arithmetic is plain C in ``tc_oracle.c`` (compiled
with gcc into ``oracle/_build``); this module is argument marshalling.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product library under
``paper_2105_00110_gb300`` never imports, links or loads anything here.

Parity status: every routine is pinned by tests against brute force on tiny
graphs, the closed forms of the paper's "Observations" section, the worked
examples of Figures 1 and 2, the Borgatti graph of Table 3, and invariants
(see tests/test_oracle.py).  No routine is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtcoracle.so")
_SRC = os.path.join(_HERE, "tc_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile tc_oracle.c (gcc, -O2, no fast-math: the quotient must be IEEE)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, i64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
            lib.og_build.restype = vp
            lib.og_build.argtypes = [vp, vp, i64, i64]
            lib.og_free.restype = None
            lib.og_free.argtypes = [vp]
            lib.og_info.restype = None
            lib.og_info.argtypes = [vp, vp, vp]
            lib.og_copy_csr.restype = None
            lib.og_copy_csr.argtypes = [vp, vp, vp]
            lib.og_edge_triangles.restype = None
            lib.og_edge_triangles.argtypes = [vp, vp]
            lib.og_fast_edge_triangles.restype = ctypes.c_int
            lib.og_fast_edge_triangles.argtypes = [vp, vp]
            lib.og_vertex_triangles.restype = ctypes.c_int
            lib.og_vertex_triangles.argtypes = [vp, vp, vp]
            lib.og_total.restype = u64
            lib.og_total.argtypes = [vp, vp, vp]
            lib.og_numer_definition.restype = None
            lib.og_numer_definition.argtypes = [vp, vp, vp, vp, vp, vp]
            lib.og_numer_algebraic.restype = ctypes.c_int
            lib.og_numer_algebraic.argtypes = [vp, vp, vp, vp]
            lib.og_sample.restype = ctypes.c_int
            lib.og_sample.argtypes = [vp, vp, i64, vp, vp, vp]
            lib.og_sample_tri.restype = ctypes.c_int
            lib.og_sample_tri.argtypes = [vp, vp, i64, vp, vp]
            lib.og_div_rn.restype = ctypes.c_double
            lib.og_div_rn.argtypes = [u64, u64]
            lib.og_div_rn_long.restype = ctypes.c_double
            lib.og_div_rn_long.argtypes = [u64, u64]
            lib.og_tc.restype = None
            lib.og_tc.argtypes = [vp, i64, u64, vp]
            ci = ctypes.c_int
            lib.og_build_mt.restype = vp
            lib.og_build_mt.argtypes = [vp, vp, i64, i64, ci]
            lib.og_edge_triangles_mt.restype = None
            lib.og_edge_triangles_mt.argtypes = [vp, vp, ci]
            lib.og_fast_edge_triangles_mt.restype = ci
            lib.og_fast_edge_triangles_mt.argtypes = [vp, vp, ci]
            lib.og_vertex_triangles_mt.restype = ci
            lib.og_vertex_triangles_mt.argtypes = [vp, vp, vp, ci]
            lib.og_numer_definition_mt.restype = None
            lib.og_numer_definition_mt.argtypes = [vp, vp, vp, vp, vp, vp, ci]
            lib.og_tc_mt.restype = None
            lib.og_tc_mt.argtypes = [vp, i64, u64, vp, ci]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class OracleGraph:
    """Canonical simple undirected graph (rows ascending) held by the oracle."""

    def __init__(self, src, dst, n: int, threads: int = 1):
        """threads > 1 runs the build and every routine of run() on that many
        host threads (same results bit for bit; the CPU timing baseline)."""
        lib = _load()
        self.threads = max(1, int(threads))
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if src.shape != dst.shape:
            raise ValueError("src/dst length mismatch")
        if self.threads > 1:
            h = lib.og_build_mt(_p(src), _p(dst), len(src), int(n), self.threads)
        else:
            h = lib.og_build(_p(src), _p(dst), len(src), int(n))
        if not h:
            raise ValueError("oracle: vertex id outside [0, n) or out of memory")
        self._h = ctypes.c_void_p(h)
        nn, mm = ctypes.c_int64(), ctypes.c_int64()
        lib.og_info(self._h, ctypes.byref(nn), ctypes.byref(mm))
        self.n, self.m = nn.value, mm.value
        self.ptr = np.empty(self.n + 1, dtype=np.int64)
        self.adj = np.empty(max(2 * self.m, 1), dtype=np.int32)
        lib.og_copy_csr(self._h, _p(self.ptr), _p(self.adj))
        self.adj = self.adj[: 2 * self.m]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.og_free(h)
            self._h = None

    def edge_triangles(self, mode: str = "definition") -> np.ndarray:
        t = np.zeros(max(2 * self.m, 1), dtype=np.uint64)
        mt = self.threads > 1
        if mode == "definition":
            if mt:
                _load().og_edge_triangles_mt(self._h, _p(t), self.threads)
            else:
                _load().og_edge_triangles(self._h, _p(t))
        elif mode == "fast":
            rc = (_load().og_fast_edge_triangles_mt(self._h, _p(t), self.threads) if mt
                  else _load().og_fast_edge_triangles(self._h, _p(t)))
            if rc != 0:
                raise RuntimeError("og_fast_edge_triangles failed (%d)" % rc)
        else:
            raise ValueError(mode)
        return t[: 2 * self.m]

    def sample(self, vertices, with_rows: bool = False):
        """Definition 1 at the given vertices only: (tri, numer[, row_t])."""
        vs = np.ascontiguousarray(vertices, dtype=np.int64)
        tri = np.zeros(len(vs), dtype=np.uint64)
        num = np.zeros(len(vs), dtype=np.uint64)
        rows = None
        if with_rows:
            deg = self.ptr[vs + 1] - self.ptr[vs]
            rows = np.zeros(max(int(deg.sum()), 1), dtype=np.uint64)
        rc = _load().og_sample(self._h, _p(vs), len(vs), _p(tri), _p(num), _p(rows))
        if rc != 0:
            raise RuntimeError("og_sample failed (%d)" % rc)
        if with_rows:
            return tri, num, rows[: int((self.ptr[vs + 1] - self.ptr[vs]).sum())]
        return tri, num

    def sample_tri(self, vertices):
        """△(v) and the rows t(v, u), u ∈ N(v) ascending, at the given vertices
        (rows concatenated in sample order): (tri, row_t)."""
        vs = np.ascontiguousarray(vertices, dtype=np.int64)
        tri = np.zeros(len(vs), dtype=np.uint64)
        deg = self.ptr[vs + 1] - self.ptr[vs]
        rows = np.zeros(max(int(deg.sum()), 1), dtype=np.uint64)
        rc = _load().og_sample_tri(self._h, _p(vs), len(vs), _p(tri), _p(rows))
        if rc != 0:
            raise RuntimeError("og_sample_tri failed (%d)" % rc)
        return tri, rows[: int(deg.sum())]

    def run(self, mode: str = "definition", algebraic: bool = True) -> dict:
        """Everything the path computes, in the caller's vertex labels.

        Keys: ptr, adj (canonical CSR), t (per adjacency entry), flag (t > 0,
        uint8), tri, total, numer (Definition 1 form), numer_alg (Proposition 2
        form), core, noncore, den (= 3 total), tc (binary64, NaN if den == 0).
        algebraic=False skips the Proposition 2 cross-form (numer_alg and
        den_alg are then None), which the CPU timing baseline leaves out.
        """
        lib = _load()
        mt = self.threads
        t = self.edge_triangles(mode)
        tb = np.ascontiguousarray(t) if len(t) else np.zeros(1, dtype=np.uint64)
        n = self.n
        tri = np.zeros(max(n, 1), dtype=np.uint64)
        rc = (lib.og_vertex_triangles_mt(self._h, _p(tb), _p(tri), mt) if mt > 1
              else lib.og_vertex_triangles(self._h, _p(tb), _p(tri)))
        if rc != 0:
            raise AssertionError("odd row sum of T")
        rem = ctypes.c_uint64()
        total = int(lib.og_total(self._h, _p(tri), ctypes.byref(rem)))
        if rem.value != 0:
            raise AssertionError("sum of vertex counts not divisible by 3")
        numer = np.zeros(max(n, 1), dtype=np.uint64)
        core = np.zeros(max(n, 1), dtype=np.uint64)
        noncore = np.zeros(max(n, 1), dtype=np.uint64)
        if mt > 1:
            lib.og_numer_definition_mt(self._h, _p(tb), _p(tri), _p(numer), _p(core), _p(noncore), mt)
        else:
            lib.og_numer_definition(self._h, _p(tb), _p(tri), _p(numer), _p(core), _p(noncore))
        numer_alg = den_alg = None
        if algebraic:
            numer_alg = np.zeros(max(n, 1), dtype=np.uint64)
            d = ctypes.c_uint64()
            if lib.og_numer_algebraic(self._h, _p(tb), _p(numer_alg), ctypes.byref(d)) != 0:
                raise AssertionError("odd algebraic numerator")
            numer_alg, den_alg = numer_alg[:n], int(d.value)
        den = 3 * total
        tc = np.zeros(max(n, 1), dtype=np.float64)
        if mt > 1:
            lib.og_tc_mt(_p(numer), n, den, _p(tc), mt)
        else:
            lib.og_tc(_p(numer), n, den, _p(tc))
        return dict(ptr=self.ptr, adj=self.adj, t=t, flag=(t > 0).astype(np.uint8),
                    tri=tri[:n], total=total, numer=numer[:n], numer_alg=numer_alg,
                    den_alg=den_alg, core=core[:n], noncore=noncore[:n],
                    den=den, tc=tc[:n])


def run(src, dst, n: int, mode: str = "definition", threads: int = 1, algebraic: bool = True) -> dict:
    return OracleGraph(src, dst, n, threads).run(mode, algebraic)


def div_rn(a: int, b: int) -> float:
    return float(_load().og_div_rn(int(a), int(b)))


def div_rn_long(a: int, b: int) -> float:
    return float(_load().og_div_rn_long(int(a), int(b)))


def tc_from_numer(numer: np.ndarray, den: int) -> np.ndarray:
    num = np.ascontiguousarray(numer, dtype=np.uint64)
    out = np.zeros(max(len(num), 1), dtype=np.float64)
    _load().og_tc(_p(num), len(num), int(den), _p(out))
    return out[: len(num)]
