"""Python binding of the GB300 triangle-centrality library (libtc_gb300.so).

Argument marshalling only: every step of the path (graph construction,
degree ordering, intersection, gather, division) runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  The binding has the
C entry points under the same names (``tc_build_csr``, ``tc_count``,
``tc_centrality``, ...) plus a small ``Graph`` convenience class.

There is no CPU fallback: if the library has not been built, or no CUDA
device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from .build import DEBUG_LIB, LIB, build  # noqa: F401

TC_OK = 0
TC_NO_TRIANGLES = 1
TC_ERR_INVALID_ARG = -1
TC_ERR_OUT_OF_MEMORY = -2
TC_ERR_CUDA = -3
TC_ERR_OVERFLOW = -4
TC_ERR_TIMEOUT = -5
TC_ERR_STATE = -6
TC_ERR_BOUNDS = -7

TC_IN_DEVICE = 1
TC_IDS_INT32 = 2

TC_STRATEGY_AUTO = 0
TC_STRATEGY_BSEARCH = 1
TC_STRATEGY_MERGE = 2
TC_STRATEGY_BITMAP = 3
TC_STRATEGY_GLOBAL = 4
STRATEGIES = {"auto": 0, "bsearch": 1, "merge": 2, "bitmap": 3, "global": 4}

EXPORTED = ["tc_build_csr", "tc_count", "tc_count_shard", "tc_load_counts", "tc_edge_triangles", "tc_centrality", "tc_divide", "tc_graph_info",
            "tc_copy_edges", "tc_get_stats", "tc_set_strategy", "tc_set_plan_params", "tc_get_plan_params",
            "tc_set_dense_core", "tc_profile_enable",
            "tc_profile_reset", "tc_profile_read", "tc_launch_count", "tc_graph_free",
            "tc_status_str", "tc_batch_build", "tc_batch_run", "tc_batch_info",
            "tc_batch_copy_edges", "tc_batch_get_stats", "tc_batch_autotune", "tc_batch_get_params",
            "tc_batch_free", "tc_csr_centrality_noalloc",
            "tc_server_create", "tc_server_submit", "tc_server_poll", "tc_server_stats", "tc_server_free",
            "tc_debug_fail_allocation", "tc_debug_allocations", "tc_debug_live_allocations",
            "tc_debug_bounds_build", "tc_debug_bounds_line"]


class TCError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s failed: %s (%d)" % (where, status_str(status), status))
        self.status = status


class RequestInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("triangles", ctypes.c_uint64), ("edges", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class GraphStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("max_degree", ctypes.c_int64), ("max_out_degree", ctypes.c_int64),
                ("sum_out_degree_sq", ctypes.c_double), ("wedges", ctypes.c_double),
                ("avg_degeneracy", ctypes.c_double),
                ("items", ctypes.c_int64 * 5), ("class_bytes", ctypes.c_double * 5),
                ("class_wedges", ctypes.c_double * 5), ("class_head", ctypes.c_double * 5),
                ("count_bytes", ctypes.c_double), ("centrality_bytes", ctypes.c_double),
                ("core_vertices", ctypes.c_int64), ("core_words", ctypes.c_double)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if not isinstance(v, (int, float)) else v
        return d


CLASS_NAMES = ["bitmap_s", "bitmap_l", "warp", "cta_list", "thread"]
# kernel name (as reported by tc_profile_read) -> item class
KERNEL_CLASS = {"count_bitmap_s": 0, "count_bitmap_l": 1, "count_warp": 2,
                "count_cta_list": 3, "count_cta_global": 3, "count_thread": 4}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


_lib = None
_lib_path = LIB


def use_library(path: str):
    """Loads the library from `path` instead of the default build (e.g. the
    bounds-checked one from build(debug=True)).  Only before the first call
    into the library."""
    global _lib_path
    if _lib is not None and os.path.abspath(path) != os.path.abspath(_lib_path):
        raise RuntimeError("the library is already loaded from " + _lib_path)
    _lib_path = path


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_lib_path):
            raise RuntimeError("libtc_gb300.so is not built: call paper_2105_00110_gb300.build()")
        L = ctypes.CDLL(_lib_path)
        vp, i64, u64, i32, u32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_int, ctypes.c_uint32)
        L.tc_build_csr.restype = i32
        L.tc_build_csr.argtypes = [vp, vp, i64, i64, u32, vp, ctypes.POINTER(vp)]
        L.tc_count.restype = i32
        L.tc_count.argtypes = [vp, vp, vp, ctypes.POINTER(u64), vp]
        L.tc_count_shard.restype = i32
        L.tc_count_shard.argtypes = [vp, i32, i32, vp, vp, ctypes.POINTER(u64), vp]
        L.tc_load_counts.restype = i32
        L.tc_load_counts.argtypes = [vp, vp, vp, ctypes.POINTER(u64), vp]
        L.tc_edge_triangles.restype = i32
        L.tc_edge_triangles.argtypes = [vp, vp, vp, ctypes.POINTER(u64), vp]
        L.tc_centrality.restype = i32
        L.tc_centrality.argtypes = [vp, vp, vp, ctypes.POINTER(u64), vp]
        L.tc_divide.restype = i32
        L.tc_divide.argtypes = [vp, i64, u64, vp, vp]
        L.tc_graph_info.restype = i32
        L.tc_graph_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.tc_copy_edges.restype = i32
        L.tc_copy_edges.argtypes = [vp, vp, vp, vp]
        L.tc_get_stats.restype = i32
        L.tc_get_stats.argtypes = [vp, ctypes.POINTER(GraphStats)]
        L.tc_set_plan_params.restype = i32
        L.tc_set_plan_params.argtypes = [vp, vp]
        L.tc_get_plan_params.restype = i32
        L.tc_get_plan_params.argtypes = [vp, vp]
        L.tc_set_strategy.restype = i32
        L.tc_set_strategy.argtypes = [vp, i32]
        L.tc_set_dense_core.restype = i32
        L.tc_set_dense_core.argtypes = [ctypes.c_longlong]
        L.tc_profile_enable.restype = i32
        L.tc_profile_enable.argtypes = [i32]
        L.tc_profile_reset.restype = i32
        L.tc_profile_reset.argtypes = []
        L.tc_profile_read.restype = i32
        L.tc_profile_read.argtypes = [ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
        L.tc_launch_count.restype = i64
        L.tc_launch_count.argtypes = []
        L.tc_debug_bounds_build.restype = i32
        L.tc_debug_bounds_build.argtypes = []
        L.tc_debug_bounds_line.restype = i64
        L.tc_debug_bounds_line.argtypes = []
        L.tc_debug_fail_allocation.restype = i32
        L.tc_debug_fail_allocation.argtypes = [i64]
        L.tc_debug_allocations.restype = i64
        L.tc_debug_allocations.argtypes = []
        L.tc_debug_live_allocations.restype = i64
        L.tc_debug_live_allocations.argtypes = []
        L.tc_graph_free.restype = None
        L.tc_graph_free.argtypes = [vp]
        L.tc_status_str.restype = ctypes.c_char_p
        L.tc_status_str.argtypes = [i32]
        L.tc_batch_build.restype = i32
        L.tc_batch_build.argtypes = [vp, vp, vp, vp, i64, u32, vp, ctypes.POINTER(vp)]
        L.tc_batch_run.restype = i32
        L.tc_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.tc_batch_info.restype = i32
        L.tc_batch_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64), vp, vp]
        L.tc_batch_copy_edges.restype = i32
        L.tc_batch_copy_edges.argtypes = [vp, vp, vp, vp]
        L.tc_batch_get_stats.restype = i32
        L.tc_batch_get_stats.argtypes = [vp, ctypes.POINTER(GraphStats)]
        L.tc_batch_autotune.restype = i32
        L.tc_batch_autotune.argtypes = [vp, i32, vp]
        L.tc_batch_get_params.restype = i32
        L.tc_batch_get_params.argtypes = [vp, vp]
        L.tc_batch_free.restype = None
        L.tc_batch_free.argtypes = [vp]
        L.tc_server_create.restype = i32
        L.tc_server_create.argtypes = [i64, i64, i32, ctypes.POINTER(vp)]
        L.tc_server_submit.restype = i32
        L.tc_server_submit.argtypes = [vp, vp, vp, i64, i64, vp, vp, ctypes.POINTER(i64)]
        L.tc_server_poll.restype = i32
        L.tc_server_poll.argtypes = [vp, ctypes.POINTER(RequestInfo), i32, ctypes.POINTER(i32), i32]
        L.tc_server_stats.restype = i32
        L.tc_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64)]
        L.tc_server_free.restype = None
        L.tc_server_free.argtypes = [vp]
        L.tc_csr_centrality_noalloc.restype = i32
        L.tc_csr_centrality_noalloc.argtypes = [vp, vp, i64, i64, vp, vp, vp, vp]
        _lib = L
    return _lib


def status_str(status: int) -> str:
    try:
        return lib().tc_status_str(int(status)).decode()
    except Exception:  # library missing
        return "status %d" % status


def _check(status: int, where: str, ok=(TC_OK, TC_NO_TRIANGLES)) -> int:
    if status not in ok:
        raise TCError(status, where)
    return status


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------- same names
def tc_build_csr(src, dst, n: int, stream=None):
    """Graph handle (ctypes.c_void_p) from pair arrays: CUDA or CPU torch
    tensors, or numpy arrays, of int32 or int64."""
    if isinstance(src, np.ndarray):
        src = torch.from_numpy(np.ascontiguousarray(src))
    if isinstance(dst, np.ndarray):
        dst = torch.from_numpy(np.ascontiguousarray(dst))
    if src.dtype != dst.dtype or src.shape != dst.shape or src.dim() != 1:
        raise ValueError("src and dst must be 1-D with the same dtype and length")
    if src.dtype not in (torch.int32, torch.int64):
        raise ValueError("ids must be int32 or int64")
    if src.is_cuda != dst.is_cuda:
        raise ValueError("src and dst must be on the same device")
    src = src.contiguous()
    dst = dst.contiguous()
    flags = (TC_IDS_INT32 if src.dtype == torch.int32 else 0) | (TC_IN_DEVICE if src.is_cuda else 0)
    h = ctypes.c_void_p()
    st = lib().tc_build_csr(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                            src.numel(), int(n), flags, _stream(stream), ctypes.byref(h))
    _check(st, "tc_build_csr", ok=(TC_OK,))
    return h


def tc_count(g, tri=None, edge_flag=None, stream=None):
    """(status, △(G)); fills tri [n] uint64 and edge_flag [m] uint8 if given."""
    total = ctypes.c_uint64()
    st = lib().tc_count(g, _dptr(tri), _dptr(edge_flag), ctypes.byref(total), _stream(stream))
    _check(st, "tc_count")
    return st, total.value


def tc_count_shard(g, shard: int, num_shards: int, tri=None, edge_flag=None, stream=None) -> int:
    """Triangles found by shard `shard` of `num_shards`; fills its partial
    tri [n] uint64 and edge_flag [m] uint8 if given."""
    part = ctypes.c_uint64()
    st = lib().tc_count_shard(g, int(shard), int(num_shards), _dptr(tri), _dptr(edge_flag), ctypes.byref(part),
                              _stream(stream))
    _check(st, "tc_count_shard", ok=(TC_OK,))
    return part.value


def tc_load_counts(g, tri, edge_flag, stream=None):
    """(status, △(G)) after loading complete counts and flags into g."""
    total = ctypes.c_uint64()
    st = lib().tc_load_counts(g, _dptr(tri), _dptr(edge_flag) if edge_flag is not None and edge_flag.numel() else None,
                              ctypes.byref(total), _stream(stream))
    _check(st, "tc_load_counts")
    return st, total.value


def allreduce_counts(tri, edge_flag, group=None):
    """The exchange step of a sharded count across processes: sums the
    partial △(v) and ORs the edge flags (a max over 0/1 bytes) in place,
    over torch.distributed (NCCL between GPUs, gloo on CPU)."""
    import torch.distributed as dist
    dist.all_reduce(tri.view(torch.int64), op=dist.ReduceOp.SUM, group=group)
    if edge_flag is not None and edge_flag.numel():
        dist.all_reduce(edge_flag, op=dist.ReduceOp.MAX, group=group)
    return tri, edge_flag


def tc_edge_triangles(g, tri=None, edge_tri=None, stream=None):
    """(status, △(G)); fills tri [n] uint64 and edge_tri [m] uint32 (t(u, v)
    per canonical edge) if given."""
    total = ctypes.c_uint64()
    st = lib().tc_edge_triangles(g, _dptr(tri), _dptr(edge_tri), ctypes.byref(total), _stream(stream))
    _check(st, "tc_edge_triangles")
    return st, total.value


def tc_centrality(g, numer=None, tc=None, stream=None):
    """(status, 3△(G)); fills numer [n] uint64 and tc [n] float64 if given."""
    den = ctypes.c_uint64()
    st = lib().tc_centrality(g, _dptr(numer), _dptr(tc), ctypes.byref(den), _stream(stream))
    _check(st, "tc_centrality")
    return st, den.value


def tc_divide(numer, den: int, out, stream=None):
    st = lib().tc_divide(_dptr(numer), numer.numel(), int(den), _dptr(out), _stream(stream))
    _check(st, "tc_divide", ok=(TC_OK,))


TC_NOALLOC_MAX_VERTICES = 65536
TC_NOALLOC_MAX_ENTRIES = 2097152


def tc_csr_centrality_noalloc(row_ptr, col, n: int, tri=None, numer=None, tc=None, stream=None):
    """Counts, numerators and TC of a small graph given as a device CSR
    (row_ptr [n+1] int64, col [nnz] int32; sorted, symmetric, no loops),
    using only the library's fixed working array: nothing is allocated.
    Outputs are caller tensors (tri/numer uint64 [n], tc float64 [n]).
    Calls on one device must not overlap in time.

    Every argument is checked here, before the library sees a pointer: a
    wrong length, dtype or device would make the kernels read or write out
    of bounds, which the C entry point cannot detect."""
    n = int(n)
    if n < 0:
        raise ValueError("n must be non-negative")
    checks = [("row_ptr", row_ptr, torch.int64, n + 1), ("col", col, torch.int32, None),
              ("tri", tri, torch.uint64, n), ("numer", numer, torch.uint64, n), ("tc", tc, torch.float64, n)]
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t, dt, size in checks:
        if t is None:
            if name in ("row_ptr", "col"):
                raise ValueError("%s is required" % name)
            continue
        if not isinstance(t, torch.Tensor) or t.dim() != 1:
            raise ValueError("%s must be a 1-D tensor" % name)
        if t.dtype != dt:
            raise ValueError("%s must be %s, got %s" % (name, dt, t.dtype))
        if size is not None and t.numel() != size:
            raise ValueError("%s must hold %d entries, got %d" % (name, size, t.numel()))
        if not t.is_cuda or t.device.index != dev:
            raise ValueError("%s must be on the current CUDA device (cuda:%s)" % (name, dev))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    st = lib().tc_csr_centrality_noalloc(_dptr(row_ptr), _dptr(col) if col.numel() else None, int(n),
                                         col.numel(), _dptr(tri), _dptr(numer), _dptr(tc),
                                         _stream(stream))
    _check(st, "tc_csr_centrality_noalloc", ok=(TC_OK,))


def tc_graph_info(g):
    n, m = ctypes.c_int64(), ctypes.c_int64()
    pu, pv = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().tc_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(pu),
                               ctypes.byref(pv)), "tc_graph_info", ok=(TC_OK,))
    return n.value, m.value, pu.value, pv.value


def tc_copy_edges(g, u, v, stream=None):
    _check(lib().tc_copy_edges(g, _dptr(u), _dptr(v), _stream(stream)), "tc_copy_edges", ok=(TC_OK,))


def tc_get_stats(g) -> dict:
    s = GraphStats()
    _check(lib().tc_get_stats(g, ctypes.byref(s)), "tc_get_stats", ok=(TC_OK,))
    return s.as_dict()


def tc_set_strategy(g, strategy):
    if isinstance(strategy, str):
        strategy = STRATEGIES[strategy]
    _check(lib().tc_set_strategy(g, int(strategy)), "tc_set_strategy", ok=(TC_OK,))


def tc_set_plan_params(g, cta_min_work: int, cta_chunk: int, warp_chunk: int):
    arr = (ctypes.c_int64 * 3)(int(cta_min_work), int(cta_chunk), int(warp_chunk))
    _check(lib().tc_set_plan_params(g, arr), "tc_set_plan_params", ok=(TC_OK,))


def tc_set_dense_core(c: int):
    """Process-wide dense-core setting for later builds: -1 chooses per graph
    (default), 0 never, c > 0 the top min(c, n) ranks."""
    _check(lib().tc_set_dense_core(int(c)), "tc_set_dense_core", ok=(TC_OK,))


def tc_get_plan_params(g):
    arr = (ctypes.c_int64 * 3)()
    _check(lib().tc_get_plan_params(g, arr), "tc_get_plan_params", ok=(TC_OK,))
    return dict(cta_min_work=arr[0], cta_chunk=arr[1], warp_chunk=arr[2])


def tc_profile_enable(on: bool = True):
    lib().tc_profile_enable(1 if on else 0)


def tc_profile_reset():
    lib().tc_profile_reset()


def tc_profile_read() -> dict:
    cap = 64
    arr = (KernelTime * cap)()
    cnt = ctypes.c_int()
    lib().tc_profile_read(arr, cap, ctypes.byref(cnt))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(cnt.value, cap))}


def tc_launch_count() -> int:
    return int(lib().tc_launch_count())


def tc_debug_fail_allocation(k: int):
    """Arms one injected device-allocation failure k allocations from now
    (k < 0 disarms); see include/tc.h."""
    lib().tc_debug_fail_allocation(int(k))


def tc_debug_bounds_build() -> bool:
    return bool(lib().tc_debug_bounds_build())


def tc_debug_bounds_line() -> int:
    return int(lib().tc_debug_bounds_line())


def tc_debug_allocations() -> int:
    return int(lib().tc_debug_allocations())


def tc_debug_live_allocations() -> int:
    return int(lib().tc_debug_live_allocations())


def tc_graph_free(g):
    if g:
        lib().tc_graph_free(g)


# ------------------------------------------------------------ convenience
class Graph:
    """Owns a tc_graph; results come back as CUDA tensors in caller labels."""

    def __init__(self, src, dst, n: int, stream=None):
        self.h = tc_build_csr(src, dst, n, stream)
        self.n, self.m, _, _ = tc_graph_info(self.h)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if self.h:
            tc_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def edges(self):
        u = torch.empty(self.m, dtype=torch.int32, device=self.device)
        v = torch.empty(self.m, dtype=torch.int32, device=self.device)
        tc_copy_edges(self.h, u, v)
        return u, v

    def stats(self) -> dict:
        return tc_get_stats(self.h)

    def set_strategy(self, s):
        tc_set_strategy(self.h, s)

    def count(self, want_flags: bool = True, stream=None):
        tri = torch.empty(self.n, dtype=torch.uint64, device=self.device)
        flags = torch.empty(self.m, dtype=torch.uint8, device=self.device) if want_flags else None
        st, total = tc_count(self.h, tri, flags, stream)
        return tri, flags, total, st

    def edge_triangles(self, stream=None):
        tri = torch.empty(self.n, dtype=torch.uint64, device=self.device)
        et = torch.empty(max(self.m, 1), dtype=torch.int32, device=self.device).view(torch.uint32)
        st, total = tc_edge_triangles(self.h, tri, et if self.m else None, stream)
        return tri, et[:self.m], total, st

    def centrality(self, stream=None):
        numer = torch.empty(self.n, dtype=torch.uint64, device=self.device)
        tc = torch.empty(self.n, dtype=torch.float64, device=self.device)
        st, den = tc_centrality(self.h, numer, tc, stream)
        return numer, tc, den, st


def triangle_centrality(src, dst, n: int, strategy=None, stream=None) -> dict:
    """One full pass: build, count, centrality.  Returns CUDA tensors."""
    g = Graph(src, dst, n, stream)
    try:
        if strategy is not None:
            g.set_strategy(strategy)
        tri, flags, total, _ = g.count(stream=stream)
        numer, tc, den, st = g.centrality(stream=stream)
        eu, ev = g.edges()
        return dict(n=g.n, m=g.m, tri=tri, flag=flags, total=total, numer=numer, tc=tc, den=den,
                    status=st, edge_u=eu, edge_v=ev, stats=g.stats())
    finally:
        g.close()


# ------------------------------------------------------------------ batches
def pack_graphs(graphs):
    """[(src, dst, n), ...] with local ids -> (src, dst, pair_offsets, num_vertices)."""
    srcs = [np.ascontiguousarray(g[0], dtype=np.int32) for g in graphs]
    dsts = [np.ascontiguousarray(g[1], dtype=np.int32) for g in graphs]
    nv = np.array([int(g[2]) for g in graphs], dtype=np.int64)
    off = np.zeros(len(graphs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(x) for x in srcs])
    src = np.concatenate(srcs) if srcs else np.zeros(0, np.int32)
    dst = np.concatenate(dsts) if dsts else np.zeros(0, np.int32)
    return src, dst, off, nv


def tc_batch_build(src, dst, pair_offsets, num_vertices, stream=None):
    if isinstance(src, np.ndarray):
        src = torch.from_numpy(np.ascontiguousarray(src))
    if isinstance(dst, np.ndarray):
        dst = torch.from_numpy(np.ascontiguousarray(dst))
    if src.dtype != dst.dtype or src.shape != dst.shape or src.dtype not in (torch.int32, torch.int64):
        raise ValueError("src/dst must be 1-D int32 or int64 of equal length")
    src, dst = src.contiguous(), dst.contiguous()
    off = np.ascontiguousarray(pair_offsets, dtype=np.int64)
    nv = np.ascontiguousarray(num_vertices, dtype=np.int64)
    if len(off) != len(nv) + 1:
        raise ValueError("pair_offsets needs num_graphs + 1 entries")
    flags = (TC_IDS_INT32 if src.dtype == torch.int32 else 0) | (TC_IN_DEVICE if src.is_cuda else 0)
    h = ctypes.c_void_p()
    st = lib().tc_batch_build(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                              ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(nv.ctypes.data),
                              len(nv), flags, _stream(stream), ctypes.byref(h))
    _check(st, "tc_batch_build", ok=(TC_OK,))
    return h


def tc_batch_run(b, tri=None, edge_flag=None, numer=None, tc=None, totals=None, stream=None):
    st = lib().tc_batch_run(b, _dptr(tri), _dptr(edge_flag), _dptr(numer), _dptr(tc), _dptr(totals),
                            _stream(stream))
    _check(st, "tc_batch_run", ok=(TC_OK,))


def tc_batch_info(b):
    G, n, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().tc_batch_info(b, ctypes.byref(G), ctypes.byref(n), ctypes.byref(m), None, None),
           "tc_batch_info", ok=(TC_OK,))
    voff = np.zeros(G.value + 1, dtype=np.int64)
    eoff = np.zeros(G.value + 1, dtype=np.int64)
    lib().tc_batch_info(b, None, None, None, ctypes.c_void_p(voff.ctypes.data), ctypes.c_void_p(eoff.ctypes.data))
    return G.value, n.value, m.value, voff, eoff


class Batch:
    """Owns a tc_batch; results are CUDA tensors in union labels."""

    def __init__(self, src, dst, pair_offsets, num_vertices, stream=None):
        self.h = tc_batch_build(src, dst, pair_offsets, num_vertices, stream)
        self.G, self.n, self.m, self.voff, self.eoff = tc_batch_info(self.h)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.out = dict(
            tri=torch.empty(max(self.n, 1), dtype=torch.uint64, device=self.device),
            flag=torch.empty(max(self.m, 1), dtype=torch.uint8, device=self.device),
            numer=torch.empty(max(self.n, 1), dtype=torch.uint64, device=self.device),
            tc=torch.empty(max(self.n, 1), dtype=torch.float64, device=self.device),
            totals=torch.empty(max(self.G, 1), dtype=torch.uint64, device=self.device))

    def close(self):
        if self.h:
            lib().tc_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, stream=None):
        o = self.out
        tc_batch_run(self.h, o["tri"], o["flag"], o["numer"], o["tc"], o["totals"], stream)
        return o

    def edges(self):
        u = torch.empty(max(self.m, 1), dtype=torch.int32, device=self.device)
        v = torch.empty(max(self.m, 1), dtype=torch.int32, device=self.device)
        _check(lib().tc_batch_copy_edges(self.h, _dptr(u), _dptr(v), _stream(None)), "tc_batch_copy_edges",
               ok=(TC_OK,))
        return u[: self.m], v[: self.m]

    def autotune(self, reps: int = 2, stream=None):
        _check(lib().tc_batch_autotune(self.h, int(reps), _stream(stream)), "tc_batch_autotune", ok=(TC_OK,))
        return self.params()

    def params(self):
        out = np.zeros(3, dtype=np.int64)
        lib().tc_batch_get_params(self.h, ctypes.c_void_p(out.ctypes.data))
        return dict(cta_min_work=int(out[0]), cta_chunk=int(out[1]), warp_chunk=int(out[2]))

    def stats(self) -> dict:
        st = GraphStats()
        _check(lib().tc_batch_get_stats(self.h, ctypes.byref(st)), "tc_batch_get_stats", ok=(TC_OK,))
        return st.as_dict()


# ----------------------------------------------------------------- serving
def _host_ptr(a, dtype):
    """Address of a contiguous host array (numpy or CPU torch) of `dtype`."""
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous() or a.dtype != dtype[1]:
            raise ValueError("expected a contiguous CPU tensor of %s" % dtype[1])
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous or a.dtype != dtype[0]:
        raise ValueError("expected a C-contiguous numpy array of %s" % dtype[0])
    return ctypes.c_void_p(a.ctypes.data)


_I32 = (np.dtype(np.int32), torch.int32)
_U64 = (np.dtype(np.uint64), torch.uint64)
_F64 = (np.dtype(np.float64), torch.float64)


def tc_server_create(memory_budget_bytes: int, max_batch_pairs: int, workers: int = 2):
    h = ctypes.c_void_p()
    _check(lib().tc_server_create(int(memory_budget_bytes), int(max_batch_pairs), int(workers),
                                  ctypes.byref(h)), "tc_server_create", ok=(TC_OK,))
    return h


def tc_server_submit(srv, src, dst, n: int, tri=None, tc=None) -> int:
    rid = ctypes.c_int64()
    st = lib().tc_server_submit(srv, _host_ptr(src, _I32), _host_ptr(dst, _I32), len(src), int(n),
                                _host_ptr(tri, _U64), _host_ptr(tc, _F64), ctypes.byref(rid))
    _check(st, "tc_server_submit", ok=(TC_OK,))
    return rid.value


def tc_server_poll(srv, cap: int = 1024, wait_ms: int = 0, buf=None):
    if buf is None or len(buf) < cap:
        buf = (RequestInfo * max(cap, 1))()
    cnt = ctypes.c_int32()
    _check(lib().tc_server_poll(srv, buf, int(cap), ctypes.byref(cnt), int(wait_ms)), "tc_server_poll",
           ok=(TC_OK,))
    return [dict(id=r.id, status=r.status, batch_size=r.batch_size, triangles=r.triangles, edges=r.edges,
                 t_submit=r.t_submit, t_start=r.t_start, t_done=r.t_done) for r in buf[:cnt.value]]


def tc_server_stats(srv) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().tc_server_stats(srv, *(ctypes.byref(x) for x in v)), "tc_server_stats", ok=(TC_OK,))
    return dict(batches=v[0].value, waiting=v[1].value, running=v[2].value, memory_in_use=v[3].value)


def tc_server_free(srv):
    lib().tc_server_free(srv)


class Server:
    """Request loop on the current device.  submit() takes host int32 pair
    arrays and returns a request id at once; poll() returns finished
    requests with their results.  The arrays of a request are kept alive
    here until it has been polled."""

    def __init__(self, memory_budget_bytes: int = 150 * 10**9, max_batch_pairs: int = 1 << 25,
                 workers: int = 2):
        self.h = None
        self.h = tc_server_create(memory_budget_bytes, max_batch_pairs, workers)
        self.live = {}
        self._buf = None

    def submit(self, src, dst, n: int, tri=None, tc=None, want_results: bool = True) -> int:
        if want_results and tri is None:
            tri = np.empty(max(int(n), 1), np.uint64)
        if want_results and tc is None:
            tc = np.empty(max(int(n), 1), np.float64)
        rid = tc_server_submit(self.h, src, dst, n, tri, tc)
        self.live[rid] = (src, dst, tri, tc, int(n))
        return rid

    def poll(self, cap: int = 4096, wait_ms: int = 0):
        if self._buf is None or len(self._buf) < cap:
            self._buf = (RequestInfo * max(cap, 1))()
        out = []
        for info in tc_server_poll(self.h, cap, wait_ms, self._buf):
            src, dst, tri, tc, n = self.live.pop(info["id"])
            info["tri"] = None if tri is None else tri[:n]
            info["tc"] = None if tc is None else tc[:n]
            out.append(info)
        return out

    def wait_all(self, timeout_s: float = 600.0):
        import time as _t
        done = []
        t_end = _t.monotonic() + timeout_s
        while self.live and _t.monotonic() < t_end:
            done += self.poll(wait_ms=100)
        return done

    def stats(self) -> dict:
        return tc_server_stats(self.h)

    def close(self):
        if self.h:
            tc_server_free(self.h)
            self.h = None
            self.live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
