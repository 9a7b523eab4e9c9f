"""Benchmark of the full triangle-centrality path on GB300.

One step = one pass of the whole path over one synthetic graph already
resident in HBM as a pair list: tc_build_csr (symmetrise, de-duplicate,
degree order, orientation, plan) + tc_count (△(v), △(G), edge flags) +
tc_centrality (exact numerators, one division) + tc_graph_free, all through
the C ABI.  value = undirected edges processed per second over the timed
steps (whole job; under torchrun every rank processes its own graph, seeded
by rank: weak scaling, no collective on the data path).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (the reference arm; there is no reference implementation to run).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s for full TC (build + count + centrality), exact"

# Workloads: name -> generator spec
WORKLOADS = {
    "rmat-s24-ef16": dict(kind="rmat", scale=24, edge_factor=16, seed=0x5EED0018),
    "rmat-s12-ef16": dict(kind="rmat", scale=12, edge_factor=16, seed=0x5EED0000),
    "rmat-s20-ef16": dict(kind="rmat", scale=20, edge_factor=16, seed=0x5EED0014),
    "rmat-s21-ef16": dict(kind="rmat", scale=21, edge_factor=16, seed=0x5EED0015),
    "rmat-s22-ef16": dict(kind="rmat", scale=22, edge_factor=16, seed=0x5EED0016),
    "grid4096-diag05-cl21": dict(kind="grid", side=4096, pdiag=0.05, gamma=2.1, mean_deg=4.0,
                                 seed=0x5EED0002),
}
DEFAULT_WORKLOAD = "rmat-s24-ef16"
BATCH_WORKLOADS = {"batched-8192": dict(kind="batch", count=8192, seed=0x5EED0003)}
SERVED_WORKLOADS = {"served-poisson": dict(kind="served", rate=2000.0, duration=60.0, pool=256,
                                           e_min=1e3, e_max=1e8, budget=150 * 10**9,
                                           max_batch_pairs=1 << 25, workers=2,
                                           sustain_duration=30.0, sustain_load=0.75, seed=0x5EED0004)}


def generate(spec: dict, rank: int = 0):
    import graphgen as gg
    seed = spec["seed"] + 0x1000 * rank
    if spec["kind"] == "rmat":
        return gg.rmat(spec["scale"], spec["edge_factor"], seed=seed)
    return gg.grid_chung_lu(spec["side"], spec["pdiag"], spec["gamma"], spec["mean_deg"], seed=seed)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------- DRAM traffic
COUNT_SOURCES = ["paper_2105_00110_gb300/csrc/tc_count.cu", "paper_2105_00110_gb300/csrc/tc_internal.cuh"]


def traffic_profile(workload: str) -> str:
    """The committed ncu summary of the count kernels' DRAM traffic on this
    workload (one kernel, one launch, small enough to capture)."""
    return os.path.join(ROOT, "profiles", "count_dram_traffic_%s.md" % workload)


def count_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in COUNT_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def dram_traffic(kernel: str, workload: str):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of `kernel`
    from the committed ncu summary, or None when that summary is for other
    count-kernel sources or another workload."""
    try:
        with open(traffic_profile(workload)) as fh:
            text = fh.read()
    except OSError:
        return None
    sha = wl = None
    rows = {}
    for line in text.splitlines():
        if line.startswith("source-sha256:"):
            sha = line.split(":", 1)[1].strip()
        elif line.startswith("workload:"):
            wl = line.split(":", 1)[1].strip()
        elif line.startswith("| count_") or line.startswith("| gather"):
            cells = [c.strip() for c in line.strip("|").split("|")]
            try:
                rows[cells[0]] = (float(cells[1]) + float(cells[2])) * 1e9
            except (ValueError, IndexError):
                pass
    if sha != count_sources_sha() or wl != workload:
        return None
    return rows.get(kernel)


# --------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0: float | None = None, t1: float | None = None) -> dict:
        """Stops sampling; keeps the samples taken between host times t0 and
        t1 (the timed region) when there are any."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        import datetime
        samples = []
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                samples.append((ts, float(r[2]), float(r[3]), float(r[4]), [x.strip() for x in r[6:10]]))
            except (ValueError, IndexError):
                continue
        inside = [x for x in samples if t0 is not None and t0 <= x[0] <= t1]
        use = inside if inside else samples
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for x in use:
            for k, name in enumerate(names):
                if x[4][k].lower().startswith("active"):
                    reasons.add(name)
        sm = [x[1] for x in use]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(x[2] for x in use) if use else None,
                "power_w_max": max(x[3] for x in use) if use else None,
                "samples": len(use), "in_timed_region": bool(inside), "reasons": sorted(reasons)}


def shard_exchange(tri, flags, group=None):
    """The exchange step of a sharded count: the partial △(v) of every rank
    summed and the edge flags OR-ed, in place (NCCL between GPUs, gloo on
    CPU).  A single process has nothing to exchange."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return tri, flags
    import paper_2105_00110_gb300 as tcg
    return tcg.allreduce_counts(tri, flags, group)


def aggregate(t_ms: float, e2e_ms: float, units: int, e2e_units: int, world: int, device=None):
    """Whole-job figures across ranks: the slowest rank's time (MAX) and the
    units all ranks processed (SUM).  Identity for a single process."""
    if world <= 1:
        return t_ms, e2e_ms, units, e2e_units
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units), float(e2e_units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), int(u[0]), int(u[1])


# ------------------------------------------------------------ our path
def run_ours(args, spec, wl_name):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2105_00110_gb300 as tcg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tcg.build()

    # sharded: every rank holds the same graph and counts its share of the
    # work items; replicas: every rank its own graph
    sharded = world > 1 and not getattr(args, "replicas", False)
    src_np, dst_np, n = generate(spec, 0 if sharded else rank)
    np_pairs = len(src_np)
    d_src = torch.from_numpy(src_np).to(dev)
    d_dst = torch.from_numpy(dst_np).to(dev)
    h_src = torch.from_numpy(src_np).pin_memory()
    h_dst = torch.from_numpy(dst_np).pin_memory()
    del src_np, dst_np
    stream = torch.cuda.current_stream(dev)

    tri = torch.empty(n, dtype=torch.uint64, device=dev)
    numer = torch.empty(n, dtype=torch.uint64, device=dev)
    tcv = torch.empty(n, dtype=torch.float64, device=dev)
    h_tc = torch.empty(n, dtype=torch.float64).pin_memory()
    h_tri = torch.empty(n, dtype=torch.uint64).pin_memory()
    flag_buf = [None]

    host_ms = {}   # host time per call of the end-to-end steps (the calls that sync their stream)

    def step(src, dst, to_host=False):
        t0 = time.perf_counter()
        g = tcg.tc_build_csr(src, dst, n, stream)
        t1 = time.perf_counter()
        m = tcg.tc_graph_info(g)[1]
        if flag_buf[0] is None or flag_buf[0].numel() < m:
            flag_buf[0] = torch.empty(max(m, 1), dtype=torch.uint8, device=dev)
        fl = flag_buf[0][:max(m, 1)] if m else None
        if sharded:
            tcg.tc_count_shard(g, rank, world, tri, fl, stream)
            shard_exchange(tri, fl)
            st, total = tcg.tc_load_counts(g, tri, fl, stream)
        else:
            st, total = tcg.tc_count(g, tri, fl, stream)
        t2 = time.perf_counter()
        tcg.tc_centrality(g, numer, tcv, stream)
        if to_host:
            h_tc.copy_(tcv, non_blocking=True)
            h_tri.copy_(tri, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()
        t3 = time.perf_counter()
        if not to_host and stats_box[0] is None:
            stats_box[0] = tcg.tc_get_stats(g)
        tcg.tc_graph_free(g)
        if to_host:
            for k, dt in (("build", t1 - t0), ("count", t2 - t1), ("centrality_and_copy_out", t3 - t2),
                          ("free", time.perf_counter() - t3)):
                host_ms[k] = host_ms.get(k, 0.0) + 1e3 * dt
        return m, total

    stats_box = [None]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---------------- device-resident timing
    # the clock sampler starts before the warm-up so that its start-up does
    # not fall into the timed region; only samples inside it are kept
    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        m, total = step(d_src, d_dst)
    stats = stats_box[0]
    tcg.tc_profile_reset()
    tcg.tc_profile_enable(True)
    launches0 = tcg.tc_launch_count()
    barrier()
    host_t0 = time.time()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    edges = 0
    for _ in range(args.steps):
        m, total = step(d_src, d_dst)
        edges += m
    ev1.record(stream)
    barrier()
    host_t1 = time.time()
    clocks = sampler.stop(host_t0, host_t1)
    tcg.tc_profile_enable(False)
    launches = tcg.tc_launch_count() - launches0
    prof = tcg.tc_profile_read()
    t_ms = ev0.elapsed_time(ev1)

    # ---------------- per-edge triangle counts: the count in edge-count mode
    # against the plain count, on one built graph (outside the timed step)
    edge_counts = None
    if world == 1 and getattr(args, "edge_counts", True):
        g = tcg.Graph(d_src, d_dst, n, stream)
        et = torch.empty(max(g.m, 1), dtype=torch.int32, device=dev).view(torch.uint32)
        times = {}
        for mode in ("count", "edges"):
            for _ in range(2):
                if mode == "count":
                    tcg.tc_count(g.h, tri, None, stream)
                else:
                    tcg.tc_edge_triangles(g.h, tri, et[:g.m], stream)
            torch.cuda.synchronize(dev)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(3):
                if mode == "count":
                    tcg.tc_count(g.h, tri, None, stream)
                else:
                    tcg.tc_edge_triangles(g.h, tri, et[:g.m], stream)
            c1.record(stream)
            torch.cuda.synchronize(dev)
            times[mode] = c0.elapsed_time(c1) / 3
        edge_counts = {"edges_per_s": g.m / (times["edges"] / 1e3), "ms_per_call": times["edges"],
                       "plain_count_ms_per_call": times["count"],
                       "sum_over_edges_equals_3_triangles": int(et[:g.m].view(torch.int32).sum().item()) == 3 * total}
        g.close()
        del et

    # ---------------- end to end from pinned host buffers
    for _ in range(max(1, args.warmup // 2)):
        step(h_src, h_dst, to_host=True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tcg.tc_profile_reset()
    tcg.tc_profile_enable(True)
    e0.record(stream)
    e2e_edges = 0
    for _ in range(args.steps):
        m2, _ = step(h_src, h_dst, to_host=True)
        e2e_edges += m2
    e1.record(stream)
    barrier()
    tcg.tc_profile_enable(False)
    e2e_prof = tcg.tc_profile_read()
    e2e_ms = e0.elapsed_time(e1)
    # the pair upload inside each end-to-end build, timed by the library
    # (explains e2e - value); kernels are the other entries
    up = e2e_prof.pop("copy_h2d_pairs", (0, 0.0))
    upload_ms = up[1] / args.steps if up[0] else None
    h2d_gbs = (2 * np_pairs * 4 / (upload_ms / 1e3) / 1e9) if upload_ms else None

    t_max, e2e_max, edges_all, e2e_edges_all = aggregate(t_ms, e2e_ms, edges, e2e_edges, world, dev)
    if sharded:   # one graph for the whole job: its edges count once
        edges_all, e2e_edges_all = edges, e2e_edges

    if rank == 0:
        peak, peak_kind = peaks()
        # the dominant kernel of the step among those with an algorithmic
        # byte model (the count classes; the build's scatter-bound kernels
        # carry none) and its algorithmic bytes per launch
        kern = {k: v for k, v in prof.items()}
        bytes_per = {name: stats["class_bytes"][c] for name, c in tcg.KERNEL_CLASS.items()}
        modelled = {k: v for k, v in kern.items() if bytes_per.get(k)}
        top = max(modelled.items(), key=lambda kv: kv[1][1]) if modelled else None
        roof = None
        if top:
            name, (launch_n, tot_ms) = top
            avg_s = tot_ms / launch_n / 1e3
            achieved = bytes_per[name] / avg_s / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1),
                    "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": dram_traffic(name, wl_name),
                    "algorithmic_bytes_per_launch": bytes_per[name],
                    "avg_launch_ms": round(tot_ms / launch_n, 4)}
        step_ms = t_max / args.steps
        kernel_ms = {k: round(v[1] / args.steps, 4) for k, v in sorted(kern.items(), key=lambda kv: -kv[1][1])}
        count_ms = sum(v for k, v in kernel_ms.items() if k.startswith("count"))
        gather_ms = sum(v for k, v in kernel_ms.items() if k.startswith("gather"))
        # the survey's per-graph roofline: B_alg = 4 Σ d_H(u)² (Procedure 1
        # streaming every N_H(u) once per higher neighbour) + 43 m + 64 n
        # compulsory bytes, over the count + centrality kernel time
        b_alg = 4.0 * stats["sum_out_degree_sq"] + 43.0 * m + 64.0 * n
        t_cc = count_ms + gather_ms
        survey_roof = None
        if t_cc > 0:
            ach = b_alg / (t_cc / 1e3) / 1e9
            survey_roof = {"model": "B_alg = 4*sum_u d_H(u)^2 + 43m + 64n per graph, t = count + centrality kernels",
                           "bytes": b_alg, "t_ms": round(t_cc, 3), "achieved": round(ach, 1), "peak": peak,
                           "unit": "GB/s", "frac": round(ach / peak, 4),
                           "note": "bytes a kernel streaming every id of N_H(u) would move; this one streams only "
                                   "the ids above the middle vertex and none of the dense core's, so frac can "
                                   "exceed 1 (the per-kernel roofline is the strict figure)"}
        # the dense core's bit-packed pass: one AND + population count per
        # 32-bit row word, core edges x words per row per count
        core_obj = None
        core_c = stats.get("core_vertices") or 0
        if core_c and "count_core_pairs" in kern:
            launch_n, tot_ms = kern["count_core_pairs"]
            words = float(stats.get("core_words") or 0.0)
            t_s = tot_ms / launch_n / 1e3
            core_obj = {"kernel": "count_core_pairs", "core_vertices": core_c, "words_per_launch": words,
                        "avg_launch_ms": round(tot_ms / launch_n, 4),
                        "achieved_gwords_per_s": round(words / t_s / 1e9, 1) if t_s > 0 else None}
        # the build (rows a1-a2) against two byte models: what it must read
        # and write at least once (pairs in; col, head records, edge_tail,
        # the canonical edge list, row_ptr/hstart/perm/work out), and what
        # this implementation moves (the radix passes over 8-byte keys, the
        # placement and run sorts, the scatter of 16- and 8-byte records at
        # 32-byte sector granularity)
        build_ms = sum(v for k, v in kernel_ms.items() if k.startswith(("build", "plan")))
        bits = max(1, int(n - 1).bit_length())
        passes = (2 * bits + 7) // 8
        b_min = 8.0 * np_pairs + 40.0 * m + 28.0 * n
        b_impl = (24.0 + 16.0 * passes) * np_pairs + 140.0 * m + 28.0 * n
        build_roof = None
        if build_ms > 0:
            build_roof = {"t_ms": round(build_ms, 3), "radix_passes": passes,
                          "compulsory_bytes": b_min, "compulsory_frac": round(b_min / (build_ms / 1e3) / 1e9 / peak, 4),
                          "implementation_bytes": b_impl,
                          "implementation_frac": round(b_impl / (build_ms / 1e3) / 1e9 / peak, 4),
                          "peak": peak, "unit": "GB/s"}
        cpu = cpu_baseline(args) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": METRIC,
            "value": edges_all / (t_max / 1e3),
            "unit": "edges/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": step_ms,
            "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": wl_name, "n": n, "m": m, "pairs": np_pairs,
                       "generator": spec, "triangles": total,
                       "l2": "inputs larger than L2 (pair list %.1f GB per step)" % (np_pairs * 8 / 1e9),
                       "parallelism": ("shard%d: every rank builds the graph, counts work items rank, "
                                       "rank + N, ...; NCCL sum of counts and OR of flags; local gather"
                                       % world) if sharded else ("replicas" if world > 1 else "single"),
                       "backend": dist.get_backend() if world > 1 else None},
            "clocks": clocks,
            "e2e": {"value": e2e_edges_all / (e2e_max / 1e3), "unit": "edges/s",
                    "h2d_bytes_per_step": 2 * np_pairs * 4,
                    "d2h_bytes_per_step": n * 8 * 2 + 8,
                    "ms_per_step": e2e_max / args.steps,
                    "upload_ms_per_step": round(upload_ms, 2) if upload_ms else None,
                    "h2d_gb_per_s_measured": round(h2d_gbs, 1) if h2d_gbs else None,
                    # pinned uploads run at 200-210 GB/s on most hosts of this
                    # kind; well below that the end-to-end figure measures the
                    # host's copy path, not the library
                    "slow_host_copies": bool(h2d_gbs) and h2d_gbs < 120.0,
                    "kernel_ms_per_step": round(sum(v[1] for v in e2e_prof.values()) / args.steps, 2),
                    "host_ms_per_step_by_call": {k: round(v / (args.steps + max(1, args.warmup // 2)), 2)
                                                 for k, v in host_ms.items()},
                    "top_kernels_ms_per_step": {k: round(v[1] / args.steps, 2) for k, v in
                                                sorted(e2e_prof.items(), key=lambda kv: -kv[1][1])[:6]}},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "phases_ms_per_step": kernel_ms,
            "count_plus_centrality_edges_per_s": (m / ((count_ms + gather_ms) / 1e3)) if count_ms else None,
            "roofline_survey_model": survey_roof,
            "dense_core": core_obj,
            "roofline_build": build_roof,
            "edge_triangles": edge_counts,
            "graph_stats": stats,
        }
        return line
    return None


# ------------------------------------------------------------ batched path
def run_batched(args, spec, wl_name):
    """Config-3 workload: one batch of `count` graphs per step (tc_batch_build
    + tc_batch_run + free), against one build/count/centrality per graph."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import graphgen as gg
    import paper_2105_00110_gb300 as tcg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tcg.build()
    graphs = gg.batch_config3(spec["count"], spec["seed"] + 0x100000 * rank)
    src, dst, off, nv = tcg.pack_graphs(graphs)
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        b = tcg.Batch(d_src, d_dst, off, nv, stream)
        b.run(stream)
        m = b.m
        b.close()
        return m

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        m = step()
    b0 = tcg.Batch(d_src, d_dst, off, nv, stream)
    stats = b0.stats()
    b0.close()
    tcg.tc_profile_reset()
    tcg.tc_profile_enable(True)
    launches0 = tcg.tc_launch_count()
    torch.cuda.synchronize(dev)
    host_t0 = time.time()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    edges = 0
    for _ in range(args.steps):
        edges += step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    host_t1 = time.time()
    clocks = sampler.stop(host_t0, host_t1)
    tcg.tc_profile_enable(False)
    launches = tcg.tc_launch_count() - launches0
    prof = tcg.tc_profile_read()
    t_ms = ev0.elapsed_time(ev1)

    # run only, replayed from a CUDA graph (the batch built once)
    b = tcg.Batch(d_src, d_dst, off, nv, stream)
    tuned = b.autotune(reps=2, stream=stream)
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        b.run(side)
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        b.run(side)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize(dev)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record()
    for _ in range(args.steps):
        graph.replay()
    r1.record()
    torch.cuda.synchronize(dev)
    replay_ms = r0.elapsed_time(r1) / args.steps
    b.close()

    # one build + count + centrality per graph, same graphs
    n_base = min(len(graphs), args.baseline_graphs)
    per = [(torch.from_numpy(g[0]).to(dev), torch.from_numpy(g[1]).to(dev), g[2]) for g in graphs[:n_base]]
    torch.cuda.synchronize(dev)
    pb0 = time.perf_counter()
    base_edges = 0
    for s_, d_, n_ in per:
        if n_ == 0:
            continue
        g = tcg.Graph(s_, d_, n_, stream)
        g.count(want_flags=True, stream=stream)
        g.centrality(stream=stream)
        base_edges += g.m
        g.close()
    torch.cuda.synchronize(dev)
    per_graph_rate = base_edges / (time.perf_counter() - pb0)

    # end to end from pinned host buffers
    h_src, h_dst = torch.from_numpy(src).pin_memory(), torch.from_numpy(dst).pin_memory()
    tot_n = int(nv.sum())
    h_tc = torch.empty(max(tot_n, 1), dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_edges = 0
    for _ in range(args.steps):
        bb = tcg.Batch(h_src, h_dst, off, nv, stream)
        o = bb.run(stream)
        h_tc[:tot_n].copy_(o["tc"][:tot_n], non_blocking=True)
        e2e_edges += bb.m
        bb.close()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    t_max, e2e_max, edges_all, e2e_all = aggregate(t_ms, e2e_ms, edges, e2e_edges, world, dev)
    if rank == 0:
        peak, peak_kind = peaks()
        # the dominant kernel among those with an algorithmic byte model (the
        # count classes); the build's run kernels, which can take longer on
        # many tiny graphs, are scatter-bound and carry none
        bytes_per = {name: stats["class_bytes"][c] for name, c in tcg.KERNEL_CLASS.items()}
        modelled = {k: v for k, v in prof.items() if bytes_per.get(k)}
        top = max(modelled.items(), key=lambda kv: kv[1][1]) if modelled else None
        roof = None
        if top and bytes_per.get(top[0]):
            name, (nl, tot) = top
            achieved = bytes_per[name] / (tot / nl / 1e3) / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": None, "algorithmic_bytes_per_launch": bytes_per[name],
                    "avg_launch_ms": round(tot / nl, 4)}
        value = edges_all / (t_max / 1e3)
        return {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl_name, "graphs": len(graphs), "vertices": tot_n, "m": m,
                       "pairs": int(len(src)), "generator": spec,
                       "l2": "inputs larger than L2 (pair list %.1f GB per step)" % (len(src) * 8 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "clocks": clocks,
            "e2e": {"value": e2e_all / (e2e_max / 1e3), "unit": "edges/s",
                    "h2d_bytes_per_step": int(len(src)) * 8 + 16 * len(nv), "d2h_bytes_per_step": tot_n * 8},
            "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": None,
            "phases_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "batched_run_replay_ms": replay_ms,
            "batched_run_replay_edges_per_s": m / (replay_ms / 1e3),
            "one_launch_per_graph_edges_per_s": per_graph_rate,
            "one_launch_per_graph_sample_graphs": n_base,
            "batched_speedup_vs_per_graph": value / per_graph_rate,
            "autotuned_params": tuned,
            "graph_stats": stats,
        }
    return None


# ------------------------------------------------------------- served path
def _pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def _mem_available():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def run_served(args, spec, wl_name):
    """Served workload: a Poisson request stream over a pre-generated pool of
    graphs in pinned host memory, through the request loop (tc_server_*).
    Every request crosses host -> device -> host.  Two phases: the stated
    arrival rate for the stated duration (offered load far beyond capacity:
    throughput is what completes inside the window, latency is that of the
    requests completed in it, the rest are dropped at the end and counted),
    then a rate of sustain_load x the measured request capacity, drained to
    the last request, whose latencies are the steady-state figures."""
    import numpy as np
    import torch

    import graphgen as gg
    import paper_2105_00110_gb300 as tcg

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    tcg.build()
    pool_seed = spec["seed"] + 0x100000 * rank
    specs = gg.served_pool_specs(spec["pool"], pool_seed, spec["e_min"], spec["e_max"])
    need = sum(8 * sp["pairs"] + 16 * (2 ** sp["scale"] if sp["kind"] == "rmat" else sp["side"] ** 2)
               for sp in specs)
    avail = _mem_available()
    if avail is not None and need > 0.4 * avail:
        raise SystemExit("served pool needs %.1f GB of pinned host memory, %.1f GB available"
                         % (need / 1e9, avail / 1e9))
    tg0 = time.perf_counter()
    pool = []
    for sp in specs:
        s_, d_, n_ = gg.served_graph(sp)
        hs = torch.from_numpy(s_).pin_memory()
        hd = torch.from_numpy(d_).pin_memory()
        # results of every request of this pool entry land here; requests of
        # the same entry write identical values
        tri = torch.empty(max(n_, 1), dtype=torch.int64).pin_memory().view(torch.uint64)
        tcv = torch.empty(max(n_, 1), dtype=torch.float64).pin_memory()
        pool.append((hs, hd, n_, tri, tcv))
        del s_, d_
    gen_s = time.perf_counter() - tg0

    def new_server():
        return tcg.Server(spec["budget"], spec["max_batch_pairs"], spec["workers"])

    # warm-up pass: every pool graph once (also gives m and triangles per entry)
    srv = new_server()
    ids = {srv.submit(hs, hd, n_, tri, tcv): i for i, (hs, hd, n_, tri, tcv) in enumerate(pool)}
    m_of, tri_of = {}, {}
    for r in srv.wait_all(900):
        m_of[ids[r["id"]]] = r["edges"]
        tri_of[ids[r["id"]]] = r["triangles"]
    srv.close()
    assert len(m_of) == len(pool), "warm-up pass incomplete"

    def run_phase(rate, duration, seed, drain):
        rng = np.random.default_rng(seed)
        k = int(rate * duration * 1.2) + 16
        arr = np.cumsum(rng.exponential(1.0 / rate, k))
        arr = arr[arr < duration]
        pick = rng.integers(0, len(pool), len(arr))
        srv = new_server()
        req_of = {}
        done = []
        lag = 0.0
        launches0 = tcg.tc_launch_count()
        t0 = time.perf_counter()
        srv_t0 = None
        j = 0
        while j < len(arr):
            now = time.perf_counter() - t0
            while j < len(arr) and arr[j] <= now:
                hs, hd, n_, tri, tcv = pool[pick[j]]
                rid = srv.submit(hs, hd, n_, tri, tcv)
                req_of[rid] = (int(pick[j]), float(arr[j]))
                lag = max(lag, now - arr[j])
                j += 1
            done += srv.poll(4096)
            if j < len(arr):
                wait = arr[j] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        t_end = time.perf_counter() - t0
        if drain:
            done += srv.wait_all(1800)
            t_end = time.perf_counter() - t0
        else:
            while True:
                got = srv.poll(4096)
                done += got
                if len(got) < 4096:
                    break
        st = srv.stats()
        launches = tcg.tc_launch_count() - launches0
        srv.close()
        # server clock: t_submit of the first request is about t = 0 here
        first = min((r["t_submit"] for r in done), default=0.0)
        window = duration if not drain else max(r["t_done"] for r in done) - first
        inside = [r for r in done if drain or r["t_done"] - first <= duration]
        lat = [1e3 * (r["t_done"] - r["t_submit"]) for r in inside]
        bad = [r for r in inside if r["status"] < 0 or r["triangles"] != tri_of[req_of[r["id"]][0]]]
        edges = sum(r["edges"] for r in inside)
        pairs = sum(len(pool[req_of[r["id"]][0]][0]) for r in inside)
        half = [1e3 * (r["t_done"] - r["t_submit"]) for r in inside if req_of[r["id"]][1] < duration / 2]
        half2 = [1e3 * (r["t_done"] - r["t_submit"]) for r in inside if req_of[r["id"]][1] >= duration / 2]
        mean_pairs = float(np.mean([len(pool[p][0]) for p in pick])) if len(pick) else 0.0
        return {
            "rate_req_s": rate, "arrivals_s": duration, "submitted": int(len(arr)),
            "completed": len(inside), "dropped_or_late": int(len(arr)) - len(inside),
            "window_s": window, "achieved_req_s": len(inside) / window,
            "achieved_edges_per_s": edges / window, "achieved_pairs_per_s": pairs / window,
            "offered_pairs_per_s": rate * mean_pairs,
            "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "max": max(lat) if lat else None},
            "p99_first_half_ms": _pct(half, 99), "p99_second_half_ms": _pct(half2, 99),
            "batch_size_mean": float(np.mean([r["batch_size"] for r in inside])) if inside else None,
            "batches": st["batches"], "submit_lag_ms_max": 1e3 * lag, "wrong_results": len(bad),
            "gpu_launches": int(launches), "edges": edges,
            "h2d_bytes": 8 * pairs, "d2h_bytes": 16 * sum(pool[req_of[r["id"]][0]][2] for r in inside),
        }

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(1.0)
    h0 = time.time()
    over = run_phase(spec["rate"], spec["duration"], pool_seed + 1, drain=False)
    h1 = time.time()
    clocks = sampler.stop(h0, h1)
    sus_rate = max(1.0, spec["sustain_load"] * over["achieved_req_s"])
    sus = run_phase(sus_rate, spec["sustain_duration"], pool_seed + 2, drain=True)
    if rank == 0:
        n_done = max(over["completed"], 1)
        return {
            "metric": METRIC + "; p50/p99 request latency", "value": over["achieved_edges_per_s"],
            "unit": "edges/s", "n_gpus": 1, "steps": over["completed"], "warmup": len(pool),
            "ms_per_step": 1e3 * over["window_s"] / n_done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl_name, "pool_graphs": len(pool),
                       "pool_pairs": int(sum(len(p[0]) for p in pool)), "generator": spec,
                       "step": "one request (host pairs in, host results out)",
                       "l2": "inputs larger than L2 (pool %.1f GB of pinned pairs, requests drawn at random)"
                             % (sum(len(p[0]) for p in pool) * 8 / 1e9),
                       "pool_generation_s": round(gen_s, 1), "parallelism": "single"},
            "clocks": clocks,
            "e2e": {"value": over["achieved_edges_per_s"], "unit": "edges/s",
                    "h2d_bytes_per_step": over["h2d_bytes"] // n_done,
                    "d2h_bytes_per_step": over["d2h_bytes"] // n_done},
            "gpu_launches": over["gpu_launches"], "roofline": None, "cpu_baseline": None,
            "latency_ms": over["latency_ms"],
            "overload": over, "sustainable": sus,
        }
    return None


# ------------------------------------------------------------- oracle side
CPU_SAMPLE_ALL = dict(kind="rmat", scale=22, edge_factor=16, seed=0x5EED0016)
CPU_SAMPLE_ONE = dict(kind="rmat", scale=19, edge_factor=16, seed=0x5EED0012)
REF_SAMPLE = dict(kind="rmat", scale=18, edge_factor=16, seed=0x5EED0010)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_pass(spec, threads=1):
    """Full triangle centrality by the oracle (build, degree-ordered listing,
    Definition 1 numerators, exact division) on `threads` host threads;
    returns (edges, seconds)."""
    import oracle
    s, d, n = generate(spec)
    t0 = time.perf_counter()
    r = oracle.run(s, d, n, "fast", threads=threads, algebraic=False)
    dt = time.perf_counter() - t0
    return len(r["adj"]) // 2, dt


def cpu_baseline(args):
    cores = host_cores()
    m_all, dt_all = oracle_pass(CPU_SAMPLE_ALL, cores)
    m_one, dt_one = oracle_pass(CPU_SAMPLE_ONE, 1)
    return {"value": m_all / dt_all, "unit": "edges/s", "cores": cores, "kind": "oracle",
            "sample": "R-MAT scale 22, edge factor 16, same (a,b,c,d) as the workload: full TC by the oracle "
                      "(canonical CSR, degree-ordered listing, Definition 1 numerators, exact division) "
                      "on all %d host threads, %.1f s" % (cores, dt_all),
            "single_thread": {"value": m_one / dt_one, "unit": "edges/s", "cores": 1,
                              "sample": "R-MAT scale 19, same generator and oracle, one thread, %.1f s" % dt_one}}


def run_reference(args, wl_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_pass(REF_SAMPLE, cores)
    tot_m, tot_t = 0, 0.0
    for _ in range(args.steps):
        m, dt = oracle_pass(REF_SAMPLE, cores)
        tot_m += m
        tot_t += dt
    val = tot_m / tot_t
    sample = ("each step: R-MAT scale 18, edge factor 16, same (a,b,c,d) as the workload, full "
              "TC by the oracle on all %d host threads (a bounded sample of %s)" % (cores, wl_name))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "edges/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": wl_name},
        "cpu_baseline": {"value": val, "unit": "edges/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------- default suite
def run_other_configs(args):
    """The other four workloads of the suite, each measured in this process
    with its own clock record, for the default run's "configs" key: R-MAT
    scale 12 and the 4096^2 grid + Chung-Lu overlay (plain single graph),
    the 8192-graph batch and the served Poisson stream."""
    import torch
    out = {}
    small = argparse.Namespace(**vars(args))
    small.no_cpu = True
    small.edge_counts = False
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "e2e", "gpu_launches", "roofline", "clocks",
            "phases_ms_per_step", "roofline_survey_model", "dense_core", "roofline_build")
    for name, steps in (("rmat-s12-ef16", max(args.steps, 20)), ("grid4096-diag05-cl21", args.steps)):
        small.steps = steps
        line = run_ours(small, WORKLOADS[name], name)
        cfg = {k: line.get(k) for k in keep}
        cfg["config"] = {k: line["config"][k] for k in ("n", "m", "pairs", "triangles")}
        cfg["phases_ms_per_step"] = dict(list(line["phases_ms_per_step"].items())[:8])
        out[name] = cfg
        torch.cuda.empty_cache()
    b = argparse.Namespace(**vars(args))
    b.steps = 3
    line = run_batched(b, BATCH_WORKLOADS["batched-8192"], "batched-8192")
    line.pop("graph_stats", None)
    line["phases_ms_per_step"] = dict(list(line["phases_ms_per_step"].items())[:8])
    out["batched-8192"] = line
    torch.cuda.empty_cache()
    line = run_served(args, SERVED_WORKLOADS["served-poisson"], "served-poisson")
    out["served-poisson"] = line
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=None,
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(SERVED_WORKLOADS),
                    help="one workload alone (default: R-MAT scale 24, then the other four configs)")
    ap.add_argument("--baseline-graphs", type=int, default=8192,
                    help="graphs timed one launch per graph (batched workloads)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-configs", action="store_true", help="default run: skip the other four configs")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: every rank counts its own graph (default for single graphs: one "
                         "graph sharded across the ranks)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    suite = args.workload is None
    wl = args.workload or DEFAULT_WORKLOAD
    if args.impl == "reference":
        run_reference(args, wl)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        # NCCL's communicator set-up lines (rank count, devices) on stderr
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        os.environ.setdefault("NCCL_DEBUG_FILE", "/dev/stderr")
        dist.init_process_group("nccl")
    if wl in SERVED_WORKLOADS:
        line = run_served(args, SERVED_WORKLOADS[wl], wl)
    elif wl in BATCH_WORKLOADS:
        line = run_batched(args, BATCH_WORKLOADS[wl], wl)
    else:
        line = run_ours(args, WORKLOADS[wl], wl)
    if suite and world == 1 and line is not None and not args.no_configs:
        line["configs"] = run_other_configs(args)
    if line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
