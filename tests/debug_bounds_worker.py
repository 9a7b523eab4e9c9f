"""Run in its own process by test_gpu_debug_bounds.py: loads the
bounds-checked build of the library (every index the count, gather and
dense-core kernels take from graph data checked against its array) and runs
the whole path on small graphs under every strategy, with and without a
dense core, in both count modes, sharded and batched, comparing each result
with the oracle.  Any failed bounds check makes the call raise
TC_ERR_BOUNDS.  Prints one line: "ok <calls>"."""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
import paper_2105_00110_gb300 as tcg  # noqa: E402


def check(src, dst, n, strategy, core):
    ref = oracle.run(src, dst, n)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ref["ptr"]))
    keep = ref["adj"] > rows
    tcg.tc_set_dense_core(core)
    g = tcg.Graph(torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda(),
                  torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda(), n)
    tcg.tc_set_dense_core(-1)
    try:
        g.set_strategy(strategy)
        tri, flags, total, _ = g.count()
        numer, tcv, _, _ = g.centrality()
        assert total == ref["total"]
        assert np.array_equal(tri.cpu().numpy().view(np.int64), ref["tri"].astype(np.int64))
        assert np.array_equal(flags.cpu().numpy(), ref["flag"][keep])
        assert np.array_equal(numer.cpu().numpy().view(np.int64), ref["numer"].astype(np.int64))
        if ref["total"]:
            assert np.array_equal(tcv.cpu().numpy().view(np.int64), ref["tc"].view(np.int64))
        tri2, et, total2, _ = g.edge_triangles()
        assert total2 == ref["total"]
        assert np.array_equal(et.cpu().numpy().view(np.int32).astype(np.int64), ref["t"][keep].astype(np.int64))
        part = torch.zeros(n, dtype=torch.int64, device="cuda")
        fl = torch.zeros(max(g.m, 1), dtype=torch.uint8, device="cuda")
        for k in range(3):
            t = torch.empty(n, dtype=torch.uint64, device="cuda")
            f = torch.empty(max(g.m, 1), dtype=torch.uint8, device="cuda")
            tcg.tc_count_shard(g.h, k, 3, t, f[:g.m] if g.m else None)
            part += t.view(torch.int64)
            fl = torch.maximum(fl, f)
        tcg.tc_load_counts(g.h, part.view(torch.uint64), fl[:g.m])
        numer3, _, _, _ = g.centrality()
        assert np.array_equal(numer3.cpu().numpy().view(np.int64), ref["numer"].astype(np.int64))
    finally:
        g.close()


def main():
    path = tcg.build(debug=True)
    tcg.use_library(path)
    assert tcg.tc_debug_bounds_build()
    graphs = [gg.rmat(10, seed=0x5EED0800), gg.rmat(12, seed=0x5EED0801), gg.barabasi_albert(3000, 6, seed=0x5EED0802),
              gg.planted_hierarchy(2000, 16, 8, 0.01, seed=0x5EED0803), gg.grid_chung_lu(side=48, seed=0x5EED0804),
              gg.complete_graph(60), gg.gnp(200, 0.15, 0x5EED0805),
              (np.zeros(0, np.int32), np.zeros(0, np.int32), 5)]
    calls = 0
    for src, dst, n in graphs:
        for strategy in ("auto", "bsearch", "merge", "bitmap", "global"):
            for core in ((0, 64, 700) if strategy in ("auto", "bitmap") else (0,)):
                check(src, dst, n, strategy, core)
                calls += 1
    batch = [gg.barabasi_albert(100 + 30 * i, 3, seed=0x5EED0810 + i) for i in range(10)]
    batch += [gg.planted_hierarchy(400, 6, 5, 0.01, seed=0x5EED0820 + i) for i in range(6)]
    b = tcg.Batch(*tcg.pack_graphs(batch))
    try:
        out = b.run()
        torch.cuda.synchronize()
        for i, (s, d, n) in enumerate(batch):
            ref = oracle.run(s, d, n)
            lo, hi = b.voff[i], b.voff[i + 1]
            assert np.array_equal(out["tri"][lo:hi].cpu().numpy().view(np.int64), ref["tri"].astype(np.int64))
            assert np.array_equal(out["tc"][lo:hi].cpu().numpy().view(np.int64), ref["tc"].view(np.int64))
    finally:
        b.close()
    assert tcg.tc_debug_bounds_line() == 0
    print("ok %d" % (calls + 1))


if __name__ == "__main__":
    main()
