"""Parity at the full bench sizes (R-MAT scale 24 and the 4096² grid with
Chung-Lu overlay), in the bench's launch configuration (device int32 pairs,
automatic strategy), where the oracle is too slow to run whole:

- on sampled vertices (uniform, by degree quantile, and the top hubs), the
  oracle's △(v), neighbour row and row of T = A² ∘ A against the GPU's
  △(v), canonical edges and per-edge counts;
- everywhere, identities that hold at any size: Σ△ = 3△(G), Σ t = 3△(G),
  △(v) = ½ Σ_u t(v, u), flag = [t > 0], the two count modes agree, and the
  numerator and the correctly rounded TC recomputed from △ and the flags;
- and, on R-MAT scale 22 and the whole 4096² grid, every output against
  the whole oracle run on the host's threads."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import bench
import oracle
import paper_2105_00110_gb300 as tcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    tcg.build()
    torch.cuda.init()


def gpu_path(s, d, n):
    g = tcg.Graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    try:
        tri, flags, total, st = g.count()
        numer, tcv, den, _ = g.centrality()
        eu, ev = g.edges()
        tri2, et, total2, _ = g.edge_triangles()
        torch.cuda.synchronize()
        return dict(n=n, m=g.m, tri=tri.view(torch.int64), flags=flags, total=total, den=den,
                    numer=numer.view(torch.int64), tc=tcv, eu=eu.long(), ev=ev.long(),
                    tri2=tri2.view(torch.int64), et=et.view(torch.int32).long(), total2=total2)
    finally:
        g.close()


def check_identities(r):
    n, total = r["n"], r["total"]
    assert total > 0 and r["den"] == 3 * total
    assert r["total2"] == total and torch.equal(r["tri2"], r["tri"])
    assert int(r["tri"].sum()) == 3 * total
    assert int(r["et"].sum()) == 3 * total
    half = torch.zeros(n, dtype=torch.int64, device="cuda")
    half.index_add_(0, r["eu"], r["et"])
    half.index_add_(0, r["ev"], r["et"])
    assert torch.equal(half, 2 * r["tri"])
    assert torch.equal(r["flags"].long(), (r["et"] > 0).long())
    w = torch.where(r["flags"] > 0, 1, 3).long()
    num = r["tri"].clone()
    num.index_add_(0, r["eu"], w * r["tri"][r["ev"]])
    num.index_add_(0, r["ev"], w * r["tri"][r["eu"]])
    assert torch.equal(num, r["numer"])
    numer = r["numer"].cpu().numpy()
    assert int(numer.max()) < 2 ** 53 and r["den"] < 2 ** 53      # exact binary64 operands
    want = numer.astype(np.float64) / np.float64(r["den"])        # one IEEE division: correctly rounded
    assert np.array_equal(r["tc"].cpu().numpy().view(np.int64), want.view(np.int64))


def check_samples(r, s, d, n, seed):
    og = oracle.OracleGraph(s, d, n)
    deg = np.diff(og.ptr)
    assert len(og.adj) == 2 * r["m"]
    rng = np.random.default_rng(seed)
    nz = np.nonzero(deg)[0]
    order = nz[np.argsort(deg[nz], kind="stable")]
    quant = order[(np.linspace(0, 1, 10)[:-1] * len(order)).astype(np.int64)]
    vs = np.unique(np.concatenate([rng.choice(nz, 40, replace=False), quant, order[-2:]]))
    tri, rows = og.sample_tri(vs)
    gtri = r["tri"].cpu().numpy()
    assert np.array_equal(gtri[vs], tri.astype(np.int64))
    eu, ev, et = r["eu"], r["ev"], r["et"]
    off = 0
    for v in vs.tolist():
        lo = og.ptr[v]
        hi = og.ptr[v + 1]
        nbr = og.adj[lo:hi].astype(np.int64)
        a = eu == v
        b = ev == v
        gu = torch.cat([ev[a], eu[b]])
        gt = torch.cat([et[a], et[b]])
        o = torch.argsort(gu)
        assert np.array_equal(gu[o].cpu().numpy(), nbr)
        assert np.array_equal(gt[o].cpu().numpy(), rows[off:off + len(nbr)].astype(np.int64))
        off += len(nbr)


@pytest.mark.parametrize("workload", ["rmat-s24-ef16", "grid4096-diag05-cl21"])
def test_full_size(workload):
    s, d, n = bench.generate(bench.WORKLOADS[workload])
    r = gpu_path(s, d, n)
    check_identities(r)
    check_samples(r, s, d, n, seed=0x5EED)


@pytest.mark.parametrize("workload", ["rmat-s22-ef16", "grid4096-diag05-cl21"])
def test_whole_graph_against_threaded_oracle(workload):
    # every vertex and edge of a large workload against the whole oracle:
    # its degree-ordered listing (pinned against the definition) run on the
    # host's threads; △(v), flags, t(u, v), numerators and TC all bit for bit
    import os
    s, d, n = bench.generate(bench.WORKLOADS[workload])
    r = gpu_path(s, d, n)
    ref = oracle.run(s, d, n, "fast", threads=os.cpu_count() or 1, algebraic=False)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ref["ptr"]))
    keep = ref["adj"] > rows
    assert r["total"] == ref["total"] and r["m"] == int(keep.sum())
    assert np.array_equal(r["eu"].cpu().numpy(), rows[keep])
    assert np.array_equal(r["ev"].cpu().numpy(), ref["adj"][keep].astype(np.int64))
    assert np.array_equal(r["tri"].cpu().numpy(), ref["tri"].astype(np.int64))
    assert np.array_equal(r["flags"].cpu().numpy(), ref["flag"][keep])
    assert np.array_equal(r["et"].cpu().numpy(), ref["t"][keep].astype(np.int64))
    assert np.array_equal(r["numer"].cpu().numpy(), ref["numer"].astype(np.int64))
    assert np.array_equal(r["tc"].cpu().numpy().view(np.int64), ref["tc"].view(np.int64))
