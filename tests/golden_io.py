"""Reader for the small text fixtures under tests/golden/.

Format: '#' comment lines (each fixture cites the figure or table it comes
from), then
  vertices <name> ...          vertex names; ids are their positions
  edge <a> <b>                 one undirected edge
  star <hub> <leaf> ...        hub adjacent to every leaf
  clique <v> ...               all pairs among the listed vertices
  expect total <int>           triangles in G
  expect n <int> / m <int>     vertex / edge count
  expect core <v> <int>        core triangle sum of v (Definition 1)
  expect noncore <v> <int>     non-core triangle sum of v
  expect tc <v> <p>[/<q>]      exact triangle centrality of v
  expect top <v>               v has the strictly largest TC
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fixtures():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


def load(name: str):
    names, edges, expect = [], [], []
    with open(os.path.join(GOLDEN, name)) as fh:
        for raw in fh:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "vertices":
                names = tok[1:]
            elif tok[0] == "edge":
                edges.append((tok[1], tok[2]))
            elif tok[0] == "star":
                edges += [(tok[1], x) for x in tok[2:]]
            elif tok[0] == "clique":
                vs = tok[1:]
                edges += [(vs[i], vs[j]) for i in range(len(vs)) for j in range(i + 1, len(vs))]
            elif tok[0] == "expect":
                expect.append(tok[1:])
            else:
                raise ValueError("bad fixture line: %r" % line)
    idx = {v: i for i, v in enumerate(names)}
    src = np.array([idx[a] for a, _ in edges], dtype=np.int32)
    dst = np.array([idx[b] for _, b in edges], dtype=np.int32)
    parsed = []
    for e in expect:
        kind = e[0]
        if kind in ("total", "n", "m"):
            parsed.append((kind, None, int(e[1])))
        elif kind in ("core", "noncore"):
            parsed.append((kind, idx[e[1]], int(e[2])))
        elif kind == "tc":
            parsed.append((kind, idx[e[1]], Fraction(e[2])))
        elif kind == "top":
            parsed.append((kind, idx[e[1]], None))
        else:
            raise ValueError(kind)
    return src, dst, len(names), names, parsed
