"""Writes bc_small.txt: exact betweenness centrality (Eq. 1, ordered pairs) of small graphs as
exact rationals, from the oracle's rational brute force only (oracle/brute.py): the literal
enumeration of shortest paths where the graph is small enough, the Bellman-criterion form of
Eq. 1 otherwise, and both (which must agree) where both run.  Nothing here comes from the
CUDA path.

    python tests/golden/make_golden.py          # rewrite the fixture
    python tests/golden/make_golden.py --check  # compare with the committed fixture
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
from oracle import brute  # noqa: E402

FIXTURE = os.path.join(HERE, "bc_small.txt")


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return outer + spokes + inner


def graphs():
    """(name, n, edges): closed-form families, the heuristics' corner cases (leaves, degree-2
    chains, a star whose centre keeps no edge after the 1-degree reduction, a K2 component,
    an isolated vertex) and two irregular graphs."""
    out = [
        ("path7", 7, [(i, i + 1) for i in range(6)]),
        ("star6", 7, [(0, i) for i in range(1, 7)]),
        ("cycle7", 7, [(i, (i + 1) % 7) for i in range(7)]),
        ("cycle8", 8, [(i, (i + 1) % 8) for i in range(8)]),
        ("k3_4", 7, [(a, b) for a in range(3) for b in range(3, 7)]),
        ("petersen", 10, petersen()),
        ("cube3", 8, [(v, v ^ (1 << k)) for v in range(8) for k in range(3) if v < v ^ (1 << k)]),
        ("bowtie", 5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
        ("star_and_cycle_with_leaf", 9, [(0, 1), (0, 2), (0, 3), (4, 5), (5, 6), (6, 7), (7, 4), (7, 8)]),
        ("k2_path_isolated", 7, [(0, 1), (2, 3), (3, 4), (4, 5)]),
        ("chain_between_triangles", 10, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 6),
                                         (6, 7), (7, 8), (8, 6), (4, 9)]),
    ]
    t = gg.random_tree(14, 3)
    su, sv = t.edges()
    out.append(("random_tree14_seed3", t.n, list(zip(su.tolist(), sv.tolist()))))
    g = gg.gnm(16, 26, 2)
    su, sv = g.edges()
    out.append(("gnm16_26_seed2", g.n, list(zip(su.tolist(), sv.tolist()))))
    return out


def exact_bc(n, edges):
    g = gg.from_edge_list(n, edges)
    bel = brute.bc_bellman(g)
    if n <= 10:
        enu = brute.bc_enumerate(g)
        assert list(enu) == list(bel), "enumeration and Bellman form disagree"
    return [Fraction(x) for x in bel]


def render():
    lines = ["# Exact betweenness centrality (Eq. 1, ordered pairs s != t, s != v != t) of small",
             "# graphs as exact rationals.  Written by tests/golden/make_golden.py from the",
             "# oracle's rational brute force (literal path enumeration for n <= 10, checked",
             "# against the Bellman-criterion form of Eq. 1; that form alone above).  One block per",
             "# graph: name, vertex count, undirected edges u-v, BC of vertices 0..n-1."]
    for name, n, edges in graphs():
        bc = exact_bc(n, edges)
        lines += [f"graph {name}", f"n {n}", "edges " + " ".join(f"{u}-{v}" for u, v in edges),
                  "bc " + " ".join(str(x) for x in bc)]
    return "\n".join(lines) + "\n"


def load(path: str = FIXTURE):
    """[(name, n, edges, bc as Fractions)] from the fixture."""
    out = []
    cur = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "graph":
            cur = {"name": rest}
        elif key == "n":
            cur["n"] = int(rest)
        elif key == "edges":
            cur["edges"] = [tuple(int(x) for x in e.split("-")) for e in rest.split()]
        elif key == "bc":
            cur["bc"] = [Fraction(x) for x in rest.split()]
            out.append((cur["name"], cur["n"], cur["edges"], cur["bc"]))
    return out


if __name__ == "__main__":
    text = render()
    if "--check" in sys.argv:
        sys.exit(0 if open(FIXTURE).read() == text else 1)
    with open(FIXTURE, "w") as f:
        f.write(text)
