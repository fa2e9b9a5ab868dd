"""Pins of the 2-degree heuristic's oracle (Sec. 3.4.2), on the CPU.

* The derived level and path count of every degree-2 vertex equal those of a plain BFS
  from it (Lemma 1 and the three-case equation), with exact integers, including counts
  past 2^64 on a grid.
* BC with the derived runs equals the exact rational brute force of Eq. 1 and the plain
  oracle, on graphs full of degree-2 vertices (cycles, paths, subdivided grids, trees).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import brute, deg2

GRAPHS = [
    gg.cycle_graph(9), gg.cycle_graph(10), gg.path_graph(12), gg.random_tree(30, 3),
    gg.subdivide_edges(gg.grid2d(5, 5, seed=1, delete_frac=0.15), 0.5, 2),
    gg.subdivide_edges(gg.complete_graph(5), 1.0, 3),
    gg.from_edge_list(6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5)]),  # triangle a-b-c
]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_derived_tree_equals_bfs(gi):
    g = GRAPHS[gi]
    adj = deg2._adj(g)
    deg = g.degrees()
    checked = 0
    for c in np.flatnonzero(deg == 2):
        a, b = adj[c]
        got = deg2.derive(adj, int(c), deg2.bfs(adj, a), deg2.bfs(adj, b))
        assert got == deg2.bfs(adj, int(c)), f"{g.name} c={c}"
        checked += 1
    assert checked > 0


def test_derived_counts_past_2_64():
    """Open 70 x 70 grid, 5% of its edges subdivided; c next to a corner: counts reach
    2^123."""
    g = gg.subdivide_edges(gg.grid2d(70, 70), 0.05, 7)
    adj = deg2._adj(g)
    c = int(min(np.flatnonzero(g.degrees() == 2), key=lambda x: min(adj[x])))
    a, b = adj[c]
    lvl, sig = deg2.derive(adj, c, deg2.bfs(adj, a), deg2.bfs(adj, b))
    want = deg2.bfs(adj, c)
    assert (lvl, sig) == want and max(sig) >= 2**64
    d, s64, ovf = oracle.sssp(g, c)  # the C oracle's modular counts agree too
    assert (d == np.array(lvl)).all()
    assert all(int(s64[v]) == sig[v] % 2**64 for v in range(g.n))
    assert all(bool(ovf[v]) == (sig[v] >= 2**64) for v in range(g.n))


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_bc_with_deg2_equals_plain(gi):
    g = GRAPHS[gi]
    got, ntri = deg2.bc_with_deg2(g)
    assert ntri > 0
    want = oracle.bc_exact(g)
    for v in range(g.n):
        assert abs(float(got[v]) - want[v]) <= 1e-9 * max(abs(want[v]), 1.0), (g.name, v)
    if g.n <= 12:
        ex = brute.bc_enumerate(g)
        assert all(got[v] == ex[v] for v in range(g.n))


def test_selection_is_disjoint():
    g = gg.subdivide_edges(gg.grid2d(8, 8, seed=3, delete_frac=0.1), 0.6, 4)
    tri = deg2.select_triples(g)
    seen = [v for t in tri for v in t]
    assert len(seen) == len(set(seen)) and len(tri) > 10
    deg = g.degrees()
    assert all(deg[c] == 2 for _, _, c in tri)


H3_GRAPHS = [
    gg.random_tree(40, 5),                                            # residual full of chains
    gg.attach_leaves(gg.cycle_graph(11), 0.5, 1),
    gg.attach_leaves(gg.subdivide_edges(gg.grid2d(5, 5, seed=1, delete_frac=0.15), 0.5, 2), 0.3, 3),
    gg.attach_leaves(gg.subdivide_edges(gg.gnm(30, 45, 4), 0.4, 5), 0.4, 6),
    gg.from_edge_list(7, [(0, 1), (1, 2), (2, 3), (3, 4), (2, 5), (5, 6)]),  # K2-free spider
    gg.from_edge_list(5, [(0, 1), (2, 3), (3, 4)]),                   # K2 component kept
    # a star (centre isolated in the residual graph, omega = 3) beside a cycle with a leaf
    gg.from_edge_list(9, [(0, 1), (0, 2), (0, 3), (4, 5), (5, 6), (6, 7), (7, 4), (7, 8)]),
]


@pytest.mark.parametrize("gi", range(len(H3_GRAPHS)))
def test_bc_deg2_with_pruning_equals_plain(gi):
    """Both heuristics at once (the paper's H3): triples chosen on the residual graph, leaf
    weights in every run; the result is exact (Eq. 1 by brute force on small graphs)."""
    g = H3_GRAPHS[gi]
    got, ntri = deg2.bc_with_deg2(g, prune=True)
    want = oracle.bc_exact(g)
    for v in range(g.n):
        assert abs(float(got[v]) - want[v]) <= 1e-9 * max(abs(want[v]), 1.0), (g.name, v)
    if g.n <= 12:
        ex = brute.bc_enumerate(g)
        assert all(got[v] == ex[v] for v in range(g.n)), g.name
    if gi < 4:
        assert ntri > 0


def test_pruning_changes_the_selection():
    """A cycle with a leaf on every vertex has no degree-2 vertex; its residual graph is the
    bare cycle, so H3 derives runs that H2 alone could not."""
    g = gg.attach_leaves(gg.cycle_graph(12), 1.0, 8, max_leaves=1)
    _, om_tri = deg2.bc_with_deg2(g, prune=True)
    assert not deg2.select_triples(g) and om_tri > 0
