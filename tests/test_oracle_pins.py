"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test fixes the oracle to something independent: the literal definition of Eq. 1
(exhaustive shortest-path enumeration in exact rationals), the Bellman-criterion form
of Eq. 1, closed forms derived from Eq. 1, an invariant, networkx, and exact integer
path counts.  Ordered-pair convention throughout: each unordered closed form is doubled.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import brute

REL = 1e-12


def close(a, b, rel=REL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= rel * np.maximum(np.abs(b), 1.0))


def all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        e = [p for i, p in enumerate(pairs) if mask >> i & 1]
        yield gg.from_edge_list(n, e) if e else gg.Graph(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32))


# ------------------------------------------------------------ Eq. 1, exhaustive
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_enumeration(n):
    """Every labelled graph on n <= 5 vertices: oracle == literal path enumeration, with
    and without 1-degree pruning."""
    for g in all_graphs(n):
        want = [float(x) for x in brute.bc_enumerate(g)]
        assert close(oracle.bc_exact(g), want), g.col_idx
        assert close(oracle.bc_exact(g, prune=True), want), g.col_idx


def test_exhaustive_n6_bellman():
    """All 32768 labelled graphs on 6 vertices vs the Bellman form of Eq. 1 (every 7th
    graph, plus all graphs with a leaf, keeps the CPU time small)."""
    for i, g in enumerate(all_graphs(6)):
        deg = g.degrees()
        if i % 7 and not (deg == 1).any():
            continue
        want = [float(x) for x in brute.bc_bellman(g)]
        assert close(oracle.bc_exact(g), want)
        assert close(oracle.bc_exact(g, prune=True), want)


def test_random_bellman(rng):
    for trial in range(40):
        n = int(rng.integers(7, 41))
        m = int(rng.integers(0, 3 * n))
        g = gg.gnm(n, m, seed=1000 + trial)
        want = [float(x) for x in brute.bc_bellman(g)]
        assert close(oracle.bc_exact(g), want)
        assert close(oracle.bc_exact(g, prune=True), want)


def test_source_subset_is_partial_sum(rng):
    """bc(sources) sums per-source dependencies: a split of the sources adds up, and a
    repeated source counts twice (multiset)."""
    g = gg.gnm(30, 60, seed=5)
    full = oracle.bc(g)
    a = oracle.bc(g, np.arange(0, 13))
    b = oracle.bc(g, np.arange(13, 30))
    assert close(a + b, full)
    twice = oracle.bc(g, np.array([4, 4], np.int32))
    once = oracle.bc(g, np.array([4], np.int32))
    assert close(twice, 2 * once)


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 3, 5, 9, 64])
def test_path(n):
    i = np.arange(n)
    assert close(oracle.bc_exact(gg.path_graph(n)), 2 * i * (n - 1 - i))
    assert close(oracle.bc_exact(gg.path_graph(n), prune=True), 2 * i * (n - 1 - i))


@pytest.mark.parametrize("n", [3, 4, 10, 200])
def test_star(n):
    want = np.zeros(n)
    want[0] = (n - 1) * (n - 2)
    assert close(oracle.bc_exact(gg.star_graph(n)), want)
    assert close(oracle.bc_exact(gg.star_graph(n), prune=True), want)


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_complete(n):
    assert close(oracle.bc_exact(gg.complete_graph(n)), np.zeros(n))


@pytest.mark.parametrize("n", [4, 5, 8, 9, 30, 31])
def test_cycle(n):
    k = n // 2
    val = (k - 1) ** 2 if n % 2 == 0 else k * (k - 1)
    assert close(oracle.bc_exact(gg.cycle_graph(n)), np.full(n, val))


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (3, 5), (4, 4)])
def test_complete_bipartite(a, b):
    want = np.concatenate([np.full(a, b * (b - 1) / a), np.full(b, a * (a - 1) / b)])
    assert close(oracle.bc_exact(gg.complete_bipartite(a, b)), want)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_hypercube(k):
    val = k * 2 ** (k - 1) - 2 ** k + 1
    assert close(oracle.bc_exact(gg.hypercube(k)), np.full(1 << k, val))


@pytest.mark.parametrize("seed", range(6))
def test_tree_component_products(seed):
    """Tree: BC(v) = sum over ordered pairs of distinct components of T - v of |Ti||Tj|."""
    n = 25
    g = gg.random_tree(n, seed)
    adj = brute.adjacency(g)
    want = np.zeros(n)
    for v in range(n):
        sizes = []
        seen = {v}
        for r in adj[v]:
            stack, cnt = [r], 0
            seen.add(r)
            while stack:
                x = stack.pop()
                cnt += 1
                for y in adj[x]:
                    if y not in seen:
                        seen.add(y)
                        stack.append(y)
            sizes.append(cnt)
        tot = sum(sizes)
        want[v] = tot * tot - sum(s * s for s in sizes)
    assert close(oracle.bc_exact(g), want)
    assert close(oracle.bc_exact(g, prune=True), want)


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("seed", range(5))
def test_distance_invariant(seed):
    """sum_v BC(v) = sum over ordered connected pairs of (d(s,t) - 1), on graphs with
    several components and isolated vertices."""
    g = gg.gnm(35, 38, seed=200 + seed)
    assert math.isclose(oracle.bc_exact(g).sum(), brute.ordered_pair_distance_sum(g), rel_tol=1e-12)


def test_networkx():
    nx = pytest.importorskip("networkx")
    for seed in range(8):
        g = gg.gnm(60, 150, seed=300 + seed)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(zip(*[x.tolist() for x in g.edges()]))
        ref = nx.betweenness_centrality(G, normalized=False)
        want = 2 * np.array([ref[v] for v in range(g.n)])
        assert close(oracle.bc_exact(g), want, rel=1e-10)
        assert close(oracle.bc_exact(g, prune=True), want, rel=1e-10)


# ----------------------------------------------------------- 1-degree pruning
def test_prune_structure():
    """Alg. 6 reading: leaves with a neighbour of degree >= 2 are removed, K2 stays,
    isolated vertices stay; omega counts removed leaves."""
    # star 0-{1,2,3}, K2 4-5, isolated 6, path 7-8-9
    g = gg.from_edge_list(10, [(0, 1), (0, 2), (0, 3), (4, 5), (7, 8), (8, 9)])
    omega, removed, res = oracle.prune_deg1(g)
    assert removed.tolist() == [0, 1, 1, 1, 0, 0, 0, 1, 0, 1]
    assert omega.tolist() == [3, 0, 0, 0, 0, 0, 0, 0, 2, 0]
    assert res.degrees().tolist() == [0, 0, 0, 0, 1, 1, 0, 0, 0, 0]


@pytest.mark.parametrize("seed", range(3))
def test_prune_equivalence_ba(seed):
    g = gg.ba_pref_attach(600, seed)
    assert close(oracle.bc_exact(g, prune=True), oracle.bc_exact(g), rel=1e-11)


def test_prune_equivalence_rmat():
    g = gg.rmat(9, 4, seed=7)  # many leaves and small components
    assert close(oracle.bc_exact(g, prune=True), oracle.bc_exact(g), rel=1e-11)


def test_prune_keeps_residual_depth_sigma():
    """Leaves are never interior to a shortest path, so depth and sigma from a residual
    source are unchanged on residual vertices."""
    g = gg.ba_pref_attach(400, 3)
    omega, removed, res = oracle.prune_deg1(g)
    for s in np.flatnonzero(removed == 0)[:20]:
        d0, s0, _ = oracle.sssp(g, int(s))
        d1, s1, _ = oracle.sssp(res, int(s))
        keep = removed == 0
        assert (d0[keep] == d1[keep]).all() and (s0[keep] == s1[keep]).all()


# ------------------------------------------------- sigma: exact integer counts
def test_sigma_grid_binomial_mod64():
    """Open w x h grid: depth = Manhattan distance, sigma = C(|dx|+|dy|, |dx|); kept mod
    2^64 with the overflow flag set exactly where the count is >= 2^64."""
    w = h = 48
    g = gg.grid2d(w, h)
    for sx, sy in [(0, 0), (17, 30), (47, 5)]:
        s = sy * w + sx
        depth, sigma, ovf = oracle.sssp(g, s)
        for v in range(w * h):
            x, y = v % w, v // w
            dx, dy = abs(x - sx), abs(y - sy)
            c = math.comb(dx + dy, dx)
            assert depth[v] == dx + dy
            assert int(sigma[v]) == c % (1 << 64)
            assert bool(ovf[v]) == (c >= (1 << 64))


def test_sigma_long_double_grid():
    """The long-double sigma carries the exact count to ~64 significant bits."""
    w = 64
    g = gg.grid2d(w, w)
    _, _, _, sl = oracle.sssp(g, 0, want_long=True)
    for v in [w * w - 1, 40 * w + 63, 63 * w + 10]:
        x, y = v % w, v // w
        c = math.comb(x + y, x)
        assert abs(float(sl[v] / np.longdouble(c)) - 1.0) < 1e-15


def test_sigma_hypercube_factorial():
    """Q_k: sigma(v) = popcount(v xor s)!."""
    k = 10
    g = gg.hypercube(k)
    s = 37
    depth, sigma, ovf = oracle.sssp(g, s)
    for v in range(1 << k):
        p = bin(v ^ s).count("1")
        assert depth[v] == p and int(sigma[v]) == math.factorial(p) and ovf[v] == 0


def test_sigma_random_vs_exact(rng):
    for trial in range(10):
        g = gg.gnm(40, 90, seed=400 + trial)
        s = int(rng.integers(0, g.n))
        depth, sigma, _ = oracle.sssp(g, s)
        d, c = brute.exact_sigma(g, s)
        assert depth.tolist() == d
        assert [int(x) for x in sigma] == c
