"""Exact rational brute force of Eq. 1 — TEST INFRASTRUCTURE (oracle side).

BC(v) = sum over ordered pairs s != t, s != v != t of sigma_st(v) / sigma_st  (Eq. 1,
Sec. 2), evaluated with ``fractions.Fraction`` so that no rounding enters.

Two independent evaluations:
  * ``bc_enumerate``: the definition taken literally — every shortest s-t path is listed
    (depth-first extension of partial paths, pruned at the BFS distance) and the paths
    through v are counted.  Exponential; meant for n <= 8.
  * ``bc_bellman``: sigma_st(v) = sigma_sv * sigma_vt when d(s,v) + d(v,t) = d(s,t), else 0
    (Bellman criterion, Lemma 2 of Sec. 3.4.2), with all-pairs BFS distances and path
    counts in exact Python integers.  Polynomial; meant for n <= ~60.
Neither shares code with the C oracle or the CUDA path.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction


def adjacency(g):
    return [list(map(int, g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]])) for v in range(g.n)]


def bfs_counts(adj, s):
    """Unweighted distances and exact shortest-path counts from s (None = unreachable)."""
    n = len(adj)
    d = [None] * n
    c = [0] * n
    d[s] = 0
    c[s] = 1
    q = deque([s])
    while q:
        v = q.popleft()
        for w in adj[v]:
            if d[w] is None:
                d[w] = d[v] + 1
                q.append(w)
            if d[w] == d[v] + 1:
                c[w] += c[v]
    return d, c


def all_shortest_paths(adj, s, t, dist):
    """Every shortest s-t path as a tuple of vertices (dist = BFS distance s->t)."""
    out = []
    stack = [(s, (s,))]
    while stack:
        v, path = stack.pop()
        if len(path) - 1 == dist:
            if v == t:
                out.append(path)
            continue
        for w in adj[v]:
            if w not in path:
                stack.append((w, path + (w,)))
    return out


def bc_enumerate(g):
    adj = adjacency(g)
    n = g.n
    bc = [Fraction(0)] * n
    for s in range(n):
        d, _ = bfs_counts(adj, s)
        for t in range(n):
            if t == s or d[t] is None:
                continue
            paths = all_shortest_paths(adj, s, t, d[t])
            total = len(paths)
            for v in range(n):
                if v == s or v == t:
                    continue
                through = sum(1 for p in paths if v in p)
                if through:
                    bc[v] += Fraction(through, total)
    return bc


def bc_bellman(g):
    adj = adjacency(g)
    n = g.n
    D, C = [], []
    for s in range(n):
        d, c = bfs_counts(adj, s)
        D.append(d)
        C.append(c)
    bc = [Fraction(0)] * n
    for s in range(n):
        for t in range(n):
            if s == t or D[s][t] is None:
                continue
            for v in range(n):
                if v == s or v == t or D[s][v] is None or D[v][t] is None:
                    continue
                if D[s][v] + D[v][t] == D[s][t]:
                    bc[v] += Fraction(C[s][v] * C[v][t], C[s][t])
    return bc


def exact_sigma(g, s):
    """Exact (unbounded) shortest-path counts and depths from s."""
    d, c = bfs_counts(adjacency(g), s)
    return [(-1 if x is None else x) for x in d], c


def ordered_pair_distance_sum(g):
    """sum over ordered connected pairs (s != t) of (d(s,t) - 1) — equals sum_v BC(v)."""
    adj = adjacency(g)
    tot = 0
    for s in range(g.n):
        d, _ = bfs_counts(adj, s)
        tot += sum(x - 1 for t, x in enumerate(d) if x is not None and t != s)
    return tot
