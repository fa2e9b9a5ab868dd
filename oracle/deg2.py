"""2-degree heuristic of Sec. 3.4.2, as plain Python (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module.

For a vertex c of degree 2 with neighbours a and b, every shortest path from c leaves
through a or b, so (Lemma 1 of Sec. 3.4.2, Bellman criterion):
  level_c(v) = 1 + min(level_a(v), level_b(v))          for v != c,
  sigma_c(v) = sigma_a(v)              if level_a(v) < level_b(v),
               sigma_b(v)              if level_a(v) > level_b(v),
               sigma_a(v) + sigma_b(v) if they are equal,
and level_c(c) = 0, sigma_c(c) = 1.  c's dependencies are then accumulated on that DAG
(Eq. 2) instead of after a traversal from c.  Integers are exact (Python ints) and
dependencies exact rationals, so this is usable on small graphs only.

Combined with the 1-degree reduction (Sec. 3.4.1, Eq. 3/4, Alg. 6), the triples are chosen
on the residual graph and every run, derived or not, carries the leaf weights omega: the
dependency recursion adds omega(v) for each successor v, a run from s counts omega(s) + 1
times, and s gains omega(s)(2 n_s - omega(s) - 3) with n_s the weighted size of its
component (the pre-increment reading of Eq. 3).
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction


def _adj(g):
    rp, ci = g.row_ptr, g.col_idx
    return [ci[rp[v]:rp[v + 1]].tolist() for v in range(g.n)]


def bfs(adj, s):
    """Level and exact path count from s (unreached: level -1, count 0)."""
    n = len(adj)
    lvl = [-1] * n
    sig = [0] * n
    lvl[s], sig[s] = 0, 1
    q = deque([s])
    while q:
        v = q.popleft()
        for w in adj[v]:
            if lvl[w] < 0:
                lvl[w] = lvl[v] + 1
                q.append(w)
            if lvl[w] == lvl[v] + 1:
                sig[w] += sig[v]
    return lvl, sig


def derive(adj, c, a_tree, b_tree):
    """Level and path count from the degree-2 vertex c, from its neighbours' trees."""
    (la, sa), (lb, sb) = a_tree, b_tree
    n = len(adj)
    lvl = [-1] * n
    sig = [0] * n
    for v in range(n):
        if v == c:
            lvl[v], sig[v] = 0, 1
        elif la[v] < 0 and lb[v] < 0:
            continue
        elif lb[v] < 0 or (la[v] >= 0 and la[v] < lb[v]):
            lvl[v], sig[v] = la[v] + 1, sa[v]
        elif la[v] < 0 or lb[v] < la[v]:
            lvl[v], sig[v] = lb[v] + 1, sb[v]
        else:
            lvl[v], sig[v] = la[v] + 1, sa[v] + sb[v]
    return lvl, sig


def dependencies(adj, s, lvl, sig, omega=None):
    """delta_s(v) for every v (Eq. 2; with leaf weights omega, Eq. 4's recursion), processing
    the DAG given by lvl / sig deepest first."""
    n = len(adj)
    om = omega if omega is not None else [0] * n
    order = sorted((v for v in range(n) if lvl[v] >= 0), key=lambda v: -lvl[v])
    delta = [Fraction(0)] * n
    for w in order:
        acc = Fraction(0)
        for v in adj[w]:
            if lvl[v] == lvl[w] + 1:
                acc += Fraction(1) / sig[v] * (1 + om[v] + delta[v])
        delta[w] = sig[w] * acc
    delta[s] = Fraction(0)
    return delta


def select_triples(g):
    """Degree-2 vertices c (in vertex order) with neighbours a, b such that no vertex is in
    two triples."""
    adj = _adj(g)
    used = [False] * g.n
    out = []
    for c in range(g.n):
        if len(adj[c]) != 2:
            continue
        a, b = adj[c]
        if used[c] or used[a] or used[b]:
            continue
        used[a] = used[b] = used[c] = True
        out.append((a, b, c))
    return out


def bc_with_deg2(g, prune: bool = False):
    """Exact BC (ordered pairs) over all sources, each selected degree-2 vertex's run taken
    from its neighbours' trees; returns (bc as Fractions, number of derived sources).
    With ``prune`` the 1-degree reduction comes first (one round, as the C oracle's
    prune_deg1) and both heuristics run on the residual graph."""
    omega = None
    if prune:
        from oracle import prune_deg1
        om, _, g = prune_deg1(g)
        omega = [int(x) for x in om]
    om = omega if omega is not None else [0] * g.n
    adj = _adj(g)
    bc = [Fraction(0)] * g.n
    triples = select_triples(g)
    derived = {c: (a, b) for a, b, c in triples}
    for s in range(g.n):
        if not adj[s] and om[s] == 0:
            continue
        if s in derived:
            a, b = derived[s]
            lvl, sig = derive(adj, s, bfs(adj, a), bfs(adj, b))
        else:
            lvl, sig = bfs(adj, s)
        d = dependencies(adj, s, lvl, sig, omega)
        for v in range(g.n):
            bc[v] += (om[s] + 1) * d[v]
        if om[s] > 0:
            n_s = sum(1 + om[v] for v in range(g.n) if lvl[v] >= 0)
            bc[s] += om[s] * (2 * n_s - om[s] - 3)
    return bc, len(triples)
