"""The oracle's pins catch plausible mistakes: each case compiles a copy of oracle/brandes.c
with one planted error (on the CPU, in a temporary directory) and checks that the pins that
do not come from the oracle reject it, while the unmodified source passes them.

Pins used (none computed by the oracle): exact rational BC of Eq. 1 by the Bellman form of
oracle/brute.py on small graphs with leaves, cycles and a K2 component, with and without
the 1-degree reduction; exact shortest-path counts C(dx + dy, dx) from a grid corner, modulo
2^64 with the overflow flag, and the Manhattan depths; and the 1-degree reduction's output
on a K2 beside a star, written out by hand from Alg. 6 (a leaf goes only when its neighbour
has degree >= 2, so the K2 stays, while BC alone cannot tell: a K2's BC is 0 either way)."""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import brute

SRC = os.path.join(os.path.dirname(oracle.__file__), "brandes.c")

# (name, text in brandes.c, replacement): one mistake each
MUTANTS = [
    ("level off by one", "w->depth[x] = dv + 1;", "w->depth[x] = dv + 2;"),
    ("predecessor test", "if (w->depth[x] == dv + 1) {", "if (w->depth[x] == dv) {"),
    ("sigma counts parents", "w->sigma[x] = before + w->sigma[v];", "w->sigma[x] = before + 1;"),
    ("no carry detection", "if (w->sigma[x] < before) w->ovf[x] = 1;", ""),
    ("no overflow propagation", "w->ovf[x] |= w->ovf[v];", ""),
    ("long sigma counts parents", "w->sigmaL[x] += w->sigmaL[v];", "w->sigmaL[x] += 1.0L;"),
    ("dropped 1 in the dependency", "(1.0L + w->delta[x] +", "(w->delta[x] +"),
    ("dropped sigma factor", "w->delta[v] += w->sigmaL[v] * coef;", "w->delta[v] += coef;"),
    ("successors for predecessors", "if (w->depth[v] == dx - 1)", "if (w->depth[v] == dx + 1)"),
    ("source counted", "if (x != s) bc[x] += ws * w->delta[x];", "bc[x] += ws * w->delta[x];"),
    ("dropped omega in Eq. 4", "(omega ? (long double)omega[x] : 0.0L)", "0.0L"),
    ("source weight without +1", "(long double)omega[s] + 1.0L : 1.0L", "(long double)omega[s] : 1.0L"),
    ("post-increment reading of Eq. 3", "om * (2.0L * ns - om - 3.0L)", "om * (2.0L * ns - om - 5.0L)"),
    ("n_s without leaves", "ns += 1.0L + (long double)omega[w->queue[i]];", "ns += 1.0L;"),
    ("K2 both ends removed", "if (row_ptr[v + 1] - row_ptr[v] >= 2) {", "if (row_ptr[v + 1] - row_ptr[v] >= 1) {"),
    ("omega as a flag", "omega[v] += 1;", "omega[v] = 1;"),
    ("arcs to removed leaves kept", "if (!removed[v]) res_col_idx[out++] = v;", "res_col_idx[out++] = v;"),
]

GRAPHS = [
    gg.attach_leaves(gg.cycle_graph(7), 0.6, 1),
    gg.from_edge_list(9, [(0, 1), (0, 2), (0, 3), (4, 5), (5, 6), (6, 7), (7, 4), (7, 8)]),
    gg.from_edge_list(6, [(0, 1), (2, 3), (3, 4), (3, 5)]),  # K2 beside a star
    gg.random_tree(12, 4),
    gg.attach_leaves(gg.gnm(12, 18, 3), 0.4, 5),
]
EXACT = [[float(x) for x in brute.bc_bellman(g)] for g in GRAPHS]
GRID = gg.grid2d(40, 40)


def pins_hold() -> bool:
    for g, want in zip(GRAPHS, EXACT):
        w = np.array(want)
        for prune in (False, True):
            got = oracle.bc_exact(g, prune=prune)
            if not np.all(np.abs(got - w) <= 1e-9 * np.maximum(np.abs(w), 1.0)):
                return False
    omega, removed, res = oracle.prune_deg1(GRAPHS[2])  # K2 {0, 1}; star 3 - {2, 4, 5}
    if omega.tolist() != [0, 0, 0, 3, 0, 0] or removed.tolist() != [0, 0, 1, 0, 1, 1]:
        return False
    if res.row_ptr.tolist() != [0, 1, 2, 2, 2, 2, 2] or res.col_idx.tolist() != [1, 0]:
        return False
    d, s, o = oracle.sssp(GRID, 0)
    for v in range(GRID.n):
        x, y = v % 40, v // 40
        c = math.comb(x + y, x)
        if d[v] != x + y or int(s[v]) != c % 2**64 or bool(o[v]) != (c >= 2**64):
            return False
    return True


def compiled(text: str, tmp: str, tag: str):
    path = os.path.join(tmp, f"brandes_{tag}.c")
    with open(path, "w") as f:
        f.write(text)
    so = os.path.join(tmp, f"liboracle_{tag}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", so, path])
    return oracle.load_from(so)


@pytest.fixture()
def swap_lib(monkeypatch):
    def use(lib):
        monkeypatch.setattr(oracle, "_lib", lib)
    return use


def test_unmodified_source_passes(swap_lib):
    with tempfile.TemporaryDirectory() as tmp:
        swap_lib(compiled(open(SRC).read(), tmp, "orig"))
        assert pins_hold()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(swap_lib, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    with tempfile.TemporaryDirectory() as tmp:
        swap_lib(compiled(src.replace(old, new), tmp, "mut"))
        assert not pins_hold(), f"the pins accept the mutant '{name}'"


# ---- the 2-degree oracle (oracle/deg2.py): mutated copies run as separate modules
DEG2_SRC = os.path.join(os.path.dirname(oracle.__file__), "deg2.py")
DEG2_MUTANTS = [
    ("tie drops b's paths", "lvl[v], sig[v] = la[v] + 1, sa[v] + sb[v]", "lvl[v], sig[v] = la[v] + 1, sa[v]"),
    ("derived level off by one", "lvl[v], sig[v] = la[v] + 1, sa[v]\n", "lvl[v], sig[v] = la[v], sa[v]\n"),
    ("tie goes to a", "elif lb[v] < 0 or (la[v] >= 0 and la[v] < lb[v]):", "elif lb[v] < 0 or (la[v] >= 0 and la[v] <= lb[v]):"),
    ("dropped omega in the recursion", "(1 + om[v] + delta[v])", "(1 + delta[v])"),
    ("source's own dependency kept", "    delta[s] = Fraction(0)\n", "\n"),
    ("source weight without +1", "bc[v] += (om[s] + 1) * d[v]", "bc[v] += d[v]"),
    ("post-increment reading of Eq. 3", "om[s] * (2 * n_s - om[s] - 3)", "om[s] * (2 * n_s - om[s] - 5)"),
    ("triples share vertices", "if used[c] or used[a] or used[b]:", "if used[c]:"),
]
DEG2_GRAPHS = [gg.cycle_graph(9), gg.subdivide_edges(gg.grid2d(4, 4, seed=1, delete_frac=0.1), 0.5, 2),
               gg.attach_leaves(gg.cycle_graph(10), 1.0, 8, max_leaves=1),
               gg.attach_leaves(gg.subdivide_edges(gg.gnm(10, 16, 4), 0.4, 5), 0.4, 6)]
DEG2_EXACT = [brute.bc_bellman(g) for g in DEG2_GRAPHS]


def deg2_module(text: str):
    import types
    m = types.ModuleType("deg2_variant")
    exec(compile(text, DEG2_SRC, "exec"), m.__dict__)
    return m


def deg2_pins_hold(m) -> bool:
    for g, want in zip(DEG2_GRAPHS, DEG2_EXACT):
        for prune in (False, True):
            got, _ = m.bc_with_deg2(g, prune=prune)
            if list(got) != list(want):
                return False
    tri = m.select_triples(gg.subdivide_edges(gg.grid2d(6, 6, seed=3, delete_frac=0.1), 0.6, 4))
    seen = [v for t in tri for v in t]
    return len(seen) == len(set(seen))


def test_deg2_unmodified_passes():
    assert deg2_pins_hold(deg2_module(open(DEG2_SRC).read()))


@pytest.mark.parametrize("name,old,new", DEG2_MUTANTS, ids=[m[0] for m in DEG2_MUTANTS])
def test_deg2_planted_mistake_is_caught(name, old, new):
    src = open(DEG2_SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    assert not deg2_pins_hold(deg2_module(src.replace(old, new))), f"the pins accept '{name}'"
