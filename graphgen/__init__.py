"""Seeded synthetic graph generators shared by the CUDA path's tests/bench and the oracle.

This module builds inputs only: it holds none of the betweenness-centrality arithmetic.
Every generator draws from ``numpy.random.Generator(PCG64(seed))`` and returns an
undirected, unweighted graph in symmetric CSR form with int32 indices, self-loops and
duplicate edges removed and every adjacency row sorted (the graph model of Sec. 2: m
unordered pairs (u, v) with u != v).

Workload shapes follow the paper's test graphs (Sec. 4.1): R-MAT with a, b, c, d =
0.57, 0.19, 0.19, 0.05, n = 2^SCALE and 2^SCALE * EF sampled edges; leaf-rich
preferential-attachment graphs as a stand-in for com-Youtube-like social graphs (53 %
degree-1 vertices, Table 1); 2-D grids with random edge deletions as a stand-in for the
long-diameter road networks (EF ~ 1.41, diameter ~ 800, Table 1).  The real data sets
are not used.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Graph", "csr_from_edges", "rmat", "ba_pref_attach", "grid2d", "erdos_renyi",
    "largest_component", "component_labels", "sample_sources", "from_edge_list",
    "path_graph", "star_graph", "complete_graph", "cycle_graph", "complete_bipartite",
    "hypercube", "random_tree", "gnm", "cached", "subdivide_edges",
]


@dataclass
class Graph:
    """Symmetric CSR: ``col_idx[row_ptr[v]:row_ptr[v+1]]`` are v's neighbours, sorted."""
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[2m]
    name: str = ""

    @property
    def m(self) -> int:
        """Undirected edges (unordered pairs)."""
        return int(self.col_idx.size // 2)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.size)

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def edges(self):
        """Unordered edges (u < v) as two int64 arrays."""
        deg = self.degrees()
        u = np.repeat(np.arange(self.n, dtype=np.int64), deg)
        v = self.col_idx.astype(np.int64)
        keep = u < v
        return u[keep], v[keep]


def _sorted_unique(key: np.ndarray) -> np.ndarray:
    key = np.sort(key)
    if key.size:
        keep = np.ones(key.size, dtype=bool)
        keep[1:] = key[1:] != key[:-1]
        key = key[keep]
    return key


def csr_from_edges(n: int, src, dst, name: str = "") -> Graph:
    """Symmetrise, drop self-loops and duplicates, sort rows, build int32 CSR."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    a = np.concatenate([src, dst])
    b = np.concatenate([dst, src])
    key = _sorted_unique(a * np.int64(n) + b)
    rows = key // n
    cols = key % n
    if key.size >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n, row_ptr.astype(np.int32), cols.astype(np.int32), name)


def from_edge_list(n: int, edges, name: str = "") -> Graph:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, e[:, 0], e[:, 1], name)


# --------------------------------------------------------------------------- R-MAT
def rmat(scale: int, ef: int, seed: int, a=0.57, b=0.19, c=0.19, permute: bool = True) -> Graph:
    """R-MAT (Chakrabarti et al.) as used in Sec. 4.1: n = 2^scale, ef * n samples.

    Each sample descends ``scale`` quadrant choices with probabilities a, b, c, d = 1-a-b-c
    (no noise).  Vertex labels are then shuffled by a seeded permutation so that the
    degree is not correlated with the id.
    """
    n = 1 << scale
    ne = ef * n
    rng = np.random.Generator(np.random.PCG64(seed))
    src = np.zeros(ne, dtype=np.int64)
    dst = np.zeros(ne, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for bit in range(scale):
        u = rng.random(ne)
        sbit = u >= ab                      # quadrants c, d
        dbit = ((u >= a) & (u < ab)) | (u >= abc)  # quadrants b, d
        src |= sbit.astype(np.int64) << bit
        dst |= dbit.astype(np.int64) << bit
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        src, dst = perm[src], perm[dst]
    return csr_from_edges(n, src, dst, f"rmat-s{scale}-ef{ef}-seed{seed}")


# ------------------------------------------------------------ preferential attachment
def ba_pref_attach(n: int, seed: int, p_single: float = 0.4, m_multi: int = 8) -> Graph:
    """Leaf-rich preferential-attachment graph.

    Starts from a triangle on vertices 0, 1, 2.  Each later vertex t draws m_t = 1 with
    probability ``p_single`` and ``m_multi`` otherwise, then links to m_t distinct
    existing vertices chosen proportionally to degree (uniform picks from the endpoint
    list; repeats are redrawn).  Connected by construction.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ms = np.where(rng.random(n) < p_single, 1, m_multi)
    total = 6 + 2 * int(ms[3:].sum())
    ends = np.empty(total, dtype=np.int64)
    ends[:6] = [0, 1, 1, 2, 2, 0]
    ne = 6
    src = [0, 1, 2]
    dst = [1, 2, 0]
    # draw uniform picks in blocks to keep the Python loop cheap
    block = rng.random(1 << 16)
    bi = 0
    for t in range(3, n):
        k = min(int(ms[t]), t)
        chosen = set()
        while len(chosen) < k:
            if bi == block.size:
                block = rng.random(1 << 16)
                bi = 0
            v = int(ends[int(block[bi] * ne)])
            bi += 1
            chosen.add(v)
        for v in sorted(chosen):
            src.append(t)
            dst.append(v)
            ends[ne] = t
            ends[ne + 1] = v
            ne += 2
    return csr_from_edges(n, np.array(src), np.array(dst), f"ba-n{n}-seed{seed}")


# ---------------------------------------------------------------------------- grid
def grid2d(w: int, h: int, seed: int | None = None, delete_frac: float = 0.0,
           lcc: bool = True) -> Graph:
    """w x h 4-neighbour open grid; vertex (x, y) has id y*w + x.

    If ``delete_frac`` > 0, exactly floor(E * delete_frac) edges chosen by a seeded
    shuffle are removed; with ``lcc`` the largest component is kept and relabelled in
    increasing original-id order.
    """
    ids = np.arange(w * h, dtype=np.int64).reshape(h, w)
    hs, hd = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    vs, vd = ids[:-1, :].ravel(), ids[1:, :].ravel()
    src = np.concatenate([hs, vs])
    dst = np.concatenate([hd, vd])
    name = f"grid-{w}x{h}"
    if delete_frac > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        e = src.size
        k = int(e * delete_frac)
        order = rng.permutation(e)
        keep = np.sort(order[k:])
        src, dst = src[keep], dst[keep]
        name += f"-del{delete_frac}-seed{seed}"
    g = csr_from_edges(w * h, src, dst, name)
    if lcc and delete_frac > 0:
        g, _ = largest_component(g)
        g.name = name + "-lcc"
    return g


def subdivide_edges(g: Graph, frac: float, seed: int) -> Graph:
    """Road-network shape: a seeded fraction of the edges (u, v) become paths u - x - v
    through a new degree-2 vertex x (ids n, n + 1, ... in edge order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    src, dst = g.edges()
    pick = rng.random(src.size) < frac
    k = int(pick.sum())
    x = g.n + np.arange(k, dtype=np.int64)
    s2 = np.concatenate([src[~pick], src[pick], x])
    d2 = np.concatenate([dst[~pick], x, dst[pick]])
    return csr_from_edges(g.n + k, s2, d2, f"{g.name}-sub{frac}-seed{seed}")


def attach_leaves(g: Graph, frac: float, seed: int, max_leaves: int = 3) -> Graph:
    """A seeded fraction of the vertices each gain 1..max_leaves pendant vertices (ids n,
    n + 1, ... in vertex order): leaf-rich inputs for the 1-degree reduction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pick = np.flatnonzero(rng.random(g.n) < frac)
    cnt = rng.integers(1, max_leaves + 1, pick.size)
    hub = np.repeat(pick, cnt).astype(np.int64)
    leaf = g.n + np.arange(hub.size, dtype=np.int64)
    src, dst = g.edges()
    return csr_from_edges(g.n + hub.size, np.concatenate([src, hub]), np.concatenate([dst, leaf]),
                          f"{g.name}-leaves{frac}-seed{seed}")


# ------------------------------------------------------------------- Erdos-Renyi
def erdos_renyi(n: int, m: int, seed: int) -> Graph:
    """G(n, M): exactly M distinct undirected edges drawn uniformly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = int((m - keys.size) * 1.1) + 16
        u = rng.integers(0, n, need)
        v = rng.integers(0, n, need)
        ok = u != v
        lo = np.minimum(u[ok], v[ok])
        hi = np.maximum(u[ok], v[ok])
        new = lo * n + hi
        keys = np.concatenate([keys, new])
        order = np.argsort(keys, kind="stable")
        sk = keys[order]
        first = np.ones(sk.size, dtype=bool)
        first[1:] = sk[1:] != sk[:-1]
        keys = keys[np.sort(order[first])]
    keys = keys[:m]
    return csr_from_edges(n, keys // n, keys % n, f"er-n{n}-m{m}-seed{seed}")


def gnm(n: int, m: int, seed: int) -> Graph:
    """Small G(n, M) without the retry loop's cost (tests); m is capped at C(n,2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.int64).reshape(-1, 2)
    m = min(m, len(pairs))
    pick = rng.choice(len(pairs), size=m, replace=False) if m else np.zeros(0, np.int64)
    e = pairs[pick]
    return csr_from_edges(n, e[:, 0], e[:, 1], f"gnm-{n}-{m}-{seed}")


# ------------------------------------------------------------------ small families
def path_graph(n: int) -> Graph:
    return csr_from_edges(n, np.arange(n - 1), np.arange(1, n), f"path-{n}")


def star_graph(n: int) -> Graph:
    """Centre 0, leaves 1..n-1."""
    return csr_from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), f"star-{n}")


def complete_graph(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return csr_from_edges(n, i, j, f"complete-{n}")


def cycle_graph(n: int) -> Graph:
    a = np.arange(n)
    return csr_from_edges(n, a, (a + 1) % n, f"cycle-{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    """Side A = 0..a-1, side B = a..a+b-1."""
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return csr_from_edges(a + b, i.ravel(), j.ravel(), f"kab-{a}-{b}")


def hypercube(k: int) -> Graph:
    n = 1 << k
    v = np.arange(n, dtype=np.int64)
    src = np.concatenate([v for _ in range(k)])
    dst = np.concatenate([v ^ (1 << i) for i in range(k)])
    return csr_from_edges(n, src, dst, f"hypercube-{k}")


def random_tree(n: int, seed: int) -> Graph:
    """Uniform random recursive tree: vertex t attaches to a uniform earlier vertex."""
    rng = np.random.Generator(np.random.PCG64(seed))
    par = np.array([rng.integers(0, t) for t in range(1, n)], dtype=np.int64)
    return csr_from_edges(n, np.arange(1, n), par, f"tree-{n}-{seed}")


# -------------------------------------------------------------- components / sources
def component_labels(g: Graph) -> np.ndarray:
    """Connected-component label per vertex (scipy's union of BFS trees)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    mat = csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    _, lab = connected_components(mat, directed=False)
    return lab


def largest_component(g: Graph):
    """Induced subgraph on the largest component, ids relabelled in increasing order.
    Returns (graph, original_ids)."""
    lab = component_labels(g)
    big = np.bincount(lab).argmax()
    keep = np.flatnonzero(lab == big).astype(np.int64)
    newid = np.full(g.n, -1, dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    u, v = g.edges()
    ok = (newid[u] >= 0) & (newid[v] >= 0)
    sub = csr_from_edges(keep.size, newid[u[ok]], newid[v[ok]], g.name + "-lcc")
    return sub, keep


def sample_sources(g: Graph, k: int, seed: int, from_lcc: bool = True) -> np.ndarray:
    """k distinct sources drawn uniformly (seeded) from the largest component, or from
    all non-isolated vertices when ``from_lcc`` is False (Sec. 4.1 footnote: sources are
    drawn among non-isolated vertices)."""
    if from_lcc:
        lab = component_labels(g)
        pool = np.flatnonzero(lab == np.bincount(lab).argmax())
    else:
        pool = np.flatnonzero(g.degrees() > 0)
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(k, pool.size)
    return np.sort(rng.choice(pool, size=k, replace=False)).astype(np.int32)


# ------------------------------------------------------------------- disk cache
def cached(tag: str, fn, *args, **kw) -> Graph:
    """Memoise an expensive generator call on disk (``$BC_GRAPH_CACHE`` or /tmp)."""
    d = os.environ.get("BC_GRAPH_CACHE", "/tmp/bc_graph_cache")
    key = hashlib.sha1(repr((tag, args, sorted(kw.items()))).encode()).hexdigest()[:16]
    path = os.path.join(d, f"{tag}-{key}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(int(z["n"]), z["row_ptr"], z["col_idx"], str(z["name"]))
    g = fn(*args, **kw)
    os.makedirs(d, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col_idx=g.col_idx, name=g.name)
    os.replace(tmp, path)
    return g
