"""BC_DETERMINISTIC: two calls with the same graph, sources and flags give bit-identical BC
(np.array_equal), on every path: the tile path at T = 64 and T = 256 (persistent kernel and
CUDA-graph level loop), the per-CTA per-source kernel and the grid-wide per-source kernel;
and each result matches the oracle within the 1e-9 tolerance.  The graphs: R-MAT scale 12
with every source (short diameter, dense levels), hubs of 10,000 and 9,000 edges (backward
work split into chunks over CTAs), and the undeleted 64 x 64 grid (long diameter, path
counts past 2^64, so the extended range is used)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1602_00963_gb300 as bc
from bcgpu import assert_bc_close, upload

pytestmark = pytest.mark.gpu

D = bc.BC_DETERMINISTIC
PATHS = {
    "tile64": bc.BC_PATH_TILED | bc.BC_TILE(64),
    "tile256-graph": bc.BC_PATH_TILED | bc.BC_TILE(256) | bc.BC_LOOP_GRAPH,
    "per-cta": bc.BC_PATH_PLAIN | bc.BC_PLAIN_CTA,
    "grid-wide": bc.BC_PATH_PLAIN | bc.BC_PLAIN_GRID,
}


def hub_chunk_graph():
    rng = np.random.Generator(np.random.PCG64(12))
    n = 14000
    e = [(0, i) for i in range(1, 10001)] + [(10001, i) for i in range(4000, 13001)]
    u = rng.integers(0, n, 9000)
    v = rng.integers(0, n, 9000)
    e += list(zip(u.tolist(), v.tolist()))
    return gg.from_edge_list(n, e)


GRAPHS = {
    "rmat12-all": lambda: (gg.rmat(12, 16, 1), None),
    "hub-chunks": lambda: (hub_chunk_graph(), np.arange(3, 14000, 97, dtype=np.int32)),
    "grid64": lambda: (gg.grid2d(64, 64), None),
}


@pytest.fixture(scope="module")
def ctx():
    c = bc.bc_ctx_create(0)
    yield c
    bc.bc_destroy(c)


@pytest.mark.parametrize("gname", list(GRAPHS))
def test_deterministic_repeats_bit_for_bit(ctx, gname):
    g, src = GRAPHS[gname]()
    h = upload(ctx, g)
    want = oracle.bc_exact(g) if src is None else oracle.bc(g, src)
    for pname, fl in PATHS.items():
        runs = []
        for _ in range(2):
            if src is None:
                got, _ = bc.bc_exact(h, g.n, fl | D)
            else:
                got, _ = bc.bc_sources(h, g.n, src, fl | D)
            runs.append(got.copy())
        assert np.array_equal(runs[0], runs[1]), f"{gname} {pname}: repeated call differs"
        assert_bc_close(runs[0], want, what=f"{gname} {pname}")
    bc.bc_destroy(h)


def test_deterministic_ignores_the_tuned_choice(ctx):
    """With the flag, a call without a path flag runs the default per-source path even after
    bc_autotune cached another configuration on the graph."""
    g = gg.rmat(12, 16, 2)
    h = upload(ctx, g)
    src = gg.sample_sources(g, 300, seed=5)
    want, _ = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN | D)
    bc.bc_autotune(h, 128, 3)
    got, st = bc.bc_sources(h, g.n, src, D)
    assert st["tile_width"] == 1  # the per-source path
    assert np.array_equal(got, want)
    bc.bc_destroy(h)
