"""Parity of the multi-source tile path (bc_tile_sssp, and bc_exact / bc_sources with
BC_PATH_TILED) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1602_00963_gb300 as bc
from bcgpu import assert_bc_close, assert_sssp_equal, upload

pytestmark = pytest.mark.gpu

TILED = bc.BC_PATH_TILED
MODES = {"persistent": 0, "launch": bc.BC_LOOP_LAUNCH, "graph": bc.BC_LOOP_GRAPH}


@pytest.fixture(scope="module")
def ctx():
    c = bc.bc_ctx_create(0)
    yield c
    bc.bc_destroy(c)


def hub_graph():
    """A hub of degree 3000 (pulled by a whole CTA), leaves, a second hub and a sparse
    random part linking them, so hubs are candidates in both sweep directions."""
    rng = np.random.Generator(np.random.PCG64(11))
    n = 6000
    e = [(0, i) for i in range(1, 3001)] + [(3001, i) for i in range(2500, 5200)]
    u = rng.integers(0, n, 6000)
    v = rng.integers(0, n, 6000)
    e += list(zip(u.tolist(), v.tolist()))
    return gg.from_edge_list(n, e)


@pytest.mark.parametrize("T", [32, 64, 128, 256])
def test_tile_sssp_rmat(ctx, T):
    g = gg.rmat(12, 16, 1)
    h = upload(ctx, g)
    src = gg.sample_sources(g, T - 3, seed=T)  # ragged tile: T - 3 lanes used
    d, s, o = bc.bc_tile_sssp(h, g.n, src, TILED | bc.BC_TILE(T))
    for i in range(0, len(src), 7):
        assert_sssp_equal((d[i], s[i], o[i]), oracle.sssp(g, int(src[i])), f"rmat12 T={T} lane {i}")
    bc.bc_destroy(h)


@pytest.mark.parametrize("mode", list(MODES))
def test_tile_sssp_grid_overflow(ctx, mode):
    g = gg.grid2d(48, 48)
    h = upload(ctx, g)
    src = np.array([0, 100, 17 * 48 + 30, 48 * 48 - 1, 1200], np.int32)
    d, s, o = bc.bc_tile_sssp(h, g.n, src, TILED | bc.BC_TILE(32) | MODES[mode])
    for i, x in enumerate(src):
        assert_sssp_equal((d[i], s[i], o[i]), oracle.sssp(g, int(x)), f"grid48 {mode} src {x}")
    bc.bc_destroy(h)


def test_tile_sssp_hubs(ctx):
    g = hub_graph()
    h = upload(ctx, g)
    src = np.array([0, 1, 3001, 4000, 5999, 17], np.int32)
    for T in (32, 256):
        d, s, o = bc.bc_tile_sssp(h, g.n, src, TILED | bc.BC_TILE(T))
        for i, x in enumerate(src):
            assert_sssp_equal((d[i], s[i], o[i]), oracle.sssp(g, int(x)), f"hub T={T} src {x}")
    bc.bc_destroy(h)


SMALL = [gg.path_graph(9), gg.star_graph(40), gg.cycle_graph(33), gg.hypercube(6),
         gg.complete_bipartite(5, 7), gg.random_tree(70, 3), gg.gnm(90, 60, 5),
         gg.from_edge_list(8, [(0, 1), (2, 3), (3, 4)])]


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_tile_exact_small(ctx, gi):
    g = SMALL[gi]
    h = upload(ctx, g)
    want = oracle.bc_exact(g)
    for T in (32, 64):
        got, st = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(T))
        assert_bc_close(got, want, what=f"{g.name} T={T}")
        got, _ = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(T) | bc.BC_PRUNE_DEG1)
        assert_bc_close(got, want, what=f"{g.name} T={T} pruned")
    bc.bc_destroy(h)


@pytest.mark.parametrize("T", [32, 64, 128, 256])
def test_tile_exact_rmat12(ctx, T):
    """R-MAT scale 12, edge factor 16, seed 1, all sources, tiles of T."""
    g = gg.rmat(12, 16, 1)
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(T))
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what=f"rmat12 T={T}")
    assert st["tile_width"] == T
    bc.bc_destroy(h)


@pytest.mark.parametrize("mode", list(MODES))
def test_tile_exact_grid_extended(ctx, mode):
    """Open 64 x 64 grid: sigma passes 2^64 (corner to corner ~2^124); the tile reruns in
    extended mode.  Plus a deleted-edge grid (largest component).  All three loop modes."""
    g = gg.grid2d(64, 64)
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(64) | MODES[mode])
    assert st["sigma_overflow_sources"] > 0
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what=f"grid64 {mode}")
    bc.bc_destroy(h)
    g = gg.grid2d(40, 40, seed=5, delete_frac=0.1)
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(32) | MODES[mode])
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what=f"grid40 deleted {mode}")
    bc.bc_destroy(h)


def test_tile_big_grid_sources(ctx):
    g = gg.grid2d(160, 160, seed=7, delete_frac=0.1)
    h = upload(ctx, g)
    src = gg.sample_sources(g, 40, seed=6)
    want = oracle.bc(g, src, nthreads=8)
    for mode in MODES.values():
        got, st = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(32) | mode)
        assert_bc_close(got, want, what=f"grid160 mode {mode}")
    bc.bc_destroy(h)


def test_tile_pruned_ba(ctx):
    g = gg.ba_pref_attach(5000, 2)
    h = upload(ctx, g)
    want = oracle.bc_exact(g, nthreads=8)
    got, _ = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(128) | bc.BC_PRUNE_DEG1)
    assert_bc_close(got, want, what="ba pruned T=128")
    got, _ = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(128))
    assert_bc_close(got, want, what="ba unpruned T=128")
    bc.bc_destroy(h)


def test_tile_hubs_exact(ctx):
    g = hub_graph()
    h = upload(ctx, g)
    src = np.arange(0, g.n, 37, dtype=np.int32)
    want = oracle.bc(g, src, nthreads=8)
    for T in (32, 256):
        for mode in MODES.values():
            got, _ = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(T) | mode)
            assert_bc_close(got, want, what=f"hubs T={T} mode={mode}")
    bc.bc_destroy(h)


def hub_chunk_graph():
    """Hubs of degree 10,000 and 9,000 (three backward chunks each) plus a sparse part."""
    rng = np.random.Generator(np.random.PCG64(12))
    n = 14000
    e = [(0, i) for i in range(1, 10001)] + [(10001, i) for i in range(4000, 13001)]
    u = rng.integers(0, n, 9000)
    v = rng.integers(0, n, 9000)
    e += list(zip(u.tolist(), v.tolist()))
    return gg.from_edge_list(n, e)


def test_tile_hub_chunks_exact(ctx):
    """Hubs of degree 10,000 and 9,000 (three chunks each, spread over CTAs, partial sums
    combined by the last chunk) plus a sparse part, at both tile widths and loop modes."""
    g = hub_chunk_graph()
    h = upload(ctx, g)
    src = np.arange(3, g.n, 211, dtype=np.int32)
    want = oracle.bc(g, src, nthreads=8)
    for T in (64, 256):
        for mode in (0, bc.BC_LOOP_LAUNCH):
            got, _ = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(T) | mode)
            assert_bc_close(got, want, what=f"hub chunks T={T} mode={mode}")
    bc.bc_destroy(h)


def test_tile_duplicates_and_plain_agree(ctx):
    g = gg.rmat(11, 8, 4)
    h = upload(ctx, g)
    src = np.array([5, 5, 5, 900, 17, 900] * 11, np.int32)
    want = oracle.bc(g, src)
    got_t, st = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(32))
    got_p, _ = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN)
    assert st["sources"] == src.size
    assert_bc_close(got_t, want, what="duplicates tiled")
    assert_bc_close(got_p, want, what="duplicates plain")
    bc.bc_destroy(h)


def test_tile_long_path_capacity_regrowth(ctx):
    """A path of 3000 vertices with 256 spread sources: every vertex sits at up to 256
    different levels of the tile, far more active-list entries than the initial
    capacity, so the tile is rerun with a larger list."""
    g = gg.path_graph(3000)
    h = upload(ctx, g)
    src = np.linspace(0, 2999, 256).astype(np.int32)
    got, st = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(256))
    assert_bc_close(got, oracle.bc(g, src), what="path3000 T=256")
    d, s, o = bc.bc_tile_sssp(h, g.n, src[:5], TILED | bc.BC_TILE(32))
    for i in range(5):
        assert_sssp_equal((d[i], s[i], o[i]), oracle.sssp(g, int(src[i])), "path sssp")
    bc.bc_destroy(h)


def test_tile_timeout_then_recovery(ctx):
    g = gg.rmat(10, 8, 9)
    h = upload(ctx, g)
    bc.bc_set_wait_limit_ms(ctx, 0)
    try:
        with pytest.raises(bc.BCError) as e:
            bc.bc_exact(h, g.n, TILED | bc.BC_TILE(32))
        assert e.value.status == bc.BC_ETIMEDOUT
    finally:
        bc.bc_set_wait_limit_ms(ctx, 20000)
    got, _ = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(32))
    assert_bc_close(got, oracle.bc_exact(g), what="after timeout")
    bc.bc_destroy(h)


def test_repeat_runs(ctx):
    """Repeated calls give identical depth, sigma and overflow flags on every path and
    bit-identical BC: every path sums in a fixed order (the tile path adds an entry's hits
    in edge order wherever the walk's 32-edge steps fall; the per-CTA kernel picks a
    vertex's thread or warp path by its degree alone; the grid-wide kernel adds fixed-point
    integers), with or without BC_DETERMINISTIC."""
    g = gg.rmat(12, 16, 1)
    h = upload(ctx, g)
    src = gg.sample_sources(g, 200, seed=3)
    for fl in (TILED | bc.BC_TILE(64), TILED | bc.BC_TILE(256) | bc.BC_LOOP_GRAPH,
               bc.BC_PATH_PLAIN | bc.BC_PLAIN_GRID):
        a, _ = bc.bc_sources(h, g.n, src, fl)
        b, _ = bc.bc_sources(h, g.n, src, fl)
        assert np.array_equal(a, b), fl
    d0 = bc.bc_tile_sssp(h, g.n, src[:40], TILED | bc.BC_TILE(64))
    d1 = bc.bc_tile_sssp(h, g.n, src[:40], TILED | bc.BC_TILE(64))
    assert all(np.array_equal(x, y) for x, y in zip(d0, d1))
    for fl in (0, bc.BC_PLAIN_GRID):
        s0 = bc.bc_sssp(h, g.n, int(src[0]), fl)
        s1 = bc.bc_sssp(h, g.n, int(src[0]), fl)
        assert all(np.array_equal(x, y) for x, y in zip(s0, s1))
    bc.bc_destroy(h)
    gh = hub_chunk_graph()
    h = upload(ctx, gh)
    src = np.arange(0, gh.n, 53, dtype=np.int32)
    a, _ = bc.bc_sources(h, gh.n, src, TILED | bc.BC_TILE(64))
    b, _ = bc.bc_sources(h, gh.n, src, TILED | bc.BC_TILE(64))
    assert np.array_equal(a, b)
    bc.bc_destroy(h)
    for gc in (gg.grid2d(48, 48), gg.gnm(3000, 9000, 4), gg.rmat(12, 16, 3)):  # past 2^64; sparse; hubs
        h = upload(ctx, gc)
        a, _ = bc.bc_exact(h, gc.n, bc.BC_PATH_PLAIN)
        b, _ = bc.bc_exact(h, gc.n, bc.BC_PATH_PLAIN)
        assert np.array_equal(a, b), gc.name
        bc.bc_destroy(h)


def test_locality_order_same_sum(ctx):
    """A call of at least four tiles runs its sources grouped by locality (distances to
    seeded landmarks); the result is the same sum as in the given order (BC_KEEP_ORDER) and
    the oracle's, with repeated and isolated sources in the list, on the graph and its
    residual (pruned) form."""
    g = gg.rmat(12, 16, 5)
    h = upload(ctx, g)
    src = np.concatenate([gg.sample_sources(g, 900, seed=2), [7, 7, 7],
                          np.flatnonzero(g.degrees() == 0)[:3]]).astype(np.int32)
    want = oracle.bc(g, src)
    for T in (32, 64):
        got, _ = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(T))
        kept, _ = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(T) | bc.BC_KEEP_ORDER)
        assert_bc_close(got, want, what=f"ordered T={T}")
        assert_bc_close(kept, want, what=f"given order T={T}")
        again, _ = bc.bc_sources(h, g.n, src, TILED | bc.BC_TILE(T))
        assert np.array_equal(got, again)
    pruned, _ = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(32) | bc.BC_PRUNE_DEG1)
    assert_bc_close(pruned, oracle.bc_exact(g), what="pruned, ordered")
    bc.bc_destroy(h)
