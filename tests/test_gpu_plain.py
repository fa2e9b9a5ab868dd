"""Parity of the per-source CUDA path (bc_sssp, bc_exact, bc_sources with
BC_PATH_PLAIN) against the CPU oracle, through the C ABI.  Each test runs both kernels of
the path: one CTA per source (the default on these small graphs) and the grid-wide kernel
(BC_PLAIN_GRID)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1602_00963_gb300 as bc
from bcgpu import assert_bc_close, assert_sssp_equal, upload

pytestmark = pytest.mark.gpu

PLAIN = bc.BC_PATH_PLAIN


@pytest.fixture(scope="module")
def ctx():
    c = bc.bc_ctx_create(0)
    yield c
    bc.bc_destroy(c)


@pytest.fixture(params=[0, bc.BC_PLAIN_GRID], ids=["cta", "grid"])
def kern(request):
    return request.param


SMALL = [
    gg.path_graph(2), gg.path_graph(17), gg.star_graph(9), gg.complete_graph(7),
    gg.cycle_graph(10), gg.cycle_graph(11), gg.complete_bipartite(3, 5), gg.hypercube(5),
    gg.random_tree(40, 1), gg.gnm(50, 20, 3), gg.gnm(60, 200, 4),
    gg.from_edge_list(8, [(0, 1), (2, 3), (3, 4)]),  # isolated vertices, K2, P3
]


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_small_exact(ctx, gi, kern):
    g = SMALL[gi]
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, PLAIN | kern)
    assert_bc_close(got, oracle.bc_exact(g), what=g.name)
    got, _ = bc.bc_exact(h, g.n, PLAIN | kern | bc.BC_PRUNE_DEG1)
    assert_bc_close(got, oracle.bc_exact(g), what=g.name + " pruned")
    bc.bc_destroy(h)


def test_sssp_rmat(ctx, kern):
    g = gg.rmat(12, 16, 1)
    h = upload(ctx, g)
    for s in [0, 5, 77, 1000, 4095]:
        assert_sssp_equal(bc.bc_sssp(h, g.n, s, kern), oracle.sssp(g, s), f"rmat12 s={s}")
    bc.bc_destroy(h)


def test_sssp_grid_overflow(ctx, kern):
    """48x48 open grid: counts pass 2^64 beyond distance ~67; sigma mod 2^64 and the
    overflow flags must match bit for bit."""
    g = gg.grid2d(48, 48)
    h = upload(ctx, g)
    for s in [0, 17 * 48 + 30, 48 * 48 - 1]:
        got = bc.bc_sssp(h, g.n, s, kern)
        want = oracle.sssp(g, s)
        assert want[2].any() or s != 0
        assert_sssp_equal(got, want, f"grid48 s={s}")
    bc.bc_destroy(h)


def test_sssp_ba_and_deleted_grid(ctx, kern):
    for g in [gg.ba_pref_attach(3000, 9), gg.grid2d(64, 64, seed=5, delete_frac=0.1)]:
        h = upload(ctx, g)
        rng = np.random.Generator(np.random.PCG64(1))
        for s in rng.choice(g.n, 6, replace=False):
            assert_sssp_equal(bc.bc_sssp(h, g.n, int(s), kern), oracle.sssp(g, int(s)), f"{g.name} s={s}")
        bc.bc_destroy(h)


def test_exact_rmat12_all_sources(ctx, kern):
    """R-MAT scale 12, edge factor 16, seed 1, all sources, no pruning, no batching."""
    g = gg.rmat(12, 16, 1)
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, PLAIN | kern)
    want = oracle.bc_exact(g, nthreads=8)
    assert_bc_close(got, want, what="rmat12 exact")
    assert st["sources"] == int((g.degrees() > 0).sum())
    assert st["teps_sources"] == st["sources"]
    assert st["edges"] == g.m
    bc.bc_destroy(h)


def test_exact_grid_extended_sigma(ctx, kern):
    """Grid with deletions: sigma overflows 2^64 and FP64; delta uses the extended-range
    sigma.  All sources of a
    40x40 grid (10% deleted, largest component); four sources of an open 120x120 grid (CTA
    state in global memory)."""
    g = gg.grid2d(40, 40, seed=5, delete_frac=0.1)
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, PLAIN | kern)
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what="grid40 exact")
    bc.bc_destroy(h)
    g = gg.grid2d(120, 120)
    h = upload(ctx, g)
    src = np.array([0, 119, 60 * 120 + 60, 120 * 120 - 1], np.int32)
    got, st = bc.bc_sources(h, g.n, src, PLAIN | kern)
    assert st["sigma_overflow_sources"] == 4
    assert st["sources"] == 4
    assert_bc_close(got, oracle.bc(g, src), what="grid120 sources")
    bc.bc_destroy(h)


def test_pruned_ba(ctx, kern):
    g = gg.ba_pref_attach(4000, 2)
    h = upload(ctx, g)
    want = oracle.bc_exact(g, nthreads=8)
    got_p, st_p = bc.bc_exact(h, g.n, PLAIN | kern | bc.BC_PRUNE_DEG1)
    got_u, st_u = bc.bc_exact(h, g.n, PLAIN | kern)
    assert_bc_close(got_p, want, what="ba pruned")
    assert_bc_close(got_u, want, what="ba unpruned")
    assert st_p["sources"] < st_u["sources"]
    assert st_p["teps_sources"] == st_u["teps_sources"]
    bc.bc_destroy(h)


def test_device_prune_matches_oracle(ctx):
    for g in [gg.ba_pref_attach(2000, 4), gg.rmat(10, 4, 2), SMALL[11]]:
        h = upload(ctx, g)
        om, rem, rrp, rci = bc.bc_prune(h, g.n, g.nnz)
        om0, rem0, res0 = oracle.prune_deg1(g)
        assert (om == om0).all() and (rem == rem0).all()
        assert (rrp == res0.row_ptr).all() and (rci == res0.col_idx).all()
        bc.bc_destroy(h)


def test_sources_multiset_and_device_ptrs(ctx, kern):
    torch = pytest.importorskip("torch")
    g = gg.rmat(10, 8, 3)
    h = upload(ctx, g)
    src = np.array([3, 3, 17, 500, 1023, 3], np.int32)
    want = oracle.bc(g, src)
    got, st = bc.bc_sources(h, g.n, src, PLAIN | kern)
    assert st["sources"] == 6
    assert_bc_close(got, want, what="multiset host")
    dsrc = torch.from_numpy(src).cuda()
    dout = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    bc.bc_sources(h, g.n, dsrc, PLAIN | kern, bc_out=dout)
    assert_bc_close(dout.cpu().numpy(), want, what="multiset device")
    bc.bc_destroy(h)


def test_invalid_inputs(ctx):
    bad = gg.Graph(3, np.array([0, 1, 1, 2], np.int32), np.array([1, 2], np.int32))  # not symmetric
    with pytest.raises(bc.BCError) as e:
        upload(ctx, bad)
    assert e.value.status == bc.BC_EINVAL
    loop = gg.Graph(2, np.array([0, 2, 2], np.int32), np.array([0, 1], np.int32))
    with pytest.raises(bc.BCError):
        upload(ctx, loop)
    g = gg.path_graph(5)
    h = upload(ctx, g)
    with pytest.raises(bc.BCError) as e:
        bc.bc_sources(h, g.n, np.array([7], np.int32), PLAIN)
    assert e.value.status == bc.BC_EINVAL
    with pytest.raises(bc.BCError) as e:
        bc.bc_sources(h, g.n, np.array([1], np.int32), PLAIN | bc.BC_PRUNE_DEG1)
    assert e.value.status == bc.BC_EINVAL
    bc.bc_destroy(h)
    # size limits of the int32 CSR, checked before any device work: nnz in [0, 2^31), even
    # (each edge stored twice), n >= 1
    rp, ci = np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32)
    for n, nnz in ((2, 2**31), (2, -2), (2, 3), (0, 0)):
        with pytest.raises(bc.BCError) as e:
            bc.bc_graph_create(ctx, n, rp, ci, nnz, 0)
        assert e.value.status == bc.BC_EINVAL, (n, nnz)


def test_wait_limit_timeout_then_recovery(ctx):
    """A zero device-wait limit makes the first grid barrier of the grid-wide kernel give
    up: the call returns BC_ETIMEDOUT (no hang, no fault) and the context stays usable.
    (The CTA kernel has no inter-CTA waits.)"""
    g = gg.rmat(10, 8, 5)
    h = upload(ctx, g)
    bc.bc_set_wait_limit_ms(ctx, 0)
    try:
        with pytest.raises(bc.BCError) as e:
            bc.bc_exact(h, g.n, PLAIN | bc.BC_PLAIN_GRID)
        assert e.value.status == bc.BC_ETIMEDOUT
        got, _ = bc.bc_exact(h, g.n, PLAIN)  # the CTA kernel is unaffected
        assert_bc_close(got, oracle.bc_exact(g), what="CTA kernel under a zero wait limit")
    finally:
        bc.bc_set_wait_limit_ms(ctx, 20000)
    got, _ = bc.bc_exact(h, g.n, PLAIN | bc.BC_PLAIN_GRID)
    assert_bc_close(got, oracle.bc_exact(g), what="after timeout")
    bc.bc_destroy(h)


DEG2_GRAPHS = [
    gg.cycle_graph(101),
    gg.from_edge_list(6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5)]),
    gg.subdivide_edges(gg.grid2d(30, 30, seed=1, delete_frac=0.1), 0.5, 2),
    gg.subdivide_edges(gg.grid2d(70, 70), 0.05, 7),  # counts past 2^64 (extended range)
    gg.subdivide_edges(gg.rmat(10, 4, 5), 0.3, 6),   # with isolated vertices and hubs
]


@pytest.mark.parametrize("gi", range(len(DEG2_GRAPHS)))
def test_deg2_heuristic_equals_plain(ctx, gi):
    """BC_DEG2 (Sec. 3.4.2): degree-2 vertices' runs derived from their neighbours' trees
    give the plain result."""
    g = DEG2_GRAPHS[gi]
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, PLAIN | bc.BC_DEG2)
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what=f"{g.name} deg2")
    assert st["sources"] == int((g.degrees() > 0).sum())
    bc.bc_destroy(h)


H3_GRAPHS = [
    gg.attach_leaves(gg.cycle_graph(60), 1.0, 8, max_leaves=1),  # degree 2 only after pruning
    gg.attach_leaves(gg.subdivide_edges(gg.grid2d(30, 30, seed=1, delete_frac=0.1), 0.5, 2), 0.3, 3),
    gg.attach_leaves(gg.subdivide_edges(gg.grid2d(70, 70), 0.05, 7), 0.2, 4),  # past 2^64
    gg.attach_leaves(gg.subdivide_edges(gg.rmat(10, 4, 5), 0.3, 6), 0.3, 9),
    gg.from_edge_list(9, [(0, 1), (0, 2), (0, 3), (4, 5), (5, 6), (6, 7), (7, 4), (7, 8)]),
]


@pytest.mark.parametrize("gi", range(len(H3_GRAPHS)))
def test_deg2_with_pruning_equals_plain(ctx, gi):
    """BC_DEG2 | BC_PRUNE_DEG1 (both heuristics, the paper's H3): triples on the residual
    graph, leaf weights in every run and the leaf term for derived sources."""
    g = H3_GRAPHS[gi]
    h = upload(ctx, g)
    got, st = bc.bc_exact(h, g.n, PLAIN | bc.BC_DEG2 | bc.BC_PRUNE_DEG1)
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what=f"{g.name} deg2 pruned")
    omega, removed, res = oracle.prune_deg1(g)
    assert st["sources"] == int(((removed == 0) & ((res.degrees() > 0) | (omega > 0))).sum())
    bc.bc_destroy(h)


NO_REUSE_GRAPHS = [gg.rmat(12, 16, 1), gg.grid2d(40, 40, seed=5, delete_frac=0.1), gg.path_graph(300)]


@pytest.mark.parametrize("gi", range(len(NO_REUSE_GRAPHS)))
def test_no_cd_reuse_same_result(ctx, gi):
    """BC_NO_CD_REUSE (the degree prefix CD scanned again per backward level, Sec. 3.1's
    reuse switched off): same BC as with the reuse (up to the atomics' order) and as the
    oracle, pruned and unpruned."""
    g = NO_REUSE_GRAPHS[gi]
    h = upload(ctx, g)
    GRID = PLAIN | bc.BC_PLAIN_GRID
    want = oracle.bc_exact(g, nthreads=8)
    for extra in (0, bc.BC_PRUNE_DEG1):
        a, _ = bc.bc_exact(h, g.n, GRID | extra)
        b, _ = bc.bc_exact(h, g.n, GRID | extra | bc.BC_NO_CD_REUSE)
        assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(a), 1.0)), (g.name, extra)
        assert_bc_close(b, want, what=f"{g.name} no CD reuse {extra}")
    bc.bc_destroy(h)


def test_no_cd_reuse_flag_rules(ctx):
    g = gg.cycle_graph(12)
    h = upload(ctx, g)
    for bad in (PLAIN, bc.BC_PATH_TILED, bc.BC_PLAIN_GRID, PLAIN | bc.BC_PLAIN_CTA,
                PLAIN | bc.BC_DEG2):
        with pytest.raises(bc.BCError) as e:
            bc.bc_exact(h, g.n, bad | bc.BC_NO_CD_REUSE)
        assert e.value.status == bc.BC_EINVAL
    bc.bc_destroy(h)


def test_deg2_flag_rules(ctx):
    g = gg.cycle_graph(12)
    h = upload(ctx, g)
    for bad in (bc.BC_PATH_TILED, bc.BC_PLAIN_GRID):
        with pytest.raises(bc.BCError) as e:
            bc.bc_exact(h, g.n, PLAIN | bc.BC_DEG2 | bad)
        assert e.value.status == bc.BC_EINVAL
    bc.bc_destroy(h)


def _edgeless(n):
    return gg.Graph(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32))


def test_degenerate_inputs(ctx):
    """An empty source list, isolated sources mixed with others (duplicates included), a
    graph without edges and a single vertex: BC is that of the oracle (zero where nothing
    is reached) and a lone root has depth 0 and one path, on every path and heuristic."""
    T = bc.BC_PATH_TILED
    paths = [PLAIN, PLAIN | bc.BC_PLAIN_GRID, T | bc.BC_TILE(32),
             T | bc.BC_TILE(64) | bc.BC_LOOP_LAUNCH, T | bc.BC_TILE(32) | bc.BC_LOOP_GRAPH]
    g = gg.from_edge_list(9, [(0, 1), (1, 2), (2, 3), (5, 6)])  # 4, 7, 8 isolated
    h = upload(ctx, g)
    src = np.array([4, 1, 7, 7, 5, 8, 1], np.int32)
    want = oracle.bc(g, src)
    for fl in paths:
        got, st = bc.bc_sources(h, g.n, np.zeros(0, np.int32), fl)
        assert not got.any() and st["sources"] == 0, fl
        got, st = bc.bc_sources(h, g.n, src, fl)
        assert st["sources"] == src.size, fl
        assert_bc_close(got, want, what=f"isolated sources {fl}")
    bc.bc_destroy(h)
    for n in (1, 5):
        g0 = _edgeless(n)
        h = upload(ctx, g0)
        for fl in (PLAIN, PLAIN | bc.BC_PLAIN_GRID, T | bc.BC_TILE(32), PLAIN | bc.BC_PRUNE_DEG1,
                   PLAIN | bc.BC_DEG2, PLAIN | bc.BC_DEG2 | bc.BC_PRUNE_DEG1):
            got, _ = bc.bc_exact(h, n, fl)
            assert not got.any(), (n, fl)
        for fl in (PLAIN, PLAIN | bc.BC_PLAIN_GRID):
            got, st = bc.bc_sources(h, n, np.array([n - 1, 0, n - 1], np.int32), fl)
            assert not got.any() and st["sources"] == 3, (n, fl)
            d, s, o = bc.bc_sssp(h, n, n - 1, fl)
            assert d.tolist() == [-1] * (n - 1) + [0], (n, fl)
            assert s.tolist() == [0] * (n - 1) + [1] and not o.any(), (n, fl)
        bc.bc_destroy(h)
