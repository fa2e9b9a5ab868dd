"""Parity at the benchmark sizes, in the launch configurations bench.py times.

* R-MAT scale 20, edge factor 16, seed 3, with the bench's sources (largest component,
  seed 4): the autotuned tile width and tile width 256 on the persistent tile kernel, and
  the per-source path, against the oracle on the same sources, BC per vertex (FP64,
  1e-9 relative); depth and sigma bit-exact on sampled lanes of a full tile.
* Grid 1024 x 1024 with 10% of its edges deleted (seed 5, largest component), sources
  seed 6: the three level-loop modes (persistent, per-level launches, CUDA graph) with
  the extended-range sigma active (sigma reaches ~2^1700 on this graph).
* Barabasi-Albert-style graph, n = 262144 (seed 2): all sources pruned (1-degree removal,
  Eq. 3 / Eq. 4) equal to all sources unpruned; unpruned on sampled sources against the
  oracle; depth and sigma bit-exact from two sources.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1602_00963_gb300 as bc
from bcgpu import assert_bc_close, assert_sssp_equal, upload

pytestmark = pytest.mark.gpu

TILED = bc.BC_PATH_TILED


@pytest.fixture(scope="module")
def ctx():
    c = bc.bc_ctx_create(0)
    yield c
    bc.bc_destroy(c)


@pytest.fixture(scope="module")
def rmat20(ctx):
    g = gg.cached("rmat", gg.rmat, 20, 16, 3)
    src = gg.sample_sources(g, 4096, seed=4)
    h = upload(ctx, g)
    yield g, src, h
    bc.bc_destroy(h)


def test_rmat20_tuned_tile_vs_oracle(rmat20):
    g, src, h = rmat20
    tune = bc.bc_autotune(h, 0, 7)
    T = tune["tile_width"] or 64
    want = oracle.bc(g, src[:T])
    got, st = bc.bc_sources(h, g.n, src[:T], TILED | bc.BC_TILE(T))
    assert st["tile_width"] == T and st["sources"] == T
    assert_bc_close(got, want, what=f"rmat20 tuned T={T}")


def test_rmat20_wide_ragged_tile_vs_oracle(rmat20):
    """T = 256 with 40 sources (a ragged tile: 216 idle lanes)."""
    g, src, h = rmat20
    s = src[64:104]
    got, _ = bc.bc_sources(h, g.n, s, TILED | bc.BC_TILE(256))
    assert_bc_close(got, oracle.bc(g, s), what="rmat20 T=256 ragged")


def test_rmat20_tile_sssp_lanes_bit_exact(rmat20):
    g, src, h = rmat20
    s = src[:40]
    d, sg, o = bc.bc_tile_sssp(h, g.n, s, TILED | bc.BC_TILE(64))
    for i in (0, 17, 39):
        assert_sssp_equal((d[i], sg[i], o[i]), oracle.sssp(g, int(s[i])), f"rmat20 lane {i}")


def test_rmat20_per_source_path_vs_oracle(rmat20):
    g, src, h = rmat20
    s = src[:12]
    got, _ = bc.bc_sources(h, g.n, s, bc.BC_PATH_PLAIN)
    assert_bc_close(got, oracle.bc(g, s), what="rmat20 per-source path")
    d, sg, o = bc.bc_sssp(h, g.n, int(s[0]))
    assert_sssp_equal((d, sg, o), oracle.sssp(g, int(s[0])), "rmat20 bc_sssp")


def test_grid1024_loop_modes_vs_oracle(ctx):
    g = gg.cached("grid", gg.grid2d, 1024, 1024, 5, 0.1)
    src = gg.sample_sources(g, 1024, seed=6)
    h = upload(ctx, g)
    s = src[:32]
    want = oracle.bc(g, s)
    modes = {"persistent": 0, "launch": bc.BC_LOOP_LAUNCH, "graph": bc.BC_LOOP_GRAPH}
    for name, m in modes.items():
        got, st = bc.bc_sources(h, g.n, s, TILED | bc.BC_TILE(32) | m)
        assert st["sigma_overflow_sources"] > 0
        assert_bc_close(got, want, what=f"grid1024 {name}")
    d, sg, o = bc.bc_tile_sssp(h, g.n, s[:6], TILED | bc.BC_TILE(32) | bc.BC_LOOP_GRAPH)
    for i in (0, 5):
        ref = oracle.sssp(g, int(s[i]))
        assert ref[2].any()  # counts beyond 2^64: the flag and sigma mod 2^64 are compared
        assert_sssp_equal((d[i], sg[i], o[i]), ref, f"grid1024 lane {i}")
    bc.bc_destroy(h)


def test_ba262144_pruned_equals_unpruned(ctx):
    g = gg.cached("ba", gg.ba_pref_attach, 262144, 2)
    h = upload(ctx, g)
    leaves = int(np.sum(g.degrees() == 1))
    assert leaves > 0.2 * g.n
    pruned, stp = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(128) | bc.BC_PRUNE_DEG1)
    full, stf = bc.bc_exact(h, g.n, TILED | bc.BC_TILE(128))
    assert stp["sources"] < stf["sources"]
    assert_bc_close(pruned, full, what="ba262144 pruned vs unpruned")
    s = gg.sample_sources(g, 48, seed=8)
    got, _ = bc.bc_sources(h, g.n, s, TILED | bc.BC_TILE(128))
    assert_bc_close(got, oracle.bc(g, s), what="ba262144 sampled sources")
    for x in s[:2]:
        d, sg, o = bc.bc_sssp(h, g.n, int(x))
        assert_sssp_equal((d, sg, o), oracle.sssp(g, int(x)), f"ba262144 source {x}")
    bc.bc_destroy(h)


def test_grid1024_per_source_cta_vs_oracle(ctx):
    """The per-CTA per-source kernel on a graph of a million vertices (BC_PLAIN_CTA): 304
    sources at a time, state in global memory, counts past 2^64 on the extended range."""
    g = gg.cached("grid", gg.grid2d, 1024, 1024, 5, 0.1)
    src = gg.sample_sources(g, 1024, seed=6)
    h = upload(ctx, g)
    s = src[:48]
    got, st = bc.bc_sources(h, g.n, s, bc.BC_PATH_PLAIN | bc.BC_PLAIN_CTA)
    assert st["sigma_overflow_sources"] == s.size
    assert_bc_close(got, oracle.bc(g, s), what="grid1024 per-source CTA")
    d, sg, o = bc.bc_sssp(h, g.n, int(s[3]), bc.BC_PLAIN_CTA)
    assert_sssp_equal((d, sg, o), oracle.sssp(g, int(s[3])), "grid1024 CTA sssp")
    bc.bc_destroy(h)
