"""Continuous-batching serving loop and autotuner, through the C ABI.

The serving test submits exact-list and sampled requests over several resident graphs at
once (so sources of different requests share tiles and tiles of different graphs overlap
on separate streams) and checks that each result equals the same request run alone
(bc_sources) and the oracle, within the BC tolerance."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1602_00963_gb300 as bc
from bcgpu import assert_bc_close, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = bc.bc_ctx_create(0)
    yield c
    bc.bc_destroy(c)


def test_mixed_requests_equal_alone(ctx):
    graphs = [gg.rmat(11, 8, 21), gg.erdos_renyi(3000, 12000, 22), gg.grid2d(50, 50, seed=23, delete_frac=0.1)]
    handles = [upload(ctx, g) for g in graphs]
    rng = np.random.Generator(np.random.PCG64(99))
    reqs = []
    for i in range(14):
        gi = i % 3
        g, h = graphs[gi], handles[gi]
        out = np.zeros(g.n, np.float64)
        if i % 2 == 0:
            k = int(rng.integers(1, 150))
            src = rng.choice(np.flatnonzero(g.degrees() > 0), size=k, replace=True).astype(np.int32)
            rid = bc.bc_stream_submit(ctx, h, out, bc.BC_REQ_EXACT_LIST, src=src)
        else:
            k = int(rng.integers(1, 90))
            seed = int(rng.integers(0, 2**40))
            rid = bc.bc_stream_submit(ctx, h, out, bc.BC_REQ_SAMPLED, k=k, seed=seed)
            src = bc.bc_sample_sources(h, k, seed)
        reqs.append((rid, gi, src, out))
    for rid, gi, src, out in reqs:
        st, res = bc.bc_stream_poll(ctx, rid, -1)
        assert st == bc.BC_OK and res["status"] == bc.BC_OK, res
        assert res["sources"] == len(src)
        assert res["latency_seconds"] >= res["queue_seconds"] >= 0
        g, h = graphs[gi], handles[gi]
        alone, _ = bc.bc_sources(h, g.n, src)
        assert_bc_close(out, alone, what=f"request {rid} mixed vs alone")
        assert_bc_close(out, oracle.bc(g, src), what=f"request {rid} vs oracle")
    for h in handles:
        bc.bc_destroy(h)


def test_tile_requests_grouped_by_locality(ctx):
    """A graph above 65,536 vertices is served with tiles; requests submitted together are
    cut into tiles by landmark profile across requests (at most 8 requests per tile, the
    oldest request always advancing).  Each result equals the request run alone and, for
    the first (12 sources), the oracle."""
    g = gg.rmat(17, 4, 41)
    h = upload(ctx, g)
    rng = np.random.Generator(np.random.PCG64(17))
    pool = np.flatnonzero(g.degrees() > 0)
    reqs = []
    for i in range(12):
        out = np.zeros(g.n)
        k = 12 if i == 0 else int(rng.integers(1, 160))
        src = rng.choice(pool, size=k, replace=False).astype(np.int32)
        reqs.append((bc.bc_stream_submit(ctx, h, out, bc.BC_REQ_EXACT_LIST, src=src), src, out))
    for i, (rid, src, out) in enumerate(reqs):
        st, res = bc.bc_stream_poll(ctx, rid, -1)
        assert st == bc.BC_OK and res["status"] == bc.BC_OK, res
        assert res["sources"] == len(src)
        alone, _ = bc.bc_sources(h, g.n, src)
        assert_bc_close(out, alone, what=f"request {rid} grouped vs alone")
        if i == 0:
            assert_bc_close(out, oracle.bc(g, src), what="grouped request vs oracle")
    bc.bc_destroy(h)


def test_sampled_is_deterministic_and_scaled(ctx):
    g = gg.rmat(10, 8, 31)
    h = upload(ctx, g)
    a = bc.bc_sample_sources(h, 40, 1234)
    b = bc.bc_sample_sources(h, 40, 1234)
    assert (a == b).all() and len(set(a.tolist())) == 40
    assert (g.degrees()[a] > 0).all()
    out = np.zeros(g.n)
    rid = bc.bc_stream_submit(ctx, h, out, bc.BC_REQ_SAMPLED, k=40, seed=1234)
    st, res = bc.bc_stream_poll(ctx, rid, -1)
    assert st == bc.BC_OK and res["status"] == bc.BC_OK
    assert abs(res["scale"] - (g.degrees() > 0).sum() / 40) < 1e-12
    assert_bc_close(out, oracle.bc(g, a), what="sampled vs oracle on the drawn list")
    bc.bc_destroy(h)


def test_cancel_poll_destroy_rules(ctx):
    g = gg.rmat(12, 16, 41)
    h = upload(ctx, g)
    outs = [np.zeros(g.n) for _ in range(6)]
    big = np.flatnonzero(g.degrees() > 0).astype(np.int32)
    ids = [bc.bc_stream_submit(ctx, h, o, bc.BC_REQ_EXACT_LIST, src=big) for o in outs]
    # a graph with requests in flight cannot be destroyed
    with pytest.raises(bc.BCError) as e:
        bc.bc_destroy(h)
    assert e.value.status == bc.BC_EAGAIN
    bc.bc_stream_cancel(ctx, ids[-1])
    statuses = []
    for rid in ids:
        st, res = bc.bc_stream_poll(ctx, rid, -1)
        statuses.append(res["status"])
    assert statuses[-1] in (bc.BC_ECANCELED, bc.BC_OK)
    assert all(s == bc.BC_OK for s in statuses[:-1])
    with pytest.raises(bc.BCError) as e:
        bc.bc_stream_poll(ctx, ids[0], 0)  # already collected
    assert e.value.status == bc.BC_ENOTFOUND
    bc.bc_destroy(h)


def test_budget_admission_completes_all():
    """A context with a small HBM budget (graph, one tile workspace and a few request
    accumulators) still completes every request, admitting them as memory allows."""
    g = gg.rmat(11, 8, 51)
    c = bc.bc_ctx_create(0, 8 << 20)
    try:
        h = upload(c, g)
        outs, ids = [], []
        for i in range(5):
            out = np.zeros(g.n)
            src = np.arange(i * 20, i * 20 + 20, dtype=np.int32)
            ids.append((bc.bc_stream_submit(c, h, out, bc.BC_REQ_EXACT_LIST, src=src), src, out))
        for rid, src, out in ids:
            st, res = bc.bc_stream_poll(c, rid, -1)
            assert res["status"] == bc.BC_OK
            assert_bc_close(out, oracle.bc(g, src), what="budgeted request")
        bc.bc_destroy(h)
    finally:
        bc.bc_destroy(c)


def test_per_cta_requests_share_calls_under_a_tight_budget():
    """Requests on a small graph (per-CTA kernel) submitted together share calls, each
    request on CTAs of its own; with an HBM budget that leaves fewer CTAs than requests,
    the requests are split over several launches.  Every result matches the oracle."""
    g = gg.rmat(11, 8, 52)
    c = bc.bc_ctx_create(0, 1200 << 10)
    try:
        h = upload(c, g)
        rng = np.random.Generator(np.random.PCG64(7))
        pool = np.flatnonzero(g.degrees() > 0)
        ids = []
        for i in range(10):
            out = np.zeros(g.n)
            src = rng.choice(pool, size=int(rng.integers(1, 12)), replace=False).astype(np.int32)
            ids.append((bc.bc_stream_submit(c, h, out, bc.BC_REQ_EXACT_LIST, src=src), src, out))
        for rid, src, out in ids:
            st, res = bc.bc_stream_poll(c, rid, -1)
            assert st == bc.BC_OK and res["status"] == bc.BC_OK, res
            assert_bc_close(out, oracle.bc(g, src), what="per-CTA request under a tight budget")
        bc.bc_destroy(h)
    finally:
        bc.bc_destroy(c)


def test_autotune_and_tuned_dispatch(ctx):
    g = gg.rmat(12, 16, 1)
    h = upload(ctx, g)
    t = bc.bc_autotune(h, 128, 5)
    assert t["tile_width"] in (0, 32, 64, 128, 256)
    assert t["probe_seconds"] > 0
    got, st = bc.bc_exact(h, g.n)  # no path flag: uses the tuned configuration
    assert st["tile_width"] == (t["tile_width"] or 1)
    assert_bc_close(got, oracle.bc_exact(g, nthreads=8), what="tuned exact")
    # serving follows the tuned kernel too (tiles or the per-CTA kernel, whichever won)
    rng = np.random.Generator(np.random.PCG64(3))
    ids = []
    for i in range(6):
        out = np.zeros(g.n)
        src = rng.choice(np.flatnonzero(g.degrees() > 0), size=int(rng.integers(1, 100)), replace=False)
        src = src.astype(np.int32)
        ids.append((bc.bc_stream_submit(ctx, h, out, bc.BC_REQ_EXACT_LIST, src=src), src, out))
    for rid, src, out in ids:
        st, res = bc.bc_stream_poll(ctx, rid, -1)
        assert st == bc.BC_OK and res["status"] == bc.BC_OK, res
        assert_bc_close(out, oracle.bc(g, src), what="request on a tuned graph")
    bc.bc_destroy(h)
