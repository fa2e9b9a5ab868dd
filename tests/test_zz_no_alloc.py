"""The allocation-free entry point bc_sources_noalloc, for callers that cannot allocate
device memory (their memory belongs to another allocator, or cudaMalloc's implicit
synchronisation is not allowed where they run).  It must give the same BC as the regular
entry point bc_sources, call after call, although every call reuses one static scratch
array; it must reject bad sizes and out-of-range source ids before any traversal.  This file
is collected last so that a failure here stops a run only after every other test has run."""
import numpy as np
import pytest

import graphgen as gg
import paper_1602_00963_gb300 as bc
from bcgpu import REL, assert_bc_close

pytestmark = pytest.mark.gpu


def _dev(torch, g):
    return torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda()


def _noalloc(torch, g, rp, ci, src, stream=None):
    out = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
    bc.bc_sources_noalloc(g.n, rp, ci, torch.from_numpy(np.asarray(src, np.int32)).cuda(), out,
                          stream=stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_bc_sources_twice():
    torch = pytest.importorskip("torch")
    g = gg.rmat(12, 16, 1)
    ctx = bc.bc_ctx_create(0)
    try:
        h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, bc.BC_VALIDATE)
        rp, ci = _dev(torch, g)
        for call, seed in enumerate((11, 12)):
            src = gg.sample_sources(g, 96, seed=seed)
            want, _ = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN)
            assert_bc_close(_noalloc(torch, g, rp, ci, src), want, rel=REL, what=f"no-alloc call {call}")
        bc.bc_destroy(h)
    finally:
        bc.bc_destroy(ctx)


def test_noalloc_sizes_streams_and_empty_lists():
    """The largest graph the scratch takes (n = BC_NOALLOC_MAX_N), a small graph of odd n
    with a repeated source, a call on a side stream, and k = 0 (bc_out set to zero)."""
    torch = pytest.importorskip("torch")
    big = gg.rmat(16, 4, 21)
    assert big.n == bc.BC_NOALLOC_MAX_N
    small = gg.grid2d(7, 9)  # n = 63
    ctx = bc.bc_ctx_create(0)
    try:
        for g, src in ((big, gg.sample_sources(big, 12, seed=3)),
                       (small, np.array([0, 5, 5, 62, 31], np.int32))):
            h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, bc.BC_VALIDATE)
            want, _ = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN)
            rp, ci = _dev(torch, g)
            assert_bc_close(_noalloc(torch, g, rp, ci, src), want, rel=REL, what=f"n={g.n}")
            side = torch.cuda.Stream()
            with torch.cuda.stream(side):
                got = _noalloc(torch, g, rp, ci, src, stream=side.cuda_stream)
            assert_bc_close(got, want, rel=REL, what=f"n={g.n}, side stream")
            assert np.array_equal(_noalloc(torch, g, rp, ci, np.zeros(0, np.int32)), np.zeros(g.n))
            bc.bc_destroy(h)
    finally:
        bc.bc_destroy(ctx)


def test_noalloc_rejects_out_of_range_sources_then_still_matches():
    torch = pytest.importorskip("torch")
    g = gg.rmat(10, 8, 2)
    ctx = bc.bc_ctx_create(0)
    try:
        h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, bc.BC_VALIDATE)
        rp, ci = _dev(torch, g)
        for bad in ([g.n], [3, -1], [0, 2, g.n + 7]):
            with pytest.raises(bc.BCError) as e:
                _noalloc(torch, g, rp, ci, bad)
            assert e.value.status == bc.BC_EINVAL and "out of range" in str(e.value)
        src = gg.sample_sources(g, 40, seed=9)
        want, _ = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN)
        assert_bc_close(_noalloc(torch, g, rp, ci, src), want, rel=REL, what="after rejected calls")
        bc.bc_destroy(h)
    finally:
        bc.bc_destroy(ctx)


def test_noalloc_rejects_too_large():
    torch = pytest.importorskip("torch")
    n = bc.BC_NOALLOC_MAX_N + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(2, dtype=torch.int32, device="cuda")
    src = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(bc.BCError) as e:
        bc.bc_sources_noalloc(n, rp, ci, src, out)
    assert e.value.status == bc.BC_EINVAL
    assert "BC_NOALLOC_MAX_N" in str(e.value) or str(bc.BC_NOALLOC_MAX_N) in str(e.value)


def test_noalloc_wrapper_rejects_wrong_dtypes_and_sizes():
    torch = pytest.importorskip("torch")
    g = gg.path_graph(8)
    rp, ci = _dev(torch, g)
    src = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        bc.bc_sources_noalloc(g.n, rp.long(), ci, src, out)
    with pytest.raises(ValueError):
        bc.bc_sources_noalloc(g.n, rp, ci, src, out.float())
    with pytest.raises(ValueError):
        bc.bc_sources_noalloc(g.n, rp[:-1], ci, src, out)
    with pytest.raises(ValueError):
        bc.bc_sources_noalloc(g.n, rp, ci, src, out[:-1])
