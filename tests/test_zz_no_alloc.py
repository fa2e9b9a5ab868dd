"""The allocation-free entry point bc_sources_noalloc, for callers that cannot allocate
device memory (their memory belongs to another allocator, or cudaMalloc's implicit
synchronisation is not allowed where they run).  It must give the same BC as the regular
entry point bc_sources, call after call, although every call reuses one static scratch
array.  This file is collected last so that a failure here stops a run only after every
other test has run."""
import numpy as np
import pytest

import graphgen as gg
import paper_1602_00963_gb300 as bc
from bcgpu import REL, assert_bc_close

pytestmark = pytest.mark.gpu


def test_noalloc_matches_bc_sources_twice():
    torch = pytest.importorskip("torch")
    g = gg.rmat(12, 16, 1)
    ctx = bc.bc_ctx_create(0)
    try:
        h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, bc.BC_VALIDATE)
        rp = torch.from_numpy(g.row_ptr).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        for call, seed in enumerate((11, 12)):
            src = gg.sample_sources(g, 96, seed=seed)
            want, _ = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN)
            out = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
            bc.bc_sources_noalloc(g.n, rp, ci, torch.from_numpy(src).cuda(), out)
            torch.cuda.synchronize()
            assert_bc_close(out.cpu().numpy(), want, rel=REL, what=f"no-alloc call {call}")
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
