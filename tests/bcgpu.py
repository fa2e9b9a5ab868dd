"""Helpers for the GPU tests: upload graphgen graphs through the C ABI and compare
results with the oracle element by element."""
import numpy as np

import paper_1602_00963_gb300 as bc

REL = 1e-9  # FP64 BC tolerance: |gpu - oracle| <= REL * max(|oracle|, 1) per vertex


def upload(ctx, g, flags=bc.BC_VALIDATE):
    return bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, flags)


def assert_bc_close(got, want, rel=REL, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want) / np.maximum(np.abs(want), 1.0)
    i = int(np.argmax(err)) if err.size else 0
    assert err.size == 0 or err[i] <= rel, (
        f"{what}: vertex {i} gpu={got[i]!r} oracle={want[i]!r} rel.err={err[i]:.3e}")


def assert_sssp_equal(got, want, what=""):
    d0, s0, o0 = got
    d1, s1, o1 = want
    bad = np.flatnonzero(d0 != d1)
    assert bad.size == 0, f"{what}: depth differs at {bad[:5]} gpu={d0[bad[:5]]} oracle={d1[bad[:5]]}"
    bad = np.flatnonzero(s0 != s1)
    assert bad.size == 0, f"{what}: sigma differs at {bad[:5]} gpu={s0[bad[:5]]} oracle={s1[bad[:5]]}"
    bad = np.flatnonzero(o0.astype(bool) != o1.astype(bool))
    assert bad.size == 0, f"{what}: overflow flag differs at {bad[:5]}"
