"""The CUDA path on the stored exact fixture (tests/golden/bc_small.txt, Eq. 1 as exact
rationals): every kernel and heuristic, through the C ABI, within 1e-9 relative."""
import os
import sys

import numpy as np
import pytest

import graphgen as gg
import paper_1602_00963_gb300 as bc
from bcgpu import assert_bc_close, upload

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden  # noqa: E402

pytestmark = pytest.mark.gpu

P, T = bc.BC_PATH_PLAIN, bc.BC_PATH_TILED
FLAGS = {"cta": P, "grid": P | bc.BC_PLAIN_GRID, "tile32": T | bc.BC_TILE(32),
         "tile256": T | bc.BC_TILE(256), "cta_pruned": P | bc.BC_PRUNE_DEG1,
         "tile_pruned": T | bc.BC_TILE(64) | bc.BC_PRUNE_DEG1, "deg2": P | bc.BC_DEG2,
         "deg2_pruned": P | bc.BC_DEG2 | bc.BC_PRUNE_DEG1}
FIX = make_golden.load()


@pytest.fixture(scope="module")
def ctx():
    c = bc.bc_ctx_create(0)
    yield c
    bc.bc_destroy(c)


@pytest.mark.parametrize("gi", range(len(FIX)))
def test_golden_all_paths(ctx, gi):
    name, n, edges, exact = FIX[gi]
    g = gg.from_edge_list(n, edges)
    want = np.array([float(x) for x in exact])
    h = upload(ctx, g)
    for key, fl in FLAGS.items():
        got, _ = bc.bc_exact(h, g.n, fl)
        assert_bc_close(got, want, what=f"{name} {key}")
    bc.bc_destroy(h)
