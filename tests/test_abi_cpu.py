"""CPU checks of the boundary: libbc.so builds for sm_103a, loads without a GPU, and
exports every function include/bc.h declares; host-side helpers of the bench."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:bc_status|void|const char \*)\s*(bc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_00963_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ["bc_ctx_create", "bc_graph_create", "bc_exact", "bc_sources", "bc_sssp",
                 "bc_stream_submit", "bc_stream_poll", "bc_stream_cancel", "bc_destroy",
                 "bc_autotune", "bc_prune", "bc_tile_sssp", "bc_last_error", "bc_sources_noalloc"]:
        assert must in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_text_without_gpu(lib):
    lib.bc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bc_version()
    buf = ctypes.create_string_buffer(256)
    lib.bc_destroy.argtypes = [ctypes.c_void_p]
    assert lib.bc_destroy(None) == 1  # BC_EINVAL, no device needed
    lib.bc_last_error(buf, ctypes.c_size_t(len(buf)))
    assert b"bc_destroy" in buf.value


def test_algorithmic_bytes_model():
    import bench
    st = {"reached_vertices": 1000, "reached_arcs": 20000}
    assert bench.algorithmic_bytes(st, 1) == 8 * 20000 + 84 * 1000
    assert bench.algorithmic_bytes(st, 64) == (8 * 20000 + 16 * 1000) / 64 + 68 * 1000 + 1000 / 4


def test_bench_deg2_triple_count_matches_the_selection_rule():
    """bench.py reports the number of derived 2-degree runs with the library's rule; it
    must agree with the oracle's statement of the same rule."""
    import bench
    import graphgen as gg
    from oracle import deg2
    for g in [gg.cycle_graph(17), gg.subdivide_edges(gg.grid2d(12, 12, seed=1, delete_frac=0.1), 0.4, 2),
              gg.random_tree(60, 4)]:
        assert bench.deg2_triples(g) == len(deg2.select_triples(g))


def test_code_hash_ignores_comments_only(tmp_path):
    """bench.py ties the committed ncu traffic figure to the tile kernel's code: editing a
    comment keeps the hash, editing code changes it."""
    import bench
    src = os.path.join(ROOT, "paper_1602_00963_gb300", "csrc", "bc_tile.cu")
    text = open(src).read()
    a = tmp_path / "a.cu"
    a.write_text(text.replace("// Warp-level work is numbered", "// Warp work is numbered"))
    b = tmp_path / "b.cu"
    import re
    changed = re.sub(r"constexpr int kHubDefault = (\d+);", r"constexpr int kHubDefault = 1\1;", text)
    assert changed != text
    b.write_text(changed)
    assert bench.code_sha1(str(a)) == bench.code_sha1(src) != bench.code_sha1(str(b))


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """include/bc.h is plain C (C11, warnings as errors) and a C program links against
    libbc.so and calls it; without a GPU only calls that need no device are made."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include "bc.h"
#include <stdio.h>
#include <string.h>
int main(void) {
  char msg[256];
  const char *v = bc_version();
  if (!v || !strstr(v, "sm_103a")) return 2;
  if (bc_destroy(NULL) != BC_EINVAL) return 3;
  bc_last_error(msg, sizeof msg);
  if (!strstr(msg, "bc_destroy")) return 4;
  if (bc_sources_noalloc(BC_NOALLOC_MAX_N + 1, NULL, NULL, 0, NULL, 0, NULL, NULL) != BC_EINVAL) return 5;
  /* size limits are checked before any device work: n in [1, max], nnz in [0, 2^31) */
  int32_t rp[2] = {0, 0}, src[1] = {0};
  double out[1];
  if (bc_sources_noalloc(0, rp, rp, 0, src, 1, out, NULL) != BC_EINVAL) return 6;
  if (bc_sources_noalloc(1, rp, rp, (int64_t)1 << 31, src, 1, out, NULL) != BC_EINVAL) return 7;
  if (bc_sources_noalloc(1, rp, rp, -1, src, 1, out, NULL) != BC_EINVAL) return 8;
  if (bc_sources_noalloc(1, rp, rp, 0, src, -1, out, NULL) != BC_EINVAL) return 9;
  if (bc_sources_noalloc(1, rp, rp, 3, src, 1, out, NULL) != BC_EINVAL) return 10; /* odd nnz */
  printf("%s\n", v);
  return 0;
}
''')
    libdir = os.path.dirname(lib._name)
    exe = tmp_path / "abi"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lbc",
                           "-o", str(exe)])
    env = dict(os.environ, LD_LIBRARY_PATH=libdir + os.pathsep + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([str(exe)], env=env, capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)


def test_committed_traffic_matches_the_current_kernel():
    """The ncu DRAM figure of the autotuner's tile width (T = 128 on the bench workload) was
    taken on the current kernel code, so the bench reports it; other widths and stale code
    give None."""
    import json
    import bench
    path = os.path.join(ROOT, "profiles", "tile_rmat20_dram_T128.json")
    j = json.load(open(path))
    assert j["tile_width"] == 128
    assert bench.ncu_traffic(128, 0.0) == float(j["dram_bytes_per_launch"])
    assert bench.ncu_traffic(32, 0.0) is None
