"""Betweenness-centrality oracle — TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference
legs may import this package.  It wraps ``brandes.c`` (plain sequential Brandes, Alg. 1
with the 1-degree variant of Eq. 3 / Eq. 4 and Alg. 6) through ctypes and shares no
code with the CUDA path.  ``brute`` holds the exact rational brute force of Eq. 1.

Parity pins (checked by ``tests/test_oracle_*.py`` under ``-m "not gpu"``): exact
rational brute force of Eq. 1 on every labelled graph with n <= 5 and random graphs up
to n = 40; closed forms (path, star, complete, even/odd cycle, complete bipartite,
hypercube, trees); the invariant sum_v BC(v) = sum over ordered connected pairs of
(d - 1); networkx x 2; pruned == unpruned; sigma on grids (binomial) and hypercubes
(popcount!) in exact integers modulo 2^64 with the overflow flag.  No function here is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile brandes.c into liboracle.so next to it (gcc, -O3, no arch flags, no fast-math:
    the floating-point operations are those of the source, in its order)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O3", "-std=c11", "-shared", "-fPIC", "-pthread",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def load_from(path: str):
    """ctypes handle of a compiled brandes.c at `path`, with its signatures declared (the
    tests also load deliberately broken copies this way, to show that the pins catch them)."""
    lib = ctypes.CDLL(path)
    lib.oracle_sssp.restype = ctypes.c_int32
    lib.oracle_sssp.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32,
                                _i32p, _u64p, _u8p, ctypes.c_void_p]
    lib.oracle_bc.restype = ctypes.c_int
    lib.oracle_bc.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int64,
                              ctypes.c_void_p, _f64p, ctypes.c_int]
    lib.oracle_prune_deg1.restype = ctypes.c_int
    lib.oracle_prune_deg1.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _u8p, _i32p,
                                      _i32p, ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_long_double_size.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_from(_LIB)
    return _lib


def _csr(g):
    return (np.ascontiguousarray(g.row_ptr, dtype=np.int32),
            np.ascontiguousarray(g.col_idx, dtype=np.int32))


def sssp(g, s: int, want_long: bool = False):
    """(depth int32[n], sigma uint64[n], ovf uint8[n][, sigmaL longdouble[n]]) from s."""
    lib = _load()
    rp, ci = _csr(g)
    depth = np.empty(g.n, np.int32)
    sigma = np.empty(g.n, np.uint64)
    ovf = np.empty(g.n, np.uint8)
    sl = None
    ptr = None
    if want_long:
        if lib.oracle_long_double_size() != np.dtype(np.longdouble).itemsize:
            raise RuntimeError("numpy longdouble does not match C long double")
        sl = np.empty(g.n, np.longdouble)
        ptr = sl.ctypes.data
    rc = lib.oracle_sssp(g.n, rp, ci, int(s), depth, sigma, ovf, ptr)
    if rc < 0:
        raise RuntimeError(f"oracle_sssp failed ({rc})")
    return (depth, sigma, ovf, sl) if want_long else (depth, sigma, ovf)


def bc(g, sources=None, omega=None, nthreads: int = 1) -> np.ndarray:
    """Sum over the (multi)set of sources of (omega[s]+1) * delta_s, plus leaf terms when
    omega is given (then g must be the residual graph).  Default sources: all vertices."""
    lib = _load()
    rp, ci = _csr(g)
    src = np.arange(g.n, dtype=np.int32) if sources is None else np.ascontiguousarray(sources, dtype=np.int32)
    om = None
    optr = None
    if omega is not None:
        om = np.ascontiguousarray(omega, dtype=np.int32)
        optr = om.ctypes.data
    out = np.zeros(g.n, np.float64)
    rc = lib.oracle_bc(g.n, rp, ci, src, src.size, optr, out, int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_bc failed ({rc})")
    return out


def prune_deg1(g):
    """(omega int32[n], removed uint8[n], residual graph) per Alg. 6 (one round)."""
    from graphgen import Graph
    lib = _load()
    rp, ci = _csr(g)
    omega = np.empty(g.n, np.int32)
    removed = np.empty(g.n, np.uint8)
    rrp = np.empty(g.n + 1, np.int32)
    rci = np.empty(max(g.nnz, 1), np.int32)
    nnz = ctypes.c_int64(0)
    lib.oracle_prune_deg1(g.n, rp, ci, omega, removed, rrp, rci, ctypes.byref(nnz))
    res = Graph(g.n, rrp, rci[: nnz.value].copy(), g.name + "-res")
    return omega, removed, res


def bc_exact(g, prune: bool = False, nthreads: int = 1) -> np.ndarray:
    """Exact BC over all sources (ordered pairs).  With ``prune`` the 1-degree heuristic
    is applied: Brandes runs on the residual graph from the non-removed vertices."""
    if not prune:
        return bc(g, None, None, nthreads)
    omega, removed, res = prune_deg1(g)
    src = np.flatnonzero(removed == 0).astype(np.int32)
    return bc(res, src, omega, nthreads)


__all__ = ["build", "sssp", "bc", "prune_deg1", "bc_exact"]
