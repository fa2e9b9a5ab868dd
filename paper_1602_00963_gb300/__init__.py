"""Python binding of libbc.so — exact betweenness centrality on one GB300.

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels behind the C ABI declared in ``include/bc.h``; the functions here carry the
same names.  Arrays may be numpy arrays (host) or CUDA torch tensors (device; the
BC_DEVICE_PTRS flag is added automatically).  There is no CPU fallback: if libbc.so is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "BCError", "load", "bc_version", "bc_last_error", "bc_ctx_create", "bc_graph_create",
    "bc_exact", "bc_sources", "bc_sssp", "bc_tile_sssp", "bc_prune", "bc_autotune",
    "bc_stream_submit", "bc_stream_poll", "bc_stream_cancel", "bc_destroy", "bc_sample_sources", "bc_sources_noalloc",
    "bc_set_wait_limit_ms", "BC_OK", "BC_EINVAL", "BC_ENOMEM", "BC_EAGAIN", "BC_ETIMEDOUT",
    "BC_ECUDA", "BC_ENOTFOUND", "BC_ECANCELED", "BC_DEVICE_PTRS", "BC_VALIDATE",
    "BC_PRUNE_DEG1", "BC_PATH_PLAIN", "BC_PATH_TILED", "BC_LOOP_LAUNCH", "BC_LOOP_GRAPH", "BC_PLAIN_GRID", "BC_DEG2", "BC_PLAIN_CTA", "BC_NO_CD_REUSE", "BC_DETERMINISTIC", "BC_KEEP_ORDER",
    "BC_TILE", "BC_REQ_EXACT_LIST", "BC_REQ_SAMPLED", "LIB_PATH",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbc.so")

BC_OK, BC_EINVAL, BC_ENOMEM, BC_EAGAIN, BC_ETIMEDOUT, BC_ECUDA, BC_ENOTFOUND, BC_ECANCELED = range(8)
BC_DEVICE_PTRS = 1 << 0
BC_VALIDATE = 1 << 1
BC_PRUNE_DEG1 = 1 << 2
BC_PATH_PLAIN = 1 << 3
BC_PATH_TILED = 1 << 4
BC_LOOP_LAUNCH = 1 << 5
BC_LOOP_GRAPH = 1 << 6
BC_PLAIN_GRID = 1 << 7
BC_DEG2 = 1 << 12
BC_PLAIN_CTA = 1 << 13
BC_NO_CD_REUSE = 1 << 14
BC_DETERMINISTIC = 1 << 15
BC_KEEP_ORDER = 1 << 16
BC_REQ_EXACT_LIST, BC_REQ_SAMPLED = 0, 1
_STATUS = {0: "BC_OK", 1: "BC_EINVAL", 2: "BC_ENOMEM", 3: "BC_EAGAIN", 4: "BC_ETIMEDOUT",
           5: "BC_ECUDA", 6: "BC_ENOTFOUND", 7: "BC_ECANCELED"}


def BC_TILE(T: int) -> int:
    return {32: 1, 64: 2, 128: 3, 256: 4}[T] << 8


class BCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class bc_stats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("sources", ctypes.c_int64),
                ("teps_sources", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("gteps", ctypes.c_double), ("max_depth", ctypes.c_int32),
                ("tile_width", ctypes.c_int32), ("sigma_overflow_sources", ctypes.c_int64),
                ("levels", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("reached_vertices", ctypes.c_int64), ("reached_arcs", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bc_tune_result(ctypes.Structure):
    _fields_ = [("tile_width", ctypes.c_int32), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("loop_mode", ctypes.c_int32), ("plain_cta", ctypes.c_int32), ("probe_seconds", ctypes.c_double),
                ("hub_degree", ctypes.c_int32), ("hub_chunk", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bc_request(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("mode", ctypes.c_int32), ("k", ctypes.c_int32),
                ("src", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("bc_out", ctypes.c_void_p)]


class bc_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("queue_seconds", ctypes.c_double),
                ("latency_seconds", ctypes.c_double), ("scale", ctypes.c_double),
                ("sources", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libbc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbc.so not found at {path}: build it with "
                           "paper_1602_00963_gb300.build.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    vp, i32, i64, u32, u64, dp = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_double)
    sig = {
        "bc_ctx_create": [ctypes.c_int, ctypes.c_size_t, u32, ctypes.POINTER(vp)],
        "bc_graph_create": [vp, i32, vp, vp, i64, u32, ctypes.POINTER(vp)],
        "bc_exact": [vp, u32, vp, vp, ctypes.POINTER(bc_stats)],
        "bc_sources": [vp, vp, i32, u32, vp, vp, ctypes.POINTER(bc_stats)],
        "bc_sssp": [vp, i32, u32, vp, vp, vp],
        "bc_tile_sssp": [vp, vp, i32, u32, vp, vp, vp],
        "bc_prune": [vp, u32, vp, vp, vp, vp, ctypes.POINTER(i64)],
        "bc_autotune": [vp, i32, u64, ctypes.POINTER(bc_tune_result)],
        "bc_stream_submit": [vp, ctypes.POINTER(bc_request), ctypes.POINTER(u64)],
        "bc_stream_poll": [vp, u64, i32, ctypes.POINTER(bc_result)],
        "bc_stream_cancel": [vp, u64],
        "bc_destroy": [vp],
        "bc_set_wait_limit_ms": [vp, i64],
        "bc_sources_noalloc": [i32, vp, vp, i64, vp, i32, vp, vp],
        "bc_sample_sources": [vp, i32, u64, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    L.bc_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    L.bc_last_error.restype = None
    L.bc_version.argtypes = []
    L.bc_version.restype = ctypes.c_char_p
    _lib = L
    return L


def bc_version() -> str:
    return load().bc_version().decode()


def bc_last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    load().bc_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(st: int):
    if st != BC_OK:
        raise BCError(st, bc_last_error())


def _is_cuda(x) -> bool:
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dev_flags(*arrays) -> int:
    kinds = {_is_cuda(a) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return BC_DEVICE_PTRS if kinds == {True} else 0


def bc_ctx_create(device: int = 0, hbm_budget_bytes: int = 0, flags: int = 0):
    h = ctypes.c_void_p()
    _check(load().bc_ctx_create(device, hbm_budget_bytes, flags, ctypes.byref(h)))
    return h


def bc_set_wait_limit_ms(ctx, ms: int):
    _check(load().bc_set_wait_limit_ms(ctx, ms))


def bc_graph_create(ctx, n: int, row_ptr, col_idx, nnz: int | None = None, flags: int = BC_VALIDATE):
    if not _is_cuda(row_ptr):
        row_ptr, col_idx = _host(row_ptr, np.int32), _host(col_idx, np.int32)
    flags |= _dev_flags(row_ptr, col_idx)
    nnz = int(col_idx.numel() if hasattr(col_idx, "numel") else col_idx.size) if nnz is None else nnz
    h = ctypes.c_void_p()
    _check(load().bc_graph_create(ctx, int(n), _ptr(row_ptr), _ptr(col_idx), nnz, flags,
                                  ctypes.byref(h)))
    return h


def bc_exact(graph, n: int, flags: int = 0, bc_out=None, stream=None):
    """Returns (bc, stats dict).  bc_out: numpy float64[n] or CUDA float64 tensor[n]."""
    if bc_out is None:
        bc_out = np.zeros(n, np.float64)
    flags |= _dev_flags(bc_out)
    st = bc_stats()
    _check(load().bc_exact(graph, flags, _ptr(bc_out), ctypes.c_void_p(stream) if stream else None,
                           ctypes.byref(st)))
    return bc_out, st.as_dict()


def bc_sources(graph, n: int, src, flags: int = 0, bc_out=None, stream=None):
    if not _is_cuda(src):
        src = _host(src, np.int32)
    if bc_out is None:
        bc_out = np.zeros(n, np.float64)
    flags |= _dev_flags(src, bc_out)
    k = int(src.numel() if hasattr(src, "numel") else src.size)
    st = bc_stats()
    _check(load().bc_sources(graph, _ptr(src), k, flags, _ptr(bc_out),
                             ctypes.c_void_p(stream) if stream else None, ctypes.byref(st)))
    return bc_out, st.as_dict()


def bc_sssp(graph, n: int, s: int, flags: int = 0):
    depth = np.empty(n, np.int32)
    sigma = np.empty(n, np.uint64)
    ovf = np.empty(n, np.uint8)
    _check(load().bc_sssp(graph, int(s), flags, _ptr(depth), _ptr(sigma), _ptr(ovf)))
    return depth, sigma, ovf


def bc_tile_sssp(graph, n: int, src, flags: int = 0):
    src = _host(src, np.int32)
    k = src.size
    depth = np.empty((k, n), np.int32)
    sigma = np.empty((k, n), np.uint64)
    ovf = np.empty((k, n), np.uint8)
    _check(load().bc_tile_sssp(graph, _ptr(src), k, flags, _ptr(depth), _ptr(sigma), _ptr(ovf)))
    return depth, sigma, ovf


def bc_prune(graph, n: int, nnz: int, flags: int = 0):
    omega = np.empty(n, np.int32)
    removed = np.empty(n, np.uint8)
    rrp = np.empty(n + 1, np.int32)
    rci = np.empty(max(nnz, 1), np.int32)
    rn = ctypes.c_int64(0)
    _check(load().bc_prune(graph, flags, _ptr(omega), _ptr(removed), _ptr(rrp), _ptr(rci),
                           ctypes.byref(rn)))
    return omega, removed, rrp, rci[: rn.value].copy()


def bc_autotune(graph, probe_sources: int = 0, seed: int = 0):
    r = bc_tune_result()
    _check(load().bc_autotune(graph, probe_sources, seed, ctypes.byref(r)))
    return r.as_dict()


def bc_stream_submit(ctx, graph, bc_out: np.ndarray, mode: int = BC_REQ_EXACT_LIST, src=None,
                     k: int = 0, seed: int = 0) -> int:
    """bc_out must stay alive until the request completes."""
    req = bc_request()
    req.graph = graph.value if isinstance(graph, ctypes.c_void_p) else graph
    req.mode = mode
    keep = None
    if mode == BC_REQ_EXACT_LIST:
        keep = _host(src, np.int32)
        req.k = keep.size
        req.src = keep.ctypes.data
    else:
        req.k = k
        req.src = None
    req.seed = seed
    req.bc_out = bc_out.ctypes.data
    rid = ctypes.c_uint64()
    _check(load().bc_stream_submit(ctx, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def bc_sample_sources(graph, k: int, seed: int):
    """The k sources a BC_REQ_SAMPLED request with this seed uses (sorted)."""
    out = np.empty(k, np.int32)
    _check(load().bc_sample_sources(graph, int(k), int(seed), _ptr(out)))
    return out


def bc_stream_poll(ctx, request_id: int, timeout_us: int = -1):
    """Returns (status, result dict); status BC_EAGAIN while the request runs."""
    r = bc_result()
    st = load().bc_stream_poll(ctx, request_id, timeout_us, ctypes.byref(r))
    if st not in (BC_OK, BC_EAGAIN):
        raise BCError(st, bc_last_error())
    return st, r.as_dict()


def bc_stream_cancel(ctx, request_id: int):
    _check(load().bc_stream_cancel(ctx, request_id))


def bc_destroy(handle):
    _check(load().bc_destroy(handle))


BC_NOALLOC_MAX_N = 65536


def bc_sources_noalloc(n: int, row_ptr, col_idx, src, bc_out, stream=None):
    """Allocation-free variant for callers that cannot allocate device memory: all
    arguments are CUDA tensors the caller owns (int32 CSR, int32 sources, float64 output);
    the library works in a static device scratch array (n <= BC_NOALLOC_MAX_N)."""
    import torch
    for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("col_idx", col_idx, torch.int32),
                        ("src", src, torch.int32), ("bc_out", bc_out, torch.float64)):
        if not _is_cuda(t):
            raise ValueError("bc_sources_noalloc takes CUDA tensors only")
        if t.dtype != dt:
            raise ValueError(f"bc_sources_noalloc: {name} must be {dt}, not {t.dtype}")
        if t.device != row_ptr.device:
            raise ValueError("bc_sources_noalloc: all tensors must be on one device")
    if row_ptr.numel() != int(n) + 1:
        raise ValueError(f"bc_sources_noalloc: row_ptr has {row_ptr.numel()} entries, not n + 1 = {int(n) + 1}")
    if bc_out.numel() < int(n):
        raise ValueError(f"bc_sources_noalloc: bc_out has {bc_out.numel()} entries, fewer than n = {int(n)}")
    _check(load().bc_sources_noalloc(int(n), _ptr(row_ptr), _ptr(col_idx), int(col_idx.numel()),
                                     _ptr(src), int(src.numel()), _ptr(bc_out),
                                     ctypes.c_void_p(stream) if stream else None))
    return bc_out
