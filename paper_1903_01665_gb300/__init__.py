"""Python binding of libfg (include/fg.h): argument marshalling only.

Every function keeps the C name and returns the C status code; arrays may be
numpy arrays (host memory) or torch tensors (host or CUDA).  All computation
runs in the CUDA library -- there is no Python or CPU fallback: if libfg.so
cannot be loaded or built, importing the binding's functions raises.

    import paper_1903_01665_gb300 as fg
    st, g = fg.fg_graph_create_coo(n, src, dst, w)
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    fg.check(fg.fg_sssp(g, 0, dist, fg.FG_VERTEX_SYNC))
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfg.so")

# status codes
FG_OK = 0
FG_ERR_INVALID_ARG = 1
FG_ERR_NEGATIVE_WEIGHT = 2
FG_ERR_OVERFLOW = 3
FG_ERR_OUT_OF_MEMORY = 4
FG_ERR_TIMEOUT = 5
FG_ERR_CUDA = 6
# modes
FG_VERTEX_SYNC = 0
FG_VERTEX_ASYNC = 1
FG_EDGE_SYNC = 2
FG_EDGE_ASYNC = 3
FG_AUTO = 4
FG_PULL = 5
FG_BUCKET = 6
MODES = {"vertex_sync": 0, "vertex_async": 1, "edge_sync": 2, "edge_async": 3, "auto": 4, "pull": 5, "bucket": 6}
MODE_NAMES = {v: k for k, v in MODES.items()}
# algorithms
FG_ALGO_SSSP = 0
FG_ALGO_BFS = 1
FG_ALGO_CC = 2
FG_INF = 2**31 - 1
FG_GRAPH_LAZY = 1
FG_GRAPH_RELABEL = 2
FG_GRAPH_KEEP_IDS = 4


class fg_options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("max_rounds", ctypes.c_int32),
                ("wait_timeout_ms", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("inject_missing_arrival", ctypes.c_int32), ("round_trace", ctypes.c_void_p),
                ("round_trace_cap", ctypes.c_int32), ("delta", ctypes.c_int32)]


class fg_stats(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("rounds", ctypes.c_int32), ("jump_passes", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("vertices_processed", ctypes.c_int64),
                ("edges_relaxed", ctypes.c_int64), ("updates", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("scanned", ctypes.c_int64), ("kernel_ms", ctypes.c_float),
                ("barriers", ctypes.c_int32), ("pull_rounds", ctypes.c_int32), ("edges_pulled", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fg_graph_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("m_sym", ctypes.c_int64),
                ("max_out_degree", ctypes.c_int32), ("n_zero_out", ctypes.c_int32),
                ("n_low", ctypes.c_int32), ("n_mid", ctypes.c_int32), ("n_high", ctypes.c_int32),
                ("n_high_chunks", ctypes.c_int32), ("n_isolated", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("relabelled", ctypes.c_int32),
                ("in_degree_gini", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fg_query(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("algo", ctypes.c_int32), ("src", ctypes.c_int32),
                ("out", ctypes.c_void_p), ("mode", ctypes.c_int32)]


class fg_batch_options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("use_cuda_graph", ctypes.c_int32),
                ("wait_timeout_ms", ctypes.c_int32), ("fuse_same_graph", ctypes.c_int32)]


class fg_batch_stats(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_float), ("launches", ctypes.c_int32), ("teams", ctypes.c_int32),
                ("ctas", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fg_server_options(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_wave", ctypes.c_int32), ("one_at_a_time", ctypes.c_int32),
                ("wait_timeout_ms", ctypes.c_int32), ("exclusive_edges", ctypes.c_int64),
                ("no_fusion", ctypes.c_int32)]


class fg_plan(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("delta", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("depth_est", ctypes.c_int32), ("degree_gini", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fg_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("wave_size", ctypes.c_int32),
                ("latency_ms", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p
_SIGNATURES = {
    "fg_graph_create_csr": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "fg_graph_create_coo": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "fg_graph_create_csr_ex": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_uint32,
                                              ctypes.POINTER(_VP)]),
    "fg_graph_create_coo_ex": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_uint32,
                                              ctypes.POINTER(_VP)]),
    "fg_graph_destroy": (ctypes.c_int, [_VP]),
    "fg_graph_info": (ctypes.c_int, [_VP, ctypes.POINTER(fg_graph_info_t)]),
    "fg_sssp": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int]),
    "fg_bfs": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int]),
    "fg_cc": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "fg_select_mode": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "fg_select_plan": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(fg_plan)]),
    "fg_run": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int32, _VP, ctypes.c_int,
                              ctypes.POINTER(fg_options), ctypes.POINTER(fg_stats)]),
    "fg_sweep": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_float)]),
    "fg_run_multi": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(_VP), ctypes.POINTER(fg_options), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(fg_stats)]),
    "fg_sssp_csr_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_int32,
                                           _VP, _VP]),
    "fg_run_batch": (ctypes.c_int, [ctypes.POINTER(fg_query), ctypes.c_int32, ctypes.POINTER(fg_batch_options),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(fg_stats),
                                    ctypes.POINTER(fg_batch_stats)]),
    "fg_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_float)]),
    "fg_server_create": (ctypes.c_int, [ctypes.POINTER(fg_server_options), ctypes.POINTER(_VP)]),
    "fg_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(fg_query), ctypes.POINTER(ctypes.c_uint64)]),
    "fg_server_poll": (ctypes.c_int32, [_VP, ctypes.POINTER(fg_completion), ctypes.c_int32]),
    "fg_server_drain": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "fg_server_destroy": (ctypes.c_int, [_VP]),
    "fg_kernel_launches": (ctypes.c_uint64, []),
    "fg_last_error": (ctypes.c_char_p, []),
    "fg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(build_if_missing: bool = True):
    """Load libfg.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if build_if_missing and not _build.is_fresh():
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libfg.so not found at {LIB_PATH}; run paper_1903_01665_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class FGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{fg_status_string(status)}: {msg}")
        self.status = status


def check(status: int):
    if status != FG_OK:
        raise FGError(status, fg_last_error())
    return status


def _ptr(x):
    """Address of an array's data: numpy (host) or torch (host or CUDA), or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _check_dtype(x, kind: str):
    if x is None:
        return
    dt = str(x.dtype)
    if kind not in dt:
        raise TypeError(f"expected {kind} array, got {dt}")


def _len(x):
    return int(x.shape[0]) if x is not None else 0


def fg_graph_create_coo(n, src, dst, w=None, flags=0):
    """Returns (status, handle).  flags: FG_GRAPH_LAZY | FG_GRAPH_RELABEL or FG_GRAPH_KEEP_IDS."""
    for a in (src, dst, w):
        _check_dtype(a, "int32")
    h = _VP()
    if flags:
        st = load().fg_graph_create_coo_ex(int(n), _len(src), _ptr(src), _ptr(dst), _ptr(w), int(flags),
                                           ctypes.byref(h))
    else:
        st = load().fg_graph_create_coo(int(n), _len(src), _ptr(src), _ptr(dst), _ptr(w), ctypes.byref(h))
    return st, (h.value if st == FG_OK else None)


def fg_graph_create_csr(n, row_off, col, w=None, flags=0):
    """Returns (status, handle).  row_off is int64[n+1]; flags as for fg_graph_create_coo."""
    _check_dtype(row_off, "int64")
    _check_dtype(col, "int32")
    _check_dtype(w, "int32")
    h = _VP()
    if flags:
        st = load().fg_graph_create_csr_ex(int(n), _len(col), _ptr(row_off), _ptr(col), _ptr(w), int(flags),
                                           ctypes.byref(h))
    else:
        st = load().fg_graph_create_csr(int(n), _len(col), _ptr(row_off), _ptr(col), _ptr(w), ctypes.byref(h))
    return st, (h.value if st == FG_OK else None)


def fg_graph_destroy(g):
    return load().fg_graph_destroy(g)


def fg_graph_info(g):
    info = fg_graph_info_t()
    st = load().fg_graph_info(g, ctypes.byref(info))
    return st, info


def fg_sssp(g, src, dist_out, mode=FG_VERTEX_SYNC):
    _check_dtype(dist_out, "int32")
    return load().fg_sssp(g, int(src), _ptr(dist_out), int(mode))


def fg_bfs(g, src, level_out, mode=FG_VERTEX_SYNC):
    _check_dtype(level_out, "int32")
    return load().fg_bfs(g, int(src), _ptr(level_out), int(mode))


def fg_cc(g, label_out, mode=FG_VERTEX_SYNC):
    _check_dtype(label_out, "int32")
    return load().fg_cc(g, _ptr(label_out), int(mode))


def fg_select_mode(g, algo):
    m = ctypes.c_int(-1)
    st = load().fg_select_mode(g, int(algo), ctypes.byref(m))
    return st, m.value


def fg_select_plan(g, algo):
    """Returns (status, fg_plan): mode, CTAs per SM, bucket width, and the model's features."""
    p = fg_plan()
    st = load().fg_select_plan(g, int(algo), ctypes.byref(p))
    return st, p


def fg_run(g, algo, src, out, mode, stream=None, max_rounds=0, wait_timeout_ms=0, blocks_per_sm=0,
           inject_missing_arrival=0, round_trace=None, delta=0):
    """Returns (status, fg_stats).  stream: a torch.cuda.Stream, a raw handle, or None."""
    _check_dtype(out, "int32")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    opt = fg_options(stream, int(max_rounds), int(wait_timeout_ms), int(blocks_per_sm),
                     int(inject_missing_arrival), _ptr(round_trace),
                     int(round_trace.shape[0]) if round_trace is not None else 0, int(delta))
    stats = fg_stats()
    st = load().fg_run(g, int(algo), int(src), _ptr(out), int(mode), ctypes.byref(opt), ctypes.byref(stats))
    return st, stats


FG_MULTI_MAX = 8


def fg_run_multi(g, algo, srcs, outs, stream=None, max_rounds=0, wait_timeout_ms=0, blocks_per_sm=0, delta=0):
    """k = len(outs) queries of one algorithm on one graph (srcs: k sources,
    ignored for CC; delta: the SSSP sweep's near-far width, 0 = default).
    Returns (status, [per-query status], fg_stats of the fused sweep)."""
    k = len(outs)
    for o in outs:
        _check_dtype(o, "int32")
    src_list = [int(x) for x in srcs] if srcs is not None else [0] * k
    if len(src_list) < k:
        raise ValueError("one source per output")
    src_arr = (ctypes.c_int32 * max(k, 1))(*src_list[:k])
    out_arr = (ctypes.c_void_p * max(k, 1))(*[_ptr(o) for o in outs])
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    opt = fg_options(stream, int(max_rounds), int(wait_timeout_ms), int(blocks_per_sm), 0, None, 0, int(delta))
    sts = (ctypes.c_int * max(k, 1))()
    stats = fg_stats()
    st = load().fg_run_multi(g, int(algo), int(k), src_arr, out_arr, ctypes.byref(opt), sts, ctypes.byref(stats))
    return st, list(sts)[:k], stats


def fg_sweep(g, mode, cur, nxt, stream=None):
    """Returns (status, updates, kernel_ms)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    upd = ctypes.c_int64(0)
    ms = ctypes.c_float(0)
    st = load().fg_sweep(g, int(mode), _ptr(cur), _ptr(nxt), stream, ctypes.byref(upd), ctypes.byref(ms))
    return st, upd.value, ms.value


def fg_run_batch(queries, stream=None, use_cuda_graph=False, wait_timeout_ms=0, fuse_same_graph=False):
    """queries: list of (graph, algo, src, out_array, mode).  Returns
    (status, [per-query status], [per-query fg_stats], fg_batch_stats)."""
    nq = len(queries)
    arr = (fg_query * nq)()
    for i, (g, algo, src, out, mode) in enumerate(queries):
        _check_dtype(out, "int32")
        arr[i] = fg_query(g, int(algo), int(src), _ptr(out), int(mode))
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    opt = fg_batch_options(stream, 1 if use_cuda_graph else 0, int(wait_timeout_ms), 1 if fuse_same_graph else 0)
    sts = (ctypes.c_int * nq)()
    stats = (fg_stats * nq)()
    bst = fg_batch_stats()
    st = load().fg_run_batch(arr, nq, ctypes.byref(opt), sts, stats, ctypes.byref(bst))
    return st, list(sts), list(stats), bst


def fg_autotune(g, algo, src=0):
    """Returns (status, best mode, [ms per mode, indexed by mode; index FG_AUTO unused])."""
    best = ctypes.c_int(-1)
    times = (ctypes.c_float * 7)()
    st = load().fg_autotune(g, int(algo), int(src), ctypes.byref(best), times)
    return st, best.value, list(times)


def fg_server_create(hbm_budget_bytes=0, max_inflight=0, max_wave=0, one_at_a_time=False, wait_timeout_ms=0,
                     exclusive_edges=0, no_fusion=False):
    """Returns (status, server handle)."""
    o = fg_server_options(int(hbm_budget_bytes), int(max_inflight), int(max_wave), 1 if one_at_a_time else 0,
                          int(wait_timeout_ms), int(exclusive_edges), 1 if no_fusion else 0)
    h = _VP()
    st = load().fg_server_create(ctypes.byref(o), ctypes.byref(h))
    return st, (h.value if st == FG_OK else None)


def fg_server_submit(server, g, algo, src, out, mode=FG_AUTO):
    """Returns (status, ticket).  out must stay alive until the request completes."""
    _check_dtype(out, "int32")
    q = fg_query(g, int(algo), int(src), _ptr(out), int(mode))
    t = ctypes.c_uint64(0)
    st = load().fg_server_submit(server, ctypes.byref(q), ctypes.byref(t))
    return st, t.value


def fg_server_poll(server, cap=4096):
    """Returns a list of completions (ticket, status, wave_size, latency_ms)."""
    buf = (fg_completion * cap)()
    n = load().fg_server_poll(server, buf, cap)
    return [(c.ticket, c.status, c.wave_size, c.latency_ms) for c in buf[:n]]


def fg_server_drain(server, timeout_ms=0):
    return load().fg_server_drain(server, int(timeout_ms))


def fg_server_destroy(server):
    return load().fg_server_destroy(server)


FG_NOALLOC_MAX_VERTICES = 1048576


def fg_sssp_csr_noalloc(n, row_off, col, w, src, dist_out, stream=None):
    """SSSP from a caller-owned device CSR without any device allocation (see include/fg.h).

    For callers that cannot allocate device memory; all arrays must be CUDA
    tensors.  Returns the status code."""
    _check_dtype(row_off, "int64")
    _check_dtype(col, "int32")
    _check_dtype(w, "int32")
    _check_dtype(dist_out, "int32")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return load().fg_sssp_csr_noalloc(int(n), _len(col), _ptr(row_off), _ptr(col), _ptr(w), int(src),
                                      _ptr(dist_out), stream)


def fg_kernel_launches() -> int:
    return int(load().fg_kernel_launches())


def fg_last_error() -> str:
    r = load().fg_last_error()
    return r.decode() if r else ""


def fg_status_string(status: int) -> str:
    r = load().fg_status_string(int(status))
    return r.decode() if r else ""
