"""Helpers of the GPU tests: create graphs through the C ABI and run queries."""
from __future__ import annotations

import contextlib

import numpy as np

import paper_1903_01665_gb300 as fg

MODES = [fg.FG_VERTEX_SYNC, fg.FG_VERTEX_ASYNC, fg.FG_EDGE_SYNC, fg.FG_EDGE_ASYNC, fg.FG_PULL, fg.FG_BUCKET]
MODE_IDS = ["vertex_sync", "vertex_async", "edge_sync", "edge_async", "pull", "bucket"]
ALGOS = {"sssp": fg.FG_ALGO_SSSP, "bfs": fg.FG_ALGO_BFS, "cc": fg.FG_ALGO_CC}


def to_csr(g):
    """Host CSR (int64 offsets) of a graphgen.Graph, stable by input order."""
    order = np.argsort(g.src, kind="stable")
    deg = np.bincount(g.src, minlength=g.n).astype(np.int64)
    row_off = np.zeros(g.n + 1, np.int64)
    np.cumsum(deg, out=row_off[1:])
    return row_off, g.dst[order].copy(), g.w[order].copy()


@contextlib.contextmanager
def graph_handle(g, kind="coo", where="host", weights=True, flags=0):
    """Create a device graph from a graphgen.Graph (creation flags: e.g.
    FG_GRAPH_RELABEL, FG_GRAPH_KEEP_IDS); destroyed on exit."""
    import torch
    w = g.w if weights else None
    if kind == "coo":
        arrs = [g.src, g.dst, w]
    else:
        arrs = list(to_csr(g))
        if not weights:
            arrs[2] = None
    if where == "device":
        arrs = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    if kind == "coo":
        st, h = fg.fg_graph_create_coo(g.n, *arrs, flags=flags)
    else:
        st, h = fg.fg_graph_create_csr(g.n, *arrs, flags=flags)
    fg.check(st)
    try:
        yield h
    finally:
        fg.check(fg.fg_graph_destroy(h))


def make_out(n, where, fill=-7):
    """An int32[n] output: "device" (torch CUDA), "host" (pageable numpy) or
    "pinned" (page-locked torch CPU tensor)."""
    import torch
    if where == "device":
        return torch.full((n,), fill, dtype=torch.int32, device="cuda")
    if where == "pinned":
        return torch.full((n,), fill, dtype=torch.int32).pin_memory()
    return np.full(n, fill, np.int32)


def as_numpy(out):
    return out.cpu().numpy() if hasattr(out, "cpu") else out


def run(h, n, algo, src, mode, where="device", **kw):
    """Run one query; returns (result as numpy int32[n], stats)."""
    out = make_out(n, where)
    st, stats = fg.fg_run(h, algo, int(src), out, mode, **kw)
    fg.check(st)
    return as_numpy(out), stats
