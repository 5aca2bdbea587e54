"""The allocation-free SSSP entry point, for callers that cannot allocate
device memory (their memory belongs to another allocator, or an allocation's
implicit synchronisation is not acceptable where they run).

It is checked through the C ABI against the ordinary entry point (graph
handle + fg_sssp, vertex-sync), exactly, on two calls in a row -- the second
call reuses the shared scratch array left behind by the first.  This file is
collected last on purpose, and passes alone in a fresh process too.
"""
import numpy as np
import pytest

import graphgen as gg
import paper_1903_01665_gb300 as fg
from tests.gpu_util import graph_handle, run, to_csr

pytestmark = pytest.mark.gpu


def _device_csr(g):
    import torch
    row_off, col, w = to_csr(g)
    return (torch.from_numpy(row_off).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(w).cuda())


def test_noalloc_matches_fg_sssp_on_two_consecutive_calls():
    import torch
    g = gg.rmat(16, seed=31)
    srcs = [int(s) for s in gg.sources(g, 2, seed=32)]
    row_off, col, w = _device_csr(g)
    with graph_handle(g) as h:
        want = [run(h, g.n, fg.FG_ALGO_SSSP, s, fg.FG_VERTEX_SYNC)[0] for s in srcs]
    for s, exp in zip(srcs, want):
        out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
        fg.check(fg.fg_sssp_csr_noalloc(g.n, row_off, col, w, s, out))
        np.testing.assert_array_equal(out.cpu().numpy(), exp)


def test_noalloc_matches_on_a_second_graph_after_the_first():
    import torch
    g = gg.grid(300, seed=33)
    row_off, col, w = _device_csr(g)
    with graph_handle(g) as h:
        exp = run(h, g.n, fg.FG_ALGO_SSSP, 7, fg.FG_VERTEX_SYNC)[0]
    for _ in range(2):
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        fg.check(fg.fg_sssp_csr_noalloc(g.n, row_off, col, w, 7, out))
        np.testing.assert_array_equal(out.cpu().numpy(), exp)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    n = fg.FG_NOALLOC_MAX_VERTICES + 1
    row_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = fg.fg_sssp_csr_noalloc(n, row_off, col[:0], None, 0, out)
    assert st == fg.FG_ERR_INVALID_ARG and "FG_NOALLOC_MAX_VERTICES" in fg.fg_last_error()
