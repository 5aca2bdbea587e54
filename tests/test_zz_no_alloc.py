"""The allocation-free SSSP entry point, for callers that cannot allocate
device memory (their memory belongs to another allocator, or an allocation's
implicit synchronisation is not acceptable where they run).

It is checked through the C ABI against the CPU oracle (Dijkstra) and against
the ordinary entry point (graph handle + fg_sssp, vertex-sync), exactly, on
two calls in a row -- the second call reuses the shared scratch array left
behind by the first.  Its error paths are exercised too: pointers that are
not this device's memory and sizes beyond its limits are rejected on the
host before any launch; an invalid CSR (decreasing offsets, an id >= n) and a
negative weight are rejected by the kernel's validation pass, which runs
before any indexed access; a finite distance >= INT32_MAX is reported as an
overflow.  The fixed round cap (n + 2) cannot be reached by valid input --
a synchronous round count never exceeds n + 1 -- so it has no test here.
This file is collected last on purpose, and passes alone in a fresh process
too.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import graph_handle, run, to_csr

pytestmark = pytest.mark.gpu


def _device_csr(g, weights=True):
    import torch
    row_off, col, w = to_csr(g)
    return (torch.from_numpy(row_off).cuda(), torch.from_numpy(col).cuda(),
            torch.from_numpy(w).cuda() if weights else None)


def _dev(a, dtype):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def test_noalloc_matches_oracle_and_fg_sssp_on_two_consecutive_calls():
    import torch
    g = gg.rmat(16, seed=31)
    srcs = [int(s) for s in gg.sources(g, 2, seed=32)]
    row_off, col, w = _device_csr(g)
    with graph_handle(g) as h:
        lib = [run(h, g.n, fg.FG_ALGO_SSSP, s, fg.FG_VERTEX_SYNC)[0] for s in srcs]
    for s, exp in zip(srcs, lib):
        rc, want = oracle.sssp(g.n, g.src, g.dst, g.w, s)
        assert rc == oracle.OK
        out = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
        fg.check(fg.fg_sssp_csr_noalloc(g.n, row_off, col, w, s, out))
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(got, exp)


def test_noalloc_matches_oracle_on_a_second_graph_after_the_first():
    import torch
    g = gg.grid(300, seed=33)
    row_off, col, w = _device_csr(g)
    rc, want = oracle.sssp(g.n, g.src, g.dst, g.w, 7)
    assert rc == oracle.OK
    for _ in range(2):
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        fg.check(fg.fg_sssp_csr_noalloc(g.n, row_off, col, w, 7, out))
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_noalloc_unit_weights_equal_bfs_levels():
    """w = NULL means unit weights: the distances are the oracle's BFS levels."""
    import torch
    g = gg.rmat(10, seed=34)
    s = int(gg.sources(g, 1, seed=35)[0])
    row_off, col, _ = _device_csr(g, weights=False)
    rc, want = oracle.bfs(g.n, g.src, g.dst, s)
    assert rc == oracle.OK
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    fg.check(fg.fg_sssp_csr_noalloc(g.n, row_off, col, None, s, out))
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    n = fg.FG_NOALLOC_MAX_VERTICES + 1
    row_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = fg.fg_sssp_csr_noalloc(n, row_off, col[:0], None, 0, out)
    assert st == fg.FG_ERR_INVALID_ARG and "FG_NOALLOC_MAX_VERTICES" in fg.fg_last_error()


def test_noalloc_rejects_host_memory_before_any_launch():
    """Host arrays are not this device's memory: rejected on the host, no kernel runs."""
    import torch
    g = gg.rmat(8, seed=36)
    row_off, col, w = to_csr(g)
    d_row, d_col, d_w = _device_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    before = fg.fg_kernel_launches()
    assert fg.fg_sssp_csr_noalloc(g.n, row_off, d_col, d_w, 0, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_sssp_csr_noalloc(g.n, d_row, d_col, d_w, 0, np.empty(g.n, np.int32)) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_sssp_csr_noalloc(g.n, d_row, col, d_w, 0, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_sssp_csr_noalloc(g.n, d_row, d_col, w, 0, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_sssp_csr_noalloc(g.n, d_row, d_col, d_w, g.n, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_sssp_csr_noalloc(g.n, d_row, d_col, d_w, -1, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_kernel_launches() == before
    assert "device memory" in fg.fg_last_error() or "source" in fg.fg_last_error()


@pytest.mark.parametrize("case", ["id_equal_n", "id_negative", "decreasing_offsets", "last_offset_not_m",
                                  "negative_weight"])
def test_noalloc_rejects_an_invalid_csr_in_its_validation_pass(case):
    """The kernel validates offsets, ids and weights before any indexed
    access, and returns FG_ERR_INVALID_ARG; a valid call afterwards still
    gives the oracle's result (the shared scratch is reset by every call)."""
    import torch
    n = 6
    row_off = [0, 2, 3, 5, 6, 7, 7]
    col = [1, 2, 3, 4, 0, 5, 2]
    w = [3, 1, 4, 1, 5, 9, 2]
    if case == "id_equal_n":
        col[3] = n
    elif case == "id_negative":
        col[0] = -1
    elif case == "decreasing_offsets":
        row_off[2], row_off[3] = 5, 3
    elif case == "last_offset_not_m":
        row_off[6] = 6
    else:
        w[5] = -2
    out = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    st = fg.fg_sssp_csr_noalloc(n, _dev(row_off, torch.int64), _dev(col, torch.int32), _dev(w, torch.int32), 0,
                                out)
    assert st == fg.FG_ERR_INVALID_ARG, fg.fg_status_string(st)
    assert "invalid CSR" in fg.fg_last_error()
    # the next valid call on the same scratch is exact
    good_row, good_col, good_w = [0, 2, 3, 5, 6, 7, 7], [1, 2, 3, 4, 0, 5, 2], [3, 1, 4, 1, 5, 9, 2]
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(good_row))
    rc, want = oracle.sssp(n, src, np.array(good_col, np.int32), np.array(good_w, np.int32), 0)
    assert rc == oracle.OK
    fg.check(fg.fg_sssp_csr_noalloc(n, _dev(good_row, torch.int64), _dev(good_col, torch.int32),
                                    _dev(good_w, torch.int32), 0, out))
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_noalloc_reports_overflow_and_not_a_shadowed_one():
    """0 -> 1 -> 2 with weights 2^31 - 2 and 5: vertex 2's distance is finite
    but >= INT32_MAX, so the call fails with FG_ERR_OVERFLOW (the oracle
    agrees).  Adding a short edge 0 -> 2 shadows the overflowing path: no
    error, and the result is the oracle's."""
    import torch
    big = 2**31 - 2
    n = 3
    src, dst, w = np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([big, 5], np.int32)
    rc, _ = oracle.sssp(n, src, dst, w, 0)
    assert rc == oracle.OVERFLOW
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = fg.fg_sssp_csr_noalloc(n, _dev([0, 1, 2, 2], torch.int64), _dev(dst, torch.int32), _dev(w, torch.int32),
                                0, out)
    assert st == fg.FG_ERR_OVERFLOW, fg.fg_status_string(st)
    src2, dst2, w2 = np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32), np.array([big, 7, 5], np.int32)
    rc, want = oracle.sssp(n, src2, dst2, w2, 0)
    assert rc == oracle.OK
    fg.check(fg.fg_sssp_csr_noalloc(n, _dev([0, 2, 3, 3], torch.int64), _dev(dst2, torch.int32),
                                    _dev(w2, torch.int32), 0, out))
    np.testing.assert_array_equal(out.cpu().numpy(), want)
