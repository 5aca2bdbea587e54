"""Error paths on the GPU, none of which faults or hangs the device: invalid
inputs rejected at creation, the overflow rule, the round cap, and a bounded
device-side wait that is made to run out (a CTA that never arrives at the
grid barrier), after which the context must still be usable."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import ALGOS, MODES, as_numpy, graph_handle, make_out, run

# host outputs: pageable numpy arrays and page-locked tensors
HOST_OUTS = ["host", "pinned"]

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("where", ["host", "device"])
def test_create_rejects_bad_inputs(where):
    import torch

    def put(a):
        a = np.asarray(a, np.int32)
        return torch.from_numpy(a).cuda() if where == "device" else a

    st, h = fg.fg_graph_create_coo(3, put([0, 1]), put([1, 3]), put([1, 1]))
    assert st == fg.FG_ERR_INVALID_ARG and h is None
    st, h = fg.fg_graph_create_coo(3, put([0, -1]), put([1, 2]), put([1, 1]))
    assert st == fg.FG_ERR_INVALID_ARG
    st, h = fg.fg_graph_create_coo(3, put([0, 1]), put([1, 2]), put([1, -5]))
    assert st == fg.FG_ERR_NEGATIVE_WEIGHT and "negative" in fg.fg_last_error()
    ro = np.array([0, 2, 1, 2], np.int64)       # decreasing offsets
    ro_t = torch.from_numpy(ro).cuda() if where == "device" else ro
    st, h = fg.fg_graph_create_csr(3, ro_t, put([1, 2]), None)
    assert st == fg.FG_ERR_INVALID_ARG
    ro = np.array([0, 1, 1, 3], np.int64)       # row_off[n] != m
    ro_t = torch.from_numpy(ro).cuda() if where == "device" else ro
    st, h = fg.fg_graph_create_csr(3, ro_t, put([1, 2]), None)
    assert st == fg.FG_ERR_INVALID_ARG


def test_query_argument_errors():
    g = gg.path(5)
    with graph_handle(g) as h:
        out = np.full(5, 99, np.int32)
        assert fg.fg_sssp(h, 5, out) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_bfs(h, -1, out) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_sssp(h, 0, out, 9) == fg.FG_ERR_INVALID_ARG
        assert np.all(out == 99)


@pytest.mark.parametrize("out_where", HOST_OUTS)
@pytest.mark.parametrize("mode", MODES)
def test_overflow_rule(mode, out_where):
    g = gg.path(3, weights=[2**30, 2**30])
    with graph_handle(g) as h:
        out = make_out(3, out_where, 99)
        st, _ = fg.fg_run(h, fg.FG_ALGO_SSSP, 0, out, mode)
        assert st == fg.FG_ERR_OVERFLOW
        assert np.all(as_numpy(out) == 99), "outputs must be untouched on error"
        st, _ = fg.fg_run(h, fg.FG_ALGO_BFS, 0, out, mode)   # BFS ignores weights
        assert st == fg.FG_OK and as_numpy(out).tolist() == [0, 1, 2]
    # dropped overflow candidates, correct result: the host's check clears it
    g = gg.Graph(3, [0, 0, 1], [1, 2, 2], [1, 1, 2**31 - 1], "shadowed")
    with graph_handle(g) as h:
        got, _ = run(h, 3, fg.FG_ALGO_SSSP, 0, mode, where=out_where)
        assert got.tolist() == [0, 1, 1]
    g = gg.path(3, weights=[2**31 - 2, 0])
    with graph_handle(g) as h:
        got, _ = run(h, 3, fg.FG_ALGO_SSSP, 0, mode, where=out_where)
        assert got.tolist() == [0, 2**31 - 2, 2**31 - 2]


@pytest.mark.parametrize("out_where", HOST_OUTS)
@pytest.mark.parametrize("mode", MODES)
def test_round_cap_returns_timeout(mode, out_where):
    g = gg.path(200)
    with graph_handle(g) as h:
        out = make_out(200, out_where, 99)
        st, _ = fg.fg_run(h, fg.FG_ALGO_SSSP, 0, out, mode, max_rounds=5)
        assert st == fg.FG_ERR_TIMEOUT and "round cap" in fg.fg_last_error()
        assert np.all(as_numpy(out) == 99)
        # the same graph with the default cap converges
        got, st = run(h, 200, fg.FG_ALGO_SSSP, 0, mode, where=out_where)
        assert got.tolist() == list(range(200))


@pytest.mark.parametrize("out_where", HOST_OUTS)
@pytest.mark.parametrize("mode", MODES)
def test_missing_arrival_times_out_and_context_survives(mode, out_where):
    g = gg.rmat(12)
    _, d = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    with graph_handle(g) as h:
        out = make_out(g.n, out_where, 99)
        st, _ = fg.fg_run(h, fg.FG_ALGO_SSSP, 0, out, mode, wait_timeout_ms=50, inject_missing_arrival=1)
        assert st == fg.FG_ERR_TIMEOUT and "timeout" in fg.fg_last_error()
        assert np.all(as_numpy(out) == 99)
        got, _ = run(h, g.n, fg.FG_ALGO_SSSP, 0, mode, where=out_where)
        np.testing.assert_array_equal(got, d)
