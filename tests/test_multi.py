"""The multi-source sweep (fg_run_multi) against the CPU oracle, bit for bit.

Up to eight SSSP or BFS queries on one graph run as one fixpoint whose rows
hold the eight values of a vertex; every slot must equal the oracle's result
for its source (Dijkstra, FIFO BFS), whatever the other slots hold: repeated
sources, sources without out-edges, unreachable parts, zero weights,
self-loops and duplicate edges, hubs that take the CTA path, fewer than
eight slots, near-far widths from 1 to INT32_MAX.  CC has no source and is
computed once for all outputs.  An overflow in one slot fails that slot
only, and leaves its output untouched.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import as_numpy, graph_handle, make_out
from tests.test_parity_small import WL

pytestmark = pytest.mark.gpu


def _want(g, algo, s):
    if algo == fg.FG_ALGO_SSSP:
        rc, r = oracle.sssp(g.n, g.src, g.dst, g.w, s)
    elif algo == fg.FG_ALGO_BFS:
        rc, r = oracle.bfs(g.n, g.src, g.dst, s)
    else:
        rc, r = oracle.cc(g.n, g.src, g.dst)
    assert rc == oracle.OK
    return r


def _sources(g, k, seed):
    """k sources: seeded ones with out-edges, a repeat, and a vertex without
    out-edges when the graph has one."""
    if g.m == 0:
        return [0] * k
    s = [int(x) for x in gg.sources(g, min(k, 6), seed=seed)]
    deg = np.bincount(g.src, minlength=g.n)
    zero = np.flatnonzero(deg == 0)
    if zero.size:
        s.append(int(zero[0]))
    s.append(s[0])   # a repeated source
    while len(s) < k:
        s.append(int(s[len(s) % max(1, len(s) - 1)]))
    return s[:k]


@pytest.mark.parametrize("name", sorted(WL))
@pytest.mark.parametrize("algo", [fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS])
def test_eight_sources_bit_exact(name, algo):
    g = WL[name]
    srcs = _sources(g, 8, seed=77)
    with graph_handle(g) as h:
        outs = [make_out(g.n, "device") for _ in srcs]
        st, sts, stats = fg.fg_run_multi(h, algo, srcs, outs)
        assert st == fg.FG_OK, fg.fg_last_error()
        assert sts == [fg.FG_OK] * len(srcs)
    for s, o in zip(srcs, outs):
        got = as_numpy(o)
        want = _want(g, algo, s)
        if not np.array_equal(got, want):
            bad = np.flatnonzero(got != want)
            raise AssertionError(f"{name} algo {algo} source {s}: {bad.size} mismatches, first v={bad[0]} "
                                 f"got={got[bad[0]]} want={want[bad[0]]}")
    assert stats.rounds >= 1 and stats.mode == -1


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_fewer_slots_and_mixed_outputs(k):
    """k < 8 slots (the others stay INF and idle); outputs in device,
    pageable host and pinned host memory."""
    g = gg.rmat(14, seed=41)
    srcs = [int(x) for x in gg.sources(g, k, seed=42)]
    wheres = ["device", "host", "pinned"]
    with graph_handle(g) as h:
        for algo in (fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS):
            outs = [make_out(g.n, wheres[j % 3]) for j in range(k)]
            st, sts, _ = fg.fg_run_multi(h, algo, srcs, outs)
            assert st == fg.FG_OK, fg.fg_last_error()
            for s, o in zip(srcs, outs):
                np.testing.assert_array_equal(as_numpy(o), _want(g, algo, s))


@pytest.mark.parametrize("delta", [1, 3, 40, 1000, 2**30, 2**31 - 1])
@pytest.mark.parametrize("name", ["grid", "rmat", "zero_weights", "heavy_path"])
def test_near_far_widths_bit_exact(name, delta):
    """The SSSP sweep's shared near-far order at widths from 1 (a split after
    nearly every value) to INT32_MAX (nothing is ever far): every slot is the
    oracle's.  Zero-weight edges keep a lowering at its source's value; the
    heavy path puts each vertex in an epoch of its own."""
    if name == "grid":
        g = gg.grid(96, seed=61)
    elif name == "rmat":
        g = gg.rmat(13, seed=62)
    elif name == "zero_weights":
        g = gg.rmat(11, seed=63)
        g = gg.Graph(g.n, g.src, g.dst, np.where(np.arange(g.m) % 3 == 0, 0, g.w).astype(np.int32), "zw")
    else:
        n = 300
        g = gg.Graph(n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32),
                     np.full(n - 1, 7_000_000, np.int32), "heavy_path")
    srcs = _sources(g, 8, seed=64)
    with graph_handle(g) as h:
        outs = [make_out(g.n, "device") for _ in srcs]
        st, sts, stats = fg.fg_run_multi(h, fg.FG_ALGO_SSSP, srcs, outs, delta=delta)
        assert st == fg.FG_OK, fg.fg_last_error()
    for s, o in zip(srcs, outs):
        np.testing.assert_array_equal(as_numpy(o), _want(g, fg.FG_ALGO_SSSP, s), err_msg=f"{name} delta {delta} src {s}")


def test_cc_is_computed_once_for_every_output():
    g = gg.disjoint_cliques([40, 1, 70, 3, 1, 33, 2], seed=5)
    want = _want(g, fg.FG_ALGO_CC, 0)
    with graph_handle(g) as h:
        outs = [make_out(g.n, w) for w in ("device", "host", "pinned", "device")]
        before = fg.fg_kernel_launches()
        st, sts, _ = fg.fg_run_multi(h, fg.FG_ALGO_CC, None, outs)
        assert st == fg.FG_OK, fg.fg_last_error()
        assert fg.fg_kernel_launches() - before <= 2   # one fixpoint (and at most a diameter probe)
    for o in outs:
        np.testing.assert_array_equal(as_numpy(o), want)


def test_cc_on_a_lazy_graph_builds_its_symmetrised_view():
    import torch
    g = gg.rmat(10, seed=43)
    st, h = fg.fg_graph_create_coo(g.n, g.src, g.dst, g.w, flags=fg.FG_GRAPH_LAZY)
    fg.check(st)
    try:
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(2)]
        fg.check(fg.fg_run_multi(h, fg.FG_ALGO_CC, None, outs)[0])
        for o in outs:
            np.testing.assert_array_equal(as_numpy(o), _want(g, fg.FG_ALGO_CC, 0))
    finally:
        fg.check(fg.fg_graph_destroy(h))


def test_overflow_fails_only_its_own_slot():
    """0 -> 1 -> 2 (2^31 - 2, then 5) and 3 -> 4: a source 0 overflows at
    vertex 2; sources 1 and 3 do not.  The failing output is untouched, the
    others are the oracle's."""
    big = 2**31 - 2
    g = gg.Graph(5, [0, 1, 3], [1, 2, 4], [big, 5, 8], "overflow5")
    with graph_handle(g) as h:
        outs = [make_out(g.n, "device", fill=-9) for _ in range(3)]
        st, sts, _ = fg.fg_run_multi(h, fg.FG_ALGO_SSSP, [0, 1, 3], outs)
        assert st == fg.FG_ERR_OVERFLOW
        assert sts == [fg.FG_ERR_OVERFLOW, fg.FG_OK, fg.FG_OK]
        assert (as_numpy(outs[0]) == -9).all()
        for s, o in zip([1, 3], outs[1:]):
            np.testing.assert_array_equal(as_numpy(o), _want(g, fg.FG_ALGO_SSSP, s))
        rc, _ = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
        assert rc == oracle.OVERFLOW
        # the same with a width of 1: vertex 1 waits far until the threshold reaches INF
        outs = [make_out(g.n, "device", fill=-9) for _ in range(3)]
        st, sts, _ = fg.fg_run_multi(h, fg.FG_ALGO_SSSP, [0, 1, 3], outs, delta=1)
        assert sts == [fg.FG_ERR_OVERFLOW, fg.FG_OK, fg.FG_OK]
        for s, o in zip([1, 3], outs[1:]):
            np.testing.assert_array_equal(as_numpy(o), _want(g, fg.FG_ALGO_SSSP, s))
        # BFS on the same graph cannot overflow
        outs = [make_out(g.n, "device") for _ in range(3)]
        fg.check(fg.fg_run_multi(h, fg.FG_ALGO_BFS, [0, 1, 3], outs)[0])
        for s, o in zip([0, 1, 3], outs):
            np.testing.assert_array_equal(as_numpy(o), _want(g, fg.FG_ALGO_BFS, s))


def test_round_cap_and_argument_errors():
    g = gg.path(100, weights=np.ones(99, np.int32))
    with graph_handle(g) as h:
        outs = [make_out(g.n, "device", fill=-4) for _ in range(2)]
        st, sts, _ = fg.fg_run_multi(h, fg.FG_ALGO_SSSP, [0, 5], outs, max_rounds=3)
        assert st == fg.FG_ERR_TIMEOUT and sts == [fg.FG_ERR_TIMEOUT] * 2
        assert all((as_numpy(o) == -4).all() for o in outs)
        before = fg.fg_kernel_launches()
        assert fg.fg_run_multi(h, fg.FG_ALGO_SSSP, [], [])[0] == fg.FG_ERR_INVALID_ARG
        nine = [make_out(g.n, "device") for _ in range(9)]
        assert fg.fg_run_multi(h, fg.FG_ALGO_SSSP, list(range(9)), nine)[0] == fg.FG_ERR_INVALID_ARG
        assert fg.fg_run_multi(h, fg.FG_ALGO_SSSP, [0, g.n], outs)[0] == fg.FG_ERR_INVALID_ARG
        assert fg.fg_run_multi(h, fg.FG_ALGO_BFS, [-1, 0], outs)[0] == fg.FG_ERR_INVALID_ARG
        assert fg.fg_run_multi(h, 7, [0, 1], outs)[0] == fg.FG_ERR_INVALID_ARG
        assert fg.fg_kernel_launches() == before


@pytest.mark.slow
@pytest.mark.parametrize("wl", ["rmat22", "grid4096"])
def test_full_size_eight_seeded_sources_bit_exact(wl):
    """The benchmark workloads at full size, the eight seeded sources of the
    benchmark in one sweep per algorithm, every slot against the oracle."""
    g = gg.rmat(22) if wl == "rmat22" else gg.grid(4096)
    srcs = [int(s) for s in gg.sources(g, 8)]
    with graph_handle(g, where="device") as h:
        for algo in (fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS):
            outs = [make_out(g.n, "device") for _ in srcs]
            st, sts, stats = fg.fg_run_multi(h, algo, srcs, outs)
            assert st == fg.FG_OK, fg.fg_last_error()
            for s, o in zip(srcs, outs):
                got = as_numpy(o)
                want = _want(g, algo, s)
                if not np.array_equal(got, want):
                    bad = np.flatnonzero(got != want)
                    raise AssertionError(f"{wl} algo {algo} source {s}: {bad.size} mismatches")
