"""The multi-core CPU baseline (oracle/omp.py) against the oracle, bit for bit.

The baseline is only reported beside the sequential oracle's figure, but a
baseline that computes something else would make that figure meaningless:
every output must be the oracle's, for any thread count, including the
error statuses (invalid ids, a negative weight, an overflowing distance).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import omp

pytestmark = pytest.mark.skipif(omp.build() is None, reason="no OpenMP in the host compiler")


def _same(g, s):
    rc, want = oracle.sssp(g.n, g.src, g.dst, g.w, s)
    rc2, got = omp.sssp(g.n, g.src, g.dst, g.w, s)
    assert rc2 == rc
    assert np.array_equal(got, want)
    rc, want = oracle.bfs(g.n, g.src, g.dst, s)
    rc2, got = omp.bfs(g.n, g.src, g.dst, s)
    assert rc2 == rc == oracle.OK
    assert np.array_equal(got, want)


def _same_cc(g):
    rc, want = oracle.cc(g.n, g.src, g.dst)
    rc2, got = omp.cc(g.n, g.src, g.dst)
    assert rc2 == rc == oracle.OK
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", range(16))
def test_small_random_graphs(seed):
    rng = np.random.Generator(np.random.PCG64(500 + seed))
    n = int(rng.integers(1, 200))
    m = int(rng.integers(0, 6 * n))
    g = gg.random_small(n, m, seed=900 + seed, wlo=0, whi=40)   # zero weights included
    for s in {0, n - 1, n // 3}:
        _same(g, s)
    _same_cc(g)


@pytest.mark.parametrize("threads", [1, 2, 7])
def test_rmat_any_thread_count(threads):
    before = omp.threads()
    omp.set_threads(threads)
    try:
        assert omp.threads() == threads
        g = gg.rmat(13)
        for s in gg.sources(g, 3):
            _same(g, int(s))
        _same_cc(g)
    finally:
        omp.set_threads(before)


def test_repeated_runs_on_a_skewed_graph():
    """Many threads on a hub-heavy graph, five times: the atomic minimum,
    the claims and the union-find hooks give the same result every time."""
    g = gg.rmat(14)
    s = int(gg.sources(g, 1)[0])
    for _ in range(5):
        _same(g, s)
        _same_cc(g)
    _same(gg.hub(5000, 3000, 20000), 0)


def test_grid_and_uniform_graphs():
    g = gg.grid(96)
    for s in gg.sources(g, 2):
        _same(g, int(s))
    _same_cc(g)
    g = gg.er()
    _same(g, 0)
    _same_cc(g)


def test_closed_form_graphs():
    for g in (gg.path(50, weights=np.arange(49, dtype=np.int32)), gg.cycle(33), gg.star(40),
              gg.complete(12), gg.full_grid(9, 13), gg.disjoint_cliques([3, 1, 5, 2])):
        _same(g, 0)
        _same_cc(g)


def test_unit_weights_are_bfs_levels():
    g = gg.rmat(11)
    s = int(gg.sources(g, 1)[0])
    rc, d = omp.sssp(g.n, g.src, g.dst, None, s)
    assert rc == omp.OK
    assert np.array_equal(d, oracle.bfs(g.n, g.src, g.dst, s)[1])


def test_single_vertex_and_no_edges():
    e = np.zeros(0, np.int32)
    assert omp.sssp(1, e, e, e, 0)[1].tolist() == [0]
    assert omp.bfs(1, e, e, 0)[1].tolist() == [0]
    assert omp.cc(1, e, e)[1].tolist() == [0]
    rc, d = omp.sssp(4, e, e, e, 2)
    assert rc == omp.OK and d.tolist() == [oracle.UNREACHED, oracle.UNREACHED, 0, oracle.UNREACHED]
    assert omp.cc(4, e, e)[1].tolist() == [0, 1, 2, 3]


def test_error_statuses_match_the_oracle():
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    assert omp.sssp(3, src, dst, np.array([1, -1], np.int32), 0)[0] == omp.NEGATIVE_WEIGHT
    assert omp.sssp(3, src, dst, np.array([1, 1], np.int32), 3)[0] == omp.INVALID
    assert omp.bfs(2, src, dst, 0)[0] == omp.INVALID          # id 2 out of range
    assert omp.cc(2, src, dst)[0] == omp.INVALID


def test_overflow_matches_the_oracle():
    """A reachable distance of exactly INT32_MAX overflows; one below does not."""
    big = np.int32(2**31 - 1 - 5)
    g_src = np.array([0, 1], np.int32)
    g_dst = np.array([1, 2], np.int32)
    for w2, status in ((5, oracle.OVERFLOW), (4, oracle.OK)):
        w = np.array([big, w2], np.int32)
        rc, want = oracle.sssp(3, g_src, g_dst, w, 0)
        rc2, got = omp.sssp(3, g_src, g_dst, w, 0)
        assert rc == status and rc2 == rc
        assert np.array_equal(got, want)


def test_graph_handle_serves_many_queries():
    """One adjacency, many queries (the form the benchmark times): every
    result is the oracle's; a bad source is rejected without touching it."""
    g = gg.rmat(12)
    with omp.Graph(g.n, g.src, g.dst, g.w) as h:
        assert h.status == omp.OK
        for s in gg.sources(g, 4):
            rc, d = h.sssp(int(s))
            assert rc == omp.OK and np.array_equal(d, oracle.sssp(g.n, g.src, g.dst, g.w, int(s))[1])
            rc, lv = h.bfs(int(s))
            assert rc == omp.OK and np.array_equal(lv, oracle.bfs(g.n, g.src, g.dst, int(s))[1])
        assert h.sssp(g.n)[0] == omp.INVALID
        assert h.bfs(-1)[0] == omp.INVALID
    bad = omp.Graph(3, np.array([0], np.int32), np.array([1], np.int32), np.array([-2], np.int32))
    assert bad.status == omp.NEGATIVE_WEIGHT
    bad.close()
