"""GPU parity of the all-active relaxation round (fg_sweep) against the
oracle's double-buffered round, bit for bit, in both variants: the vertex
variant of Alg. 1 over the degree buckets and the edge variant of Alg. 2 over
the staged edge stream.

States cover a source's first rounds, random finite values with unreached
vertices mixed in, next already below cur, ragged edge counts around the
1024-edge tile (and below 4 edges), overflow, and -- at the benchmark's size
-- the R-MAT scale-22 state the benchmark times.  The update count depends
on the schedule, so only its bounds are checked.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import graph_handle

pytestmark = pytest.mark.gpu

INF = oracle.UNREACHED
SWEEP_MODES = [(fg.FG_VERTEX_SYNC, "vertex"), (fg.FG_EDGE_SYNC, "edge")]


def gpu_sweep(h, mode, cur, nxt):
    import torch
    c = torch.from_numpy(np.ascontiguousarray(cur, np.int32)).cuda()
    x = torch.from_numpy(np.ascontiguousarray(nxt, np.int32)).cuda()
    st, upd, ms = fg.fg_sweep(h, mode, c, x)
    return st, x.cpu().numpy(), upd, ms


def check(g, h, cur, nxt, expect_status=oracle.OK):
    rc, want, lowered = oracle.sweep(g.n, g.src, g.dst, g.w, cur, nxt)
    assert rc == expect_status
    n_cand = 0
    if g.m:
        cu = np.asarray(cur, np.int64)[g.src]
        n_cand = int(np.count_nonzero(cu != INF))
    for mode, name in SWEEP_MODES:
        st, got, upd, _ = gpu_sweep(h, mode, cur, nxt)
        want_st = fg.FG_OK if expect_status == oracle.OK else fg.FG_ERR_OVERFLOW
        assert st == want_st, (name, st, fg.fg_last_error())
        if not np.array_equal(got, want):
            bad = np.flatnonzero(got != want)
            raise AssertionError(f"{name}: {bad.size} mismatches, v={bad[0]} got={got[bad[0]]} want={want[bad[0]]}")
        assert lowered <= upd <= n_cand, (name, lowered, upd, n_cand)


def first_rounds(g, s, k):
    cur = np.full(g.n, INF, np.int32)
    cur[s] = 0
    for _ in range(k):
        rc, cur, _ = oracle.sweep(g.n, g.src, g.dst, g.w, cur, cur)
        assert rc == oracle.OK
    return cur


GRAPHS = {
    "er_16k": lambda: gg.er(16384, 131072, seed=11),
    "rmat_12": lambda: gg.rmat(12, seed=12),
    "grid_64": lambda: gg.grid(64, seed=13),
    "self_loops_dups_zero_w": lambda: gg.random_small(300, 2500, seed=14, wlo=0, whi=20),
    "star_3000": lambda: gg.star(3000, weights=(np.arange(2999) * 31) % 1000 + 1),
    "m_1": lambda: gg.Graph(3, [0], [2], [5], "m1"),
    "m_3": lambda: gg.Graph(4, [0, 0, 2], [1, 3, 3], [1, 2, 3], "m3"),
    "no_edges": lambda: gg.Graph(10, [], [], [], "empty10"),
}
for _m in (1024, 1025, 1027, 2048 + 3, 4095):
    GRAPHS[f"ragged_m_{_m}"] = (lambda m: lambda: gg.random_small(700, m, seed=m, wlo=0, whi=50))(_m)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_sweep_states(name):
    g = GRAPHS[name]()
    rng = np.random.Generator(np.random.PCG64(99))
    with graph_handle(g) as h:
        s = int(g.src[0]) if g.m else 0
        # the source's first three rounds (Jacobi: next starts as cur)
        cur = first_rounds(g, s, 0)
        for _ in range(3):
            check(g, h, cur, cur)
            _, cur, _ = oracle.sweep(g.n, g.src, g.dst, g.w, cur, cur)
        # random finite values, a quarter unreached; next is cur or below it
        cur = rng.integers(0, 1 << 20, g.n).astype(np.int32)
        cur[rng.random(g.n) < 0.25] = INF
        check(g, h, cur, cur)
        nxt = np.minimum(cur, rng.integers(0, 1 << 20, g.n).astype(np.int32))
        check(g, h, cur, nxt)


def test_sweep_overflow_applies_the_other_edges():
    big = 2**31 - 1
    g = gg.Graph(5, [0, 0, 1, 3], [1, 2, 4, 4], [10, 1, 7, 2], "of")
    with graph_handle(g) as h:
        cur = np.array([big - 5, INF, INF, 4, INF], np.int32)
        check(g, h, cur, cur, expect_status=oracle.OVERFLOW)


def test_sweep_rejects_bad_arguments():
    import torch
    g = gg.rmat(8, seed=3)
    with graph_handle(g) as h:
        c = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        assert fg.fg_sweep(h, fg.FG_VERTEX_ASYNC, c, c.clone())[0] == fg.FG_ERR_INVALID_ARG
        assert fg.fg_sweep(h, fg.FG_EDGE_SYNC, np.zeros(g.n, np.int32), c)[0] == fg.FG_ERR_INVALID_ARG


def bench_state(g, s, k=3):
    """The benchmark's timed state: k rounds from s, then every vertex still
    unreached set to 2^30 so that every vertex and edge is active."""
    cur = first_rounds(g, s, k)
    cur[cur == INF] = 1 << 30
    return cur


def test_sweep_rmat22_benchmark_state():
    g = gg.rmat(22)
    s = int(gg.sources(g, 1)[0])
    cur = bench_state(g, s)
    with graph_handle(g) as h:
        check(g, h, cur, cur)
