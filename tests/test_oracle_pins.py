"""Pins of the CPU oracle against references other than itself (no GPU needed).

SSSP (Alg. 1/2 fixpoint) is pinned by Floyd-Warshall, brute-force simple-path
enumeration, scipy.sparse.csgraph Dijkstra, closed forms (path prefix sums,
unit grid = Manhattan distance, star = edge weights) and the fixpoint
invariants.  BFS (Alg. 3) by brute force, scipy unweighted shortest paths,
closed forms (grid, directed cycle, complete graph) and invariants.  CC by
scipy weak components, DFS component counts, disjoint cliques and the
one-label-per-component invariants.  The Jacobi round count by path/star
closed forms and by its definition through hop counts.  The all-active round
(one double-buffered relaxation from a given state) by a hand example, by
hop-limited brute-force path enumeration after k rounds, and by iterating it
to the Floyd-Warshall distances in the hop-count number of rounds.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import pins

INF = oracle.UNREACHED


def _to_int64_dist(d):
    d = np.asarray(d, np.int64).copy()
    return d


# ---------------------------------------------------------------- SSSP
@pytest.mark.parametrize("seed", range(12))
def test_sssp_vs_floyd_warshall(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    n = int(rng.integers(2, 65))
    m = int(rng.integers(0, 4 * n))
    g = gg.random_small(n, m, seed=1000 + seed, wlo=0, whi=30)
    fw = pins.floyd_warshall(n, g.src, g.dst, g.w)
    for s in {0, n - 1, n // 2}:
        rc, dist = oracle.sssp(n, g.src, g.dst, g.w, s)
        assert rc == oracle.OK
        exp = np.where(fw[s] >= pins.BIG, INF, fw[s])
        np.testing.assert_array_equal(dist, exp)


@pytest.mark.parametrize("seed", range(20))
def test_sssp_bfs_vs_brute_force(seed):
    rng = np.random.Generator(np.random.PCG64(200 + seed))
    n = int(rng.integers(1, 9))
    m = int(rng.integers(0, 3 * n + 1))
    g = gg.random_small(n, m, seed=2000 + seed, wlo=0, whi=9)
    s = int(rng.integers(0, n))
    bw, bh = pins.brute_force_paths(n, g.src.tolist(), g.dst.tolist(), g.w.tolist(), s)
    rc, dist = oracle.sssp(n, g.src, g.dst, g.w, s)
    assert rc == oracle.OK
    assert dist.tolist() == [INF if x is None else x for x in bw]
    rc, level = oracle.bfs(n, g.src, g.dst, s)
    assert rc == oracle.OK
    assert level.tolist() == [INF if x is None else x for x in bh]


@pytest.mark.parametrize("which", ["er", "rmat"])
def test_sssp_bfs_vs_scipy(which):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    if which == "er":
        g = gg.er(3000, 24000, seed=31)
    else:
        g = gg.rmat(11, 8, seed=32)  # self-loops and duplicates present
    u, v, w = pins.dedup_min(g.n, g.src, g.dst, g.w)
    A = sp.csr_matrix((w.astype(np.float64), (u, v)), shape=(g.n, g.n))
    B = sp.csr_matrix((np.ones(u.size), (u, v)), shape=(g.n, g.n))
    for s in gg.sources(g, 3, seed=33):
        s = int(s)
        ref = csgraph.dijkstra(A, directed=True, indices=s)
        ref = np.where(np.isinf(ref), INF, ref).astype(np.int64)
        rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, s)
        assert rc == oracle.OK
        np.testing.assert_array_equal(dist, ref)
        refh = csgraph.shortest_path(B, directed=True, unweighted=True, indices=s)
        refh = np.where(np.isinf(refh), INF, refh).astype(np.int64)
        rc, level = oracle.bfs(g.n, g.src, g.dst, s)
        assert rc == oracle.OK
        np.testing.assert_array_equal(level, refh)


def test_sssp_path_prefix_sums():
    w = [5, 0, 7, 1, 1000, 3]
    g = gg.path(7, weights=w)
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.OK
    assert dist.tolist() == np.concatenate([[0], np.cumsum(w)]).tolist()
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 3)   # upstream vertices unreachable
    assert dist.tolist() == [INF, INF, INF, 0, 1, 1001, 1004]


def test_sssp_star_equals_edge_weights():
    w = np.array([9, 3, 0, 77, 12], np.int32)
    g = gg.star(6, weights=w)
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.OK
    assert dist.tolist() == [0] + w.tolist()
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 2)   # a leaf: nothing reachable
    assert dist.tolist() == [INF, INF, 0, INF, INF, INF]


@pytest.mark.parametrize("rows,cols,r0,c0", [(7, 9, 0, 0), (16, 5, 8, 2), (1, 12, 0, 11)])
def test_unit_grid_manhattan(rows, cols, r0, c0):
    g = gg.full_grid(rows, cols)
    s = r0 * cols + c0
    r, c = np.divmod(np.arange(rows * cols), cols)
    manhattan = np.abs(r - r0) + np.abs(c - c0)
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, s)
    assert rc == oracle.OK
    np.testing.assert_array_equal(dist, manhattan)
    rc, level = oracle.bfs(g.n, g.src, g.dst, s)
    np.testing.assert_array_equal(level, manhattan)
    rc, label = oracle.cc(g.n, g.src, g.dst)
    assert np.all(label == 0)


def test_unit_weights_sssp_equals_bfs():
    g = gg.rmat(10, 8, seed=41)
    ones = np.ones(g.m, np.int32)
    for s in gg.sources(g, 4, seed=42):
        _, d = oracle.sssp(g.n, g.src, g.dst, ones, int(s))
        _, l = oracle.bfs(g.n, g.src, g.dst, int(s))
        np.testing.assert_array_equal(d, l)


def test_sssp_invariants_medium():
    g = gg.rmat(14, 16, seed=43)
    for s in gg.sources(g, 2, seed=44):
        s = int(s)
        rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, s)
        assert rc == oracle.OK
        pins.check_sssp_invariants(g.n, g.src, g.dst, g.w, s, dist)
        _, level = oracle.bfs(g.n, g.src, g.dst, s)
        np.testing.assert_array_equal(dist == INF, level == INF)


def test_sssp_overflow_and_negative():
    g = gg.path(3, weights=[2**30, 2**30])            # dist[2] = 2^31 > INT32_MAX
    rc, _ = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.OVERFLOW
    g = gg.path(2, weights=[2**31 - 1])               # exactly INT32_MAX is not representable
    rc, _ = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.OVERFLOW
    g = gg.path(3, weights=[2**31 - 2, 0])             # largest finite distance
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.OK and dist.tolist() == [0, 2**31 - 2, 2**31 - 2]
    # an overflowing edge that does not decide any distance is not an error
    g = gg.Graph(3, [0, 0, 1], [1, 2, 2], [1, 1, 2**31 - 1], "shadowed")
    rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.OK and dist.tolist() == [0, 1, 1]
    g = gg.path(3, weights=[4, -1])
    rc, _ = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    assert rc == oracle.NEGATIVE_WEIGHT


def test_invalid_arguments():
    rc, _ = oracle.sssp(3, [0, 5], [1, 2], [1, 1], 0)
    assert rc == oracle.INVALID
    rc, _ = oracle.bfs(3, [0], [1], 3)
    assert rc == oracle.INVALID


def test_single_vertex_and_no_edges():
    for f in (lambda: oracle.sssp(1, [], [], [], 0), lambda: oracle.bfs(1, [], [], 0)):
        rc, out = f()
        assert rc == oracle.OK and out.tolist() == [0]
    rc, out = oracle.cc(4, [], [])
    assert out.tolist() == [0, 1, 2, 3]


# ---------------------------------------------------------------- BFS
@pytest.mark.parametrize("n,s", [(10, 0), (10, 7), (1, 0), (33, 32)])
def test_bfs_directed_cycle(n, s):
    g = gg.cycle(n)
    rc, level = oracle.bfs(g.n, g.src, g.dst, s)
    assert rc == oracle.OK
    assert level.tolist() == [(v - s) % n for v in range(n)]


def test_bfs_complete_graph():
    g = gg.complete(12)
    rc, level = oracle.bfs(g.n, g.src, g.dst, 5)
    assert level.tolist() == [1] * 5 + [0] + [1] * 6


def test_bfs_invariants_grid_with_shortcuts():
    g = gg.grid(64, seed=45)
    s = int(gg.sources(g, 1, seed=46)[0])
    rc, level = oracle.bfs(g.n, g.src, g.dst, s)
    assert rc == oracle.OK
    pins.check_bfs_invariants(g.n, g.src, g.dst, s, level)


# ---------------------------------------------------------------- CC
def test_cc_disjoint_cliques():
    g = gg.disjoint_cliques([5, 1, 7, 3, 2], seed=47)
    rc, label = oracle.cc(g.n, g.src, g.dst)
    assert rc == oracle.OK
    for ids in g.blocks:
        assert set(label[ids].tolist()) == {min(ids)}


@pytest.mark.parametrize("which", ["rmat", "grid", "er"])
def test_cc_vs_scipy_and_dfs(which):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = {"rmat": lambda: gg.rmat(12, 2, seed=48),
         "grid": lambda: gg.grid(40, p_del=0.3, shortcut_frac=0.0005, seed=49),
         "er": lambda: gg.er(4000, 3000, seed=50)}[which]()
    rc, label = oracle.cc(g.n, g.src, g.dst)
    assert rc == oracle.OK
    pins.check_cc_invariants(g.n, g.src, g.dst, label)
    A = sp.csr_matrix((np.ones(g.m), (g.src, g.dst)), shape=(g.n, g.n))
    ncomp, comp = csgraph.connected_components(A, directed=True, connection="weak")
    minid = np.full(ncomp, g.n, np.int64)
    np.minimum.at(minid, comp, np.arange(g.n))
    np.testing.assert_array_equal(label, minid[comp])
    assert len(np.unique(label)) == pins.dfs_component_count(g.n, g.src, g.dst) == ncomp


# ---------------------------------------------------------------- Jacobi round counts
def test_jacobi_rounds_closed_forms():
    g = gg.path(9)
    r, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, 0)
    assert r == 9          # 8 rounds that change a distance, then one that does not
    g = gg.star(50)
    r, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, 0)
    assert r == 2
    r, _ = oracle.jacobi_rounds(1, [], [], [], 0)
    assert r == 1
    g = gg.full_grid(6, 11)
    r, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, 0, unit=True)
    assert r == 5 + 10 + 1  # eccentricity of a corner, plus the no-change round


@pytest.mark.parametrize("seed", range(6))
def test_jacobi_rounds_vs_definition(seed):
    g = gg.random_small(40, 150, seed=3000 + seed, wlo=0, whi=12)
    r, dist = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, 0)
    _, ref = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    np.testing.assert_array_equal(dist, ref)
    assert r == pins.sync_rounds_from_distances(g.n, g.src, g.dst, g.w, 0, ref)


# ---------------------------------------------------------------- one all-active round
def _init_state(n, s):
    cur = np.full(n, INF, np.int32)
    cur[s] = 0
    return cur


def test_sweep_hand_example():
    # 0 -5-> 1 -7-> 2, 3 -1-> 2 with vertex 3 unreached: one double-buffered
    # round from (0: 0) reaches 1 only; a round that read its own writes
    # would also reach 2.
    src, dst, w = [0, 1, 3], [1, 2, 2], [5, 7, 1]
    cur = _init_state(4, 0)
    rc, nxt, low = oracle.sweep(4, src, dst, w, cur, cur)
    assert rc == oracle.OK and nxt.tolist() == [0, 5, INF, INF] and low == 1
    rc, nxt2, low = oracle.sweep(4, src, dst, w, nxt, nxt)
    assert rc == oracle.OK and nxt2.tolist() == [0, 5, 12, INF] and low == 1
    # next below cur is kept; only lower candidates are written
    rc, nxt3, low = oracle.sweep(4, src, dst, w, nxt2, [0, 3, 20, 9])
    assert nxt3.tolist() == [0, 3, 12, 9] and low == 1


@pytest.mark.parametrize("seed", range(10))
def test_sweep_rounds_vs_hop_limited_brute_force(seed):
    rng = np.random.Generator(np.random.PCG64(400 + seed))
    n = int(rng.integers(1, 9))
    g = gg.random_small(n, int(rng.integers(0, 3 * n + 1)), seed=4000 + seed, wlo=0, whi=9)
    s = int(rng.integers(0, n))
    cur = _init_state(n, s)
    for k in range(1, n + 1):
        rc, cur, _ = oracle.sweep(n, g.src, g.dst, g.w, cur, cur)
        assert rc == oracle.OK
        exp = pins.brute_force_hop_limited(n, g.src.tolist(), g.dst.tolist(), g.w.tolist(), s, k)
        assert cur.tolist() == [INF if x is None else x for x in exp], k


@pytest.mark.parametrize("seed", range(6))
def test_sweep_iterated_reaches_floyd_warshall(seed):
    g = gg.random_small(40, 160, seed=4100 + seed, wlo=0, whi=20)
    fw = pins.floyd_warshall(g.n, g.src, g.dst, g.w)
    cur = _init_state(g.n, 0)
    sweeps = 0
    while True:
        rc, nxt, low = oracle.sweep(g.n, g.src, g.dst, g.w, cur, cur)
        assert rc == oracle.OK
        sweeps += 1
        assert low == int(np.count_nonzero(nxt < cur))
        cur = nxt
        if low == 0:
            break
    np.testing.assert_array_equal(cur, np.where(fw[0] >= pins.BIG, INF, fw[0]))
    assert sweeps == pins.sync_rounds_from_distances(g.n, g.src, g.dst, g.w, 0, cur)


def test_sweep_overflow_and_errors():
    big = 2**31 - 1
    # 0 -> 1 overflows (dropped, status OVERFLOW), 0 -> 2 is still applied
    rc, nxt, low = oracle.sweep(3, [0, 0], [1, 2], [10, 1], [big - 5, INF, INF], [big - 5, INF, INF])
    assert rc == oracle.OVERFLOW and nxt.tolist() == [big - 5, INF, big - 4] and low == 1
    assert oracle.sweep(2, [0], [1], [-1], [0, INF], [0, INF])[0] == oracle.NEGATIVE_WEIGHT
    assert oracle.sweep(2, [0], [2], [1], [0, INF], [0, INF])[0] == oracle.INVALID
    rc, nxt, low = oracle.sweep(3, [], [], [], [0, INF, 4], [0, 7, 4])
    assert rc == oracle.OK and nxt.tolist() == [0, 7, 4] and low == 0
