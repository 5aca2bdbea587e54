"""GPU parity, bit-exact against the CPU oracle, on graphs the oracle finishes
in seconds: every algorithm in all four modes, through the C ABI.

Each result is the unique fixpoint of Alg. 1/2 (SSSP), Alg. 3 (BFS) or of
min-label propagation (CC), so every mode must reproduce the oracle exactly.
The synchronous modes' round counts must also equal the Jacobi round count.
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests import pins
from tests.gpu_util import ALGOS, MODE_IDS, MODES, graph_handle, run
from tests.test_golden import HAND, parse_fixture

pytestmark = pytest.mark.gpu


def hand_graph(path):
    f = parse_fixture(path)
    return gg.Graph(f["n"], f["src"], f["dst"], f["w"], os.path.basename(path))


def adversarial():
    """Small graphs with the method's degenerate cases."""
    out = {}
    out["single_vertex"] = gg.Graph(1, [], [], [], "single")
    out["no_edges"] = gg.Graph(10, [], [], [], "empty10")
    out["self_loops_dups_zero_w"] = gg.random_small(300, 2500, seed=17, wlo=0, whi=20)
    out["path_1500"] = gg.path(1500, weights=np.arange(1, 1500) % 7)
    out["cycle_257"] = gg.cycle(257)
    out["star_5000"] = gg.star(5000, weights=(np.arange(4999) * 37) % 1000 + 1)
    out["hub_150k"] = gg.hub(200_000, 150_000, 200_000, seed=3)
    out["cliques_isolated"] = gg.disjoint_cliques([40, 1, 70, 3, 1, 33, 2], seed=5)
    # two components, the second unreachable from 0; vertex 9 has no out-edges
    out["unreachable"] = gg.Graph(10, [0, 1, 2, 5, 6, 7, 8], [1, 2, 9, 6, 7, 5, 9], [3, 1, 4, 1, 5, 9, 2], "unreach")
    out["full_grid_40x70"] = gg.full_grid(40, 70)
    return out


def workloads():
    out = {os.path.basename(p): hand_graph(p) for p in HAND}
    out.update(adversarial())
    out["er_16384"] = gg.er()
    out["rmat_10"] = gg.rmat(10)
    out["rmat_14"] = gg.rmat(14)
    out["grid_64"] = gg.grid(64)
    out["grid_300"] = gg.grid(300, seed=9)
    return out


WL = workloads()


def sources_of(g):
    if g.m == 0:
        return [0]
    s = [0] + [int(x) for x in gg.sources(g, 2, seed=1234)]
    deg = np.bincount(g.src, minlength=g.n)
    zero = np.flatnonzero(deg == 0)
    if zero.size:
        s.append(int(zero[0]))       # a source with no out-edges
    return sorted(set(s))


@pytest.fixture(scope="module")
def expected():
    cache = {}

    def get(name, algo, s):
        key = (name, algo, s)
        if key not in cache:
            g = WL[name]
            if algo == "sssp":
                rc, r = oracle.sssp(g.n, g.src, g.dst, g.w, s)
            elif algo == "bfs":
                rc, r = oracle.bfs(g.n, g.src, g.dst, s)
            else:
                rc, r = oracle.cc(g.n, g.src, g.dst)
            assert rc == oracle.OK
            cache[key] = r
        return cache[key]
    return get


@pytest.mark.parametrize("name", sorted(WL))
def test_all_modes_match_oracle(name, expected):
    g = WL[name]
    with graph_handle(g) as h:
        for algo in ("sssp", "bfs", "cc"):
            srcs = [0] if algo == "cc" else sources_of(g)
            for s in srcs:
                exp = expected(name, algo, s)
                for mode, mid in zip(MODES, MODE_IDS):
                    got, st = run(h, g.n, ALGOS[algo], s, mode)
                    if not np.array_equal(got, exp):
                        bad = np.flatnonzero(got != exp)
                        raise AssertionError(f"{name} {algo} src={s} {mid}: {bad.size} mismatches, first "
                                             f"v={bad[0]} got={got[bad[0]]} want={exp[bad[0]]}")


@pytest.mark.parametrize("name", ["hand_7v.txt", "hand_zero_cycle.txt", "er_16384", "rmat_14", "grid_64",
                                  "path_1500", "self_loops_dups_zero_w"])
def test_sync_round_counts_equal_jacobi(name):
    g = WL[name]
    with graph_handle(g) as h:
        for s in sources_of(g):
            r_sssp, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, s)
            r_bfs, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, s, unit=True)
            for mode in (0, 2):   # vertex-sync, edge-sync
                _, st = run(h, g.n, ALGOS["sssp"], s, mode)
                assert st.rounds == r_sssp, (name, s, mode, st.rounds, r_sssp)
                _, st = run(h, g.n, ALGOS["bfs"], s, mode)
                assert st.rounds == r_bfs, (name, s, mode, st.rounds, r_bfs)


@pytest.mark.parametrize("kind,where,out_where", [("coo", "device", "host"), ("csr", "host", "device"),
                                                  ("csr", "device", "host"), ("coo", "host", "pinned")])
def test_input_forms_and_host_outputs(kind, where, out_where):
    g = gg.rmat(12, seed=77)
    s = int(gg.sources(g, 1, seed=78)[0])
    _, d = oracle.sssp(g.n, g.src, g.dst, g.w, s)
    _, lv = oracle.bfs(g.n, g.src, g.dst, s)
    _, lab = oracle.cc(g.n, g.src, g.dst)
    with graph_handle(g, kind=kind, where=where) as h:
        for mode in MODES:
            got, _ = run(h, g.n, ALGOS["sssp"], s, mode, where=out_where)
            np.testing.assert_array_equal(got, d)
            got, _ = run(h, g.n, ALGOS["bfs"], s, mode, where=out_where)
            np.testing.assert_array_equal(got, lv)
            got, _ = run(h, g.n, ALGOS["cc"], 0, mode, where=out_where)
            np.testing.assert_array_equal(got, lab)


def test_null_weights_mean_unit_weights():
    g = gg.rmat(11, seed=5)
    _, lv = oracle.bfs(g.n, g.src, g.dst, 0)
    with graph_handle(g, weights=False) as h:
        for mode in MODES:
            got, _ = run(h, g.n, ALGOS["sssp"], 0, mode)
            np.testing.assert_array_equal(got, lv)


def test_graph_info():
    import paper_1903_01665_gb300 as fg
    g = gg.rmat(12)
    deg = np.bincount(g.src, minlength=g.n)
    with graph_handle(g) as h:
        st, info = fg.fg_graph_info(h)
        assert st == fg.FG_OK
        assert info.n == g.n and info.m == g.m and info.m_sym == 2 * g.m
        assert info.max_out_degree == deg.max()
        assert info.n_zero_out == int((deg == 0).sum())
        assert info.n_low == int(((deg >= 1) & (deg < 32)).sum())
        assert info.n_mid == int(((deg >= 32) & (deg < 1024)).sum())
        assert info.n_high == int((deg >= 1024).sum())
        assert info.n_high_chunks == int(((deg[deg >= 1024] + 2047) // 2048).sum())
        indeg = np.bincount(g.dst, minlength=g.n)
        assert info.n_isolated == int(((deg + indeg) == 0).sum())


def test_select_mode_runs_and_auto_matches():
    import paper_1903_01665_gb300 as fg
    g = gg.rmat(13)
    _, d = oracle.sssp(g.n, g.src, g.dst, g.w, 0)
    with graph_handle(g) as h:
        for algo in (0, 1, 2):
            st, m = fg.fg_select_mode(h, algo)
            assert st == fg.FG_OK and m in (0, 1, 2, 3, 5, 6)
        got, st = run(h, g.n, ALGOS["sssp"], 0, fg.FG_AUTO)
        np.testing.assert_array_equal(got, d)
        assert st.mode in (0, 1, 2, 3, 5, 6)


def test_invariants_on_results():
    g = gg.grid(128, seed=21)
    with graph_handle(g) as h:
        for mode in MODES:
            d, _ = run(h, g.n, ALGOS["sssp"], 5, mode)
            pins.check_sssp_invariants(g.n, g.src, g.dst, g.w, 5, d)
            lv, _ = run(h, g.n, ALGOS["bfs"], 5, mode)
            pins.check_bfs_invariants(g.n, g.src, g.dst, 5, lv)
            lab, _ = run(h, g.n, ALGOS["cc"], 0, mode)
            pins.check_cc_invariants(g.n, g.src, g.dst, lab)


@pytest.mark.parametrize("delta", [1, 7, 500, 2**30])
def test_bucket_mode_any_width(delta):
    """The bucketed SSSP reaches the same fixpoint whatever the bucket width:
    1 (one distance per bucket), small, and one bucket holding everything."""
    for g in (gg.grid(96, seed=31), gg.rmat(12, seed=32), gg.random_small(300, 2500, seed=33, wlo=0, whi=20)):
        s = int(gg.sources(g, 1, seed=34)[0])
        _, d = oracle.sssp(g.n, g.src, g.dst, g.w, s)
        with graph_handle(g) as h:
            got, st = run(h, g.n, ALGOS["sssp"], s, fg.FG_BUCKET, delta=delta)
            np.testing.assert_array_equal(got, d)
            assert st.mode == fg.FG_BUCKET


def test_edge_async_dense_generations_stream():
    """Edge-async generations whose worklist holds a quarter of the edges or
    more stream the whole edge list (stats.scanned counts the streamed edge
    sources); the result stays the oracle's in all three algorithms, on a
    skewed graph (dense middle generations) and a grid (CC's all-active
    first generation, sparse wavefronts after)."""
    for g in (gg.rmat(13, seed=41), gg.grid(80, seed=42)):
        s = int(gg.sources(g, 1, seed=43)[0])
        _, d = oracle.sssp(g.n, g.src, g.dst, g.w, s)
        _, lv = oracle.bfs(g.n, g.src, g.dst, s)
        _, lab = oracle.cc(g.n, g.src, g.dst)
        with graph_handle(g) as h:
            for algo, want in (("sssp", d), ("bfs", lv), ("cc", lab)):
                got, st = run(h, g.n, ALGOS[algo], s, fg.FG_EDGE_ASYNC)
                np.testing.assert_array_equal(got, want, err_msg=f"{g.name} {algo}")
                if algo == "cc" or g.name.startswith("rmat"):
                    assert st.scanned > 0, (g.name, algo)


def _info(h):
    st, info = fg.fg_graph_info(h)
    fg.check(st)
    return info


def test_lazy_graph_builds_parts_on_first_use():
    """FG_GRAPH_LAZY: the CSR alone at creation; the edge sources on the first
    edge-based query, the symmetrised view on the first CC query (and in a
    batch); every result stays the oracle's."""
    g = gg.rmat(12, seed=51)
    s = int(gg.sources(g, 1, seed=52)[0])
    want = {"sssp": oracle.sssp(g.n, g.src, g.dst, g.w, s)[1], "bfs": oracle.bfs(g.n, g.src, g.dst, s)[1],
            "cc": oracle.cc(g.n, g.src, g.dst)[1]}
    with graph_handle(g) as hf:
        full = _info(hf)
    st, h = fg.fg_graph_create_coo(g.n, g.src, g.dst, g.w, flags=fg.FG_GRAPH_LAZY)
    fg.check(st)
    try:
        b0 = _info(h).device_bytes
        assert b0 < full.device_bytes and _info(h).n_isolated == -1
        got, _ = run(h, g.n, ALGOS["sssp"], s, fg.FG_VERTEX_SYNC)
        np.testing.assert_array_equal(got, want["sssp"])
        assert _info(h).device_bytes == b0            # vertex modes read the CSR only
        got, _ = run(h, g.n, ALGOS["bfs"], s, fg.FG_EDGE_ASYNC)
        np.testing.assert_array_equal(got, want["bfs"])
        b1 = _info(h).device_bytes
        assert b1 >= b0 + 4 * g.m                     # the edge sources
        lab = np.zeros(g.n, np.int32)
        st_, sts, _, _ = fg.fg_run_batch([(h, fg.FG_ALGO_CC, 0, lab, fg.FG_EDGE_SYNC)])
        fg.check(st_)
        fg.check(sts[0])
        np.testing.assert_array_equal(lab, want["cc"])
        assert _info(h).n_isolated == full.n_isolated
        assert _info(h).device_bytes == full.device_bytes
        for algo in ("sssp", "bfs", "cc"):
            for mode in MODES:
                got, _ = run(h, g.n, ALGOS[algo], s, mode)
                np.testing.assert_array_equal(got, want[algo], err_msg=f"{algo} mode {mode}")
    finally:
        fg.check(fg.fg_graph_destroy(h))
    # the edge variant of the all-active round on a fresh lazy graph
    import torch
    st, h = fg.fg_graph_create_coo(g.n, g.src, g.dst, g.w, flags=fg.FG_GRAPH_LAZY)
    fg.check(st)
    try:
        cur = np.where(want["sssp"] == fg.FG_INF, 1 << 30, want["sssp"]).astype(np.int32)
        _, exp, _ = oracle.sweep(g.n, g.src, g.dst, g.w, cur, cur)
        nxt = torch.from_numpy(cur.copy()).cuda()
        st, _, _ = fg.fg_sweep(h, fg.FG_EDGE_SYNC, torch.from_numpy(cur).cuda(), nxt)
        fg.check(st)
        np.testing.assert_array_equal(nxt.cpu().numpy(), exp)
    finally:
        fg.check(fg.fg_graph_destroy(h))


def _gini_exact(deg):
    d = np.sort(deg.astype(np.float64))
    n = d.size
    i = np.arange(1, n + 1)
    return float((2 * (i * d).sum()) / (n * d.sum()) - (n + 1) / n) if d.sum() else 0.0


@pytest.mark.parametrize("kind", ["rmat", "grid", "er"])
def test_selection_model_features_and_picks(kind):
    """fg_select_plan on a skewed shallow graph (R-MAT 16), a uniform deep one
    (a 256^2 grid) and a uniform shallow one (ER): the degree Gini agrees
    with the exact one from the degrees, the depth estimate classifies the
    graph, the picks follow the documented rules, FG_AUTO runs the plan's
    mode with its CTAs per SM, and its results are the oracle's."""
    import paper_1903_01665_gb300 as fg
    g = {"rmat": lambda: gg.rmat(16, seed=8), "grid": lambda: gg.grid(256, seed=8),
         "er": lambda: gg.er(20000, 160000, seed=8)}[kind]()
    deg = np.bincount(g.src, minlength=g.n)
    s = int(gg.sources(g, 1, seed=9)[0])
    with graph_handle(g) as h:
        plans = {}
        for algo in (0, 1, 2):
            st, p = fg.fg_select_plan(h, algo)
            assert st == fg.FG_OK and p.tuned == 0
            plans[algo] = p
        p = plans[0]
        assert abs(p.degree_gini - _gini_exact(deg)) < 0.06
        deep, skew = p.depth_est > 32, p.degree_gini > 0.5
        assert (deep, skew) == {"rmat": (False, True), "grid": (True, False), "er": (False, False)}[kind]
        if kind == "rmat":
            want = {0: fg.FG_EDGE_ASYNC, 1: fg.FG_PULL, 2: fg.FG_VERTEX_ASYNC if g.n >= 1 << 19 else fg.FG_BUCKET}
        elif kind == "grid":
            want = {0: fg.FG_VERTEX_SYNC, 1: fg.FG_VERTEX_SYNC, 2: fg.FG_PULL}
        else:
            want = {0: fg.FG_EDGE_SYNC, 1: fg.FG_VERTEX_SYNC, 2: fg.FG_EDGE_SYNC}
        assert {a: plans[a].mode for a in plans} == want
        assert all(plans[a].blocks_per_sm == 2 for a in plans)   # every graph here has < 3 M edges
        for algo, name in ((0, "sssp"), (1, "bfs"), (2, "cc")):
            got, st = run(h, g.n, ALGOS[name], s, fg.FG_AUTO)
            assert st.mode == want[algo]
            assert st.grid_blocks <= 2 * 152
            if name == "sssp":
                exp = oracle.sssp(g.n, g.src, g.dst, g.w, s)[1]
            elif name == "bfs":
                exp = oracle.bfs(g.n, g.src, g.dst, s)[1]
            else:
                exp = oracle.cc(g.n, g.src, g.dst)[1]
            np.testing.assert_array_equal(got, exp)
