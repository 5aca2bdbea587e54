"""Renumbered graphs (FG_GRAPH_RELABEL, and skewed graphs by default) against
the CPU oracle, bit for bit.

A renumbered graph holds its vertices in internal ids ordered by in-degree
class; every call still takes and returns original ids.  So every result on
such a graph must equal the oracle's on the original graph: sources are
translated, outputs permuted back (device, pageable and pinned host), and CC
labels stay each component's smallest original id.  Covered: every mode of
every algorithm on the small workloads with renumbering forced, the same
skewed graphs with it switched off, the multi-source sweeps, batches (fused
and unfused, with CC and staged host outputs), the server, fg_sweep against
the oracle's round, input as CSR, lazy graphs, overflow, and the creation
rule and fg_graph_info fields.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import ALGOS, MODE_IDS, MODES, as_numpy, graph_handle, make_out, run
from tests.test_parity_small import WL, sources_of

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


def _binned_gini(deg):
    """The Gini coefficient of degrees in power-of-two bins, from its
    definition: 1 - 2 x the area under the Lorenz curve (vertices by
    increasing degree against their share of the edges), linear in a bin."""
    deg = np.asarray(deg, np.int64)
    b = np.where(deg > 0, np.floor(np.log2(np.maximum(deg, 1))).astype(np.int64) + 1, 0)
    cnt = np.bincount(b, minlength=33).astype(float)
    tot = np.bincount(b, weights=deg, minlength=33).astype(float)
    if cnt.sum() == 0 or tot.sum() == 0:
        return 0.0
    x = np.concatenate([[0.0], np.cumsum(cnt) / cnt.sum()])
    y = np.concatenate([[0.0], np.cumsum(tot) / tot.sum()])
    return 1.0 - 2.0 * np.sum((x[1:] - x[:-1]) * (y[1:] + y[:-1]) / 2)


@pytest.mark.parametrize("name", sorted(WL))
def test_renumbered_all_modes_match_oracle(name):
    g = WL[name]
    with graph_handle(g, flags=fg.FG_GRAPH_RELABEL) as h:
        st, info = fg.fg_graph_info(h)
        assert st == fg.FG_OK and info.relabelled == 1
        for algo in ("sssp", "bfs", "cc"):
            for s in ([0] if algo == "cc" else sources_of(g)):
                want = _want(g, ALGOS[algo], s)
                for mode, mid in zip(MODES, MODE_IDS):
                    got, _ = run(h, g.n, ALGOS[algo], s, mode)
                    if not np.array_equal(got, want):
                        bad = np.flatnonzero(got != want)
                        raise AssertionError(f"{name} {algo} src={s} {mid}: {bad.size} mismatches, first "
                                             f"v={bad[0]} got={got[bad[0]]} want={want[bad[0]]}")


@pytest.mark.parametrize("name", ["rmat_10", "rmat_14", "hub_150k", "star_5000"])
def test_skewed_graphs_with_ids_kept_match_oracle(name):
    g = WL[name]
    with graph_handle(g, flags=fg.FG_GRAPH_KEEP_IDS) as h:
        assert fg.fg_graph_info(h)[1].relabelled == 0
        for algo in ("sssp", "bfs", "cc"):
            for s in ([0] if algo == "cc" else sources_of(g)):
                want = _want(g, ALGOS[algo], s)
                for mode in MODES:
                    np.testing.assert_array_equal(run(h, g.n, ALGOS[algo], s, mode)[0], want)


def test_creation_rule_and_info_fields():
    """Skewed in-degrees (R-MAT) are renumbered by default, a grid is not;
    the flags force either way; in_degree_gini is the binned Gini of the
    in-degrees (the same formula as the out-degree one)."""
    r = gg.rmat(12, seed=71)
    grid = gg.grid(64, seed=72)
    for g, default in ((r, 1), (grid, 0)):
        gini = _binned_gini(np.bincount(g.dst, minlength=g.n))
        assert (gini > 0.5) == bool(default)
        for flags, want in ((0, default), (fg.FG_GRAPH_RELABEL, 1), (fg.FG_GRAPH_KEEP_IDS, 0),
                            (fg.FG_GRAPH_LAZY, default)):
            with graph_handle(g, flags=flags) as h:
                st, info = fg.fg_graph_info(h)
                assert st == fg.FG_OK and info.relabelled == want, (g.name, flags)
                if not flags & fg.FG_GRAPH_KEEP_IDS:
                    assert abs(info.in_degree_gini - gini) < 1e-5
                else:
                    assert info.in_degree_gini == 0.0


@pytest.mark.parametrize("kind,where,out_where", [("coo", "device", "host"), ("csr", "host", "pinned"),
                                                  ("csr", "device", "device")])
def test_renumbered_input_forms_and_outputs(kind, where, out_where):
    g = gg.rmat(13, seed=73)
    s = int(gg.sources(g, 1, seed=74)[0])
    with graph_handle(g, kind=kind, where=where, flags=fg.FG_GRAPH_RELABEL) as h:
        for algo in (fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS, fg.FG_ALGO_CC):
            for mode in (fg.FG_VERTEX_SYNC, fg.FG_EDGE_ASYNC):
                got, _ = run(h, g.n, algo, s, mode, where=out_where)
                np.testing.assert_array_equal(got, _want(g, algo, s))


def test_renumbered_cc_labels_are_smallest_original_ids():
    """Cliques whose smallest original id is not their highest-degree
    vertex: the renumbering puts hubs first, the labels must not follow."""
    rng = np.random.default_rng(75)
    n = 3000
    perm = rng.permutation(n).astype(np.int32)   # scatter the cliques' members over the id range
    src, dst = [], []
    start = 0
    for size in (1, 2, 17, 300, 5, 1200, 3, 40):
        members = perm[start:start + size]
        hub = members[-1]
        for v in members[:-1]:   # a star around the last member, both ways
            src += [v, hub]
            dst += [hub, v]
        start += size
    g = gg.Graph(n, np.array(src, np.int32), np.array(dst, np.int32), np.ones(len(src), np.int32), "stars")
    want = _want(g, fg.FG_ALGO_CC, 0)
    with graph_handle(g, flags=fg.FG_GRAPH_RELABEL) as h:
        for mode in MODES:
            np.testing.assert_array_equal(run(h, g.n, fg.FG_ALGO_CC, 0, mode)[0], want)


@pytest.mark.parametrize("algo", [fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS, fg.FG_ALGO_CC])
def test_renumbered_multi_source_sweeps(algo):
    g = gg.rmat(14, seed=76)
    srcs = [int(x) for x in gg.sources(g, 6, seed=77)] + [0, 0]
    with graph_handle(g, flags=fg.FG_GRAPH_RELABEL) as h:
        outs = [make_out(g.n, ["device", "host", "pinned"][j % 3]) for j in range(8)]
        st, sts, _ = fg.fg_run_multi(h, algo, srcs if algo != fg.FG_ALGO_CC else None, outs)
        assert st == fg.FG_OK, fg.fg_last_error()
        for s, o in zip(srcs, outs):
            np.testing.assert_array_equal(as_numpy(o), _want(g, algo, s))


def test_renumbered_multi_source_overflow_fails_only_its_slot():
    big = 2**31 - 2
    g = gg.Graph(5, [0, 1, 3, 4, 4, 4], [1, 2, 4, 2, 1, 3], [big, 5, 8, 1, 1, 1], "overflow5")
    with graph_handle(g, flags=fg.FG_GRAPH_RELABEL) as h:
        outs = [make_out(g.n, "device", fill=-9) for _ in range(3)]
        st, sts, _ = fg.fg_run_multi(h, fg.FG_ALGO_SSSP, [0, 1, 3], outs)
        assert sts == [fg.FG_ERR_OVERFLOW, fg.FG_OK, fg.FG_OK]
        assert (as_numpy(outs[0]) == -9).all()
        for s, o in zip([1, 3], outs[1:]):
            np.testing.assert_array_equal(as_numpy(o), _want(g, fg.FG_ALGO_SSSP, s))
        out = make_out(g.n, "device", fill=-9)
        st, _ = fg.fg_run(h, fg.FG_ALGO_SSSP, 0, out, fg.FG_VERTEX_SYNC)
        assert st == fg.FG_ERR_OVERFLOW and (as_numpy(out) == -9).all()


@pytest.mark.parametrize("fuse", [False, True])
def test_renumbered_batch_fused_and_unfused(fuse):
    """A batch over renumbered and plain graphs: single queries (the kernel
    writes original order), fused sweeps, CC (smallest original ids in the
    kernel), host outputs staged on the device."""
    graphs = [gg.rmat(12, seed=78), gg.grid(48, seed=79), gg.rmat(11, seed=80)]
    flags = [fg.FG_GRAPH_RELABEL, fg.FG_GRAPH_RELABEL, 0]
    import contextlib
    with contextlib.ExitStack() as es:
        hs = [es.enter_context(graph_handle(g, flags=f)) for g, f in zip(graphs, flags)]
        qs, want = [], []
        for gi, (g, h) in enumerate(zip(graphs, hs)):
            srcs = [int(x) for x in gg.sources(g, 3, seed=81 + gi)]
            for j, s in enumerate(srcs):
                for algo in (fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS):
                    out = make_out(g.n, "host" if (j + algo) % 2 else "device")
                    qs.append((h, algo, s, out, fg.FG_AUTO))
                    want.append((out, _want(g, algo, s)))
            for j in range(2):
                out = make_out(g.n, "pinned" if j else "device")
                qs.append((h, fg.FG_ALGO_CC, 0, out, fg.FG_AUTO))
                want.append((out, _want(g, fg.FG_ALGO_CC, 0)))
        st, sts, _, bstats = fg.fg_run_batch(qs, fuse_same_graph=fuse)
        assert st == fg.FG_OK, fg.fg_last_error()
        assert all(x == fg.FG_OK for x in sts)
        for out, w in want:
            np.testing.assert_array_equal(as_numpy(out), w)


def test_renumbered_server_results_match_oracle():
    g = gg.rmat(12, seed=83)
    srcs = [int(x) for x in gg.sources(g, 5, seed=84)]
    with graph_handle(g, flags=fg.FG_GRAPH_RELABEL) as h:
        st, srv = fg.fg_server_create()
        fg.check(st)
        try:
            outs, tickets, want = [], [], []
            for s in srcs:
                for algo in (fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS, fg.FG_ALGO_CC):
                    out = make_out(g.n, "device")
                    st, t = fg.fg_server_submit(srv, h, algo, s, out, fg.FG_AUTO)
                    fg.check(st)
                    outs.append(out)
                    tickets.append(t)
                    want.append(_want(g, algo, s))
            assert fg.fg_server_drain(srv, 120000) == fg.FG_OK
            comps = fg.fg_server_poll(srv, cap=len(tickets) + 8)
            assert sorted(c[0] for c in comps) == sorted(tickets)
            assert all(c[1] == fg.FG_OK for c in comps)
        finally:
            fg.check(fg.fg_server_destroy(srv))
        for out, w in zip(outs, want):
            np.testing.assert_array_equal(as_numpy(out), w)


@pytest.mark.parametrize("mode", [fg.FG_VERTEX_SYNC, fg.FG_EDGE_SYNC])
def test_renumbered_sweep_matches_oracle_round(mode):
    import torch
    g = gg.rmat(13, seed=85)
    rng = np.random.default_rng(86)
    cur = np.where(rng.random(g.n) < 0.3, rng.integers(0, 10**6, g.n), 2**31 - 1).astype(np.int32)
    nxt0 = np.where(rng.random(g.n) < 0.5, rng.integers(0, 10**6, g.n), 2**31 - 1).astype(np.int32)
    rc, want, _ = oracle.sweep(g.n, g.src, g.dst, g.w, cur, nxt0)
    assert rc == oracle.OK
    with graph_handle(g, flags=fg.FG_GRAPH_RELABEL) as h:
        c = torch.from_numpy(cur).cuda()
        nx = torch.from_numpy(nxt0.copy()).cuda()
        st, _, _ = fg.fg_sweep(h, mode, c, nx)
        assert st == fg.FG_OK, fg.fg_last_error()
        np.testing.assert_array_equal(nx.cpu().numpy(), want)
        np.testing.assert_array_equal(c.cpu().numpy(), cur)   # the caller's cur is not touched


def test_renumbered_lazy_graph_builds_its_views():
    g = gg.rmat(12, seed=87)
    s = int(gg.sources(g, 1, seed=88)[0])
    with graph_handle(g, flags=fg.FG_GRAPH_LAZY | fg.FG_GRAPH_RELABEL) as h:
        for algo in (fg.FG_ALGO_CC, fg.FG_ALGO_SSSP, fg.FG_ALGO_BFS):
            for mode in (fg.FG_EDGE_SYNC, fg.FG_PULL, fg.FG_VERTEX_ASYNC):
                np.testing.assert_array_equal(run(h, g.n, algo, s, mode)[0], _want(g, algo, s))
        st, plan = fg.fg_select_plan(h, fg.FG_ALGO_SSSP)
        assert st == fg.FG_OK
