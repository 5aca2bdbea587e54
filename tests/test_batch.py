"""Batched queries on the GPU (one persistent launch per algorithm x mode,
teams of CTAs per query): every result must equal the oracle's, for mixed
graphs of uneven size, mixed algorithms and modes, host and device outputs,
direct launches and a CUDA-graph launch; FG_AUTO after the autotuner."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import graph_handle

pytestmark = pytest.mark.gpu


def _graphs():
    return [gg.rmat(10, seed=1), gg.rmat(13, seed=2), gg.rmat(16, seed=3), gg.grid(64, seed=4),
            gg.grid(256, seed=5), gg.er(4000, 30000, seed=6), gg.path(3000)]


def _expected(g, algo, s):
    if algo == 0:
        return oracle.sssp(g.n, g.src, g.dst, g.w, s)[1]
    if algo == 1:
        return oracle.bfs(g.n, g.src, g.dst, s)[1]
    return oracle.cc(g.n, g.src, g.dst)[1]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(use_graph):
    import torch
    from contextlib import ExitStack
    graphs = _graphs()
    rng = np.random.Generator(np.random.PCG64(7))
    with ExitStack() as stack:
        handles = [stack.enter_context(graph_handle(g)) for g in graphs]
        queries, want = [], []
        for gi, (g, h) in enumerate(zip(graphs, handles)):
            srcs = [int(x) for x in gg.sources(g, 3, seed=100 + gi)]
            for k, s in enumerate(srcs):
                for algo in (0, 1, 2):
                    mode = int(rng.choice([0, 1, 2, 3, 5]))
                    if (k + algo) % 2:
                        out = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
                    else:
                        out = np.full(g.n, -5, np.int32)
                    queries.append((h, algo, s, out, mode))
                    want.append(_expected(g, algo, s))
        st, sts, stats, bst = fg.fg_run_batch(queries, use_cuda_graph=use_graph)
        assert st == fg.FG_OK, fg.fg_last_error()
        assert all(x == fg.FG_OK for x in sts)
        assert bst.launches >= 1 and bst.teams >= 1
        for (h, algo, s, out, mode), exp, stt in zip(queries, want, stats):
            got = out.cpu().numpy() if hasattr(out, "cpu") else out
            np.testing.assert_array_equal(got, exp, err_msg=f"algo={algo} mode={mode} src={s}")
            assert stt.mode == mode


def test_batch_auto_after_autotune_and_overflow_status():
    import torch
    g = gg.rmat(14, seed=9)
    bad = gg.path(3, weights=[2**30, 2**30])
    with graph_handle(g) as h, graph_handle(bad) as hb:
        s = int(gg.sources(g, 1, seed=3)[0])
        for algo in (0, 1, 2):
            st, best, times = fg.fg_autotune(h, algo, s)
            tried = (0, 1, 2, 3, 6) if algo == fg.FG_ALGO_SSSP else (0, 1, 2, 3, 5, 6)
            assert st == fg.FG_OK and best in tried and all(times[m] > 0 for m in tried)
            assert times[fg.FG_AUTO] == 0 and times[best] == min(times[m] for m in tried)
            assert all(times[m] == 0 for m in range(7) if m not in tried)
            st, m = fg.fg_select_mode(h, algo)
            assert m == best
            st, plan = fg.fg_select_plan(h, algo)
            assert st == fg.FG_OK and plan.tuned == 1 and plan.mode == best and plan.blocks_per_sm in (0, 2)
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
        ob = np.full(3, 99, np.int32)
        q = [(h, a, s, outs[a], fg.FG_AUTO) for a in (0, 1, 2)] + [(hb, 0, 0, ob, 0)]
        st, sts, stats, _ = fg.fg_run_batch(q)
        assert st == fg.FG_ERR_OVERFLOW
        assert sts == [fg.FG_OK, fg.FG_OK, fg.FG_OK, fg.FG_ERR_OVERFLOW]
        assert np.all(ob == 99)
        for a in (0, 1, 2):
            np.testing.assert_array_equal(outs[a].cpu().numpy(), _expected(g, a, s))


@pytest.mark.parametrize("use_graph", [False, True])
def test_fused_batch_matches_oracle(use_graph):
    """fuse_same_graph: the SSSP and BFS queries of a graph run as
    multi-source sweeps of up to 8 sources (11 sources: a sweep of 8 and one
    of 3), its CC queries as one computation; a graph's lone query keeps its
    own mode.  Every output (device, pageable and pinned host; repeated
    sources) must be the oracle's."""
    import torch
    from contextlib import ExitStack
    graphs = _graphs()
    with ExitStack() as stack:
        handles = [stack.enter_context(graph_handle(g)) for g in graphs]
        queries, want, fused = [], [], []
        for gi, (g, h) in enumerate(zip(graphs, handles)):
            srcs = [int(x) for x in gg.sources(g, 10, seed=200 + gi)]
            srcs.append(srcs[0])   # a repeat
            plan = [(0, s) for s in srcs] + [(1, s) for s in srcs[:3]] + [(2, 0)] * 3
            if gi == 2:
                plan = [(1, srcs[1])]   # a lone query on its graph
            for k, (algo, s) in enumerate(plan):
                where = k % 3
                if where == 0:
                    out = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
                elif where == 1:
                    out = np.full(g.n, -5, np.int32)
                else:
                    out = torch.full((g.n,), -5, dtype=torch.int32).pin_memory()
                queries.append((h, algo, s, out, fg.FG_VERTEX_ASYNC))
                want.append(_expected(g, algo, s))
                fused.append(algo != 2 and gi != 2)
        st, sts, stats, bst = fg.fg_run_batch(queries, use_cuda_graph=use_graph, fuse_same_graph=True)
        assert st == fg.FG_OK, fg.fg_last_error()
        assert all(x == fg.FG_OK for x in sts)
        for (h, algo, s, out, mode), exp, stt, fu in zip(queries, want, stats, fused):
            got = out.cpu().numpy() if hasattr(out, "cpu") else out
            np.testing.assert_array_equal(got, exp, err_msg=f"algo={algo} src={s}")
            assert stt.mode == (-1 if fu else mode)
        assert bst.launches == 3   # the multi-source sweeps (SSSP and BFS in one kernel), CC, the lone query


def test_fused_batch_overflow_fails_only_its_slot():
    """A fused sweep with sources 0 and 1 on 0 -> 1 -> 2 (2^30, 2^30): source
    0 overflows at vertex 2, source 1 does not; the overflowed host output is
    untouched, the other is the oracle's, and the other graph's queries are
    unaffected."""
    import torch
    g = gg.rmat(12, seed=9)
    bad = gg.path(3, weights=[2**30, 2**30])
    with graph_handle(g) as h, graph_handle(bad) as hb:
        s = [int(x) for x in gg.sources(g, 2, seed=5)]
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(2)]
        ob = [np.full(3, 99, np.int32), np.full(3, 98, np.int32)]
        q = [(h, 0, s[0], outs[0], 0), (h, 0, s[1], outs[1], 0), (hb, 0, 0, ob[0], 0), (hb, 0, 1, ob[1], 0)]
        st, sts, _, _ = fg.fg_run_batch(q, fuse_same_graph=True)
        assert st == fg.FG_ERR_OVERFLOW
        assert sts == [fg.FG_OK, fg.FG_OK, fg.FG_ERR_OVERFLOW, fg.FG_OK]
        assert np.all(ob[0] == 99)
        np.testing.assert_array_equal(ob[1], _expected(bad, 0, 1))
        for j in range(2):
            np.testing.assert_array_equal(outs[j].cpu().numpy(), _expected(g, 0, s[j]))
