"""The query server (continuous batching) on the GPU: every request served
in a mix with others must return exactly the CPU oracle's result for its
query (Dijkstra, FIFO BFS, union-find CC), whatever wave it ran in; the HBM
budget and the one-at-a-time baseline change scheduling only."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1903_01665_gb300 as fg
from tests.gpu_util import graph_handle

pytestmark = pytest.mark.gpu


def _requests(graphs, count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    srcs = [gg.sources(g, 16, seed=seed + i) for i, g in enumerate(graphs)]
    reqs = []
    for _ in range(count):
        gi = int(rng.integers(0, len(graphs)))
        u = rng.random()
        algo = 0 if u < 0.4 else (1 if u < 0.8 else 2)
        reqs.append((gi, algo, int(srcs[gi][rng.integers(0, len(srcs[gi]))])))
    return reqs


def _serve(handles, graphs, reqs, host_every=0, **opts):
    import torch
    outs, tickets = [], {}
    # outputs first, then the requests in a tight loop: a burst that queues
    # (a request alone on an idle device runs the plain per-query kernel)
    for i, (gi, algo, s) in enumerate(reqs):
        n = graphs[gi].n
        if host_every and i % host_every == 0:
            outs.append(torch.full((n,), -3, dtype=torch.int32).pin_memory())
        else:
            outs.append(torch.full((n,), -3, dtype=torch.int32, device="cuda"))
    st, srv = fg.fg_server_create(**opts)
    assert st == fg.FG_OK, fg.fg_last_error()
    try:
        for i, (gi, algo, s) in enumerate(reqs):
            st, t = fg.fg_server_submit(srv, handles[gi], algo, s, outs[i], fg.FG_AUTO)
            assert st == fg.FG_OK, fg.fg_last_error()
            tickets[t] = i
        assert fg.fg_server_drain(srv, 120000) == fg.FG_OK
        comps = fg.fg_server_poll(srv, cap=len(reqs) + 8)
    finally:
        assert fg.fg_server_destroy(srv) == fg.FG_OK
    assert len(comps) == len(reqs)
    assert all(c[1] == fg.FG_OK for c in comps)
    return outs, comps


@pytest.fixture(scope="module")
def setup():
    from contextlib import ExitStack
    graphs = [gg.rmat(12, seed=21), gg.rmat(15, seed=22), gg.grid(128, seed=23), gg.er(4000, 30000, seed=24)]
    with ExitStack() as stack:
        handles = [stack.enter_context(graph_handle(g)) for g in graphs]
        yield graphs, handles


def _alone(graphs, handles, reqs):
    """The oracle's result of every distinct request (graph, algorithm, source)."""
    want = {}
    for gi, algo, s in set(reqs):
        g = graphs[gi]
        if algo == fg.FG_ALGO_SSSP:
            rc, res = oracle.sssp(g.n, g.src, g.dst, g.w, s)
        elif algo == fg.FG_ALGO_BFS:
            rc, res = oracle.bfs(g.n, g.src, g.dst, s)
        else:
            rc, res = oracle.cc(g.n, g.src, g.dst)
        assert rc == oracle.OK
        want[(gi, algo, s)] = res
    return want


def test_results_in_the_mix_equal_results_alone(setup):
    graphs, handles = setup
    reqs = _requests(graphs, 300, seed=5)
    outs, comps = _serve(handles, graphs, reqs, host_every=7, max_inflight=4, max_wave=32)
    want = _alone(graphs, handles, reqs)
    for (gi, algo, s), out in zip(reqs, outs):
        np.testing.assert_array_equal(out.cpu().numpy(), want[(gi, algo, s)])
    assert max(c[2] for c in comps) > 1, "requests submitted in a burst should share waves"
    assert all(c[3] > 0 for c in comps)


def test_large_graphs_run_alone_and_match(setup):
    """Without fusion, requests on graphs with at least exclusive_edges edges
    run alone (wave size 1) on the whole device between the waves; every
    result is the oracle's."""
    graphs, handles = setup
    reqs = _requests(graphs, 120, seed=8)
    cut = graphs[1].m   # rmat-15 and larger run alone
    outs, comps = _serve(handles, graphs, reqs, max_inflight=3, max_wave=16, exclusive_edges=cut, no_fusion=True)
    want = _alone(graphs, handles, reqs)
    for (gi, algo, s), out in zip(reqs, outs):
        np.testing.assert_array_equal(out.cpu().numpy(), want[(gi, algo, s)])
    ticket_to_req = {}
    by_ticket = {c[0]: c for c in comps}
    first = min(by_ticket)
    for i, (gi, algo, s) in enumerate(reqs):
        ticket_to_req[first + i] = (gi, algo)
    for t, c in by_ticket.items():
        gi, algo = ticket_to_req[t]
        edges = 2 * graphs[gi].m if algo == 2 else graphs[gi].m
        if edges >= cut:
            assert c[2] == 1, "a large-graph request must run alone"


def test_tiny_budget_serves_one_per_wave(setup):
    graphs, handles = setup
    reqs = _requests(graphs, 40, seed=6)
    outs, comps = _serve(handles, graphs, reqs, hbm_budget_bytes=1, max_inflight=2)
    assert all(c[2] == 1 for c in comps)
    want = _alone(graphs, handles, reqs)
    for (gi, algo, s), out in zip(reqs, outs):
        np.testing.assert_array_equal(out.cpu().numpy(), want[(gi, algo, s)])


def test_one_at_a_time_baseline(setup):
    graphs, handles = setup
    reqs = _requests(graphs, 40, seed=7)
    outs, comps = _serve(handles, graphs, reqs, one_at_a_time=True)
    assert all(c[2] == 1 for c in comps)
    want = _alone(graphs, handles, reqs)
    for (gi, algo, s), out in zip(reqs, outs):
        np.testing.assert_array_equal(out.cpu().numpy(), want[(gi, algo, s)])


def test_large_graph_requests_fuse_by_graph_and_algorithm(setup):
    """With fusion (the default), a large-graph request runs on the whole
    device together with the later pending requests of its graph and
    algorithm: up to 8 SSSP or BFS requests in one multi-source sweep, the
    pending CC requests in one computation.  A burst on large graphs only
    must produce fused groups, and every result must be the oracle's."""
    graphs, handles = setup
    reqs = _requests(graphs, 200, seed=9)
    outs, comps = _serve(handles, graphs, reqs, host_every=5, max_inflight=2, max_wave=32, exclusive_edges=1)
    want = _alone(graphs, handles, reqs)
    for (gi, algo, s), out in zip(reqs, outs):
        np.testing.assert_array_equal(out.cpu().numpy(), want[(gi, algo, s)])
    by_ticket = {c[0]: c for c in comps}
    first = min(by_ticket)
    sizes = {0: [], 1: [], 2: []}
    for i, (gi, algo, s) in enumerate(reqs):
        sizes[algo].append(by_ticket[first + i][2])
    assert max(sizes[0]) > 1 and max(sizes[1]) > 1, "a burst should fuse SSSP and BFS requests"
    assert max(sizes[0]) <= 8 and max(sizes[1]) <= 8


def test_fusion_off_serves_the_same_results(setup):
    graphs, handles = setup
    reqs = _requests(graphs, 120, seed=10)
    outs, comps = _serve(handles, graphs, reqs, max_inflight=2, max_wave=16, no_fusion=True)
    want = _alone(graphs, handles, reqs)
    for (gi, algo, s), out in zip(reqs, outs):
        np.testing.assert_array_equal(out.cpu().numpy(), want[(gi, algo, s)])
