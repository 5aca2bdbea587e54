"""Planted mistakes: each plausible slip in the oracle must fail at least one pin.

The mutation is applied to a copy of the oracle's C source in a temporary
directory (the oracle itself is untouched), compiled, and run through a
compact version of the pins of ``test_oracle_pins.py``.
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import pins

INF = oracle.UNREACHED

MUTANTS = {
    "dropped_weight_term": [("int64_t cand = it.key + (w ? (int64_t)a.wt[k] : 1);",
                             "int64_t cand = it.key + 1;")],
    "heap_order_flipped": [("if (h->a[parent].key <= key) break;",
                            "if (h->a[parent].key >= key) break;")],
    "edges_transposed": [("a->start[src[e] + 1]++;", "a->start[dst[e] + 1]++;"),
                         ("int64_t slot = fill[src[e]]++;", "int64_t slot = fill[dst[e]]++;"),
                         ("a->to[slot] = dst[e];", "a->to[slot] = src[e];")],
    "bfs_level_not_incremented": [("level[t] = level[u] + 1;", "level[t] = level[u];")],
    "cc_root_not_min_id": [("label[v] = minid[uf_find(parent, v)];",
                            "label[v] = uf_find(parent, v);")],
    "overflow_bound_off_by_one": [("else if (d[v] >= (int64_t)INT32_MAX)",
                                   "else if (d[v] > (int64_t)INT32_MAX)")],
    "jacobi_reads_write_buffer": [("if (cur[src[e]] == INT64_MAX) continue;",
                                   "if (next[src[e]] == INT64_MAX) continue;"),
                                  ("int64_t cand = cur[src[e]] + ((unit || !w) ? 1 : (int64_t)w[e]);",
                                   "int64_t cand = next[src[e]] + ((unit || !w) ? 1 : (int64_t)w[e]);")],
    "sweep_reads_write_buffer": [("if (cur[src[e]] == UNREACHED) continue;",
                                  "if (next[src[e]] == UNREACHED) continue;"),
                                 ("int64_t cand = (int64_t)cur[src[e]] + (w ? (int64_t)w[e] : 1);",
                                  "int64_t cand = (int64_t)next[src[e]] + (w ? (int64_t)w[e] : 1);")],
    "sweep_drops_weight": [("int64_t cand = (int64_t)cur[src[e]] + (w ? (int64_t)w[e] : 1);",
                            "int64_t cand = (int64_t)cur[src[e]] + 1;")],
    "sweep_counts_writes": [("count += next[v] < before[v];", "count += next[v] <= before[v];")],
    "dijkstra_skips_zero_weight": [("if (cand < d[t]) {", "if (cand < d[t] && cand != it.key) {")],
}


def run_pins(lib):
    """Return the names of the pins that fail for this oracle build."""
    failed = []

    def check(name, fn):
        try:
            fn()
        except AssertionError:
            failed.append(name)

    def fw():
        for seed in range(4):
            g = gg.random_small(20, 70, seed=500 + seed, wlo=0, whi=9)
            d = pins.floyd_warshall(g.n, g.src, g.dst, g.w)
            rc, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 0, lib=lib)
            assert rc == oracle.OK
            assert np.array_equal(dist, np.where(d[0] >= pins.BIG, INF, d[0]))

    def brute():
        for seed in range(6):
            g = gg.random_small(7, 14, seed=600 + seed, wlo=0, whi=5)
            bw, bh = pins.brute_force_paths(g.n, g.src.tolist(), g.dst.tolist(), g.w.tolist(), 0)
            _, dist = oracle.sssp(g.n, g.src, g.dst, g.w, 0, lib=lib)
            _, lev = oracle.bfs(g.n, g.src, g.dst, 0, lib=lib)
            assert dist.tolist() == [INF if x is None else x for x in bw]
            assert lev.tolist() == [INF if x is None else x for x in bh]

    def cycle():
        g = gg.cycle(9)
        _, lev = oracle.bfs(g.n, g.src, g.dst, 4, lib=lib)
        assert lev.tolist() == [(v - 4) % 9 for v in range(9)]

    def cliques():
        g = gg.disjoint_cliques([4, 6, 3], seed=9)
        _, lab = oracle.cc(g.n, g.src, g.dst, lib=lib)
        for ids in g.blocks:
            assert set(lab[ids].tolist()) == {min(ids)}

    def overflow():
        g = gg.path(2, weights=[2**31 - 1])
        rc, _ = oracle.sssp(g.n, g.src, g.dst, g.w, 0, lib=lib)
        assert rc == oracle.OVERFLOW

    def rounds():
        g = gg.path(9)
        r, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, 0, lib=lib)
        assert r == 9

    def sweep():
        src, dst, w = [0, 1, 3], [1, 2, 2], [5, 7, 1]
        cur = np.array([0, INF, INF, INF], np.int32)
        rc, nxt, low = oracle.sweep(4, src, dst, w, cur, cur, lib=lib)
        assert rc == oracle.OK and nxt.tolist() == [0, 5, INF, INF] and low == 1

    def invariants():
        g = gg.rmat(10, 8, seed=77)
        s = int(gg.sources(g, 1, seed=78)[0])
        _, dist = oracle.sssp(g.n, g.src, g.dst, g.w, s, lib=lib)
        pins.check_sssp_invariants(g.n, g.src, g.dst, g.w, s, dist)
        _, lab = oracle.cc(g.n, g.src, g.dst, lib=lib)
        pins.check_cc_invariants(g.n, g.src, g.dst, lab)

    for name, fn in [("floyd_warshall", fw), ("brute_force", brute), ("cycle", cycle),
                     ("cliques", cliques), ("overflow", overflow), ("rounds", rounds),
                     ("sweep", sweep), ("invariants", invariants)]:
        check(name, fn)
    return failed


def test_unmutated_oracle_passes_all_pins():
    assert run_pins(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    text = open(oracle._SRC).read()
    for old, new in MUTANTS[name]:
        assert old in text, f"mutation anchor missing: {old}"
        text = text.replace(old, new)
    src = tmp_path / "oracle_mutant.c"
    src.write_text(text)
    out = str(tmp_path / f"liboracle_{name}.so")
    import subprocess
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", str(src), "-o", out],
                   check=True, capture_output=True)
    lib = oracle.load_variant(out)
    failed = run_pins(lib)
    assert failed, f"mutant {name} survived every pin"
    os.remove(out)
