"""The seeded input recipe: determinism (stored SHA-256) and the shape of each workload."""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STORED = json.load(open(os.path.join(GOLDEN, "graphgen_hashes.json")))


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


MAKERS = {
    "er-16384-131072": lambda: gg.er(),
    "rmat-12": lambda: gg.rmat(12),
    "rmat-22": lambda: gg.rmat(22),
    "grid-64": lambda: gg.grid(64),
    "grid-4096": lambda: gg.grid(4096),
}


@pytest.mark.parametrize("name", sorted(MAKERS))
def test_stored_hash(name):
    g = MAKERS[name]()
    rec = STORED[name]
    assert (g.n, g.m) == (rec["n"], rec["m"])
    assert sha(g.src, g.dst, g.w) == rec["edges"]
    assert sha(gg.sources(g, 8)) == rec["sources8"]


def test_splitmix64_reference_values():
    # splitmix64 seeded with 1234567: published first outputs of the reference generator
    assert gg.splitmix64(1234567, 0) == 6457827717110365317
    assert gg.splitmix64(1234567, 1) == 3203168211198807973


def test_er_shape():
    g = gg.er()
    assert g.n == 16384 and g.m == 131072
    assert np.all(g.src != g.dst)
    assert np.unique(g.src.astype(np.int64) * g.n + g.dst).size == g.m
    assert g.w.min() >= 1 and g.w.max() <= 100
    deg = np.bincount(g.src, minlength=g.n)
    assert deg.max() <= 30          # near-uniform, mean 8


def test_rmat_shape_small():
    g = gg.rmat(14)
    assert g.n == 1 << 14 and g.m == 16 << 14
    assert g.w.min() >= 1 and g.w.max() <= 1000
    deg = np.bincount(g.src, minlength=g.n)
    assert deg.max() > 50 * deg.mean()   # power-law skew
    assert deg[0] == deg.max()           # a = 0.57 makes vertex 0 the hub
    assert np.any(g.src == g.dst)        # self-loops kept
    # quadrant frequencies of the top bit: P(src top bit = 0) = a + b = 0.76
    top = (g.src >> 13) & 1
    assert abs((top == 0).mean() - 0.76) < 0.01


def test_rmat_permutation_is_relabelling():
    a = gg.rmat(10, permute_seed=0)
    b = gg.rmat(10, permute_seed=99)
    da = np.sort(np.bincount(a.src, minlength=a.n))
    db = np.sort(np.bincount(b.src, minlength=b.n))
    np.testing.assert_array_equal(da, db)


def test_grid_shape():
    side = 64
    g = gg.grid(side, p_del=0.02, seed=3)
    nsc = gg.grid_shortcut_pairs(side)
    full = 4 * side * (side - 1)
    assert g.m % 2 == 0
    # every edge has its reverse (symmetric like a road network)
    fwd = set(zip(g.src.tolist(), g.dst.tolist()))
    assert all((v, u) in fwd for u, v in fwd)
    grid_edges = g.m - 2 * nsc
    kept = grid_edges / full
    assert 0.95 < kept < 1.0
    r0, c0 = np.divmod(g.src[:grid_edges], side)
    r1, c1 = np.divmod(g.dst[:grid_edges], side)
    assert np.all(np.abs(r0 - r1) + np.abs(c0 - c1) == 1)
    assert g.w.min() >= 1 and g.w.max() <= 10000
    assert gg.grid_shortcut_pairs(4096) == 33546


def test_sources_have_out_edges():
    g = gg.rmat(12)
    s = gg.sources(g, 8)
    assert len(set(s.tolist())) == 8
    deg = np.bincount(g.src, minlength=g.n)
    assert np.all(deg[s] > 0)
