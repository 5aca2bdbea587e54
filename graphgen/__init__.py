"""Seeded synthetic inputs shared by the oracle runs, the tests and the benchmark.

This module draws graphs and source vertices only; it holds none of the
relaxation arithmetic.  The C generators in ``gen.c`` are counter-based
(splitmix64), so every array is a pure function of its seed on any machine.

Workload recipes (the paper's own inputs -- USA road networks, orkut,
sinaweibo and its rand/rmat instances, Table "Benchmark characteristics",
Sec. 4.1 -- are not available; these shapes stand in for their classes):

* ``er``    -- G(n, m) directed, no self-loops/duplicates, weights U[1,100]
               (the "rand" class: near-uniform degree, small diameter).
* ``rmat``  -- R-MAT a,b,c,d = .57,.19,.19,.05, edge factor 16, self-loops
               and duplicates kept, weights U[1,1000] (the "rmat"/social
               class: power-law degree skew).
* ``grid``  -- 4-neighbour 2-D grid, 2 % of neighbour pairs deleted, 0.1 %
               random shortcut pairs, weights U[1,10000] (the road class:
               degree <= 5, large diameter).
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

# Default seeds of the named workloads.
SEED_ER = 0x1903_0166_5001
SEED_RMAT = 0x1903_0166_5002
SEED_GRID = 0x1903_0166_5003
SEED_SOURCES = 0x1903_0166_5004


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (gcc, OpenMP if present)."""
    lock_path = _LIB + ".lock"
    with open(lock_path, "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
        if fresh and not force:
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
        try:
            subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.gg_er.restype = ctypes.c_int64
    lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                          ctypes.c_int32, i32p, i32p, i32p]
    lib.gg_rmat.restype = None
    lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                            ctypes.c_uint64, i32p, i32p, i32p]
    lib.gg_grid.restype = ctypes.c_int64
    lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p]
    lib.gg_sources.restype = ctypes.c_int32
    lib.gg_sources.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, ctypes.c_int32,
                               ctypes.c_uint64, i32p]
    lib.gg_splitmix64.restype = ctypes.c_uint64
    lib.gg_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class Graph:
    """A directed edge list (COO, generation order) plus its vertex count."""

    def __init__(self, n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray, name: str):
        self.n = int(n)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.w = np.ascontiguousarray(w, dtype=np.int32)
        self.name = name

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def __repr__(self) -> str:
        return f"Graph({self.name}, n={self.n}, m={self.m})"


def er(n: int = 16384, m: int = 131072, seed: int = SEED_ER, wlo: int = 1, whi: int = 100) -> Graph:
    lib = _load()
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); w = np.empty(m, np.int32)
    r = lib.gg_er(n, m, seed, wlo, whi, _p(src), _p(dst), _p(w))
    if r < 0:
        raise ValueError("G(n,m) impossible for these sizes")
    return Graph(n, src, dst, w, f"er-{n}-{m}")


def rmat(scale: int = 22, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = SEED_RMAT, wlo: int = 1, whi: int = 1000,
         permute_seed: int = 0) -> Graph:
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); w = np.empty(m, np.int32)
    lib.gg_rmat(scale, m, a, b, c, seed, wlo, whi, permute_seed, _p(src), _p(dst), _p(w))
    return Graph(n, src, dst, w, f"rmat-{scale}")


def grid_shortcut_pairs(side: int, frac: float = 0.001) -> int:
    """Number of undirected shortcut pairs: frac of the full grid's undirected pairs."""
    full_directed = 4 * side * (side - 1)
    return int(round(frac * full_directed / 2))


def grid(side: int = 4096, p_del: float = 0.02, shortcut_frac: float = 0.001,
         seed: int = SEED_GRID, wlo: int = 1, whi: int = 10000, n_short: int | None = None) -> Graph:
    lib = _load()
    if n_short is None:
        n_short = grid_shortcut_pairs(side, shortcut_frac)
    cap = 4 * side * (side - 1) + 2 * n_short
    src = np.empty(cap, np.int32); dst = np.empty(cap, np.int32); w = np.empty(cap, np.int32)
    m = lib.gg_grid(side, p_del, n_short, seed, wlo, whi, cap, _p(src), _p(dst), _p(w))
    if m < 0:
        raise RuntimeError("grid buffer too small")
    return Graph(side * side, src[:m].copy(), dst[:m].copy(), w[:m].copy(), f"grid-{side}")


def sources(g: Graph, k: int = 8, seed: int = SEED_SOURCES) -> np.ndarray:
    """k distinct sources, uniform over vertices with out-degree > 0."""
    lib = _load()
    out = np.empty(k, np.int32)
    got = lib.gg_sources(g.n, g.m, _p(g.src), k, seed, _p(out))
    if got < 0:
        raise MemoryError
    return out[:got].copy()


def splitmix64(state: int, i: int) -> int:
    return int(_load().gg_splitmix64(state, i))


# ---- small structured graphs for edge cases (structure only) ----

def _mk(n, edges, name, w=None):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if w is None:
        w = np.ones(e.shape[0], np.int32)
    return Graph(n, e[:, 0], e[:, 1], np.asarray(w, np.int32), name)


def path(n: int, weights=None) -> Graph:
    """0 -> 1 -> ... -> n-1."""
    edges = [(i, i + 1) for i in range(n - 1)]
    return _mk(n, edges, f"path-{n}", weights)


def cycle(n: int) -> Graph:
    edges = [(i, (i + 1) % n) for i in range(n)]
    return _mk(n, edges, f"cycle-{n}")


def star(n: int, weights=None) -> Graph:
    """Hub 0 with out-edges to 1..n-1."""
    edges = [(0, i) for i in range(1, n)]
    return _mk(n, edges, f"star-{n}", weights)


def complete(n: int, seed: int = 7, wlo: int = 1, whi: int = 100) -> Graph:
    edges = [(i, j) for i in range(n) for j in range(n) if i != j]
    rng = np.random.Generator(np.random.PCG64(seed))
    return _mk(n, edges, f"complete-{n}", rng.integers(wlo, whi + 1, len(edges)))


def full_grid(rows: int, cols: int) -> Graph:
    """4-neighbour grid, both directions, unit weights, no deletions."""
    edges = []
    for r in range(rows):
        for c in range(cols):
            u = r * cols + c
            if c + 1 < cols:
                edges += [(u, u + 1), (u + 1, u)]
            if r + 1 < rows:
                edges += [(u, u + cols), (u + cols, u)]
    return _mk(rows * cols, edges, f"fullgrid-{rows}x{cols}")


def disjoint_cliques(sizes, seed: int = 11) -> Graph:
    """Cliques of the given sizes on consecutive ids, then ids shuffled by a seeded permutation.

    Returns the graph; ``.blocks`` holds each clique's vertex ids.
    """
    n = int(sum(sizes))
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n)
    edges, blocks, base = [], [], 0
    for s in sizes:
        ids = [int(perm[base + i]) for i in range(s)]
        blocks.append(ids)
        edges += [(a, b) for a in ids for b in ids if a < b]  # one direction only
        base += s
    g = _mk(n, edges if edges else np.zeros((0, 2)), f"cliques-{len(sizes)}")
    g.blocks = blocks
    return g


def random_small(n: int, m: int, seed: int, wlo: int = 0, whi: int = 20,
                 self_loops: bool = True, dups: bool = True) -> Graph:
    """Tiny random multigraph (numpy PCG64), for brute-force and Floyd-Warshall cases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    if not self_loops:
        keep = u != v
        u, v = u[keep], v[keep]
    if not dups and u.size:
        key = u * n + v
        _, first = np.unique(key, return_index=True)
        first.sort()
        u, v = u[first], v[first]
    w = rng.integers(wlo, whi + 1, u.size)
    return Graph(n, u, v, w, f"small-{n}-{m}-{seed}")


def hub(n: int, hub_degree: int, extra_m: int, seed: int = 5, wlo: int = 1, whi: int = 1000) -> Graph:
    """Vertex 0 with hub_degree out-edges to random targets, plus extra_m random edges."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hs = np.zeros(hub_degree, np.int64)
    hd = rng.integers(0, n, hub_degree)
    es = rng.integers(0, n, extra_m)
    ed = rng.integers(0, n, extra_m)
    src = np.concatenate([hs, es]); dst = np.concatenate([hd, ed])
    w = rng.integers(wlo, whi + 1, src.size)
    return Graph(n, src, dst, w, f"hub-{n}-{hub_degree}")


# ---- the batched workload: 64 resident graphs of uneven size, 512 queries

SEED_BATCH = 0x1903_0166_5005


def batched_graphs(seed: int = SEED_BATCH):
    """32 R-MAT graphs of scale 10 + (i mod 11) and 32 grids of side
    256 * 2^(i mod 4) (2 % deletions, 0.1 % shortcuts), weights U[1,1000]."""
    out = []
    for i in range(32):
        out.append(rmat(10 + (i % 11), seed=seed + i, whi=1000))
    for i in range(32):
        out.append(grid(256 << (i % 4), seed=seed + 100 + i, whi=1000))
    return out


def batched_queries(graphs, per_graph: int = 8, seed: int = SEED_BATCH):
    """per_graph seeded sources per graph, alternating SSSP (0) and BFS (1):
    a list of (graph index, algorithm, source)."""
    q = []
    for gi, g in enumerate(graphs):
        srcs = sources(g, per_graph, seed=seed + 1000 + gi)
        for k, s in enumerate(srcs):
            q.append((gi, k % 2, int(s)))
    return q
