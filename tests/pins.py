"""Independent references used to pin the oracle (tests only).

Each one reaches the fixpoint's result by a different route than the oracle:
Floyd-Warshall (all-pairs dynamic programming), brute-force enumeration of
simple paths, scipy.sparse.csgraph, and the invariant checks that any
fixpoint of the relaxation must satisfy (Sec. 2: no edge can still lower a
value, and every reached value is attained through some edge).
"""
from __future__ import annotations

import numpy as np

INF = 2**31 - 1
BIG = np.int64(1) << 62


def floyd_warshall(n, src, dst, w):
    """All-pairs shortest distances (int64, BIG = no path) by the O(n^3) recurrence."""
    d = np.full((n, n), BIG, dtype=np.int64)
    np.fill_diagonal(d, 0)
    for u, v, x in zip(np.asarray(src), np.asarray(dst), np.asarray(w)):
        if x < d[u, v]:
            d[u, v] = x
    for k in range(n):
        via = d[:, k:k + 1] + d[k:k + 1, :]
        via[d[:, k] >= BIG, :] = BIG
        via[:, d[k, :] >= BIG] = BIG
        np.minimum(d, via, out=d)
    return d


def brute_force_paths(n, src, dst, w, s):
    """Minimum weight and minimum hop count over all simple paths from s (tiny n only)."""
    adj = [[] for _ in range(n)]
    for u, v, x in zip(src, dst, w):
        adj[int(u)].append((int(v), int(x)))
    best_w = [None] * n
    best_h = [None] * n
    best_w[s] = 0
    best_h[s] = 0
    onpath = [False] * n

    def walk(u, acc_w, hops):
        onpath[u] = True
        for v, x in adj[u]:
            if onpath[v]:
                continue
            cw, ch = acc_w + x, hops + 1
            if best_w[v] is None or cw < best_w[v]:
                best_w[v] = cw
            if best_h[v] is None or ch < best_h[v]:
                best_h[v] = ch
            walk(v, cw, ch)
        onpath[u] = False

    walk(s, 0, 0)
    return best_w, best_h


def dedup_min(n, src, dst, w):
    """Collapse duplicate (u,v) pairs to their minimum weight and drop self-loops."""
    src = np.asarray(src, np.int64); dst = np.asarray(dst, np.int64); w = np.asarray(w, np.int64)
    keep = src != dst
    src, dst, w = src[keep], dst[keep], w[keep]
    if src.size == 0:
        return src, dst, w
    key = src * n + dst
    order = np.lexsort((w, key))
    key, w = key[order], w[order]
    first = np.ones(key.size, bool)
    first[1:] = key[1:] != key[:-1]
    key, w = key[first], w[first]
    return key // n, key % n, w


def check_sssp_invariants(n, src, dst, w, s, dist):
    """Fixpoint conditions of Alg. 1/2: dist[s]=0, no edge relaxes, each reached v is tight."""
    dist = np.asarray(dist, np.int64)
    src = np.asarray(src, np.int64); dst = np.asarray(dst, np.int64); w = np.asarray(w, np.int64)
    assert dist[s] == 0
    fin = dist[src] < INF
    cand = dist[src] + w
    assert np.all(dist[dst[fin]] <= cand[fin]), "some edge can still be relaxed"
    tight = np.zeros(n, bool)
    eq = fin & (dist[dst] == cand)
    tight[dst[eq]] = True
    reached = dist < INF
    reached[s] = False
    assert np.all(tight[reached]), "a reached vertex has no tight in-edge"


def check_bfs_invariants(n, src, dst, s, level):
    level = np.asarray(level, np.int64)
    src = np.asarray(src, np.int64); dst = np.asarray(dst, np.int64)
    assert level[s] == 0
    fin = level[src] < INF
    assert np.all(level[dst[fin]] <= level[src[fin]] + 1)
    tight = np.zeros(n, bool)
    eq = fin & (level[dst] == level[src] + 1)
    tight[dst[eq]] = True
    reached = level < INF
    reached[s] = False
    assert np.all(tight[reached])


def check_cc_invariants(n, src, dst, label):
    label = np.asarray(label, np.int64)
    src = np.asarray(src, np.int64); dst = np.asarray(dst, np.int64)
    assert np.all(label[src] == label[dst]), "an edge joins two labels"
    ids = np.arange(n)
    assert np.all(label <= ids)
    assert np.all(label[label] == label), "a label is not its own component's representative"


def dfs_component_count(n, src, dst):
    """Number of weak components by iterative DFS over the undirected adjacency."""
    adj = [[] for _ in range(n)]
    for u, v in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        adj[u].append(v)
        adj[v].append(u)
    seen = [False] * n
    count = 0
    for r in range(n):
        if seen[r]:
            continue
        count += 1
        stack = [r]
        seen[r] = True
        while stack:
            u = stack.pop()
            for v in adj[u]:
                if not seen[v]:
                    seen[v] = True
                    stack.append(v)
    return count


def sync_rounds_from_distances(n, src, dst, w, s, dist):
    """Jacobi round count from the definition: 1 + max over reached v of the fewest
    hops among shortest paths to v (computed by BFS over the tight-edge subgraph)."""
    dist = np.asarray(dist, np.int64)
    adj = [[] for _ in range(n)]
    for u, v, x in zip(np.asarray(src).tolist(), np.asarray(dst).tolist(), np.asarray(w).tolist()):
        if dist[u] < INF and dist[u] + x == dist[v]:
            adj[u].append(v)
    hops = [-1] * n
    hops[s] = 0
    q = [s]
    for u in q:
        for v in adj[u]:
            if hops[v] < 0:
                hops[v] = hops[u] + 1
                q.append(v)
    return 1 + max(hops)


def brute_force_hop_limited(n, src, dst, w, s, k):
    """Minimum weight over simple paths from s with at most k edges (None = no
    such path), by enumeration.  With w >= 0 a walk never beats its simple
    sub-path, so this is what k double-buffered rounds from (s: 0, else
    unreached) must hold (tiny n only)."""
    adj = [[] for _ in range(n)]
    for u, v, x in zip(src, dst, w):
        adj[int(u)].append((int(v), int(x)))
    best = [None] * n
    best[s] = 0
    stack = [(s, 0, 0, 1 << s)]
    while stack:
        u, dist, hops, seen = stack.pop()
        if hops == k:
            continue
        for v, x in adj[u]:
            if seen >> v & 1:
                continue
            nd = dist + x
            if best[v] is None or nd < best[v]:
                best[v] = nd
            stack.append((v, nd, hops + 1, seen | (1 << v)))
    return best
