/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, sequential, obviously-correct definitions of what the fixpoint
 * relaxation computes.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * What the method computes (Sec. 2, Algorithms 1-3):
 *   SSSP  -- Algorithms 1 and 2 repeat MIN(t.dist, p.dist + w(p,t)) over
 *            every edge until no dist changes.  With w >= 0 that fixpoint is
 *            the shortest-path distance, so the oracle is textbook Dijkstra
 *            (binary heap, lazy deletion) in 64-bit sums.
 *   BFS   -- Algorithm 3 sets t.dist = lev+1 for out-neighbours of the
 *            vertices at level lev, for lev = 0, 1, ...; the fixpoint is the
 *            hop distance, so the oracle is a FIFO-queue BFS.
 *   CC    -- the paper benchmarks connected components (Sec. 4.1) but prints
 *            no algorithm; min-label propagation over the undirected
 *            neighbour iterator (Table "foreach iterators", nbrs) converges to
 *            the smallest vertex id of each component, so the oracle is
 *            union-find (path halving, union by size) followed by a
 *            per-component minimum.
 *   Jacobi round count -- the synchronous variant's round count, defined
 *            by double-buffered Bellman-Ford: D_r = min(D_{r-1}, min over
 *            edges of D_{r-1}[u] + w), counted until the first round that
 *            changes nothing (inclusive).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   - "unreached" is INT32_MAX for all three outputs (Alg. 1 uses MAX_INT,
 *     Alg. 3 uses 1234567890).
 *   - The source is an argument (the paper fixes point zero).
 *   - Weights must be >= 0; w == 0 is allowed.  BFS and CC ignore weights.
 *   - Overflow: if some vertex's exact shortest distance is finite but
 *     >= INT32_MAX, the query fails with status ORACLE_OVERFLOW.
 *   - CC works on the symmetrised graph (each edge also read backwards);
 *     the label is the minimum vertex id of the component.
 *   - Self-loops and duplicate edges are kept.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_INVALID 1
#define ORACLE_NEGATIVE_WEIGHT 2
#define ORACLE_OVERFLOW 3
#define ORACLE_NOMEM 4

#define UNREACHED INT32_MAX

/* Out-adjacency (CSR) built by a counting sort of the edge list. */
typedef struct {
    int64_t *start; /* n + 1 */
    int32_t *to;
    int32_t *wt;    /* may be NULL */
} adjacency;

static void adj_free(adjacency *a) {
    free(a->start); free(a->to); free(a->wt);
}

static int adj_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const int32_t *w, adjacency *a) {
    a->start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    a->to = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    a->wt = w ? (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t)) : NULL;
    if (!a->start || !a->to || (w && !a->wt)) { adj_free(a); return ORACLE_NOMEM; }
    for (int64_t e = 0; e < m; e++) a->start[src[e] + 1]++;
    for (int32_t v = 0; v < n; v++) a->start[v + 1] += a->start[v];
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t) + 1);
    if (!fill) { adj_free(a); return ORACLE_NOMEM; }
    memcpy(fill, a->start, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; e++) {
        int64_t slot = fill[src[e]]++;
        a->to[slot] = dst[e];
        if (w) a->wt[slot] = w[e];
    }
    free(fill);
    return ORACLE_OK;
}

static int check_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    if (n <= 0 || m < 0 || (m > 0 && (!src || !dst))) return ORACLE_INVALID;
    for (int64_t e = 0; e < m; e++)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORACLE_INVALID;
    return ORACLE_OK;
}

/* ---------------- binary min-heap of (key, vertex) ---------------- */
typedef struct { int64_t key; int32_t v; } heap_item;
typedef struct { heap_item *a; int64_t size, cap; } heap;

static int heap_push(heap *h, int64_t key, int32_t v) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        heap_item *na = (heap_item *)realloc(h->a, (size_t)nc * sizeof(heap_item));
        if (!na) return ORACLE_NOMEM;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->size++;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (h->a[parent].key <= key) break;
        h->a[i] = h->a[parent];
        i = parent;
    }
    h->a[i].key = key; h->a[i].v = v;
    return ORACLE_OK;
}

static heap_item heap_pop(heap *h) {
    heap_item top = h->a[0];
    heap_item last = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        int64_t skey = last.key;
        if (l < h->size && h->a[l].key < skey) { s = l; skey = h->a[l].key; }
        if (r < h->size && h->a[r].key < skey) { s = r; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

/*
 * SSSP from s: Dijkstra with 64-bit tentative distances.  dist[v] =
 * shortest distance, UNREACHED if no path.  Returns ORACLE_OVERFLOW if a
 * finite distance is >= INT32_MAX (those entries are written UNREACHED).
 */
int or_sssp(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w,
            int32_t s, int32_t *dist) {
    int rc = check_edges(n, m, src, dst);
    if (rc) return rc;
    if (s < 0 || s >= n || !dist) return ORACLE_INVALID;
    if (w) for (int64_t e = 0; e < m; e++) if (w[e] < 0) return ORACLE_NEGATIVE_WEIGHT;
    adjacency a;
    if ((rc = adj_build(n, m, src, dst, w, &a))) return rc;
    int64_t *d = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    heap h = {0, 0, 0};
    if (!d || !done) { free(d); free(done); adj_free(&a); return ORACLE_NOMEM; }
    for (int32_t v = 0; v < n; v++) d[v] = INT64_MAX;
    d[s] = 0;
    rc = heap_push(&h, 0, s);
    while (rc == ORACLE_OK && h.size > 0) {
        heap_item it = heap_pop(&h);
        if (done[it.v] || it.key != d[it.v]) continue;   /* stale entry */
        done[it.v] = 1;
        for (int64_t k = a.start[it.v]; k < a.start[it.v + 1]; k++) {
            int32_t t = a.to[k];
            int64_t cand = it.key + (w ? (int64_t)a.wt[k] : 1);
            if (cand < d[t]) {
                d[t] = cand;
                if ((rc = heap_push(&h, cand, t))) break;
            }
        }
    }
    int overflow = 0;
    for (int32_t v = 0; v < n; v++) {
        if (d[v] == INT64_MAX) dist[v] = UNREACHED;
        else if (d[v] >= (int64_t)INT32_MAX) { dist[v] = UNREACHED; overflow = 1; }
        else dist[v] = (int32_t)d[v];
    }
    free(h.a); free(d); free(done); adj_free(&a);
    if (rc) return rc;
    return overflow ? ORACLE_OVERFLOW : ORACLE_OK;
}

/* BFS from s: level[v] = fewest edges on a path s -> v, UNREACHED if none. */
int or_bfs(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t s,
           int32_t *level) {
    int rc = check_edges(n, m, src, dst);
    if (rc) return rc;
    if (s < 0 || s >= n || !level) return ORACLE_INVALID;
    adjacency a;
    if ((rc = adj_build(n, m, src, dst, NULL, &a))) return rc;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) { adj_free(&a); return ORACLE_NOMEM; }
    for (int32_t v = 0; v < n; v++) level[v] = UNREACHED;
    int64_t head = 0, tail = 0;
    level[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t k = a.start[u]; k < a.start[u + 1]; k++) {
            int32_t t = a.to[k];
            if (level[t] == UNREACHED) {
                level[t] = level[u] + 1;
                queue[tail++] = t;
            }
        }
    }
    free(queue); adj_free(&a);
    return ORACLE_OK;
}

static int32_t uf_find(int32_t *parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];   /* path halving */
        x = parent[x];
    }
    return x;
}

/* CC: label[v] = minimum vertex id in v's component of the undirected graph. */
int or_cc(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *label) {
    int rc = check_edges(n, m, src, dst);
    if (rc) return rc;
    if (!label) return ORACLE_INVALID;
    int32_t *parent = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *size = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *minid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!parent || !size || !minid) { free(parent); free(size); free(minid); return ORACLE_NOMEM; }
    for (int32_t v = 0; v < n; v++) { parent[v] = v; size[v] = 1; }
    for (int64_t e = 0; e < m; e++) {
        int32_t ru = uf_find(parent, src[e]), rv = uf_find(parent, dst[e]);
        if (ru == rv) continue;
        if (size[ru] < size[rv]) { int32_t t = ru; ru = rv; rv = t; }
        parent[rv] = ru;
        size[ru] += size[rv];
    }
    for (int32_t v = 0; v < n; v++) minid[v] = INT32_MAX;
    for (int32_t v = 0; v < n; v++) {
        int32_t r = uf_find(parent, v);
        if (v < minid[r]) minid[r] = v;
    }
    for (int32_t v = 0; v < n; v++) label[v] = minid[uf_find(parent, v)];
    free(parent); free(size); free(minid);
    return ORACLE_OK;
}

/*
 * Jacobi (double-buffered) Bellman-Ford from s, run until a round changes
 * nothing.  Writes the distances and returns the number of rounds executed,
 * the final no-change round included; negative values are error codes.
 * unit != 0 ignores w (every edge weighs 1), which gives the level-synchronous
 * BFS round count.  Hitting the cap max_rounds returns -ORACLE_INVALID.
 */
int64_t or_jacobi_rounds(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                         const int32_t *w, int32_t s, int unit, int64_t max_rounds,
                         int32_t *dist) {
    int rc = check_edges(n, m, src, dst);
    if (rc) return -rc;
    if (s < 0 || s >= n) return -ORACLE_INVALID;
    int64_t *cur = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!cur || !next) { free(cur); free(next); return -ORACLE_NOMEM; }
    for (int32_t v = 0; v < n; v++) cur[v] = INT64_MAX;
    cur[s] = 0;
    int64_t rounds = 0;
    for (;;) {
        if (rounds >= max_rounds) { free(cur); free(next); return -ORACLE_INVALID; }
        rounds++;
        memcpy(next, cur, (size_t)n * sizeof(int64_t));
        int changed = 0;
        for (int64_t e = 0; e < m; e++) {
            if (cur[src[e]] == INT64_MAX) continue;
            int64_t cand = cur[src[e]] + ((unit || !w) ? 1 : (int64_t)w[e]);
            if (cand < next[dst[e]]) { next[dst[e]] = cand; changed = 1; }
        }
        int64_t *t = cur; cur = next; next = t;
        if (!changed) break;
    }
    if (dist)
        for (int32_t v = 0; v < n; v++)
            dist[v] = (cur[v] == INT64_MAX || cur[v] >= INT32_MAX) ? UNREACHED : (int32_t)cur[v];
    free(cur); free(next);
    return rounds;
}

/*
 * One relaxation round from a given state, every vertex active: the body of
 * Algorithm 1 (over CSR) and Algorithm 2 (over the edge list) applied once,
 * double-buffered.  For every edge u->v with cur[u] finite, the candidate
 * cur[u] + w (64-bit) lowers next[v] if smaller.  A candidate that reaches
 * INT32_MAX is not written and makes the call return ORACLE_OVERFLOW (the
 * other edges are still applied).  *lowered receives the number of vertices
 * whose next value went down.  cur and next must not overlap.
 */
int or_sweep(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w,
             const int32_t *cur, int32_t *next, int64_t *lowered) {
    int rc = check_edges(n, m, src, dst);
    if (rc) return rc;
    if (!cur || !next) return ORACLE_INVALID;
    for (int64_t e = 0; e < m; e++)
        if (w && w[e] < 0) return ORACLE_NEGATIVE_WEIGHT;
    int32_t *before = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!before) return ORACLE_NOMEM;
    memcpy(before, next, (size_t)n * sizeof(int32_t));
    int overflow = 0;
    for (int64_t e = 0; e < m; e++) {
        if (cur[src[e]] == UNREACHED) continue;
        int64_t cand = (int64_t)cur[src[e]] + (w ? (int64_t)w[e] : 1);
        if (cand >= INT32_MAX) { overflow = 1; continue; }
        if (cand < next[dst[e]]) next[dst[e]] = (int32_t)cand;
    }
    int64_t count = 0;
    for (int32_t v = 0; v < n; v++) count += next[v] < before[v];
    free(before);
    if (lowered) *lowered = count;
    return overflow ? ORACLE_OVERFLOW : ORACLE_OK;
}
