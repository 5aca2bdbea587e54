/*
 * MULTI-CORE CPU BASELINE -- test infrastructure only; NOT the oracle.
 *
 * The paper compares Falcon's generated CUDA code with the OpenMP code that
 * Falcon generates for multi-core CPUs from the same programs (Sec. 4,
 * experimental setup and Table "CPU/GPU" results): a parallel loop over the
 * points or edges that applies MIN(t.dist, p.dist + w) with an atomic, run
 * until nothing changes.  This file is such a program, written here so that
 * the benchmark can report a multi-core host figure beside the sequential
 * oracle's: the same results, on all host cores.
 *
 *   ofr_sssp -- frontier Bellman-Ford: each round expands, in parallel, the
 *               vertices lowered in the round before, lowering targets in
 *               place with a 64-bit compare-and-swap minimum (Alg. 1's MIN
 *               applied by many threads); a vertex lowered in a round is put
 *               on the next frontier once (a per-vertex round stamp).
 *   ofr_bfs  -- level-synchronous top-down BFS (Alg. 3): the vertices at
 *               level lev claim their unvisited out-neighbours with a
 *               compare-and-swap from "unreached" to lev + 1.
 *   ofr_cc   -- weakly connected components by lock-free union-find over
 *               the edge list: a root is only ever hooked under a smaller
 *               id (compare-and-swap on the root's parent), so each tree's
 *               root is its smallest id, which is the label the oracle
 *               defines (minimum vertex id of the component).
 *
 * Status codes and the readings (unreached = INT32_MAX, weights >= 0, a
 * finite distance >= INT32_MAX is an overflow, self-loops and duplicates
 * kept) are the oracle's.  ofr_graph_build makes the adjacency once (a
 * parallel counting sort) for any number of SSSP and BFS queries, as the GPU
 * library's graph handle does; ofr_sssp and ofr_bfs build, query and free
 * in one call, as the oracle does.  The tests compare every function with
 * the oracle.  It shares no code with the oracle or with the CUDA library.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OFR_OK 0
#define OFR_INVALID 1
#define OFR_NEGATIVE_WEIGHT 2
#define OFR_OVERFLOW 3
#define OFR_NOMEM 4

#define UNREACHED INT32_MAX
#define FAR64 INT64_MAX

#define LD(p) __atomic_load_n((p), __ATOMIC_RELAXED)
#define ST(p, v) __atomic_store_n((p), (v), __ATOMIC_RELAXED)

int ofr_threads(void) { return omp_get_max_threads(); }
void ofr_set_threads(int t) {
    if (t > 0) omp_set_num_threads(t);
}

/* ---------------- input checks ---------------- */
static int check_input(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w) {
    if (n <= 0 || m < 0 || (m > 0 && (!src || !dst))) return OFR_INVALID;
    int bad = 0, neg = 0;
#pragma omp parallel for schedule(static) reduction(| : bad, neg)
    for (int64_t e = 0; e < m; e++) {
        bad |= src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n;
        if (w) neg |= w[e] < 0;
    }
    if (bad) return OFR_INVALID;
    return neg ? OFR_NEGATIVE_WEIGHT : OFR_OK;
}

/* ---------------- adjacency by a parallel counting sort ---------------- */
typedef struct {
    int64_t *start; /* n + 1 */
    int32_t *to;
    int32_t *wt;    /* NULL when unweighted */
} csr;

static void csr_free(csr *g) {
    free(g->start); free(g->to); free(g->wt);
}

/* inclusive prefix sum of a[0..len) over the team: each thread sums its
   block, the block totals are scanned once, then each block adds its
   offset */
static int scan_inclusive(int64_t *a, int64_t len) {
    const int nt = omp_get_max_threads();
    int64_t *part = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
    if (!part) return OFR_NOMEM;
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int64_t lo = len * t / T, hi = len * (t + 1) / T;
        int64_t s = 0;
        for (int64_t i = lo; i < hi; i++) { s += a[i]; a[i] = s; }
        part[t + 1] = s;
#pragma omp barrier
#pragma omp single
        for (int k = 1; k <= T; k++) part[k] += part[k - 1];
        const int64_t off = part[t];
        for (int64_t i = lo; i < hi; i++) a[i] += off;
    }
    free(part);
    return OFR_OK;
}

/* Each thread owns a contiguous range of source ids and streams the whole
   edge list, counting (then placing) only the edges whose source it owns:
   no atomics, no shared counters, rows in edge-list order.  Every thread
   reads the edge list once per pass; random atomic increments on shared
   counters were several times slower (one serialised cache miss each). */
static int csr_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w, csr *g) {
    g->start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->to = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    g->wt = w ? (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t)) : NULL;
    int64_t *cur = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!g->start || !g->to || (w && !g->wt) || !cur) { free(cur); csr_free(g); return OFR_NOMEM; }
#pragma omp parallel
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int32_t lo = (int32_t)((int64_t)n * t / T), hi = (int32_t)((int64_t)n * (t + 1) / T);
        int64_t *cnt = g->start + 1;
        for (int64_t e = 0; e < m; e++) {
            const int32_t u = src[e];
            if (u >= lo && u < hi) cnt[u]++;
        }
    }
    if (scan_inclusive(g->start + 1, n)) { free(cur); csr_free(g); return OFR_NOMEM; }
#pragma omp parallel
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int32_t lo = (int32_t)((int64_t)n * t / T), hi = (int32_t)((int64_t)n * (t + 1) / T);
        for (int32_t v = lo; v < hi; v++) cur[v] = g->start[v];
        for (int64_t e = 0; e < m; e++) {
            const int32_t u = src[e];
            if (u >= lo && u < hi) {
                const int64_t slot = cur[u]++;
                g->to[slot] = dst[e];
                if (w) g->wt[slot] = w[e];
            }
        }
    }
    free(cur);
    return OFR_OK;
}

/* ---------------- frontiers: per-thread buffers, gathered after a round ---------------- */
typedef struct {
    int32_t *a;
    int64_t n, cap;
    int oom;
} vec;

static inline void vec_push(vec *v, int32_t x) {
    if (v->n == v->cap) {
        const int64_t nc = v->cap ? 2 * v->cap : 4096;
        int32_t *na = (int32_t *)realloc(v->a, (size_t)nc * sizeof(int32_t));
        if (!na) { v->oom = 1; return; }
        v->a = na;
        v->cap = nc;
    }
    v->a[v->n++] = x;
}

typedef struct {
    int nt;          /* threads of every parallel region of the query */
    vec *loc;        /* [nt] this round's discoveries, by thread */
    int64_t *off;    /* [nt + 1] */
    int32_t *cur, *next;   /* [n] each */
    int64_t ncur;
} frontier;

static int frontier_init(frontier *f, int32_t n) {
    f->nt = omp_get_max_threads();
    f->loc = (vec *)calloc((size_t)f->nt, sizeof(vec));
    f->off = (int64_t *)calloc((size_t)f->nt + 1, sizeof(int64_t));
    f->cur = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    f->next = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    f->ncur = 0;
    return (f->loc && f->off && f->cur && f->next) ? OFR_OK : OFR_NOMEM;
}

static void frontier_free(frontier *f) {
    if (f->loc)
        for (int t = 0; t < f->nt; t++) free(f->loc[t].a);
    free(f->loc); free(f->off); free(f->cur); free(f->next);
}

/* the threads' discoveries become the next frontier (each vertex at most
   once: the callers push a vertex only from the one thread that claimed it
   for this round) */
static int frontier_advance(frontier *f) {
    int oom = 0;
    f->off[0] = 0;
    for (int t = 0; t < f->nt; t++) {
        f->off[t + 1] = f->off[t] + f->loc[t].n;
        oom |= f->loc[t].oom;
    }
    if (oom) return OFR_NOMEM;
#pragma omp parallel for schedule(static, 1) num_threads(f->nt)
    for (int t = 0; t < f->nt; t++)
        if (f->loc[t].n) memcpy(f->next + f->off[t], f->loc[t].a, (size_t)f->loc[t].n * sizeof(int32_t));
    int32_t *x = f->cur;
    f->cur = f->next;
    f->next = x;
    f->ncur = f->off[f->nt];
    for (int t = 0; t < f->nt; t++) f->loc[t].n = 0;
    return OFR_OK;
}

/* ---------------- SSSP: frontier Bellman-Ford, in-place atomic minimum ---------------- */
static int sssp_core(const csr *gp, int32_t n, int32_t s, int32_t *dist) {
    const csr g = *gp;
    int rc;
    int64_t *d = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *stamp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    frontier f;
    rc = frontier_init(&f, n);
    if (rc || !d || !stamp) {
        frontier_free(&f); free(d); free(stamp);
        return OFR_NOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; v++) { d[v] = FAR64; stamp[v] = 0; }
    d[s] = 0;
    f.cur[0] = s;
    f.ncur = 1;
    int32_t round = 0;
    while (f.ncur > 0) {
        round++;
        const int64_t fn = f.ncur;
#pragma omp parallel num_threads(f.nt)
        {
            vec *mine = &f.loc[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < fn; i++) {
                const int32_t u = f.cur[i];
                const int64_t du = LD(&d[u]);
                for (int64_t e = g.start[u]; e < g.start[u + 1]; e++) {
                    const int32_t v = g.to[e];
                    const int64_t nd = du + (g.wt ? g.wt[e] : 1);
                    int64_t old = LD(&d[v]);
                    while (nd < old) {
                        if (__atomic_compare_exchange_n(&d[v], &old, nd, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
                            /* lowered: on the next frontier once per round */
                            if (__atomic_exchange_n(&stamp[v], round, __ATOMIC_RELAXED) != round) vec_push(mine, v);
                            break;
                        }
                    }
                }
            }
        }
        if ((rc = frontier_advance(&f))) break;
    }
    if (!rc) {
        int over = 0;
#pragma omp parallel for schedule(static) reduction(| : over)
        for (int32_t v = 0; v < n; v++) {
            const int64_t x = d[v];
            if (x == FAR64) {
                dist[v] = UNREACHED;
            } else if (x >= (int64_t)INT32_MAX) {
                dist[v] = UNREACHED;
                over = 1;
            } else {
                dist[v] = (int32_t)x;
            }
        }
        rc = over ? OFR_OVERFLOW : OFR_OK;
    }
    frontier_free(&f); free(d); free(stamp);
    return rc;
}

/* ---------------- BFS: level-synchronous, claims by compare-and-swap ---------------- */
static int bfs_core(const csr *gp, int32_t n, int32_t s, int32_t *level) {
    const csr g = *gp;
    int rc;
    frontier f;
    if ((rc = frontier_init(&f, n))) { frontier_free(&f); return rc; }
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; v++) level[v] = UNREACHED;
    level[s] = 0;
    f.cur[0] = s;
    f.ncur = 1;
    for (int32_t lev = 0; f.ncur > 0; lev++) {
        const int64_t fn = f.ncur;
#pragma omp parallel num_threads(f.nt)
        {
            vec *mine = &f.loc[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < fn; i++) {
                const int32_t u = f.cur[i];
                for (int64_t e = g.start[u]; e < g.start[u + 1]; e++) {
                    const int32_t v = g.to[e];
                    if (LD(&level[v]) != UNREACHED) continue;
                    int32_t expect = UNREACHED;
                    if (__atomic_compare_exchange_n(&level[v], &expect, lev + 1, 0, __ATOMIC_RELAXED,
                                                    __ATOMIC_RELAXED))
                        vec_push(mine, v);
                }
            }
        }
        if ((rc = frontier_advance(&f))) break;
    }
    frontier_free(&f);
    return rc;
}

/* ---------------- public entry points ---------------- */
/* A graph built once for many queries (the adjacency of its edge list,
   weights kept when given). */
typedef struct ofr_graph {
    int32_t n;
    csr g;
} ofr_graph;

int ofr_graph_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w,
                    ofr_graph **out) {
    if (!out) return OFR_INVALID;
    *out = NULL;
    int rc = check_input(n, m, src, dst, w);
    if (rc) return rc;
    ofr_graph *h = (ofr_graph *)calloc(1, sizeof(ofr_graph));
    if (!h) return OFR_NOMEM;
    h->n = n;
    if ((rc = csr_build(n, m, src, dst, w, &h->g))) { free(h); return rc; }
    *out = h;
    return OFR_OK;
}

void ofr_graph_free(ofr_graph *h) {
    if (!h) return;
    csr_free(&h->g);
    free(h);
}

/* SSSP on a built graph (unit weights if it was built without them) */
int ofr_graph_sssp(const ofr_graph *h, int32_t s, int32_t *dist) {
    if (!h || s < 0 || s >= h->n || !dist) return OFR_INVALID;
    return sssp_core(&h->g, h->n, s, dist);
}

int ofr_graph_bfs(const ofr_graph *h, int32_t s, int32_t *level) {
    if (!h || s < 0 || s >= h->n || !level) return OFR_INVALID;
    return bfs_core(&h->g, h->n, s, level);
}

/* one query from an edge list: build, query, free */
int ofr_sssp(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w, int32_t s,
             int32_t *dist) {
    ofr_graph *h;
    int rc = ofr_graph_build(n, m, src, dst, w, &h);
    if (rc) return rc;
    rc = ofr_graph_sssp(h, s, dist);
    ofr_graph_free(h);
    return rc;
}

int ofr_bfs(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t s, int32_t *level) {
    ofr_graph *h;
    int rc = ofr_graph_build(n, m, src, dst, NULL, &h);
    if (rc) return rc;
    rc = ofr_graph_bfs(h, s, level);
    ofr_graph_free(h);
    return rc;
}

/* ---------------- CC: lock-free union-find, roots hooked under smaller ids ---------------- */
/* Root of x with path halving.  Parents only ever move to ancestors (a
   tree is never split, and an ancestor has a smaller id than its
   descendants), so a concurrent stale halving still points x at an
   ancestor; only roots are hooked, and only by compare-and-swap. */
static inline int32_t uf_find(int32_t *p, int32_t x) {
    for (;;) {
        const int32_t px = LD(&p[x]);
        if (px == x) return x;
        const int32_t ppx = LD(&p[px]);
        if (ppx != px) ST(&p[x], ppx);
        x = ppx;
    }
}

int ofr_cc(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *label) {
    int rc = check_input(n, m, src, dst, NULL);
    if (rc) return rc;
    if (!label) return OFR_INVALID;
    int32_t *p = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!p) return OFR_NOMEM;
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; v++) p[v] = v;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t e = 0; e < m; e++) {
        for (;;) {
            const int32_t ru = uf_find(p, src[e]), rv = uf_find(p, dst[e]);
            if (ru == rv) break;
            const int32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
            int32_t expect = hi;
            /* fails only if hi stopped being a root meanwhile: look again */
            if (__atomic_compare_exchange_n(&p[hi], &expect, lo, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) break;
        }
    }
    /* every root is its tree's smallest id, so the root is the label */
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; v++) label[v] = uf_find(p, v);
    free(p);
    return OFR_OK;
}
