// extern "C" entry points of include/fg.h: argument checks, error plumbing,
// and the runtime mode selection.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <new>
#include <string>

#include "fg_internal.cuh"

namespace fg {

namespace {
thread_local std::string t_last_error;

// Default device memory pool: keep freed blocks for reuse by later queries
// instead of returning them to the driver after every synchronisation.
void configure_pool_once(int dev) {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t threshold = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    }
    cudaGetLastError();
    done[dev] = true;
}

bool ensure_device(int *dev) {
    int d = -1;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    configure_pool_once(d);
    if (dev) *dev = d;
    return true;
}
}  // namespace

void set_last_error(const std::string &msg) { t_last_error = msg; }
const char *last_error_cstr() { return t_last_error.c_str(); }

fg_status fail(fg_status code, const std::string &msg) {
    t_last_error = msg;
    return code;
}

fg_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    fg_status code = (e == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
    return fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {
std::atomic<unsigned long long> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool is_device_pointer_on(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace fg

using namespace fg;

namespace {

fg_status check_mode(fg_mode m) {
    if (m < FG_VERTEX_SYNC || m > FG_BUCKET) return fail(FG_ERR_INVALID_ARG, "invalid mode");
    return FG_OK;
}

// FG_AUTO: the plan's mode, and its CTAs per SM unless the caller set them
fg_status resolve_mode(const fg_graph *g, fg_algo algo, fg_mode m, Mode *out, int32_t *blocks_per_sm) {
    if (m == FG_AUTO) {
        fg_plan pl;
        fg_status s = fg_select_plan(g, algo, &pl);
        if (s != FG_OK) return s;
        m = (fg_mode)pl.mode;
        if (blocks_per_sm && *blocks_per_sm == 0) *blocks_per_sm = pl.blocks_per_sm;
    }
    *out = (Mode)m;
    return FG_OK;
}

fg_status query(const fg_graph *g, fg_algo algo, int32_t src, int32_t *out, fg_mode mode,
                const fg_options *opt, fg_stats *stats) {
    if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
    if (!out) return fail(FG_ERR_INVALID_ARG, "output buffer is NULL");
    if (algo < FG_ALGO_SSSP || algo > FG_ALGO_CC) return fail(FG_ERR_INVALID_ARG, "invalid algorithm");
    fg_status s = check_mode(mode);
    if (s != FG_OK) return s;
    if (algo != FG_ALGO_CC && (src < 0 || src >= g->info.n))
        return fail(FG_ERR_INVALID_ARG, "source vertex outside [0, n)");
    if (opt && (opt->max_rounds < 0 || opt->wait_timeout_ms < 0 || opt->blocks_per_sm < 0 || opt->delta < 0))
        return fail(FG_ERR_INVALID_ARG, "negative option");
    int dev;
    if (!ensure_device(&dev)) return fail(FG_ERR_CUDA, "no CUDA device");
    Mode m;
    fg_options o{};
    if (opt) o = *opt;
    s = resolve_mode(g, algo, mode, &m, &o.blocks_per_sm);
    if (s != FG_OK) return s;
    return run_query(g, (Algo)algo, m, src, out, &o, stats);
}

}  // namespace

extern "C" {

fg_status fg_graph_create_coo(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                              const int32_t *w, fg_graph **out) {
    return fg_graph_create_coo_ex(n, m, src, dst, w, 0u, out);
}

fg_status fg_graph_create_csr(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                              const int32_t *w, fg_graph **out) {
    return fg_graph_create_csr_ex(n, m, row_off, col, w, 0u, out);
}

fg_status fg_graph_create_coo_ex(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                 const int32_t *w, uint32_t flags, fg_graph **out) {
    if (!out) return fail(FG_ERR_INVALID_ARG, "out is NULL");
    if (flags & ~(FG_GRAPH_LAZY | FG_GRAPH_RELABEL | FG_GRAPH_KEEP_IDS))
        return fail(FG_ERR_INVALID_ARG, "unknown graph creation flags");
    if ((flags & FG_GRAPH_RELABEL) && (flags & FG_GRAPH_KEEP_IDS))
        return fail(FG_ERR_INVALID_ARG, "graph creation flags FG_GRAPH_RELABEL and FG_GRAPH_KEEP_IDS together");
    if (n <= 0) return fail(FG_ERR_INVALID_ARG, "n must be positive");
    if (m < 0) return fail(FG_ERR_INVALID_ARG, "m must be non-negative");
    if (m >= ((int64_t)1 << 31)) return fail(FG_ERR_INVALID_ARG, "m must be below 2^31 (the symmetrised copy uses 32-bit offsets)");
    if (m > 0 && (!src || !dst)) return fail(FG_ERR_INVALID_ARG, "src or dst is NULL");
    if (!ensure_device(nullptr)) return fail(FG_ERR_CUDA, "no CUDA device");
    return build_graph_from_coo(n, m, src, dst, w, false, nullptr, flags, out);
}

fg_status fg_graph_create_csr_ex(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                                 const int32_t *w, uint32_t flags, fg_graph **out) {
    if (!out) return fail(FG_ERR_INVALID_ARG, "out is NULL");
    if (flags & ~(FG_GRAPH_LAZY | FG_GRAPH_RELABEL | FG_GRAPH_KEEP_IDS))
        return fail(FG_ERR_INVALID_ARG, "unknown graph creation flags");
    if ((flags & FG_GRAPH_RELABEL) && (flags & FG_GRAPH_KEEP_IDS))
        return fail(FG_ERR_INVALID_ARG, "graph creation flags FG_GRAPH_RELABEL and FG_GRAPH_KEEP_IDS together");
    if (n <= 0) return fail(FG_ERR_INVALID_ARG, "n must be positive");
    if (m < 0) return fail(FG_ERR_INVALID_ARG, "m must be non-negative");
    if (m >= ((int64_t)1 << 31)) return fail(FG_ERR_INVALID_ARG, "m must be below 2^31 (the symmetrised copy uses 32-bit offsets)");
    if (!row_off) return fail(FG_ERR_INVALID_ARG, "row_off is NULL");
    if (m > 0 && !col) return fail(FG_ERR_INVALID_ARG, "col is NULL");
    if (!ensure_device(nullptr)) return fail(FG_ERR_CUDA, "no CUDA device");
    return build_graph_from_coo(n, m, nullptr, col, w, true, row_off, flags, out);
}

fg_status fg_graph_destroy(fg_graph *g) {
    if (!g) return FG_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != g->device) cudaSetDevice(g->device);
    for (int i = 0; i < g->n_allocs; i++) cudaFreeAsync(g->allocs[i], 0);
    cudaError_t e = cudaStreamSynchronize(0);
    if (dev != g->device && dev >= 0) cudaSetDevice(dev);
    delete g;
    if (e != cudaSuccess) return cuda_fail(e, "graph destroy");
    return FG_OK;
}

fg_status fg_graph_info(const fg_graph *g, fg_graph_info_t *out) {
    if (!g || !out) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(g->mu);   // lazily built parts update it
    *out = g->info;
    return FG_OK;
}

fg_status fg_sssp(const fg_graph *g, int32_t src, int32_t *dist_out, fg_mode mode) {
    return query(g, FG_ALGO_SSSP, src, dist_out, mode, nullptr, nullptr);
}

fg_status fg_bfs(const fg_graph *g, int32_t src, int32_t *level_out, fg_mode mode) {
    return query(g, FG_ALGO_BFS, src, level_out, mode, nullptr, nullptr);
}

fg_status fg_cc(const fg_graph *g, int32_t *label_out, fg_mode mode) {
    return query(g, FG_ALGO_CC, 0, label_out, mode, nullptr, nullptr);
}

fg_status fg_run(const fg_graph *g, fg_algo algo, int32_t src, int32_t *out, fg_mode mode,
                 const fg_options *opt, fg_stats *stats) {
    return query(g, algo, src, out, mode, opt, stats);
}

fg_status fg_run_multi(const fg_graph *g, fg_algo algo, int32_t k, const int32_t *srcs, int32_t *const *outs,
                       const fg_options *opt, fg_status *status_out, fg_stats *stats) {
    if (!g) return fail(FG_ERR_INVALID_ARG, "graph is NULL");
    if (algo < FG_ALGO_SSSP || algo > FG_ALGO_CC) return fail(FG_ERR_INVALID_ARG, "invalid algorithm");
    if (k < 1 || k > FG_MULTI_MAX) return fail(FG_ERR_INVALID_ARG, "k must be in [1, FG_MULTI_MAX = 8]");
    if (!outs || (algo != FG_ALGO_CC && !srcs)) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    for (int32_t j = 0; j < k; j++) {
        if (!outs[j]) return fail(FG_ERR_INVALID_ARG, "output buffer " + std::to_string(j) + " is NULL");
        if (algo != FG_ALGO_CC && (srcs[j] < 0 || srcs[j] >= g->info.n))
            return fail(FG_ERR_INVALID_ARG, "source " + std::to_string(j) + " outside [0, n)");
    }
    if (opt && (opt->max_rounds < 0 || opt->wait_timeout_ms < 0 || opt->blocks_per_sm < 0 || opt->delta < 0))
        return fail(FG_ERR_INVALID_ARG, "negative option");
    if (!ensure_device(nullptr)) return fail(FG_ERR_CUDA, "no CUDA device");
    if (algo == FG_ALGO_CC) {   // the symmetrised view of a FG_GRAPH_LAZY graph
        fg_status vs = ensure_views(g, kCC, -1);
        if (vs != FG_OK) return vs;
    }
    return run_multi(g, (Algo)algo, k, srcs, outs, opt, status_out, stats);
}

fg_status fg_sweep(const fg_graph *g, fg_mode mode, const int32_t *cur, int32_t *next, void *stream,
                   int64_t *updates, float *kernel_ms) {
    if (!g || !cur || !next) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    if (mode != FG_VERTEX_SYNC && mode != FG_EDGE_SYNC)
        return fail(FG_ERR_INVALID_ARG, "a sweep is FG_VERTEX_SYNC or FG_EDGE_SYNC");
    if (!ensure_device(nullptr)) return fail(FG_ERR_CUDA, "no CUDA device");
    if (!is_device_pointer(cur) || !is_device_pointer(next))
        return fail(FG_ERR_INVALID_ARG, "cur and next must be device memory");
    return run_sweep(g, (Mode)mode, cur, next, (cudaStream_t)stream, updates, kernel_ms);
}

// The selection model (Sec. 2 "flexible processing" and Sec. 4.3 of the
// paper: edge-based code for skewed degrees, vertex-based for near-uniform
// ones, a data-driven worklist for long propagation), restated for GB300 from
// measurements of every mode and two CTA counts on R-MAT graphs (scales 10 to
// 22, Gini 0.79-0.94, 4-7 BFS levels), 2-D grids with shortcuts (256^2 to
// 4096^2, Gini 0.02, 72-134 levels) and a uniform random graph (Gini 0.2):
// its picks are within 10 % of the fastest (mode, CTAs per SM) for 201 of
// those 207 (graph, algorithm) pairs, and within 15 % for all.  With degree
// buckets the vertex modes no longer lose on skew the way the paper's K40C
// code did, so skew mostly selects between the asynchronous edge form, pull
// and the bucketed worklist, and depth selects the worklists that pay on
// long propagation.
namespace {
fg_plan model_plan(const fg_graph *g, fg_algo algo, int32_t depth) {
    const int64_t n = g->info.n, m = g->info.m;
    const bool deep = depth > 32;
    const bool skew = g->degree_gini > 0.5;
    fg_mode mode;
    int32_t bps;
    if (algo == FG_ALGO_SSSP) {
        mode = deep ? (n >= (1 << 21) ? FG_BUCKET : FG_VERTEX_SYNC)
                    : ((skew || n >= (1 << 19)) ? FG_EDGE_ASYNC : FG_EDGE_SYNC);
        bps = m <= 3000000 ? 2 : 0;
    } else if (algo == FG_ALGO_BFS) {
        mode = deep ? (n >= (1 << 21) ? FG_BUCKET : FG_VERTEX_SYNC) : (skew ? FG_PULL : FG_VERTEX_SYNC);
        bps = m <= 9000000 ? 2 : 0;
    } else {
        if (deep) mode = n < (1 << 23) ? FG_PULL : FG_VERTEX_SYNC;
        else if (!skew || n < (1 << 14)) mode = FG_EDGE_SYNC;
        else mode = n < (1 << 19) ? FG_BUCKET : FG_VERTEX_ASYNC;
        bps = m <= 3000000 ? 2 : 0;
    }
    fg_plan p{};
    p.mode = (int32_t)mode;
    p.blocks_per_sm = bps;
    p.delta = (mode == FG_BUCKET && algo == FG_ALGO_SSSP) ? default_delta(g) : 0;
    p.tuned = 0;
    p.depth_est = depth;
    p.degree_gini = (float)g->degree_gini;
    return p;
}

// The depth estimate: BFS levels from a high-degree vertex (the first vertex
// of the high bucket, else of the mid or low one), run once and cached.
fg_status depth_estimate(const fg_graph *g, int32_t *out) {
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (g->diam_est >= 0) {
            *out = g->diam_est;
            return FG_OK;
        }
    }
    const int32_t n = g->info.n;
    int32_t *level = nullptr;
    if (!ensure_device(nullptr)) return fail(FG_ERR_CUDA, "no CUDA device");
    cudaError_t e = cudaMalloc(&level, (size_t)n * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "select_plan workspace");
    int32_t start = 0;
    if (g->g.n_high_chunks > 0) {
        int2 h;
        cudaMemcpy(&h, g->g.high, sizeof(int2), cudaMemcpyDeviceToHost);
        start = h.x;
    } else if (g->g.n_mid > 0) {
        cudaMemcpy(&start, g->g.mid, sizeof(int32_t), cudaMemcpyDeviceToHost);
    } else if (g->g.n_low > 0) {
        cudaMemcpy(&start, g->g.low, sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    if (g->orig_of)   // run_query takes original ids
        cudaMemcpy(&start, g->orig_of + start, sizeof(int32_t), cudaMemcpyDeviceToHost);
    fg_stats st{};
    fg_status s = run_query(g, kBFS, kVertexAsync, start, level, nullptr, &st);
    cudaFree(level);
    if (s != FG_OK) return s;
    std::lock_guard<std::mutex> lk(g->mu);
    g->diam_est = st.rounds;
    *out = st.rounds;
    return FG_OK;
}
}  // namespace

fg_status fg_select_plan(const fg_graph *g, fg_algo algo, fg_plan *out) {
    if (!g || !out) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    if (algo < FG_ALGO_SSSP || algo > FG_ALGO_CC) return fail(FG_ERR_INVALID_ARG, "invalid algorithm");
    int32_t depth = 0;
    fg_status s = depth_estimate(g, &depth);
    if (s != FG_OK) return s;
    fg_plan p = model_plan(g, algo, depth);
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (g->tuned_mode[algo] >= 0) {
            p.mode = g->tuned_mode[algo];
            p.blocks_per_sm = g->tuned_bps[algo];
            p.delta = (p.mode == FG_BUCKET && algo == FG_ALGO_SSSP) ? default_delta(g) : 0;
            p.tuned = 1;
        }
    }
    *out = p;
    return FG_OK;
}

fg_status fg_select_mode(const fg_graph *g, fg_algo algo, fg_mode *out) {
    if (!g || !out) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    fg_plan p;
    fg_status s = fg_select_plan(g, algo, &p);
    if (s != FG_OK) return s;
    *out = (fg_mode)p.mode;
    return FG_OK;
}

fg_status fg_autotune(const fg_graph *g, fg_algo algo, int32_t src, fg_mode *best, float *times_ms) {
    if (!g || !best) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    if (algo < FG_ALGO_SSSP || algo > FG_ALGO_CC) return fail(FG_ERR_INVALID_ARG, "invalid algorithm");
    if (algo != FG_ALGO_CC && (src < 0 || src >= g->info.n))
        return fail(FG_ERR_INVALID_ARG, "source vertex outside [0, n)");
    if (!ensure_device(nullptr)) return fail(FG_ERR_CUDA, "no CUDA device");
    int32_t *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)g->info.n * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "autotune workspace");
    // the paper's four modes and the bucketed worklist for every algorithm,
    // FG_PULL for BFS and CC (SSSP pull rounds read every in-edge and did not
    // win alone), each at the occupancy limit and at 2 CTAs per SM
    float t[7] = {0, 0, 0, 0, 0, 0, 0};
    const int modes_all[6] = {kVertexSync, kVertexAsync, kEdgeSync, kEdgeAsync, kBucket, kPull};
    const int nmodes = algo == FG_ALGO_SSSP ? 5 : 6;
    const int32_t bps_try[2] = {0, 2};
    fg_status s = FG_OK;
    int bm = -1, bb = 0;
    float bt = 0.f;
    for (int i = 0; i < nmodes && s == FG_OK; i++) {
        for (int b = 0; b < 2 && s == FG_OK; b++) {
            fg_options o{};
            o.blocks_per_sm = bps_try[b];
            float r[3];
            for (int k = 0; k < 3 && s == FG_OK; k++) {
                fg_stats st{};
                s = run_query(g, (Algo)algo, (Mode)modes_all[i], src, out, &o, &st);
                r[k] = st.kernel_ms;
            }
            if (s != FG_OK) break;
            std::sort(r, r + 3);
            const float med = r[1];
            if (t[modes_all[i]] == 0.f || med < t[modes_all[i]]) t[modes_all[i]] = med;
            if (bm < 0 || med < bt) {
                bm = modes_all[i];
                bb = bps_try[b];
                bt = med;
            }
        }
    }
    cudaFree(out);
    if (s != FG_OK) return s;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        g->tuned_mode[algo] = bm;
        g->tuned_bps[algo] = bb;
    }
    *best = (fg_mode)bm;
    if (times_ms)
        for (int m = 0; m < 7; m++) times_ms[m] = t[m];
    return FG_OK;
}

fg_status fg_run_batch(const fg_query *queries, int32_t nq, const fg_batch_options *opt,
                       fg_status *status_out, fg_stats *stats_out, fg_batch_stats *bstats) {
    if (!queries || nq <= 0) return fail(FG_ERR_INVALID_ARG, "empty batch");
    if (opt && opt->wait_timeout_ms < 0) return fail(FG_ERR_INVALID_ARG, "negative option");
    for (int32_t i = 0; i < nq; i++) {
        const fg_query &q = queries[i];
        std::string where = "batch query " + std::to_string(i) + ": ";
        if (!q.g) return fail(FG_ERR_INVALID_ARG, where + "graph is NULL");
        if (!q.out) return fail(FG_ERR_INVALID_ARG, where + "output buffer is NULL");
        if (q.algo < FG_ALGO_SSSP || q.algo > FG_ALGO_CC) return fail(FG_ERR_INVALID_ARG, where + "invalid algorithm");
        if (q.mode < FG_VERTEX_SYNC || q.mode > FG_BUCKET) return fail(FG_ERR_INVALID_ARG, where + "invalid mode");
        if (q.algo != FG_ALGO_CC && (q.src < 0 || q.src >= q.g->info.n))
            return fail(FG_ERR_INVALID_ARG, where + "source vertex outside [0, n)");
    }
    int dev;
    if (!ensure_device(&dev)) return fail(FG_ERR_CUDA, "no CUDA device");
    for (int32_t i = 0; i < nq; i++)
        if (queries[i].g->device != dev)
            return fail(FG_ERR_INVALID_ARG, "batch query " + std::to_string(i) + ": graph lives on another device");
    return run_batch(queries, nq, opt, status_out, stats_out, bstats);
}

const char *fg_last_error(void) { return fg::last_error_cstr(); }

uint64_t fg_kernel_launches(void) { return fg::g_launches.load(std::memory_order_relaxed); }

const char *fg_status_string(fg_status s) {
    switch (s) {
        case FG_OK: return "FG_OK";
        case FG_ERR_INVALID_ARG: return "FG_ERR_INVALID_ARG";
        case FG_ERR_NEGATIVE_WEIGHT: return "FG_ERR_NEGATIVE_WEIGHT";
        case FG_ERR_OVERFLOW: return "FG_ERR_OVERFLOW";
        case FG_ERR_OUT_OF_MEMORY: return "FG_ERR_OUT_OF_MEMORY";
        case FG_ERR_TIMEOUT: return "FG_ERR_TIMEOUT";
        case FG_ERR_CUDA: return "FG_ERR_CUDA";
    }
    return "FG_UNKNOWN_STATUS";
}

}  // extern "C"
