// Single-query entry of the fixpoint sweep: one persistent cooperative
// kernel per query, the whole grid as one team; the multi-source sweep (up
// to 8 queries on one graph in one launch); plus the all-active sweep used
// for roofline measurements and the overflow test.
#include <algorithm>

#include "fg_multi.cuh"

namespace fg {

namespace {

template <int ALGO, int MODE>
__global__ void __launch_bounds__(kBlock, min_blocks<MODE>()) fixpoint_kernel(Params p) {
    const Team t{(int)blockIdx.x, (int)gridDim.x, &p.ctrl->bar_count};
    uint32_t ring_used;
    fixpoint_prologue<ALGO, MODE>(ring_used);
    query_body<ALGO, MODE>(p, t, ring_used);
}

// One all-active sweep: vertex variant over the buckets, edge variant over
// the COO (staged edge stream).  Ordinary launch (no grid barrier).  The
// vertex variant is held to 32 registers, 8 CTAs per SM: all 64 warps of an
// SM in flight for its latency-bound gathers (at 40 registers, 6 CTAs, its
// all-active round ran 3 % slower under ncu); the edge variant keeps 6 CTAs
// at 40 registers.
constexpr unsigned long long kSweepTimeoutNs = 2000000000ull;
template <int MODE>
__global__ void __launch_bounds__(kBlock, MODE == kVertexSync ? 8 : 6)
    sweep_kernel(View g, const int32_t *cur, int32_t *next, Ctrl *c) {
    const Team t{(int)blockIdx.x, (int)gridDim.x, nullptr};
    Acc a;
    SweepOp op{g.w, cur, next};
    if constexpr (MODE == kVertexSync) {
        expand_vertices(t, g.row_off, g.col, g.low, g.n_low, g.mid, g.n_mid, g.high, g.n_high_chunks, op, NoPush{},
                        a);
    } else {
        uint32_t used = 0;
        rings_init(edge_rings<true>());
        stream_all_edges<true>(t, used, g, op, a, c, kSweepTimeoutNs);
    }
    unsigned long long eu = block_sum(a.updates);
    int of = block_sum(a.overflow);
    if (threadIdx.x == 0) {
        if (eu) atomicAdd(&c->st_updates, eu);
        if (of) atomicOr(&c->status, kStOverflow);
    }
}

// FG_ERR_OVERFLOW test: some edge u->v with dist[u] finite and dist[v] still
// INF means v's true distance is finite but >= INT32_MAX.
__global__ void overflow_check_kernel(View g, const int32_t *D, int *flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.m; e += (int64_t)gridDim.x * blockDim.x) {
        if (__ldg(D + g.src[e]) != kInf && __ldg(D + g.col[e]) == kInf) {
            *flag = 1;
            return;
        }
    }
}

// ================================================================ host side
using KernelFn = void (*)(Params);

KernelFn kernel_for(Algo algo, Mode mode) {
#define FG_K(A, M) \
    if (algo == A && mode == M) return fixpoint_kernel<A, M>;
    FG_K(kSSSP, kVertexSync) FG_K(kSSSP, kVertexAsync) FG_K(kSSSP, kEdgeSync) FG_K(kSSSP, kEdgeAsync)
    FG_K(kBFS, kVertexSync) FG_K(kBFS, kVertexAsync) FG_K(kBFS, kEdgeSync) FG_K(kBFS, kEdgeAsync)
    FG_K(kCC, kVertexSync) FG_K(kCC, kVertexAsync) FG_K(kCC, kEdgeSync) FG_K(kCC, kEdgeAsync)
    FG_K(kSSSP, kPull) FG_K(kBFS, kPull) FG_K(kCC, kPull)
    FG_K(kSSSP, kBucket) FG_K(kBFS, kBucket) FG_K(kCC, kBucket)
    FG_K(kSSSP, kMulti) FG_K(kBFS, kMulti)
#undef FG_K
    return nullptr;
}

struct DeviceProps {
    int sms = 0;
    bool coop = false;
};

DeviceProps device_props(int dev) {
    static std::mutex mu;
    static DeviceProps cache[64];
    static bool have[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && have[dev]) return cache[dev];
    DeviceProps p;
    cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    p.coop = coop != 0;
    if (dev >= 0 && dev < 64) { cache[dev] = p; have[dev] = true; }
    return p;
}

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}


}  // namespace

void overflow_check_launch(const View &g, const int32_t *D, int *flag, cudaStream_t st) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    overflow_check_kernel<<<std::max(1, sms) * 8, kBlock, 0, st>>>(g, D, flag);
    count_launch();
}

void ms_overflow_check_launch(const View &g, const int32_t *D, int k, int *flag, cudaStream_t st) {
    ms_overflow_check_kernel<<<std::max(1, device_props(current_device()).sms) * 8, kBlock, 0, st>>>(g, D, k, flag);
    count_launch();
}

void ms_output_launch(const int32_t *D, int32_t n, int k, const MsOuts &outs, const int32_t *new_of,
                      cudaStream_t st) {
    ms_output_kernel<<<std::max(1, device_props(current_device()).sms) * 8, kBlock, 0, st>>>(D, n, k, outs,
                                                                                             new_of);
    count_launch();
}

// ---------------------------------------------------------------- renumbered graphs
namespace {
// out[v] = res[idx[v]]: with idx = new_of, an internal-order result in
// original order; with idx = orig_of, the reverse
__global__ void k_gather_out(int32_t n, const int32_t *__restrict__ res, const int32_t *__restrict__ idx,
                             int32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = res[idx[v]];
}
__global__ void k_fill_inf(int32_t n, int32_t *x) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        x[v] = kInf;
}
// mn[L] = the smallest original id among the vertices labelled L
__global__ void k_cc_min_orig(int32_t n, const int32_t *__restrict__ lab, const int32_t *__restrict__ orig_of,
                              int32_t *mn) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    cc_min_orig_warp(warp, nwarps, n, [&](int64_t u) { return lab[u]; }, orig_of, mn);
}
// out[v] = mn[lab[new_of[v]]]: every vertex labelled with its component's smallest original id
__global__ void k_cc_out(int32_t n, const int32_t *__restrict__ lab, const int32_t *__restrict__ new_of,
                         const int32_t *__restrict__ mn, int32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = mn[lab[new_of[v]]];
}
}  // namespace

void set_relabel(const fg_graph *G, Params &p) {
    p.new_of = G->new_of;
    p.orig_of = G->orig_of;
}

fg_status relabel_output(const fg_graph *G, Algo algo, const int32_t *res, int32_t *out, cudaStream_t st) {
    const int32_t n = G->info.n;
    const bool direct = is_device_pointer_on(out, G->device);
    const int64_t tmp_n = (direct ? 0 : (int64_t)n) + (algo == kCC ? (int64_t)n : 0);
    int32_t *tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (tmp_n > 0) e = cudaMallocAsync((void **)&tmp, (size_t)tmp_n * sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "output permutation workspace");
    int32_t *dst = direct ? out : tmp;
    const int grid = std::max(1, device_props(G->device).sms) * 8;
    if (algo == kCC) {
        int32_t *mn = tmp + (direct ? 0 : n);
        k_fill_inf<<<grid, kBlock, 0, st>>>(n, mn);
        k_cc_min_orig<<<grid, kBlock, 0, st>>>(n, res, G->orig_of, mn);
        k_cc_out<<<grid, kBlock, 0, st>>>(n, res, G->new_of, mn, dst);
        count_launch();
        count_launch();
        count_launch();
    } else {
        k_gather_out<<<grid, kBlock, 0, st>>>(n, res, G->new_of, dst);
        count_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && !direct) e = cudaMemcpyAsync(out, dst, (size_t)n * sizeof(int32_t), cudaMemcpyDefault, st);
    if (tmp) cudaFreeAsync(tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "output permutation");
    return FG_OK;
}

namespace {
int64_t wl_cap_of(const View &g, Mode mode, int k) {
    if (mode == kVertexAsync || mode == kBucket) {
        if (k == kWlLow) return std::max(g.n_low, 1);
        if (k == kWlMid) return std::max(g.n_mid, 1);
        return 2 * (int64_t)std::max(g.n_high_chunks, 1);
    }
    if (mode == kEdgeAsync) return k == 0 ? std::max(g.n_nz, 1) : 1;
    return 0;
}
}  // namespace

// Bytes of one query's device state (control block, value buffers, stamps,
// worklists, edge offsets, warp-tile flags, far lists), each piece 256-byte
// aligned.
size_t query_workspace_bytes(const View &g, Algo algo, Mode mode) {
    const int32_t n = g.n;
    if (mode == kMulti) {
        if (algo == kBFS)   // control block, reached-by masks, three frontier mask arrays
            return Workspace::need(1, sizeof(Ctrl)) + Workspace::need(msb_pad(n), 1) +
                   Workspace::need(3 * msb_pad(n), 1);
        // control block, rows of 8 values, stamps, far-pending epochs
        return Workspace::need(1, sizeof(Ctrl)) + Workspace::need((int64_t)n * 8, 4) + 2 * Workspace::need(n, 4);
    }
    const bool sync = (mode == kVertexSync || mode == kEdgeSync || mode == kPull);
    size_t need = Workspace::need(1, sizeof(Ctrl)) + Workspace::need(n, 4);
    if (sync && algo != kBFS) need += 3 * Workspace::need(n, 4);
    const int64_t nwt = (g.m + kWTile - 1) / kWTile;   // edge-sync: one flag per 128-edge warp tile
    if (mode == kEdgeSync) need += Workspace::need(nwt, 4);
    if (algo == kBFS) need += Workspace::need(((int64_t)n + 31) / 32, 4);
    if (!sync) {
        if (algo != kBFS) need += Workspace::need(n, 4);
        for (int k = 0; k < 3; k++) need += 2 * Workspace::need(wl_cap_of(g, mode, k), 4);
        if (mode == kEdgeAsync) need += 2 * Workspace::need(wl_cap_of(g, mode, 0), 4);
        if (mode == kBucket && algo == kSSSP) need += 3 * Workspace::need(n, 4);
    }
    return need;
}

// Lays one query's state out from base (query_workspace_bytes bytes) into p.
void carve_query_workspace(char *base, const View &g, Algo algo, Mode mode, Params &p) {
    Workspace ws;
    ws.base = base;
    const int32_t n = g.n;
    const bool sync = (mode == kVertexSync || mode == kEdgeSync || mode == kPull);
    const int64_t nwt = (g.m + kWTile - 1) / kWTile;
    p.g = g;
    p.ctrl = ws.take<Ctrl>(1);
    if (mode == kMulti) {
        if (algo == kBFS) {
            p.A = reinterpret_cast<int32_t *>(ws.take<uint8_t>(msb_pad(n)));
            p.S0 = reinterpret_cast<int32_t *>(ws.take<uint8_t>(3 * msb_pad(n)));
        } else {
            p.A = ws.take<int32_t>((int64_t)n * 8);
            p.S0 = ws.take<int32_t>(n);
            p.far_mark = ws.take<int32_t>(n);
        }
        return;
    }
    p.A = ws.take<int32_t>(n);
    if (sync && algo != kBFS) {
        p.B = ws.take<int32_t>(n);
        p.S0 = ws.take<int32_t>(n);
        p.S1 = ws.take<int32_t>(n);
    }
    if (mode == kEdgeSync) p.eflag = ws.take<int32_t>(nwt);
    if (algo == kBFS) p.vis = ws.take<uint32_t>(((int64_t)n + 31) / 32);
    if (!sync) {
        if (algo != kBFS) p.S0 = ws.take<int32_t>(n);
        for (int par = 0; par < 2; par++)
            for (int k = 0; k < 3; k++) p.wl[par][k] = ws.take<int32_t>(wl_cap_of(g, mode, k));
        for (int k = 0; k < 3; k++) p.wl_cap[k] = (int32_t)wl_cap_of(g, mode, k);
        if (mode == kEdgeAsync) {
            p.lb_off[0] = ws.take<uint32_t>(wl_cap_of(g, mode, 0));
            p.lb_off[1] = ws.take<uint32_t>(wl_cap_of(g, mode, 0));
        }
        if (mode == kBucket && algo == kSSSP) {
            p.far[0] = ws.take<int32_t>(n);
            p.far[1] = ws.take<int32_t>(n);
            p.far_mark = ws.take<int32_t>(n);
            p.far_cap = n;
        }
    }
}

// Default round cap of a multi-source sweep.  Without a width a round count
// never exceeds n + 1 (every round extends the settled hop count of every
// slot).  With the near-far order (SSSP) the rounds of one epoch that lower
// something are at most the vertex-slot pairs the epoch settles, and each
// epoch ends with one round that lowers nothing: 2 k n + 2 bounds the sum.
int32_t ms_default_rounds(int32_t n, int k, bool near_far) {
    const int64_t cap = near_far ? 2 * (int64_t)k * n + 2 : (int64_t)n + 2;
    return cap > INT32_MAX ? INT32_MAX : (int32_t)cap;
}

// bucket mode: 5 x the mean edge weight x the mean out-degree unless the
// caller sets it.  A narrower bucket relaxes fewer edges but needs more
// generations, each a grid barrier: on the 4096^2 road-like grid a width of
// the mean weight relaxes each edge about once yet runs 3x more generations
// and takes twice as long; 5x sits at the measured optimum there, and on
// skewed low-diameter graphs any width above a few mean weights does as well.
int32_t default_delta(const fg_graph *G) {
    const double deg = G->info.n > 0 ? (double)G->info.m / (double)G->info.n : 1.0;
    const double d = 5.0 * G->w_mean * std::max(1.0, deg);
    return d >= (double)(kInf / 2) ? kInf / 2 : std::max(1, (int32_t)(d + 0.5));
}

fg_status run_query(const fg_graph *G, Algo algo, Mode mode, int32_t source, int32_t *out,
                    const fg_options *opt, fg_stats *stats) {
    if (kernel_for(algo, mode)) {   // the parts of a FG_GRAPH_LAZY graph this query reads
        fg_status vs = ensure_views(G, algo, (int)mode);
        if (vs != FG_OK) return vs;
    }
    const View &g = (algo == kCC) ? G->s : G->g;
    const int32_t n = g.n;
    cudaStream_t st = opt && opt->stream ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != G->device) return fail(FG_ERR_INVALID_ARG, "the current device is not the graph's device");
    DeviceProps dp = device_props(dev);
    if (!dp.coop) return fail(FG_ERR_CUDA, "device does not support cooperative launches");
    KernelFn fn = kernel_for(algo, mode);
    if (!fn) return fail(FG_ERR_INVALID_ARG, "invalid algorithm or mode");

    int per_sm = 0;
#ifdef FG_L1_CARVEOUT
    cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout, FG_L1_CARVEOUT);
#endif
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBlock, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (opt && opt->blocks_per_sm > 0) per_sm = std::min(per_sm, (int)opt->blocks_per_sm);
    int grid = std::min(per_sm * dp.sms, kMaxGrid);
    if (grid < 1) return fail(FG_ERR_CUDA, "kernel does not fit on an SM");

    // per-query state, carved from one stream-ordered allocation
    const size_t need = query_workspace_bytes(g, algo, mode);
    char *wsbase = nullptr;
    e = cudaMallocAsync((void **)&wsbase, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "query workspace");
    Params p;
    carve_query_workspace(wsbase, g, algo, mode, p);
    if (mode == kPull) p.tv = (algo == kCC) ? G->s : G->t;
    p.delta = (opt && opt->delta > 0) ? opt->delta : default_delta(G);
    struct {
        char *base;
    } ws{wsbase};
    p.source = source;
    set_relabel(G, p);
    p.max_rounds = (opt && opt->max_rounds > 0) ? opt->max_rounds : (n > INT32_MAX - 2 ? INT32_MAX : n + 2);
    int tmo = (opt && opt->wait_timeout_ms > 0) ? opt->wait_timeout_ms : 1000;
    p.timeout_ns = (unsigned long long)tmo * 1000000ull;
    p.inject_missing_arrival = (opt && opt->inject_missing_arrival) ? 1 : 0;
    if (opt && opt->round_trace && opt->round_trace_cap > 0) {
        if (!is_device_pointer(opt->round_trace)) {
            cudaFreeAsync(ws.base, st);
            return fail(FG_ERR_INVALID_ARG, "round_trace must be device memory");
        }
        p.trace = reinterpret_cast<unsigned long long *>(opt->round_trace);
        p.trace_cap = opt->round_trace_cap;
    }

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    fg_status status = FG_OK;
    std::string msg;
    Ctrl hc;
    e = cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) {
        void *args[] = {&p};
        e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kBlock), args, 0, st);
        if (e == cudaSuccess) count_launch();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        status = (e == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
        msg = std::string("fixpoint kernel: ") + cudaGetErrorString(e);
        cudaGetLastError();
    }
    const int32_t *result = (hc.result_in_b && p.B) ? p.B : p.A;
    if (status == FG_OK) {
        if (hc.status & kStTimeout) {
            status = FG_ERR_TIMEOUT;
            msg = "a device-side wait exceeded the timeout";
        } else if (hc.status & kStRoundCap) {
            status = FG_ERR_TIMEOUT;
            msg = "round cap reached before the fixpoint";
        } else if (hc.status & kStWorklist) {
            status = FG_ERR_CUDA;
            msg = "internal error: worklist capacity exceeded";
        } else if ((hc.status & kStOverflow) && algo == kSSSP) {
            int *flag = reinterpret_cast<int *>(p.ctrl);   // reuse the control block
            int hf = 0;
            const fg_status ss = ensure_src(G);   // the check reads the edge sources
            if (ss != FG_OK) {
                status = ss;
                msg = fg_last_error();
            }
            e = cudaMemsetAsync(flag, 0, sizeof(int), st);
            if (e == cudaSuccess && ss == FG_OK) {
                overflow_check_kernel<<<dp.sms * 8, kBlock, 0, st>>>(g, result, flag);
                count_launch();
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                status = FG_ERR_CUDA;
                msg = std::string("overflow check: ") + cudaGetErrorString(e);
            } else if (hf) {
                status = FG_ERR_OVERFLOW;
                msg = "a finite shortest distance is >= INT32_MAX";
            }
        }
    }
    if (status == FG_OK && G->new_of) {   // internal order to original order
        status = relabel_output(G, algo, result, out, st);
        if (status != FG_OK) msg = fg_last_error();
    } else if (status == FG_OK) {
        e = cudaMemcpyAsync(out, result, (size_t)n * sizeof(int32_t), cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            status = FG_ERR_CUDA;
            msg = std::string("result copy: ") + cudaGetErrorString(e);
        }
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFreeAsync(ws.base, st);
    if (stats) {
        stats->mode = (int32_t)mode;
        stats->rounds = hc.rounds;
        stats->jump_passes = hc.jump_passes;
        stats->grid_blocks = grid;
        stats->vertices_processed = (int64_t)hc.st_vertices;
        stats->edges_relaxed = (int64_t)hc.st_edges;
        stats->updates = (int64_t)hc.st_updates;
        stats->pushes = (int64_t)hc.st_pushes;
        stats->scanned = (int64_t)hc.st_scanned;
        stats->barriers = hc.barriers;
        stats->pull_rounds = hc.pull_rounds;
        stats->edges_pulled = (int64_t)hc.st_pulled;
        stats->kernel_ms = ms;
    }
    if (status != FG_OK) return fail(status, msg);
    return FG_OK;
}

// Up to kMsMax queries of one algorithm on one graph.  SSSP and BFS run as
// one multi-source sweep (one launch); CC has no source, so it runs once and
// its result is copied to every output.  Per-slot status: only an overflow
// (SSSP) can differ between slots.
fg_status run_multi(const fg_graph *G, Algo algo, int32_t k, const int32_t *srcs, int32_t *const *outs,
                    const fg_options *opt, fg_status *status_out, fg_stats *stats) {
    cudaStream_t st = opt && opt->stream ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    auto all = [&](fg_status x) {
        if (status_out)
            for (int j = 0; j < k; j++) status_out[j] = x;
        return x;
    };
    if (algo == kCC) {
        fg_mode m;
        fg_status s = fg_select_mode(G, FG_ALGO_CC, &m);
        if (s == FG_OK) s = run_query(G, kCC, (Mode)m, 0, outs[0], opt, stats);
        if (s != FG_OK) return all(s);
        cudaError_t e = cudaSuccess;
        for (int j = 1; j < k && e == cudaSuccess; j++)
            e = cudaMemcpyAsync(outs[j], outs[0], (size_t)G->s.n * sizeof(int32_t), cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return all(cuda_fail(e, "result copies"));
        return all(FG_OK);
    }
    const View &g = G->g;
    const int32_t n = g.n;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != G->device) return all(fail(FG_ERR_INVALID_ARG, "the current device is not the graph's device"));
    DeviceProps dp = device_props(dev);
    if (!dp.coop) return all(fail(FG_ERR_CUDA, "device does not support cooperative launches"));
    KernelFn fn = kernel_for(algo, kMulti);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBlock, 0);
    if (e != cudaSuccess) return all(cuda_fail(e, "occupancy query"));
    if (opt && opt->blocks_per_sm > 0) per_sm = std::min(per_sm, (int)opt->blocks_per_sm);
    const int grid = std::min(per_sm * dp.sms, kMaxGrid);
    if (grid < 1) return all(fail(FG_ERR_CUDA, "kernel does not fit on an SM"));

    // one allocation: the query state, then device staging of host outputs
    bool on_dev[kMsMax] = {};
    int n_host = 0;
    for (int j = 0; j < k; j++) {
        on_dev[j] = is_device_pointer(outs[j]);
        n_host += !on_dev[j];
    }
    const size_t qbytes = query_workspace_bytes(g, algo, kMulti);
    const size_t sbytes = Workspace::need(n, 4);
    char *base = nullptr;
    e = cudaMallocAsync((void **)&base, qbytes + (size_t)n_host * sbytes, st);
    if (e != cudaSuccess) return all(cuda_fail(e, "multi-source workspace"));
    Params p;
    carve_query_workspace(base, g, algo, kMulti, p);
    p.ms_k = k;
    p.ms_bfs = algo == kBFS ? 1 : 0;
    set_relabel(G, p);
    p.delta = (opt && opt->delta > 0) ? opt->delta : default_delta(G);   // the SSSP sweep's near-far width
    int32_t *dout[kMsMax] = {};
    for (int j = 0, h = 0; j < k; j++) {
        p.ms_src[j] = srcs[j];
        dout[j] = on_dev[j] ? outs[j] : reinterpret_cast<int32_t *>(base + qbytes + (size_t)(h++) * sbytes);
        p.ms_out[j] = dout[j];
    }
    p.max_rounds = (opt && opt->max_rounds > 0) ? opt->max_rounds : ms_default_rounds(n, k, algo == kSSSP);
    const int tmo = (opt && opt->wait_timeout_ms > 0) ? opt->wait_timeout_ms : 1000;
    p.timeout_ns = (unsigned long long)tmo * 1000000ull;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    fg_status status = FG_OK;
    std::string msg;
    Ctrl hc{};
    e = cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) {
        void *args[] = {&p};
        e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kBlock), args, 0, st);
        if (e == cudaSuccess) count_launch();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        status = (e == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
        msg = std::string("multi-source kernel: ") + cudaGetErrorString(e);
        cudaGetLastError();
    } else if (hc.status & kStTimeout) {
        status = FG_ERR_TIMEOUT;
        msg = "a device-side wait exceeded the timeout";
    } else if (hc.status & kStRoundCap) {
        status = FG_ERR_TIMEOUT;
        msg = "round cap reached before the fixpoint";
    } else if (!hc.done) {
        status = FG_ERR_CUDA;
        msg = "internal error: the multi-source sweep ended without a fixpoint";
    }
    fg_status slot[kMsMax];
    for (int j = 0; j < kMsMax; j++) slot[j] = status;
    if (status == FG_OK && (hc.status & kStOverflow)) {
        // which sources overflowed; the kernel wrote no output, so write the others'
        int *flag = reinterpret_cast<int *>(p.ctrl);
        int hf = 0;
        e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        if (e == cudaSuccess) {
            ms_overflow_check_launch(g, p.A, k, flag, st);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        MsOuts ok_outs{};
        for (int j = 0; j < k; j++) {
            if ((hf >> j) & 1) slot[j] = FG_ERR_OVERFLOW;
            else ok_outs.p[j] = dout[j];
        }
        if (e == cudaSuccess && hf != (1 << k) - 1) {
            ms_output_launch(p.A, n, k, ok_outs, p.new_of, st);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            for (int j = 0; j < k; j++) slot[j] = FG_ERR_CUDA;
            msg = std::string("overflow check: ") + cudaGetErrorString(e);
        } else if (hf) {
            msg = "a finite shortest distance is >= INT32_MAX";
        }
    }
    for (int j = 0; j < k && e == cudaSuccess; j++)
        if (slot[j] == FG_OK && !on_dev[j])
            e = cudaMemcpyAsync(outs[j], dout[j], (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        for (int j = 0; j < k; j++) slot[j] = FG_ERR_CUDA;
        msg = std::string("result copy: ") + cudaGetErrorString(e);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFreeAsync(base, st);
    if (stats) {
        *stats = fg_stats{};
        stats->mode = -1;
        stats->rounds = hc.rounds;
        stats->grid_blocks = grid;
        stats->vertices_processed = (int64_t)hc.st_vertices;
        stats->edges_relaxed = (int64_t)hc.st_edges;
        stats->updates = (int64_t)hc.st_updates;
        stats->scanned = (int64_t)hc.st_scanned;
        stats->barriers = hc.barriers;
        stats->kernel_ms = ms;
    }
    fg_status first = FG_OK;
    for (int j = 0; j < k; j++) {
        if (status_out) status_out[j] = slot[j];
        if (first == FG_OK) first = slot[j];
    }
    if (first != FG_OK) return fail(first, msg);
    return FG_OK;
}

fg_status run_sweep(const fg_graph *G, Mode mode, const int32_t *cur, int32_t *next, cudaStream_t st,
                    int64_t *updates, float *kernel_ms) {
    const View &g = G->g;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != G->device) return fail(FG_ERR_INVALID_ARG, "the current device is not the graph's device");
    if (mode == kEdgeSync) {   // the edge variant streams the edge sources
        fg_status ss = ensure_src(G);
        if (ss != FG_OK) return ss;
    }
    DeviceProps dp = device_props(dev);
    // a renumbered graph: the caller's arrays to internal order around the round
    const int32_t n = g.n;
    int32_t *icur = nullptr, *inext = nullptr;
    int32_t *const user_next = next;
    const int pgrid = std::max(1, dp.sms) * 8;
    if (G->new_of) {
        cudaError_t e0 = cudaMallocAsync((void **)&icur, 2 * (size_t)n * sizeof(int32_t), st);
        if (e0 != cudaSuccess) return cuda_fail(e0, "sweep permutation workspace");
        inext = icur + n;
        k_gather_out<<<pgrid, kBlock, 0, st>>>(n, cur, G->orig_of, icur);
        k_gather_out<<<pgrid, kBlock, 0, st>>>(n, next, G->orig_of, inext);
        count_launch();
        count_launch();
        cur = icur;
        next = inext;
    }
    auto fn = (mode == kVertexSync) ? sweep_kernel<kVertexSync> : sweep_kernel<kEdgeSync>;
    int per_sm = 0;
#ifdef FG_L1_CARVEOUT
    cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout, FG_L1_CARVEOUT);
#endif
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBlock, 0);
    int grid = std::max(1, per_sm * dp.sms);
    Ctrl *c = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&c, sizeof(Ctrl), st);
    if (e != cudaSuccess) {
        if (icur) cudaFreeAsync(icur, st);
        return cuda_fail(e, "sweep workspace");
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    Ctrl hc;
    e = cudaMemsetAsync(c, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) {
        fn<<<grid, kBlock, 0, st>>>(g, cur, next, c);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
    if (e == cudaSuccess && icur) {   // next back to original order
        k_gather_out<<<pgrid, kBlock, 0, st>>>(n, inext, G->new_of, user_next);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, c, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFreeAsync(c, st);
    if (icur) cudaFreeAsync(icur, st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep");
    if (updates) *updates = (int64_t)hc.st_updates;
    if (kernel_ms) *kernel_ms = ms;
    if (hc.status & kStTimeout) return fail(FG_ERR_TIMEOUT, "sweep: an edge tile copy did not complete");
    if (hc.status & kStOverflow) return fail(FG_ERR_OVERFLOW, "sweep: a candidate reached INT32_MAX");
    return FG_OK;
}

}  // namespace fg
