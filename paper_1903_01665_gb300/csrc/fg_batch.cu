// Batched queries: many sources over many resident graphs in one launch per
// (algorithm, mode) kind present -- the runtime counterpart of the paper's
// barrier-free kernels on separate streams (Sec. 3.2) and of its
// independent parallel sections (Sec. 3.4).
//
// Each launch is a persistent cooperative kernel whose CTAs are split into
// teams; every team pulls queries from the queue of its size class and runs
// the whole fixpoint of each with a team-local barrier (a one-CTA team needs
// only __syncthreads).  The team size of a query comes from its edge count,
// the CTA budget of each kind and class from its estimated work.  Kinds run
// concurrently on forked streams, optionally captured in one CUDA graph.
#include <algorithm>
#include <map>
#include <vector>

#include "fg_multi.cuh"

namespace fg {

namespace {

struct BatchArgs {
    const int4 *cta_team;     // per CTA: team, rank in team, team size, class
    unsigned *team_bar;       // 2 per team: arrivals, generation
    int *team_q;              // per team: the queue slot it is working on
    int *cls_next;            // per class: next queue slot
    const int *cls_begin;     // per class: queue range in `order`
    const int *cls_end;
    const int *order;         // query indices, by class, largest work first
    const Params *params;     // per query of the batch
    Ctrl *bctrl;              // status of the queue barriers
    unsigned long long timeout_ns;
};

template <int ALGO, int MODE>
__global__ void __launch_bounds__(kBlock, min_blocks<MODE>()) batch_kernel(BatchArgs b) {
    const int4 ct = b.cta_team[blockIdx.x];
    const Team t{ct.y, ct.z, b.team_bar + 2 * ct.x};
    const int cls = ct.w;
    uint32_t ring_used;
    fixpoint_prologue<ALGO, MODE>(ring_used);
    for (;;) {
        if (t.rank == 0 && threadIdx.x == 0) b.team_q[ct.x] = b.cls_begin[cls] + atomicAdd(&b.cls_next[cls], 1);
        if (!team_sync(t, b.bctrl, b.timeout_ns)) return;
        const int qi = __ldcg(&b.team_q[ct.x]);
        if (qi >= b.cls_end[cls]) return;
        query_body<ALGO, MODE>(b.params[b.order[qi]], t, ring_used);
        if (!team_sync(t, b.bctrl, b.timeout_ns)) return;
    }
}

using BatchFn = void (*)(BatchArgs);

// kind = algo * 8 + mode
BatchFn batch_kernel_for(int kind) {
    switch (kind) {
        case kSSSP * 8 + kVertexSync: return batch_kernel<kSSSP, kVertexSync>;
        case kSSSP * 8 + kVertexAsync: return batch_kernel<kSSSP, kVertexAsync>;
        case kSSSP * 8 + kEdgeSync: return batch_kernel<kSSSP, kEdgeSync>;
        case kSSSP * 8 + kEdgeAsync: return batch_kernel<kSSSP, kEdgeAsync>;
        case kBFS * 8 + kVertexSync: return batch_kernel<kBFS, kVertexSync>;
        case kBFS * 8 + kVertexAsync: return batch_kernel<kBFS, kVertexAsync>;
        case kBFS * 8 + kEdgeSync: return batch_kernel<kBFS, kEdgeSync>;
        case kBFS * 8 + kEdgeAsync: return batch_kernel<kBFS, kEdgeAsync>;
        case kCC * 8 + kVertexSync: return batch_kernel<kCC, kVertexSync>;
        case kCC * 8 + kVertexAsync: return batch_kernel<kCC, kVertexAsync>;
        case kCC * 8 + kEdgeSync: return batch_kernel<kCC, kEdgeSync>;
        case kCC * 8 + kEdgeAsync: return batch_kernel<kCC, kEdgeAsync>;
        case kSSSP * 8 + kPull: return batch_kernel<kSSSP, kPull>;
        case kBFS * 8 + kPull: return batch_kernel<kBFS, kPull>;
        case kCC * 8 + kPull: return batch_kernel<kCC, kPull>;
        case kSSSP * 8 + kBucket: return batch_kernel<kSSSP, kBucket>;
        case kBFS * 8 + kBucket: return batch_kernel<kBFS, kBucket>;
        case kCC * 8 + kBucket: return batch_kernel<kCC, kBucket>;
    }
    return nullptr;
}

// CTAs a query's team gets: one per ~128K edges, a power of two in [1, 128].
int team_size_for(int64_t m) {
    int s = 1;
    while (s < 128 && (int64_t)s * (1 << 17) < m) s <<= 1;
    return s;
}

// relative work of a query (SSSP relaxes each edge several times)
double work_of(int algo, const View &v) {
    return (double)v.m * (algo == kSSSP ? 4.0 : 1.0) + (double)v.n;
}

struct KindPlan {
    int kind = 0;
    std::vector<int> queries;                 // indices into the batch
    std::vector<int> class_size;              // team size per class
    std::vector<std::vector<int>> class_q;    // queries per class, largest work first
    std::vector<int> class_teams;             // teams per class
    double work = 0;
    int ctas = 0;
};

}  // namespace

// Plans, allocates and enqueues a batch on opt->stream; nothing waits.  The
// results reach device outputs directly; host outputs go to device staging
// and, if enqueue_host_copies, are copied back on the stream (their contents
// are then unspecified for a failed query).  cta_fraction scales the CTA
// budget so that several batches can be resident at once.
fg_status batch_launch(const fg_query *qs, int32_t nq, const fg_batch_options *opt, double cta_fraction,
                       bool enqueue_host_copies, Ctrl *h_ctrls_pinned, BatchJob &job) {
    job.nq = nq;
    job.qs.assign(qs, qs + nq);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t st = opt && opt->stream ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    job.st = st;
    const int tmo = (opt && opt->wait_timeout_ms > 0) ? opt->wait_timeout_ms : 1000;
    int sms = 0, coop = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(FG_ERR_CUDA, "device does not support cooperative launches");

    // ---- resolve modes, group by kind, plan teams
    std::vector<Mode> &mode = job.mode;
    std::vector<const View *> &view = job.view;
    mode.resize(nq);
    view.resize(nq);
    std::map<int, KindPlan> kinds;
    double total_work = 0;
    for (int i = 0; i < nq; i++) {
        const fg_query &q = qs[i];
        fg_mode m = (fg_mode)q.mode;
        if (m == FG_AUTO) {
            fg_status s = fg_select_mode(q.g, (fg_algo)q.algo, &m);
            if (s != FG_OK) return s;
        }
        mode[i] = (Mode)m;
        fg_status vs = ensure_views(q.g, (Algo)q.algo, (int)m);   // lazily built parts, transposed view
        if (vs != FG_OK) return vs;
        view[i] = (q.algo == FG_ALGO_CC) ? &q.g->s : &q.g->g;
        KindPlan &kp = kinds[q.algo * 8 + (int)m];
        kp.kind = q.algo * 8 + (int)m;
        kp.queries.push_back(i);
        double w = work_of(q.algo, *view[i]);
        kp.work += w;
        total_work += w;
    }
    for (auto &kv : kinds) {
        KindPlan &kp = kv.second;
        std::map<int, std::vector<int>> by_size;
        // a kind with few queries (at most 8) gives each a larger team (a lone
        // query the whole budget); otherwise the size follows its edge count
        int per_sm0 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm0, (const void *)batch_kernel_for(kp.kind), kBlock, 0);
        const int cap0 = std::max(1, (int)(std::max(1, std::min(per_sm0 * sms, kMaxGrid)) * cta_fraction *
                                           std::max(kp.work / std::max(total_work, 1.0), 0.0)));
        int share = 1;
        if (kp.queries.size() <= 8)
            while (share * 2 <= cap0 / (int)kp.queries.size()) share *= 2;
        for (int i : kp.queries) by_size[std::max(team_size_for(view[i]->m), share)].push_back(i);
        std::vector<double> cw;
        for (auto &c : by_size) {
            std::vector<int> v = c.second;
            std::sort(v.begin(), v.end(), [&](int a, int b) {
                return work_of(qs[a].algo, *view[a]) > work_of(qs[b].algo, *view[b]);
            });
            double w = 0;
            for (int i : v) w += work_of(qs[i].algo, *view[i]);
            kp.class_size.push_back(c.first);
            kp.class_q.push_back(v);
            cw.push_back(w);
        }
        int per_sm = 0;
        BatchFn fn = batch_kernel_for(kp.kind);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBlock, 0);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        int capacity = std::max(1, std::min(per_sm * sms, kMaxGrid));
        capacity = std::max(1, (int)(capacity * cta_fraction));
        int min_ctas = 0;
        for (int s : kp.class_size) min_ctas += std::min(s, capacity);
        int budget = (int)(capacity * (kp.work / std::max(total_work, 1.0)));
        budget = std::min(capacity, std::max(budget, min_ctas));
        // one team per class, the rest of the budget by class work
        int used = 0;
        for (size_t c = 0; c < kp.class_size.size(); c++) {
            kp.class_size[c] = std::min(kp.class_size[c], capacity);
            kp.class_teams.push_back(1);
            used += kp.class_size[c];
        }
        const int rest = std::max(0, budget - used);
        for (size_t c = 0; c < kp.class_size.size(); c++) {
            int extra = (int)(rest * (cw[c] / std::max(kp.work, 1.0)) / kp.class_size[c]);
            extra = std::min(extra, (int)kp.class_q[c].size() - 1);
            kp.class_teams[c] += std::max(0, extra);
        }
        kp.ctas = 0;
        for (size_t c = 0; c < kp.class_size.size(); c++) kp.ctas += kp.class_teams[c] * kp.class_size[c];
    }

    // ---- one device allocation: zeroed region | tables | query workspaces | staging
    size_t zero_bytes = Workspace::need(1, sizeof(Ctrl)) + Workspace::need(nq, sizeof(Ctrl));
    size_t table_bytes = Workspace::need(nq, sizeof(Params)) + Workspace::need(nq, sizeof(int));
    for (auto &kv : kinds) {
        KindPlan &kp = kv.second;
        int teams = 0;
        for (int t : kp.class_teams) teams += t;
        const int nc = (int)kp.class_size.size();
        zero_bytes += Workspace::need(2 * teams, 4) + Workspace::need(teams, 4) + Workspace::need(nc, 4);
        table_bytes += Workspace::need(kp.ctas, sizeof(int4)) + 2 * Workspace::need(nc, 4);
    }
    std::vector<bool> dev_out(nq);
    size_t ws_bytes = 0;
    for (int i = 0; i < nq; i++) {
        ws_bytes += query_workspace_bytes(*view[i], (Algo)qs[i].algo, mode[i]);
        dev_out[i] = is_device_pointer(qs[i].out);
        if (!dev_out[i]) ws_bytes += Workspace::need(view[i]->n, 4);
    }
    const size_t total = zero_bytes + table_bytes + ws_bytes;
    job.device_bytes = total;
    cudaError_t e = cudaMallocAsync((void **)&job.base, total, st);
    if (e != cudaSuccess) {
        job.base = nullptr;
        return cuda_fail(e, "batch workspace");
    }
    char *base = job.base;

    // host image of the tables, copied in one transfer
    std::vector<char> img(table_bytes, 0);
    Workspace zw{base}, tw{base + zero_bytes}, hw{img.data()}, qw{base + zero_bytes + table_bytes};
    Ctrl *bctrl = zw.take<Ctrl>(1);
    job.d_ctrls = zw.take<Ctrl>(nq);
    Params *d_params = tw.take<Params>(nq);
    Params *h_params = hw.take<Params>(nq);
    int *d_order = tw.take<int>(nq);
    int *h_order = hw.take<int>(nq);
    job.staging.assign(nq, nullptr);
    for (int i = 0; i < nq; i++) {
        char *w = qw.base + qw.off;
        qw.off += query_workspace_bytes(*view[i], (Algo)qs[i].algo, mode[i]);
        Params p;
        carve_query_workspace(w, *view[i], (Algo)qs[i].algo, mode[i], p);
        if (mode[i] == kPull) p.tv = (qs[i].algo == FG_ALGO_CC) ? qs[i].g->s : qs[i].g->t;
        p.delta = default_delta(qs[i].g);
        p.ctrl = job.d_ctrls + i;
        p.source = qs[i].algo == FG_ALGO_CC ? 0 : qs[i].src;
        p.max_rounds = view[i]->n > INT32_MAX - 2 ? INT32_MAX : view[i]->n + 2;
        p.timeout_ns = (unsigned long long)tmo * 1000000ull;
        if (dev_out[i]) {
            p.out = qs[i].out;
        } else {
            job.staging[i] = qw.take<int32_t>(view[i]->n);
            p.out = job.staging[i];
        }
        h_params[i] = p;
    }
    job.params.assign(h_params, h_params + nq);
    std::vector<BatchArgs> args;
    std::vector<int> kind_ctas;
    std::vector<BatchFn> kind_fn;
    int order_pos = 0;
    for (auto &kv : kinds) {
        KindPlan &kp = kv.second;
        const int nc = (int)kp.class_size.size();
        int teams = 0;
        for (int t : kp.class_teams) teams += t;
        BatchArgs a;
        a.team_bar = zw.take<unsigned>(2 * teams);
        a.team_q = zw.take<int>(teams);
        a.cls_next = zw.take<int>(nc);
        int4 *d_ct = tw.take<int4>(kp.ctas);
        int4 *h_ct = hw.take<int4>(kp.ctas);
        int *d_cb = tw.take<int>(nc), *h_cb = hw.take<int>(nc);
        int *d_ce = tw.take<int>(nc), *h_ce = hw.take<int>(nc);
        int cta = 0, team = 0;
        for (int c = 0; c < nc; c++) {
            h_cb[c] = order_pos;
            for (int i : kp.class_q[c]) h_order[order_pos++] = i;
            h_ce[c] = order_pos;
            for (int k = 0; k < kp.class_teams[c]; k++, team++)
                for (int r = 0; r < kp.class_size[c]; r++) h_ct[cta++] = make_int4(team, r, kp.class_size[c], c);
        }
        a.cta_team = d_ct;
        a.cls_begin = d_cb;
        a.cls_end = d_ce;
        a.order = d_order;
        a.params = d_params;
        a.bctrl = bctrl;
        a.timeout_ns = (unsigned long long)tmo * 1000000ull;
        args.push_back(a);
        kind_ctas.push_back(kp.ctas);
        kind_fn.push_back(batch_kernel_for(kp.kind));
        job.teams += teams;
        job.ctas += kp.ctas;
    }

    // ---- enqueue: fork one stream per kind, join, optionally as a CUDA graph
    const int nk = (int)args.size();
    job.launches = nk;
    job.ks.assign(nk, nullptr);
    job.kev.assign(nk, nullptr);
    const bool use_graph = opt && opt->use_cuda_graph;
    auto ck = [&](cudaError_t err, const char *what) {
        if (err != cudaSuccess && job.status == FG_OK) {
            job.status = (err == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
            job.msg = std::string(what) + ": " + cudaGetErrorString(err);
        }
        return err == cudaSuccess;
    };
    ck(cudaEventCreateWithFlags(&job.fork, cudaEventDisableTiming), "event");
    ck(cudaEventCreate(&job.ev0), "event");
    ck(cudaEventCreate(&job.ev1), "event");
    ck(cudaEventCreateWithFlags(&job.done, cudaEventDisableTiming), "event");
    for (int k = 0; k < nk; k++) {
        ck(cudaStreamCreateWithFlags(&job.ks[k], cudaStreamNonBlocking), "stream");
        ck(cudaEventCreateWithFlags(&job.kev[k], cudaEventDisableTiming), "event");
    }
    ck(cudaMemcpyAsync(base + zero_bytes, img.data(), table_bytes, cudaMemcpyHostToDevice, st), "table upload");
    ck(cudaEventRecord(job.ev0, st), "event");
    // the launches are recorded on `cs`: the caller's stream itself, or for a
    // CUDA graph a private stream (the legacy default stream cannot capture)
    cudaStream_t cs = st;
    if (job.status == FG_OK && use_graph) {
        ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
        ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "capture");
    }
    ck(cudaMemsetAsync(base, 0, zero_bytes, cs), "memset");
    ck(cudaEventRecord(job.fork, cs), "event");
    for (int k = 0; k < nk && job.status == FG_OK; k++) {
        ck(cudaStreamWaitEvent(job.ks[k], job.fork, 0), "fork");
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kind_ctas[k]);
        cfg.blockDim = dim3(kBlock);
        cfg.stream = job.ks[k];
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (ck(cudaLaunchKernelEx(&cfg, kind_fn[k], args[k]), "batch launch")) count_launch();
        ck(cudaEventRecord(job.kev[k], job.ks[k]), "event");
        ck(cudaStreamWaitEvent(cs, job.kev[k], 0), "join");
    }
    if (use_graph && cs != st) {
        cudaError_t ce = cudaStreamEndCapture(cs, &job.graph);
        if (job.status == FG_OK) ck(ce, "capture");
        if (job.status == FG_OK) ck(cudaGraphInstantiate(&job.exec, job.graph, 0), "graph instantiate");
        if (job.status == FG_OK) ck(cudaGraphLaunch(job.exec, st), "graph launch");
        cudaStreamDestroy(cs);
    }
    ck(cudaEventRecord(job.ev1, st), "event");
    job.h_ctrls = h_ctrls_pinned;
    if (!job.h_ctrls) {
        job.own_ctrls.resize(nq);
        job.h_ctrls = job.own_ctrls.data();
    }
    ck(cudaMemcpyAsync(job.h_ctrls, job.d_ctrls, nq * sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "status copy");
    if (enqueue_host_copies) {
        for (int i = 0; i < nq; i++)
            if (job.staging[i])
                ck(cudaMemcpyAsync(qs[i].out, job.staging[i], (size_t)view[i]->n * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, st), "result copy");
        job.host_copies_done = true;
    }
    ck(cudaEventRecord(job.done, st), "event");
    if (job.status != FG_OK) return fail(job.status, job.msg);
    return FG_OK;
}

// Waits for a launched batch, reports every query and releases the batch.
fg_status batch_finish(BatchJob &job, fg_status *status_out, fg_stats *stats_out, fg_batch_stats *bstats) {
    const int nq = job.nq;
    cudaStream_t st = job.st;
    auto ck = [&](cudaError_t err, const char *what) {
        if (err != cudaSuccess && job.status == FG_OK) {
            job.status = (err == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
            job.msg = std::string(what) + ": " + cudaGetErrorString(err);
        }
        return err == cudaSuccess;
    };
    if (job.done) ck(cudaEventSynchronize(job.done), "batch");
    float ms = 0.f;
    if (job.status == FG_OK && job.ev0 && job.ev1) cudaEventElapsedTime(&ms, job.ev0, job.ev1);
    fg_status first_err = FG_OK;
    std::string first_msg;
    for (int i = 0; i < nq && job.status == FG_OK; i++) {
        const Ctrl &hc = job.h_ctrls[i];
        const fg_query &q = job.qs[i];
        const Params &p = job.params[i];
        fg_status qs_st = FG_OK;
        if (hc.status & kStTimeout) qs_st = FG_ERR_TIMEOUT;
        else if (hc.status & kStRoundCap) qs_st = FG_ERR_TIMEOUT;
        else if (hc.status & kStWorklist) qs_st = FG_ERR_CUDA;
        else if (!hc.done) qs_st = FG_ERR_TIMEOUT;
        else if ((hc.status & kStOverflow) && q.algo == FG_ALGO_SSSP) {
            int *flag = reinterpret_cast<int *>(p.ctrl);
            int hf = 0;
            ck(cudaMemsetAsync(flag, 0, sizeof(int), st), "memset");
            overflow_check_launch(*job.view[i], p.out, flag, st);
            ck(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
            ck(cudaStreamSynchronize(st), "overflow check");
            if (hf) qs_st = FG_ERR_OVERFLOW;
        }
        if (qs_st == FG_OK && job.staging[i] && !job.host_copies_done)
            ck(cudaMemcpyAsync(q.out, job.staging[i], (size_t)job.view[i]->n * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, st), "result copy");
        if (status_out) status_out[i] = qs_st;
        if (qs_st != FG_OK && first_err == FG_OK) {
            first_err = qs_st;
            first_msg = "batch query " + std::to_string(i) + " failed: " + fg_status_string(qs_st);
        }
        if (stats_out) {
            fg_stats &s = stats_out[i];
            s = fg_stats{};
            s.mode = (int32_t)job.mode[i];
            s.rounds = hc.rounds;
            s.jump_passes = hc.jump_passes;
            s.vertices_processed = (int64_t)hc.st_vertices;
            s.edges_relaxed = (int64_t)hc.st_edges;
            s.updates = (int64_t)hc.st_updates;
            s.pushes = (int64_t)hc.st_pushes;
            s.scanned = (int64_t)hc.st_scanned;
            s.barriers = hc.barriers;
            s.pull_rounds = hc.pull_rounds;
            s.edges_pulled = (int64_t)hc.st_pulled;
        }
    }
    if (job.status != FG_OK && status_out)
        for (int i = 0; i < nq; i++) status_out[i] = job.status;
    ck(cudaStreamSynchronize(st), "result copies");
    if (job.exec) cudaGraphExecDestroy(job.exec);
    if (job.graph) cudaGraphDestroy(job.graph);
    for (size_t k = 0; k < job.ks.size(); k++) {
        if (job.kev[k]) cudaEventDestroy(job.kev[k]);
        if (job.ks[k]) cudaStreamDestroy(job.ks[k]);
    }
    if (job.fork) cudaEventDestroy(job.fork);
    if (job.ev0) cudaEventDestroy(job.ev0);
    if (job.ev1) cudaEventDestroy(job.ev1);
    if (job.done) cudaEventDestroy(job.done);
    if (job.base) cudaFreeAsync(job.base, st);
    job.exec = nullptr;
    job.graph = nullptr;
    job.ks.clear();
    job.kev.clear();
    job.fork = job.ev0 = job.ev1 = job.done = nullptr;
    job.base = nullptr;
    if (bstats) {
        bstats->kernel_ms = ms;
        bstats->launches = job.launches;
        bstats->teams = job.teams;
        bstats->ctas = job.ctas;
    }
    if (job.status != FG_OK) return fail(job.status, job.msg);
    if (first_err != FG_OK) return fail(first_err, first_msg);
    return FG_OK;
}

fg_status run_batch(const fg_query *qs, int32_t nq, const fg_batch_options *opt, fg_status *status_out,
                    fg_stats *stats_out, fg_batch_stats *bstats) {
    BatchJob job;
    fg_status s = batch_launch(qs, nq, opt, 1.0, false, nullptr, job);
    fg_status f = batch_finish(job, status_out, stats_out, bstats);
    return s != FG_OK ? s : f;
}

}  // namespace fg
