// Batched queries: many sources over many resident graphs in one launch per
// (algorithm, mode) kind present -- the runtime counterpart of the paper's
// barrier-free kernels on separate streams (Sec. 3.2) and of its
// independent parallel sections (Sec. 3.4).
//
// The queries are first grouped into units: each query alone, or -- with
// fusion -- the queries on one graph merged (SSSP/BFS into multi-source
// sweeps of up to 8 sources, CC into one computation for all its outputs).
// Each launch is a persistent cooperative kernel whose CTAs are split into
// teams; every team pulls units from the queue of its size class and runs
// the whole fixpoint of each with a team-local barrier (a one-CTA team needs
// only __syncthreads).  The team size of a unit comes from its edge count,
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
    const int *order;         // unit indices, by class, largest work first
    const Params *params;     // per unit of the batch
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
        case kAnyAlgo * 8 + kMulti: return batch_kernel<kAnyAlgo, kMulti>;
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

// relative work of a unit: a fused sweep of k sources costs a fraction of k
// separate sweeps (R-MAT 22, 8 sources: SSSP about 2x one query, BFS about 4x)
double unit_work(const BatchUnit &u, const View &v) {
    const double one = work_of(u.algo, v);
    if (u.mode != kMulti) return one;
    const double k = (double)u.q.size();
    return one * (1.0 + (k - 1.0) * (u.algo == kSSSP ? 0.15 : 0.45));
}

struct KindPlan {
    int kind = 0;
    std::vector<int> queries;                 // units of the batch of this kind
    std::vector<int> class_size;              // team size per class
    std::vector<std::vector<int>> class_q;    // units per class, largest work first
    std::vector<int> class_teams;             // teams per class
    double work = 0;
    int ctas = 0;
};

}  // namespace

// Groups the batch's queries into units.  Without fusion every query is a
// unit of its own.  With fusion, queries on the same graph are merged: CC
// queries into one unit (CC has no source: one result for every output),
// SSSP and BFS queries into multi-source sweeps of up to 8 sources (a lone
// query stays a plain unit in its own mode).  Units keep the order of their
// first query.
static std::vector<BatchUnit> plan_units(const fg_query *qs, int32_t nq, const std::vector<Mode> &mode,
                                         bool fuse) {
    std::vector<BatchUnit> units;
    if (!fuse) {
        for (int i = 0; i < nq; i++) {
            BatchUnit u;
            u.g = qs[i].g;
            u.algo = (Algo)qs[i].algo;
            u.mode = mode[i];
            u.q.push_back(i);
            units.push_back(u);
        }
        return units;
    }
    std::map<std::pair<const fg_graph *, int>, std::vector<int>> groups;
    std::vector<std::pair<const fg_graph *, int>> order;
    for (int i = 0; i < nq; i++) {
        auto key = std::make_pair(qs[i].g, (int)qs[i].algo);
        auto it = groups.find(key);
        if (it == groups.end()) {
            order.push_back(key);
            groups[key].push_back(i);
        } else {
            it->second.push_back(i);
        }
    }
    for (auto &key : order) {
        const std::vector<int> &qi = groups[key];
        const Algo algo = (Algo)key.second;
        if (algo == kCC || qi.size() == 1) {
            BatchUnit u;
            u.g = key.first;
            u.algo = algo;
            u.mode = mode[qi[0]];
            u.q = qi;
            units.push_back(u);
            continue;
        }
        for (size_t b = 0; b < qi.size(); b += 8) {
            BatchUnit u;
            u.g = key.first;
            u.algo = algo;
            const size_t e = std::min(qi.size(), b + 8);
            u.q.assign(qi.begin() + (long)b, qi.begin() + (long)e);
            u.mode = u.q.size() >= 2 ? kMulti : mode[u.q[0]];
            units.push_back(u);
        }
    }
    return units;
}

// Plans, allocates and enqueues a batch on opt->stream; nothing waits.  The
// results reach device outputs directly; host outputs go to device staging
// and, if enqueue_host_copies, are copied back on the stream (their contents
// are then unspecified for a failed query), as are the copies of a shared
// CC result to its other outputs.  cta_fraction scales the CTA budget so
// that several batches can be resident at once.  fuse merges queries on the
// same graph (plan_units).
fg_status batch_launch(const fg_query *qs, int32_t nq, const fg_batch_options *opt, double cta_fraction,
                       bool enqueue_host_copies, bool fuse, Ctrl *h_ctrls_pinned, BatchJob &job) {
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

    // ---- resolve modes, form units, group them by kind, plan teams
    std::vector<Mode> mode(nq);
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
    }
    job.units = plan_units(qs, nq, mode, fuse);
    const int nu = (int)job.units.size();
    std::vector<BatchUnit> &units = job.units;
    std::vector<const View *> &view = job.view;
    view.resize(nu);
    job.qmode.assign(nq, kVertexSync);
    job.qunit.assign(nq, 0);
    std::map<int, KindPlan> kinds;
    double total_work = 0;
    for (int u = 0; u < nu; u++) {
        const BatchUnit &un = units[u];
        view[u] = (un.algo == kCC) ? &un.g->s : &un.g->g;
        for (int i : un.q) {
            job.qmode[i] = un.mode;
            job.qunit[i] = u;
        }
        // every multi-source sweep, SSSP or BFS, in one kernel (one launch)
        const int kind = un.mode == kMulti ? kAnyAlgo * 8 + kMulti : un.algo * 8 + (int)un.mode;
        KindPlan &kp = kinds[kind];
        kp.kind = kind;
        kp.queries.push_back(u);
        const double w = unit_work(un, *view[u]);
        kp.work += w;
        total_work += w;
    }
    for (auto &kv : kinds) {
        KindPlan &kp = kv.second;
        std::map<int, std::vector<int>> by_size;
        // a kind with few units (at most 8) gives each a larger team (a lone
        // unit the whole budget); otherwise the size follows its edge count
        int per_sm0 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm0, (const void *)batch_kernel_for(kp.kind), kBlock, 0);
        const int cap0 = std::max(1, (int)(std::max(1, std::min(per_sm0 * sms, kMaxGrid)) * cta_fraction *
                                           std::max(kp.work / std::max(total_work, 1.0), 0.0)));
        int share = 1;
        if (kp.queries.size() <= 8)
            while (share * 2 <= cap0 / (int)kp.queries.size()) share *= 2;
        for (int u : kp.queries) by_size[std::max(team_size_for(view[u]->m), share)].push_back(u);
        std::vector<double> cw;
        for (auto &c : by_size) {
            std::vector<int> v = c.second;
            std::sort(v.begin(), v.end(), [&](int a, int b) {
                return unit_work(units[a], *view[a]) > unit_work(units[b], *view[b]);
            });
            double w = 0;
            for (int u : v) w += unit_work(units[u], *view[u]);
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

    // ---- one device allocation: zeroed region | tables | unit workspaces | staging
    size_t zero_bytes = Workspace::need(1, sizeof(Ctrl)) + Workspace::need(nu, sizeof(Ctrl));
    size_t table_bytes = Workspace::need(nu, sizeof(Params)) + Workspace::need(nu, sizeof(int));
    for (auto &kv : kinds) {
        KindPlan &kp = kv.second;
        int teams = 0;
        for (int t : kp.class_teams) teams += t;
        const int nc = (int)kp.class_size.size();
        zero_bytes += Workspace::need(2 * teams, 4) + Workspace::need(teams, 4) + Workspace::need(nc, 4);
        table_bytes += Workspace::need(kp.ctas, sizeof(int4)) + 2 * Workspace::need(nc, 4);
    }
    job.staged.assign(nq, false);
    size_t ws_bytes = 0;
    for (int u = 0; u < nu; u++) {
        ws_bytes += query_workspace_bytes(*view[u], units[u].algo, units[u].mode);
        if (units[u].algo == kCC && units[u].g->orig_of)   // the labels' smallest original ids
            ws_bytes += Workspace::need(view[u]->n, 4);
    }
    for (int i = 0; i < nq; i++) {
        job.staged[i] = !is_device_pointer(qs[i].out);
        if (job.staged[i]) ws_bytes += Workspace::need(view[job.qunit[i]]->n, 4);
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
    job.d_ctrls = zw.take<Ctrl>(nu);
    Params *d_params = tw.take<Params>(nu);
    Params *h_params = hw.take<Params>(nu);
    int *d_order = tw.take<int>(nu);
    int *h_order = hw.take<int>(nu);
    job.dout.assign(nq, nullptr);
    for (int u = 0; u < nu; u++) {
        const BatchUnit &un = units[u];
        char *w = qw.base + qw.off;
        qw.off += query_workspace_bytes(*view[u], un.algo, un.mode);
        Params p;
        carve_query_workspace(w, *view[u], un.algo, un.mode, p);
        set_relabel(un.g, p);
        if (un.algo == kCC && un.g->orig_of) p.cc_min = qw.take<int32_t>(view[u]->n);
        h_params[u] = p;
    }
    for (int i = 0; i < nq; i++)
        job.dout[i] = job.staged[i] ? qw.take<int32_t>(view[job.qunit[i]]->n) : qs[i].out;
    for (int u = 0; u < nu; u++) {
        const BatchUnit &un = units[u];
        Params &p = h_params[u];
        if (un.mode == kPull) p.tv = (un.algo == kCC) ? un.g->s : un.g->t;
        p.delta = default_delta(un.g);
        p.ctrl = job.d_ctrls + u;
        p.source = un.algo == kCC ? 0 : qs[un.q[0]].src;
        p.max_rounds = view[u]->n > INT32_MAX - 2 ? INT32_MAX : view[u]->n + 2;
        p.timeout_ns = (unsigned long long)tmo * 1000000ull;
        if (un.mode == kMulti) {
            p.ms_k = (int32_t)un.q.size();
            p.ms_bfs = un.algo == kBFS ? 1 : 0;
            p.max_rounds = ms_default_rounds(view[u]->n, p.ms_k, un.algo == kSSSP);
            for (size_t j = 0; j < un.q.size(); j++) {
                p.ms_src[j] = qs[un.q[j]].src;
                p.ms_out[j] = job.dout[un.q[j]];
            }
        } else {
            p.out = job.dout[un.q[0]];
        }
    }
    job.params.assign(h_params, h_params + nu);
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
            for (int u : kp.class_q[c]) h_order[order_pos++] = u;
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
        job.own_ctrls.resize(nu);
        job.h_ctrls = job.own_ctrls.data();
    }
    ck(cudaMemcpyAsync(job.h_ctrls, job.d_ctrls, nu * sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "status copy");
    if (enqueue_host_copies) {
        for (int u = 0; u < nu; u++) {
            const BatchUnit &un = units[u];
            const size_t bytes = (size_t)view[u]->n * sizeof(int32_t);
            for (size_t j = 0; j < un.q.size(); j++) {
                const int i = un.q[j];
                if (un.mode != kMulti && j > 0)   // the unit's one result, to its other outputs
                    ck(cudaMemcpyAsync(qs[i].out, job.dout[un.q[0]], bytes, cudaMemcpyDefault, st), "result copy");
                else if (job.staged[i])
                    ck(cudaMemcpyAsync(qs[i].out, job.dout[i], bytes, cudaMemcpyDeviceToHost, st), "result copy");
            }
        }
        job.host_copies_done = true;
    }
    ck(cudaEventRecord(job.done, st), "event");
    if (job.status != FG_OK) return fail(job.status, job.msg);
    return FG_OK;
}

// Waits for a launched batch, reports every query and releases the batch.
fg_status batch_finish(BatchJob &job, fg_status *status_out, fg_stats *stats_out, fg_batch_stats *bstats) {
    const int nq = job.nq;
    const int nu = (int)job.units.size();
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
    std::vector<fg_status> qst(nq, FG_OK);
    for (int u = 0; u < nu && job.status == FG_OK; u++) {
        const Ctrl &hc = job.h_ctrls[u];
        const BatchUnit &un = job.units[u];
        const Params &p = job.params[u];
        const View &v = *job.view[u];
        const size_t bytes = (size_t)v.n * sizeof(int32_t);
        fg_status us = FG_OK;
        if (hc.status & kStTimeout) us = FG_ERR_TIMEOUT;
        else if (hc.status & kStRoundCap) us = FG_ERR_TIMEOUT;
        else if (hc.status & kStWorklist) us = FG_ERR_CUDA;
        else if (!hc.done) us = FG_ERR_TIMEOUT;
        for (int i : un.q) qst[i] = us;
        if (us == FG_OK && (hc.status & kStOverflow) && un.algo == kSSSP) {
            int *flag = reinterpret_cast<int *>(p.ctrl);
            int hf = 0;
            ck(cudaMemsetAsync(flag, 0, sizeof(int), st), "memset");
            if (un.mode == kMulti) {
                ms_overflow_check_launch(v, p.A, p.ms_k, flag, st);
            } else {   // on the result in internal order (p.out holds it in original order)
                overflow_check_launch(v, p.new_of ? ((hc.result_in_b && p.B) ? p.B : p.A) : p.out, flag, st);
            }
            ck(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
            ck(cudaStreamSynchronize(st), "overflow check");
            if (un.mode == kMulti) {
                // the sweep wrote no output: write those of the sources that did not overflow
                MsOuts ok{};
                for (size_t j = 0; j < un.q.size(); j++) {
                    if ((hf >> j) & 1) qst[un.q[j]] = FG_ERR_OVERFLOW;
                    else ok.p[j] = job.dout[un.q[j]];
                }
                ms_output_launch(p.A, v.n, p.ms_k, ok, p.new_of, st);
                if (job.host_copies_done)   // the early copies carried no result: copy again
                    for (size_t j = 0; j < un.q.size(); j++) {
                        const int i = un.q[j];
                        if (qst[i] == FG_OK && job.staged[i])
                            ck(cudaMemcpyAsync(job.qs[i].out, job.dout[i], bytes, cudaMemcpyDeviceToHost, st),
                               "result copy");
                    }
            } else if (hf) {
                for (int i : un.q) qst[i] = FG_ERR_OVERFLOW;
            }
        }
        if (!job.host_copies_done)
            for (size_t j = 0; j < un.q.size(); j++) {
                const int i = un.q[j];
                if (qst[i] != FG_OK) continue;
                if (un.mode != kMulti && j > 0)
                    ck(cudaMemcpyAsync(job.qs[i].out, job.dout[un.q[0]], bytes, cudaMemcpyDefault, st),
                       "result copy");
                else if (job.staged[i])
                    ck(cudaMemcpyAsync(job.qs[i].out, job.dout[i], bytes, cudaMemcpyDeviceToHost, st),
                       "result copy");
            }
        if (stats_out)
            for (int i : un.q) {
                fg_stats &s = stats_out[i];
                s = fg_stats{};
                s.mode = un.mode == kMulti ? -1 : (int32_t)un.mode;
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
    ck(cudaStreamSynchronize(st), "result copies");
    if (job.status != FG_OK)
        for (int i = 0; i < nq; i++) qst[i] = job.status;
    fg_status first_err = FG_OK;
    std::string first_msg;
    for (int i = 0; i < nq; i++) {
        if (status_out) status_out[i] = qst[i];
        if (qst[i] != FG_OK && first_err == FG_OK) {
            first_err = qst[i];
            first_msg = "batch query " + std::to_string(i) + " failed: " + fg_status_string(qst[i]);
        }
    }
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
    const bool fuse = opt && opt->fuse_same_graph;
    fg_status s = batch_launch(qs, nq, opt, 1.0, false, fuse, nullptr, job);
    fg_status f = batch_finish(job, status_out, stats_out, bstats);
    return s != FG_OK ? s : f;
}

}  // namespace fg
