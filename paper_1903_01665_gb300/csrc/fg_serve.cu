// Query server with continuous batching.
//
// Requests (SSSP / BFS / CC on resident graphs) are submitted from any host
// thread and queued.  A native worker thread admits them in waves: whenever a
// wave slot is free and the HBM budget of the in-flight waves' query state
// allows, the oldest pending request and the later ones of the same kind
// (graph, algorithm, mode; up to max_wave) are launched as one batch on the
// slot's stream (fg_batch.cu), so waves overlap on the device and requests
// arriving while others run start as soon as a slot and memory free up.
// Completion = the wave's results are in the callers' outputs; latency is
// measured from submission to completion.
//
// A request on a large graph (exclusive_edges) is not batched with other
// graphs' requests: it runs on the whole device as soon as the waves
// admitted before it have finished (the queue stays first come, first
// served) -- alone with the plain per-query kernel, or, with fusion, together
// with the later pending requests of the same graph and algorithm: up to 8
// SSSP or BFS requests as one multi-source sweep, every pending CC request
// as one computation copied to each output.  On such graphs one query fills
// the device, and fusing the queries' sweeps is what still saves work.
// Waves of smaller graphs fuse the same way inside the batch (fg_batch.cu).
//
// In one-at-a-time mode the worker serves the queue strictly one request at
// a time with the plain per-query kernel (the baseline).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

#include "fg_internal.cuh"

using Clock = std::chrono::steady_clock;

struct fg_server {
    fg_server_options opt{};
    int device = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_ticket = 1;

    struct Req {
        uint64_t ticket;
        fg_query q;
        Clock::time_point t_submit;
        size_t bytes;
        bool exclusive;           // runs alone on the whole device
        int32_t bps;              // FG_AUTO: the plan's CTAs per SM for a query run alone (0 = default)
    };
    struct Wave {
        fg::BatchJob job;
        std::vector<Req> reqs;
        size_t bytes = 0;
        int slot = 0;
    };
    std::deque<Req> pending;
    std::vector<std::unique_ptr<Wave>> inflight;
    std::deque<fg_completion> done;
    size_t bytes_inflight = 0;
    uint64_t n_submitted = 0, n_completed = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> after_legacy;   // per slot: legacy-stream work before a wave
    std::vector<bool> slot_busy;
    fg::Ctrl *pinned = nullptr;   // per slot: max_wave control blocks read back by the waves
};

namespace fg {
namespace {

size_t request_bytes(const fg_query &q, Mode m) {
    const View &v = (q.algo == FG_ALGO_CC) ? q.g->s : q.g->g;
    size_t b = query_workspace_bytes(v, (Algo)q.algo, m) + 4096;
    if (!is_device_pointer(q.out)) b += Workspace::need(v.n, 4);
    return b;
}

void complete(fg_server *s, const fg_server::Req &r, fg_status st, int wave_size, Clock::time_point now) {
    fg_completion c;
    c.ticket = r.ticket;
    c.status = (int32_t)st;
    c.wave_size = wave_size;
    c.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
    s->done.push_back(c);
    s->n_completed++;
}

// Orders the slot's stream after everything enqueued on the legacy default
// stream so far (e.g. the caller initialising its outputs before submitting);
// the slot streams are non-blocking and would otherwise overtake that work.
void after_legacy_work(fg_server *s, int slot) {
    cudaEventRecord(s->after_legacy[slot], (cudaStream_t)0);
    cudaStreamWaitEvent(s->streams[slot], s->after_legacy[slot], 0);
}

void serve_one_at_a_time(fg_server *s, std::unique_lock<std::mutex> &lk) {
    fg_server::Req r = s->pending.front();
    s->pending.pop_front();
    lk.unlock();
    fg_mode m = (fg_mode)r.q.mode;
    fg_status st = FG_OK;
    if (m == FG_AUTO) st = fg_select_mode(r.q.g, (fg_algo)r.q.algo, &m);
    if (st == FG_OK) {
        after_legacy_work(s, 0);
        fg_options o{};
        o.stream = s->streams[0];
        o.wait_timeout_ms = s->opt.wait_timeout_ms;
        o.blocks_per_sm = r.bps;
        st = run_query(r.q.g, (Algo)r.q.algo, (Mode)m, r.q.algo == FG_ALGO_CC ? 0 : r.q.src, r.q.out, &o, nullptr);
    }
    lk.lock();
    complete(s, r, st, 1, Clock::now());
}

// Runs a group of requests on one graph and algorithm alone on the whole
// device: one request with the plain per-query kernel, several SSSP/BFS as
// one multi-source sweep, several CC as one computation copied to each.
void serve_group_alone(fg_server *s, std::unique_lock<std::mutex> &lk, const std::vector<fg_server::Req> &reqs) {
    lk.unlock();
    after_legacy_work(s, 0);
    fg_options o{};
    o.stream = s->streams[0];
    o.wait_timeout_ms = s->opt.wait_timeout_ms;
    const fg_query &q0 = reqs[0].q;
    const int k = (int)reqs.size();
    std::vector<fg_status> sts(k, FG_OK);
    if (k == 1 || q0.algo == FG_ALGO_CC) o.blocks_per_sm = reqs[0].bps;
    if (k == 1) {
        sts[0] = run_query(q0.g, (Algo)q0.algo, (Mode)q0.mode, q0.algo == FG_ALGO_CC ? 0 : q0.src, q0.out, &o,
                           nullptr);
    } else if (q0.algo == FG_ALGO_CC) {
        fg_status st = run_query(q0.g, kCC, (Mode)q0.mode, 0, q0.out, &o, nullptr);
        cudaError_t e = cudaSuccess;
        const size_t bytes = (size_t)q0.g->s.n * sizeof(int32_t);
        for (int j = 1; j < k && st == FG_OK && e == cudaSuccess; j++)
            e = cudaMemcpyAsync(reqs[j].q.out, q0.out, bytes, cudaMemcpyDefault, s->streams[0]);
        if (st == FG_OK && e == cudaSuccess) e = cudaStreamSynchronize(s->streams[0]);
        if (st == FG_OK && e != cudaSuccess) st = cuda_fail(e, "result copies");
        for (int j = 0; j < k; j++) sts[j] = st;
    } else {
        int32_t srcs[8];
        int32_t *outs[8];
        for (int j = 0; j < k; j++) {
            srcs[j] = reqs[j].q.src;
            outs[j] = reqs[j].q.out;
        }
        run_multi(q0.g, (Algo)q0.algo, k, srcs, outs, &o, sts.data(), nullptr);
    }
    lk.lock();
    const Clock::time_point now = Clock::now();
    for (int j = 0; j < k; j++) complete(s, reqs[j], sts[j], k, now);
}

// The head request of the queue and the later pending requests that can
// join it: same graph and algorithm (and mode, without fusion), up to `cap`;
// they are taken out of the queue.
std::vector<fg_server::Req> take_group(fg_server *s, size_t cap, bool want_exclusive) {
    std::vector<fg_server::Req> out;
    const fg_query head = s->pending.front().q;
    const bool fuse = !s->opt.no_fusion;
    size_t window = std::min(s->pending.size(), (size_t)s->opt.max_wave * 8);   // requests scanned
    for (size_t i = 0; i < window && i < s->pending.size() && out.size() < cap;) {
        const fg_server::Req &r = s->pending[i];
        if (r.exclusive != want_exclusive || r.q.g != head.g || r.q.algo != head.algo ||
            (!fuse && r.q.mode != head.mode)) {
            i++;
            continue;
        }
        out.push_back(r);
        s->pending.erase(s->pending.begin() + (long)i);
        window--;
    }
    return out;
}

void worker_main(fg_server *s) {
    cudaSetDevice(s->device);
    const int max_inflight = s->opt.max_inflight;
    const int max_wave = s->opt.max_wave;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->pending.empty() && s->inflight.empty()) {
            if (s->stop) break;
            s->cv.wait(lk);
            continue;
        }
        if (s->opt.one_at_a_time) {
            if (!s->pending.empty()) serve_one_at_a_time(s, lk);
            s->cv.notify_all();
            continue;
        }
        // collect finished waves
        for (size_t i = 0; i < s->inflight.size();) {
            fg_server::Wave *w = s->inflight[i].get();
            if (cudaEventQuery(w->job.done) == cudaErrorNotReady) {
                i++;
                continue;
            }
            cudaGetLastError();
            std::vector<fg_status> sts(w->reqs.size(), FG_OK);
            lk.unlock();
            fg_status bst = batch_finish(w->job, sts.data(), nullptr, nullptr);
            lk.lock();
            const Clock::time_point now = Clock::now();
            for (size_t k = 0; k < w->reqs.size(); k++)
                complete(s, w->reqs[k], bst != FG_OK && sts[k] == FG_OK ? bst : sts[k], (int)w->reqs.size(), now);
            s->bytes_inflight -= w->bytes;
            s->slot_busy[w->slot] = false;
            s->inflight.erase(s->inflight.begin() + i);
        }
        // admit new waves while a slot and the HBM budget allow
        while (!s->pending.empty() && (int)s->inflight.size() < max_inflight) {
            if (s->pending.front().exclusive) {
                if (!s->inflight.empty()) break;   // after the waves before it
                if (s->opt.no_fusion) {
                    serve_one_at_a_time(s, lk);
                } else {
                    const size_t cap = s->pending.front().q.algo == FG_ALGO_CC ? (size_t)max_wave : 8;
                    std::vector<fg_server::Req> grp = take_group(s, cap, true);
                    serve_group_alone(s, lk, grp);
                }
                continue;
            }
            // a lone request on an idle device: the plain per-query kernel
            // (a batch of one costs its planning and staging for nothing)
            if (s->pending.size() == 1 && s->inflight.empty()) {
                serve_one_at_a_time(s, lk);
                continue;
            }
            int slot = 0;
            while (s->slot_busy[slot]) slot++;
            // A wave holds requests of one kind (graph, algorithm; and mode
            // without fusion): the oldest pending request and the later ones
            // of its kind.  Mixed waves finish with their slowest kind while
            // the CTAs of the others idle, and mix hot sets in each SM's L1;
            // with fusion, the batch merges the wave's requests into
            // multi-source sweeps (SSSP, BFS) and one computation (CC).
            std::unique_ptr<fg_server::Wave> w(new fg_server::Wave());
            size_t bytes = 0;
            const fg_query head = s->pending.front().q;
            const bool fuse = !s->opt.no_fusion;
            size_t window = std::min(s->pending.size(), (size_t)max_wave * 8);   // requests scanned
            for (size_t i = 0; i < window && i < s->pending.size() && (int)w->reqs.size() < max_wave;) {
                const fg_server::Req &r = s->pending[i];
                if (r.exclusive || r.q.g != head.g || r.q.algo != head.algo || (!fuse && r.q.mode != head.mode)) {
                    i++;
                    continue;
                }
                const bool fits = s->bytes_inflight + bytes + r.bytes <= (size_t)s->opt.hbm_budget_bytes;
                const bool alone = s->inflight.empty() && w->reqs.empty();   // always make progress
                if (!fits && !alone) break;
                bytes += r.bytes;
                w->reqs.push_back(r);
                s->pending.erase(s->pending.begin() + (long)i);
                window--;   // the scan window shrinks with the queue; i now names the next request
            }
            if (w->reqs.empty()) break;
            w->bytes = bytes;
            w->slot = slot;
            s->slot_busy[slot] = true;
            s->bytes_inflight += bytes;
            std::vector<fg_query> qs;
            for (auto &r : w->reqs) qs.push_back(r.q);
            fg_batch_options bo{};
            bo.stream = s->streams[slot];
            bo.wait_timeout_ms = s->opt.wait_timeout_ms;
            fg_server::Wave *wp = w.get();
            s->inflight.push_back(std::move(w));
            lk.unlock();
            after_legacy_work(s, slot);
            // a wave shares the device with the waves already running
            const double fraction = 1.0 / (double)s->inflight.size();
            fg_status ls = batch_launch(qs.data(), (int32_t)qs.size(), &bo, fraction, true, fuse,
                                        s->pinned + (size_t)slot * max_wave, wp->job);
            lk.lock();
            if (ls != FG_OK) {
                // nothing useful is running for this wave: report it now
                lk.unlock();
                batch_finish(wp->job, nullptr, nullptr, nullptr);
                lk.lock();
                const Clock::time_point now = Clock::now();
                for (auto &r : wp->reqs) complete(s, r, ls, (int)wp->reqs.size(), now);
                s->bytes_inflight -= wp->bytes;
                s->slot_busy[wp->slot] = false;
                for (size_t i = 0; i < s->inflight.size(); i++)
                    if (s->inflight[i].get() == wp) {
                        s->inflight.erase(s->inflight.begin() + i);
                        break;
                    }
            }
        }
        s->cv.notify_all();
        if (!s->inflight.empty()) s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" {

fg_status fg_server_create(const fg_server_options *opt, fg_server **out) {
    if (!out) return fail(FG_ERR_INVALID_ARG, "out is NULL");
    fg_server_options o{};
    if (opt) o = *opt;
    if (o.hbm_budget_bytes < 0 || o.max_inflight < 0 || o.max_wave < 0 || o.wait_timeout_ms < 0)
        return fail(FG_ERR_INVALID_ARG, "negative option");
    if (o.hbm_budget_bytes == 0) o.hbm_budget_bytes = (int64_t)8 << 30;
    if (o.exclusive_edges == 0) o.exclusive_edges = (int64_t)1 << 25;
    // two waves in flight: a new wave starts while one runs; more made the
    // waves' kernels crowd each other's SMs (L1, CTA budget) and cost
    // throughput on the R-MAT 20-22 + grid mix
    if (o.max_inflight == 0) o.max_inflight = 2;
    if (o.max_wave == 0) o.max_wave = 64;
    if (o.one_at_a_time) o.max_inflight = 1;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(FG_ERR_CUDA, "no CUDA device");
    }
    fg_server *s = new (std::nothrow) fg_server();
    if (!s) return fail(FG_ERR_OUT_OF_MEMORY, "host allocation failed");
    s->opt = o;
    s->device = dev;
    s->streams.assign(o.max_inflight, nullptr);
    s->after_legacy.assign(o.max_inflight, nullptr);
    s->slot_busy.assign(o.max_inflight, false);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < o.max_inflight && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->after_legacy[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&s->pinned, sizeof(Ctrl) * (size_t)o.max_inflight * o.max_wave);
    if (e != cudaSuccess) {
        for (auto st : s->streams)
            if (st) cudaStreamDestroy(st);
        for (auto ev : s->after_legacy)
            if (ev) cudaEventDestroy(ev);
        delete s;
        return cuda_fail(e, "server setup");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return FG_OK;
}

fg_status fg_server_submit(fg_server *s, const fg_query *q, uint64_t *ticket) {
    if (!s || !q) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    if (!q->g || !q->out) return fail(FG_ERR_INVALID_ARG, "graph or output is NULL");
    if (q->algo < FG_ALGO_SSSP || q->algo > FG_ALGO_CC) return fail(FG_ERR_INVALID_ARG, "invalid algorithm");
    if (q->mode < FG_VERTEX_SYNC || q->mode > FG_BUCKET) return fail(FG_ERR_INVALID_ARG, "invalid mode");
    if (q->algo != FG_ALGO_CC && (q->src < 0 || q->src >= q->g->info.n))
        return fail(FG_ERR_INVALID_ARG, "source vertex outside [0, n)");
    if (q->g->device != s->device) return fail(FG_ERR_INVALID_ARG, "graph lives on another device");
    fg_query qq = *q;
    fg_mode m = (fg_mode)qq.mode;
    int32_t bps = 0;
    if (m == FG_AUTO) {
        fg_plan pl;
        fg_status st = fg_select_plan(qq.g, (fg_algo)qq.algo, &pl);
        if (st != FG_OK) return st;
        m = (fg_mode)pl.mode;
        bps = pl.blocks_per_sm;
    }
    qq.mode = (int32_t)m;
    {   // a FG_GRAPH_LAZY graph builds the parts this request reads now, so
        // that the request's workspace size is known and no wave builds them
        fg_status vs = ensure_views(qq.g, (Algo)qq.algo, (int)m);
        if (vs != FG_OK) return vs;
    }
    const int64_t edges = (qq.algo == FG_ALGO_CC) ? qq.g->s.m : qq.g->g.m;
    const bool exclusive = s->opt.exclusive_edges > 0 && edges >= s->opt.exclusive_edges;
    fg_server::Req r{0, qq, Clock::now(), request_bytes(qq, (Mode)m), exclusive, bps};
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(FG_ERR_INVALID_ARG, "server is shutting down");
        r.ticket = s->next_ticket++;
        s->pending.push_back(r);
        s->n_submitted++;
    }
    s->cv.notify_all();
    if (ticket) *ticket = r.ticket;
    return FG_OK;
}

int32_t fg_server_poll(fg_server *s, fg_completion *out, int32_t cap) {
    if (!s || !out || cap <= 0) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    int32_t n = 0;
    while (n < cap && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

fg_status fg_server_drain(fg_server *s, int32_t timeout_ms) {
    if (!s) return fail(FG_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto pred = [&] { return s->n_completed == s->n_submitted; };
    if (timeout_ms > 0) {
        if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
            return fail(FG_ERR_TIMEOUT, "requests still running after the drain timeout");
    } else {
        s->cv.wait(lk, pred);
    }
    return FG_OK;
}

fg_status fg_server_destroy(fg_server *s) {
    if (!s) return FG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto ev : s->after_legacy)
        if (ev) cudaEventDestroy(ev);
    if (s->pinned) cudaFreeHost(s->pinned);
    delete s;
    return FG_OK;
}

}  // extern "C"
