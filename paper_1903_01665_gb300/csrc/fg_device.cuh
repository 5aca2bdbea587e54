// Device code of the fixpoint relaxation sweep, shared by the single-query
// kernels (fg_fixpoint.cu) and the batched kernel (fg_batch.cu).
//
// The four variants of Sec. 3.1-3.3 run as persistent cooperative kernels:
// init, every round and the convergence test happen on the device, rounds
// separated by bounded barriers.  Everything here is parameterised by a Team:
// the CTAs that run one query together (the whole grid for a single query; a
// slice of the grid, down to one CTA, for a query of a batch).
//
//   vertex-sync  : Alg. 1 -- every round scans the vertices (dense activity
//                  words, degree-bucketed lists) and expands those that
//                  changed in the previous round; reads cur, MIN into next
//                  (double-buffered, Jacobi), barrier, swap.
//   edge-sync    : Alg. 2 -- every round streams the edges (src,dst,w) in
//                  1024-edge tiles by bulk copy (TMA) into a shared-memory
//                  ring and relaxes those whose source changed; rounds with
//                  few changes stream only the flagged tiles.
//   vertex-async : data-driven (Sec. 3.3) -- worklists of vertices by degree
//                  class, in-place atomic MIN, changed targets appended through
//                  per-warp buffers, until the worklist is empty.
//   edge-async   : the worklist's out-edges, load-balanced edge-parallel by a
//                  prefix sum of the items' degrees, in place.
//
// BFS uses Alg. 3's level filter (dist == lev, plain store of lev+1); CC is
// min-label propagation on the symmetrised graph plus pointer jumping
// (label[v] = label[label[v]]).
#pragma once

#include <algorithm>

#include "fg_internal.cuh"

namespace fg {
namespace {


struct Acc {
    unsigned long long edges = 0, verts = 0, updates = 0, pushes = 0, scanned = 0, pulled = 0;
    int changed = 0;
    int overflow = 0;
};

__device__ __forceinline__ int32_t warp_min(int32_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// minimum over the CTA, returned to every thread
__device__ __forceinline__ int32_t block_min(int32_t x) {
    __shared__ int32_t sh[kWarps];
    x = warp_min(x);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    int32_t r = sh[0];
#pragma unroll
    for (int i = 1; i < kWarps; i++) r = min(r, sh[i]);
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T block_sum(T x) {
    __shared__ T sh[kWarps];
    x = warp_sum(x);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    T r = 0;
    if (threadIdx.x < 32) {
        r = lane_id() < (unsigned)kWarps ? sh[lane_id()] : (T)0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// ================================================================ edge ops
// Each op provides:
//   active(u, val, rq) -- is u expanded this round; its value.  An op may
//                      lower u's own value here (CC pointer jumping); it then
//                      sets rq if u must be re-queued for the next generation.
//   own(u, val)     -- once per expanded vertex (sync: carry cur[u] into next)
//   cand(val, e, c, a) -- the candidate value of edge e from a source value
//                      val (false: dropped, e.g. >= INT32_MAX)
//   probe(v)        -- the target's current value, to compare against
//   commit(v, c, pv, a) -- apply a candidate; true if v must be appended to
//                      the worklist.
// Splitting a relaxation into cand / probe / commit lets the expansions
// issue the loads of several edges before using any of them.

// Synchronous SSSP / CC: Jacobi round r reads cur, lowers next.
template <int ALGO>
struct SyncOp {
    const int32_t *__restrict__ w;
    const int32_t *cur;
    int32_t *next;
    const int32_t *scur;
    int32_t *snext;
    int32_t r;
    bool two;          // apply the second filter (running minimum) in this round

    // cur and scur are the previous round's: not written during the round
    __device__ __forceinline__ bool active(int32_t u, int32_t &val, bool &) const {
        if (ldca(scur + u) != r) return false;
        val = ldca(cur + u);
        return true;
    }
    __device__ __forceinline__ void own(int32_t u, int32_t val) const { red_min(next + u, val); }
    __device__ __forceinline__ int32_t refresh(int32_t, int32_t val) const { return val; }
    __device__ __forceinline__ bool cand(int32_t val, uint32_t e, int32_t &c, Acc &a) const {
        if (ALGO == kSSSP) {
            uint32_t x = (uint32_t)val + (uint32_t)ld_edge(w + e);
            if (x >= (uint32_t)kInf) { a.overflow = 1; return false; }
            c = (int32_t)x;
        } else {
            c = val;
        }
        return true;
    }
    // staged-stream interface: the activity word and the value are loaded
    // together (no dependent load), the weight comes from shared memory
    __device__ __forceinline__ void load_act(int32_t u, int32_t &s, int32_t &v) const {
        s = ldca(scur + u);
        v = ldca(cur + u);
    }
    __device__ __forceinline__ bool is_act(int32_t s, int32_t) const { return s == r; }
    __device__ __forceinline__ bool cand_w(int32_t val, int32_t wv, int32_t &c, Acc &a) const {
        if (ALGO == kSSSP) {
            uint32_t x = (uint32_t)val + (uint32_t)wv;
            if (x >= (uint32_t)kInf) { a.overflow = 1; return false; }
            c = (int32_t)x;
        } else {
            c = val;
        }
        return true;
    }
    __device__ __forceinline__ int32_t probe(int32_t v) const { return ldca(cur + v); }
    // v changes this round iff some candidate is below its previous-round
    // value, so any such candidate may mark it: the MIN needs no return value.
    __device__ __forceinline__ bool commit(int32_t v, int32_t c, int32_t pv, Acc &a) const {
        if (c < pv) {
            red_min(next + v, c);
            stcg(snext + v, r + 1);
            a.changed++;
            a.updates++;
        }
        return false;
    }
    // Second filter: a candidate below cur[v] is checked against next[v],
    // the running minimum of this round (read through L2), and only one that
    // beats it is applied.  next[v] below cur[v] means an earlier candidate
    // went below cur[v] and marked v, so only the first one writes the mark.
    // (R-MAT 22 CC's all-active first round: most of its 67 M MINs skipped.)
    // It pays where many candidates meet at one target (dense rounds of
    // skewed graphs); a round after few changes skips the extra load.
    static constexpr bool kNextProbe = true;
    __device__ __forceinline__ int32_t probe_next(int32_t v) const { return two ? ldcg(next + v) : kInf; }
    __device__ __forceinline__ bool commit2(int32_t v, int32_t c, int32_t pv, int32_t nv, Acc &a) const {
        if (c < pv && c < nv) {
            red_min(next + v, c);
            if (nv >= pv) stcg(snext + v, r + 1);
            a.changed++;
            a.updates++;
        }
        return false;
    }
};

// Level-synchronous BFS (Alg. 3): in place, filter dist == lev.
struct BfsSyncOp {
    static constexpr bool kNextProbe = false;
    int32_t *L;
    int32_t lev;
    uint32_t *vis;     // visited bitmap: the probe's 32x denser copy of "L[v] != INF"

    __device__ __forceinline__ bool active(int32_t u, int32_t &val, bool &) const {
        val = lev;
        return ldcg(L + u) == lev;
    }
    __device__ __forceinline__ void own(int32_t, int32_t) const {}
    __device__ __forceinline__ int32_t refresh(int32_t, int32_t val) const { return val; }
    __device__ __forceinline__ bool cand(int32_t, uint32_t, int32_t &c, Acc &) const {
        c = lev + 1;
        return true;
    }
    // A source's level was set in an earlier round, so L1 is exact for it.
    // The probe may also go through L1: a stale copy can only show INF for a
    // vertex another thread set to lev+1 in this round, and then the store
    // below writes that same level again (the counters count it twice; the
    // result and the no-change test are unaffected).
    __device__ __forceinline__ void load_act(int32_t u, int32_t &s, int32_t &v) const {
        v = ldca(L + u);
        s = v;
    }
    __device__ __forceinline__ bool is_act(int32_t, int32_t v) const { return v == lev; }
    __device__ __forceinline__ bool cand_w(int32_t, int32_t, int32_t &c, Acc &) const {
        c = lev + 1;
        return true;
    }
    // The probe reads the visited bitmap (n/8 bytes, mostly L1 hits) instead
    // of the level array: a visited vertex has a level <= lev + 1 and cannot
    // be lowered.  A stale copy misses only bits set in this round, whose
    // vertices then get the same level stored again.
    __device__ __forceinline__ int32_t probe(int32_t v) const { return vis_test(vis, v) ? 0 : kInf; }
    __device__ __forceinline__ bool commit(int32_t v, int32_t c, int32_t pv, Acc &a) const {
        if (pv > c) {
            stcg(L + v, c);
            red_or(vis + (v >> 5), 1u << (v & 31));
            a.changed++;
            a.updates++;
        }
        return false;
    }
};

// Asynchronous SSSP / CC: in place, push on decrease, dedup by generation stamp.
template <int ALGO>
struct AsyncOp {
    static constexpr bool kNextProbe = false;
    const int32_t *__restrict__ w;
    int32_t *D;
    int32_t *stamp;
    int32_t gen;
    // edge-async: refresh a staged window's values before each sub-tile
    static constexpr bool kRefreshWindow = (ALGO == kSSSP);

    __device__ __forceinline__ bool active(int32_t u, int32_t &val, bool &rq) const {
        val = ldcg(D + u);
        if (ALGO == kCC) {
            // pointer jumping: follow label[label[...]] while it decreases
            int32_t l = val;
#pragma unroll 1
            for (int k = 0; k < 8; k++) {
                int32_t ll = ldcg(D + l);
                if (ll >= l) break;
                l = ll;
            }
            if (l < val) {
                // u's other edges may be relaxed elsewhere with the old label,
                // so u is queued again to pass the new one to all neighbours
                if (atomicMin(D + u, l) > l) rq = atomicExch(stamp + u, gen + 1) != gen + 1;
                val = l;
            }
        }
        return true;
    }
    __device__ __forceinline__ void own(int32_t, int32_t) const {}
    // in place: the latest value, read just before the vertex is expanded
    __device__ __forceinline__ int32_t refresh(int32_t u, int32_t val) const { return min(val, ldcg(D + u)); }
    __device__ __forceinline__ bool cand(int32_t val, uint32_t e, int32_t &c, Acc &a) const {
        if (ALGO == kSSSP) {
            uint32_t x = (uint32_t)val + (uint32_t)ld_edge(w + e);
            if (x >= (uint32_t)kInf) { a.overflow = 1; return false; }
            c = (int32_t)x;
        } else {
            c = val;
        }
        return true;
    }
    // Values only decrease, so an L1 copy (possibly stale, never below the
    // current value) rejects most candidates without an L2 access; the few
    // it lets through are checked again against L2 before the update.
    __device__ __forceinline__ int32_t probe(int32_t v) const { return ldca(D + v); }
    // A candidate below the value just read lowers v or loses to an even
    // lower one; either way v has changed in this generation and is queued
    // (once, by the stamp) for the next.
    __device__ __forceinline__ bool commit(int32_t v, int32_t c, int32_t pv, Acc &a) const {
        if (c < pv && c < ldcg(D + v)) {
            red_min(D + v, c);
            a.updates++;
            return atomicExch(stamp + v, gen + 1) != gen + 1;
        }
        return false;
    }
};

// Dense vertex-async SSSP generation: every vertex is tested instead of the
// worklist's items; a vertex is expanded if it was queued for this
// generation (stamp g) or lowered during it (stamp g + 1, queued for the
// next as well): a relaxation with a current distance is always valid.
#ifndef FG_VA_DENSE_DIV
#define FG_VA_DENSE_DIV 4
#endif
struct AsyncScanOp : AsyncOp<kSSSP> {
    __device__ __forceinline__ bool active(int32_t u, int32_t &val, bool &) const {
        if (ldca(stamp + u) < gen) return false;
        val = ldcg(D + u);
        return val != kInf;
    }
};

// Bucketed SSSP (near-far): as AsyncOp, but a target whose new distance is
// not below the threshold T goes to the far list of the current epoch (once
// per epoch, by far_mark) instead of the next generation's worklist.
struct BucketOp : AsyncOp<kSSSP> {
    int32_t T;
    int32_t epoch;
    int32_t *far;
    int32_t *far_mark;
    int *far_size;
    int32_t far_cap;
    Ctrl *ctrl;

    __device__ __forceinline__ bool commit(int32_t v, int32_t c, int32_t pv, Acc &a) const {
        if (c < pv && c < ldcg(D + v)) {
            red_min(D + v, c);
            a.updates++;
            if (c < T) return atomicExch(stamp + v, gen + 1) != gen + 1;
            if (atomicExch(far_mark + v, epoch) != epoch) {
                // warp-aggregated append of the lanes that got here together
                const unsigned am = __activemask();
                const int leader = __ffs(am) - 1;
                int base = 0;
                if ((int)lane_id() == leader) base = atomicAdd(far_size, __popc(am));
                base = __shfl_sync(am, base, leader) + __popc(am & lanemask_lt());
                if (base < far_cap) far[base] = v;
                else atomicOr(&ctrl->status, kStWorklist);
            }
        }
        return false;
    }
};

// Asynchronous BFS: frontier queue; a vertex is claimed once by CAS from INF.
struct BfsAsyncOp {
    static constexpr bool kNextProbe = false;
    int32_t *L;
    int32_t gen;
    uint32_t *vis;     // visited bitmap; a vertex is claimed by setting its bit
    static constexpr bool kRefreshWindow = false;

    __device__ __forceinline__ bool active(int32_t, int32_t &val, bool &) const {
        val = gen;
        return true;
    }
    __device__ __forceinline__ void own(int32_t, int32_t) const {}
    __device__ __forceinline__ int32_t refresh(int32_t, int32_t val) const { return val; }
    __device__ __forceinline__ bool cand(int32_t, uint32_t, int32_t &c, Acc &) const {
        c = gen + 1;
        return true;
    }
    // a vertex, once claimed, stays claimed: an L1 copy of its bitmap word
    // that shows the bit is exact, one that does not may be stale and the
    // atomic OR decides; its one winner stores the level and queues it
    __device__ __forceinline__ int32_t probe(int32_t v) const { return vis_test(vis, v) ? 0 : kInf; }
    __device__ __forceinline__ bool commit(int32_t v, int32_t c, int32_t pv, Acc &a) const {
        if (pv != kInf) return false;
        const uint32_t bit = 1u << (v & 31);
        if (atomicOr(vis + (v >> 5), bit) & bit) return false;
        stcg(L + v, c);
        a.updates++;
        return true;
    }
};

// One full sweep with every vertex active (roofline measurement).
struct SweepOp {
    static constexpr bool kNextProbe = false;
    const int32_t *__restrict__ w;
    const int32_t *cur;
    int32_t *next;

    // cur is read-only during the sweep; a stale (larger) probe of next only
    // lets through a candidate the atomic MIN then rejects
    __device__ __forceinline__ bool active(int32_t u, int32_t &val, bool &) const {
        val = ldca(cur + u);
        return val != kInf;
    }
    __device__ __forceinline__ void own(int32_t, int32_t) const {}
    __device__ __forceinline__ int32_t refresh(int32_t, int32_t val) const { return val; }
    __device__ __forceinline__ bool cand(int32_t val, uint32_t e, int32_t &c, Acc &a) const {
        uint32_t x = (uint32_t)val + (uint32_t)ld_edge(w + e);
        if (x >= (uint32_t)kInf) { a.overflow = 1; return false; }
        c = (int32_t)x;
        return true;
    }
    __device__ __forceinline__ void load_act(int32_t u, int32_t &s, int32_t &v) const {
        v = ldca(cur + u);
        s = v;
    }
    __device__ __forceinline__ bool is_act(int32_t, int32_t v) const { return v != kInf; }
    __device__ __forceinline__ bool cand_w(int32_t val, int32_t wv, int32_t &c, Acc &a) const {
        uint32_t x = (uint32_t)val + (uint32_t)wv;
        if (x >= (uint32_t)kInf) { a.overflow = 1; return false; }
        c = (int32_t)x;
        return true;
    }
    __device__ __forceinline__ int32_t probe(int32_t v) const { return ldca(next + v); }
    // a write per candidate below the probed value: at least the number of
    // lowered values, at most the number of edges
    __device__ __forceinline__ bool commit(int32_t v, int32_t c, int32_t pv, Acc &a) const {
        if (c < pv) {
            red_min(next + v, c);
            a.updates++;
        }
        return false;
    }
};

// ================================================================ appenders
struct NoPush {
    __device__ __forceinline__ void operator()(bool, int32_t, Acc &) const {}
    __device__ __forceinline__ void flush() const {}
};

// Per-warp staging buffer of worklist appends in shared memory: appends go
// to the warp's buffer (ballot + prefix, no atomics) and reach the global
// list in blocks, one atomicAdd on the list's size per block, so that
// thousands of warps do not serialise on one counter.
constexpr int kPushBuf = 256;
struct WarpBuf {
    int32_t item[kPushBuf];
    int count;
};

__device__ __forceinline__ void warp_flush(WarpBuf *b, int cnt, int32_t *list, int *size, int32_t cap, Ctrl *c) {
    __syncwarp();
    int base = 0;
    if (lane_id() == 0) base = atomicAdd(size, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = (int)lane_id(); i < cnt; i += 32) {
        int pos = base + i;
        if (pos < cap) list[pos] = b->item[i];
        else atomicOr(&c->status, kStWorklist);
    }
    __syncwarp();
}

__device__ __forceinline__ void buffered_append(bool want, int32_t v, WarpBuf *b, int32_t *list, int *size,
                                                int32_t cap, Ctrl *c) {
    unsigned bal = __ballot_sync(0xffffffffu, want);
    if (bal == 0) return;
    int n = __popc(bal);
    int cnt = b->count;
    if (cnt + n > kPushBuf) {
        warp_flush(b, cnt, list, size, cap, c);
        cnt = 0;
    }
    if (want) b->item[cnt + __popc(bal & lanemask_lt())] = v;
    __syncwarp();
    if (lane_id() == 0) b->count = cnt + n;
    __syncwarp();
}

__device__ __forceinline__ void buffered_flush(WarpBuf *b, int32_t *list, int *size, int32_t cap, Ctrl *c) {
    int cnt = b->count;
    if (cnt > 0) warp_flush(b, cnt, list, size, cap, c);
    __syncwarp();
    if (lane_id() == 0) b->count = 0;
    __syncwarp();
}

// vertex-async: append to the class list of the target's out-degree
struct ClassPush {
    const uint32_t *__restrict__ row_off;
    const uint8_t *__restrict__ vclass;   // 0 no out-edge, 1 low, 2 mid, 3 high
    int32_t *low, *mid;
    int2 *high;
    int *size;          // [3]
    int32_t cap_low, cap_mid, cap_high;
    WarpBuf *buf_low, *buf_mid;           // this warp's staging buffers
    Ctrl *c;

    __device__ __forceinline__ void operator()(bool want, int32_t v, Acc &a) const {
        int cls = -1;
        if (want) {
            cls = (int)__ldg(vclass + v) - 1;
            if (cls >= 0) a.pushes++;
        }
        if (__ballot_sync(0xffffffffu, cls >= 0) == 0) return;
        buffered_append(cls == kWlLow, v, buf_low, low, &size[kWlLow], cap_low, c);
        buffered_append(cls == kWlMid, v, buf_mid, mid, &size[kWlMid], cap_mid, c);
        if (cls == kWlHigh) {
            uint32_t b = __ldg(row_off + v), d = __ldg(row_off + v + 1) - b;
            int nck = (int)((d + kChunk - 1) / kChunk);
            int base = atomicAdd(&size[kWlHigh], nck);
            if (base + nck <= cap_high) {
                for (int k = 0; k < nck; k++) high[base + k] = make_int2(v, (int32_t)(b + (uint32_t)k * kChunk));
            } else {
                atomicOr(&c->status, kStWorklist);
            }
        }
    }
    __device__ __forceinline__ void flush() const {
        buffered_flush(buf_low, low, &size[kWlLow], cap_low, c);
        buffered_flush(buf_mid, mid, &size[kWlMid], cap_mid, c);
    }
};

// edge-async: the worklist with each item's global edge offset.  A warp's
// staged block of items reserves its slots and its edges in one 64-bit
// atomicAdd on (edges << 32 | items), so the next generation's load balance
// needs no separate prefix pass over the worklist.
struct LbPush {
    const uint32_t *__restrict__ row_off;
    const uint8_t *__restrict__ vclass;
    int32_t *list;
    uint32_t *off;
    unsigned long long *pack;
    int32_t cap;
    WarpBuf *buf;
    Ctrl *c;

    __device__ __forceinline__ void flush_block(int cnt) const {
        __syncwarp();
        const unsigned lane = lane_id();
        constexpr int kPer = kPushBuf / 32;   // contiguous items per lane
        uint32_t deg[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const int i = (int)lane * kPer + k;
            deg[k] = 0;
            if (i < cnt) {
                const int32_t v = buf->item[i];
                deg[k] = __ldg(row_off + v + 1) - __ldg(row_off + v);
            }
            sum += deg[k];
        }
        const uint32_t incl = warp_inclusive_scan(sum);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(pack, ((unsigned long long)total << 32) | (unsigned)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t ibase = (uint32_t)base, ebase = (uint32_t)(base >> 32);
        uint32_t run = ebase + incl - sum;
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const int i = (int)lane * kPer + k;
            if (i < cnt) {
                const uint32_t pos = ibase + (uint32_t)i;
                if (pos < (uint32_t)cap) {
                    list[pos] = buf->item[i];
                    off[pos] = run;
                } else {
                    atomicOr(&c->status, kStWorklist);
                }
            }
            run += deg[k];
        }
        __syncwarp();
    }
    __device__ __forceinline__ void operator()(bool want, int32_t v, Acc &a) const {
        bool ok = false;
        if (want) {
            ok = __ldg(vclass + v) != 0;
            if (ok) a.pushes++;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (bal == 0) return;
        const int n = __popc(bal);
        int cnt = buf->count;
        if (cnt + n > kPushBuf) {
            flush_block(cnt);
            cnt = 0;
        }
        if (ok) buf->item[cnt + __popc(bal & lanemask_lt())] = v;
        __syncwarp();
        if (lane_id() == 0) buf->count = cnt + n;
        __syncwarp();
    }
    __device__ __forceinline__ void flush() const {
        const int cnt = buf->count;
        if (cnt > 0) flush_block(cnt);
        __syncwarp();
        if (lane_id() == 0) buf->count = 0;
        __syncwarp();
    }
};

// ================================================================ batched relaxation
constexpr int kU = 4;   // edges per thread per loop iteration

// Relax up to kU edges per thread: every load of the batch is issued before
// any result is used.  All lanes of the warp call it (the appends are
// warp-collective); lanes with in[j] == false take no part in edge j.
template <class OP, class PUSH, int N>
__device__ __forceinline__ void relax_batch(const int32_t *__restrict__ col, const OP &op, const PUSH &push,
                                            const uint32_t (&e)[N], const int32_t (&val)[N],
                                            const bool (&in)[N], Acc &a) {
    int32_t v[N], c[N], pv[N];
    bool ok[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        v[j] = 0;
        c[j] = 0;
        ok[j] = in[j];
        if (ok[j]) {
            v[j] = ld_edge(col + e[j]);
            ok[j] = op.cand(val[j], e[j], c[j], a);
        }
    }
#pragma unroll
    for (int j = 0; j < N; j++) pv[j] = ok[j] ? op.probe(v[j]) : 0;
    bool want[N];
    if constexpr (OP::kNextProbe) {
        int32_t nv[N];
#pragma unroll
        for (int j = 0; j < N; j++) nv[j] = (ok[j] && c[j] < pv[j]) ? op.probe_next(v[j]) : 0;
#pragma unroll
        for (int j = 0; j < N; j++) want[j] = ok[j] && op.commit2(v[j], c[j], pv[j], nv[j], a);
    } else {
#pragma unroll
        for (int j = 0; j < N; j++) want[j] = ok[j] && op.commit(v[j], c[j], pv[j], a);
    }
#pragma unroll
    for (int j = 0; j < N; j++) push(want[j], v[j], a);
}

// Edges of up to 32 rows, given per lane as (row start, degree < 32, value),
// redistributed over the warp: a warp-wide prefix sum of the degrees, and each
// lane finds the owner row of its edge by a 5-step shuffle search, so that the
// edge loads of a batch are contiguous.
template <class OP, class PUSH>
__device__ __forceinline__ void relax_rows_of_warp(const int32_t *__restrict__ col, const OP &op, const PUSH &push,
                                                   uint32_t rb, uint32_t d, int32_t vv, Acc &a) {
    const unsigned lane = lane_id();
    uint32_t incl = warp_inclusive_scan(d);
    uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t excl = incl - d;
    if (lane == 0) a.edges += total;
    for (uint32_t k0 = 0; k0 < total; k0 += 32 * kU) {
        uint32_t e[kU];
        int32_t val[kU];
        bool in[kU];
#pragma unroll
        for (int j = 0; j < kU; j++) {
            uint32_t k = k0 + 32 * j + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                uint32_t pv = __shfl_sync(0xffffffffu, incl, owner + step - 1);
                if (pv <= k) owner += step;
            }
            uint32_t ob = __shfl_sync(0xffffffffu, rb, owner);
            uint32_t oe = __shfl_sync(0xffffffffu, excl, owner);
            val[j] = __shfl_sync(0xffffffffu, vv, owner);
            e[j] = ob + (k - oe);
            in[j] = k < total;
        }
        relax_batch(col, op, push, e, val, in, a);
    }
}

// Synchronous low-degree path: the warp scans 128 consecutive vertex ids per
// step with 128-bit loads of the activity word (round stamp, or BFS level),
// compacts the active vertices with 1..31 out-edges into shared memory, and
// relaxes their edges 32 rows at a time.  Mid and high vertices are expanded
// from their bucket lists; vertices without out-edges have nothing to expand.
template <class OP>
__device__ __forceinline__ void expand_low_dense(const Team &t, const uint32_t *__restrict__ row_off, const int32_t *__restrict__ col,
                                                 const int32_t *actw, int32_t act_val, int32_t n, const OP &op,
                                                 Acc &a) {
    __shared__ uint32_t s_rb[kWarps][128];
    __shared__ uint32_t s_d[kWarps][128];
    __shared__ int32_t s_v[kWarps][128];
    const unsigned lane = lane_id();
    const int wid = threadIdx.x >> 5;
    const int64_t gw = (t.rank * (int64_t)kBlock + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)t.size * kWarps;
    for (int64_t w0 = gw * 128; w0 < n; w0 += nw * 128) {
        const int64_t v0 = w0 + 4 * lane;
        if (lane == 0) a.scanned += min((int64_t)128, (int64_t)n - w0);
        int32_t st[4];
        if (v0 + 3 < n) {
            int4 t = __ldcg(reinterpret_cast<const int4 *>(actw + v0));
            st[0] = t.x; st[1] = t.y; st[2] = t.z; st[3] = t.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) st[j] = (v0 + j < n) ? ldcg(actw + v0 + j) : act_val - 1;
        }
        bool act[4];
        uint32_t rb[4], d[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            act[j] = st[j] == act_val;
            rb[j] = 0;
            d[j] = 0;
            if (act[j]) {
                rb[j] = __ldg(row_off + v0 + j);
                d[j] = __ldg(row_off + v0 + j + 1) - rb[j];
                act[j] = d[j] >= 1 && d[j] < (uint32_t)kLowMax;
            }
        }
        unsigned cnt_lane = act[0] + act[1] + act[2] + act[3];
        unsigned any = __ballot_sync(0xffffffffu, cnt_lane != 0);
        if (!any) continue;
        unsigned incl = warp_inclusive_scan(cnt_lane);
        unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned slot = incl - cnt_lane;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (act[j]) {
                int32_t val;
                bool rq;
                op.active((int32_t)(v0 + j), val, rq);
                op.own((int32_t)(v0 + j), val);
                s_rb[wid][slot] = rb[j];
                s_d[wid][slot] = d[j];
                s_v[wid][slot] = val;
                slot++;
            }
        }
        __syncwarp();
        if (lane == 0) a.verts += tot;
        for (unsigned g0 = 0; g0 < tot; g0 += 32) {
            unsigned k = g0 + lane;
            uint32_t r0 = 0, dd = 0;
            int32_t vv = 0;
            if (k < tot) {
                r0 = s_rb[wid][k];
                dd = s_d[wid][k];
                vv = s_v[wid][k];
            }
            relax_rows_of_warp(col, op, NoPush{}, r0, dd, vv, a);
        }
        __syncwarp();
    }
}

// ================================================================ expansions
// Block-wide compaction helper: every thread offers at most one index; the
// offered indices are gathered in shared memory (order not kept).
__device__ __forceinline__ int block_compact(bool offer, int32_t idx, int32_t *s_list, int *s_n) {
    if (threadIdx.x == 0) *s_n = 0;
    __syncthreads();
    unsigned bal = __ballot_sync(0xffffffffu, offer);
    int base = 0;
    if (lane_id() == 0 && bal) base = atomicAdd(s_n, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (offer) s_list[base + __popc(bal & lanemask_lt())] = idx;
    __syncthreads();
    return *s_n;
}

// Bucketed vertex expansion: high chunks by whole CTAs, mid vertices by warps,
// low vertices by threads with the warp's edges redistributed over its lanes.
// Activity is tested for many items at once (256 chunks per CTA, 32 mid
// vertices per warp) so that inactive items cost one parallel load.
template <class OP, class PUSH>
__device__ __forceinline__ void expand_vertices(const Team &t, const uint32_t *__restrict__ row_off, const int32_t *__restrict__ col,
                                                const int32_t *low, int n_low, const int32_t *mid, int n_mid,
                                                const int2 *high, int n_high, const OP &op, const PUSH &push,
                                                Acc &a) {
    __shared__ int32_t s_list[kBlock];
    __shared__ int32_t s_cval[kBlock];
    __shared__ int s_n;
    const unsigned lane = lane_id();
    // high-degree chunks: dealt to the CTAs round-robin, one CTA per chunk
    const int64_t G = t.size;
    for (int64_t base = t.rank; base < n_high; base += G * kBlock) {
        const int64_t ci = base + (int64_t)threadIdx.x * G;
        bool act = false, rq = false;
        int32_t cval = 0, cv = 0;
        if (ci < n_high) {
            cv = ldcg(&high[ci].x);
            const int32_t cb = ldcg(&high[ci].y);
            act = op.active(cv, cval, rq);
            if (act && (uint32_t)cb == __ldg(row_off + cv)) {
                op.own(cv, cval);
                a.verts++;
            }
        }
        push(rq, cv, a);
        s_cval[threadIdx.x] = cval;
        const int na = block_compact(act, (int32_t)threadIdx.x, s_list, &s_n);
        for (int i = 0; i < na; i++) {
            const int t = s_list[i];
            const int64_t cj = base + (int64_t)t * G;
            const int32_t vtx = ldcg(&high[cj].x);
            const uint32_t e0 = (uint32_t)ldcg(&high[cj].y);
            const uint32_t e1 = min(e0 + (uint32_t)kChunk, __ldg(row_off + vtx + 1));
            const int32_t vv = op.refresh(vtx, s_cval[t]);
            if (threadIdx.x == 0) a.edges += e1 - e0;
            for (uint32_t eb = e0; eb < e1; eb += kBlock * kU) {
                uint32_t e[kU];
                int32_t val[kU];
                bool in[kU];
#pragma unroll
                for (int j = 0; j < kU; j++) {
                    e[j] = eb + j * kBlock + threadIdx.x;
                    in[j] = e[j] < e1;
                    val[j] = vv;
                }
                relax_batch(col, op, push, e, val, in, a);
            }
        }
        __syncthreads();
    }
    const int gw = (int)((t.rank * (unsigned)kBlock + threadIdx.x) >> 5);
    const int nw = (int)(t.size * (unsigned)kWarps);
    // mid-degree vertices: a warp tests 32 at once, then expands the active
    // ones one after the other with all its lanes
    for (int base = gw; base < n_mid; base += nw * 32) {
        const int i = base + (int)lane * nw;
        int32_t u = 0, vv = 0;
        bool act = false, rq = false;
        if (i < n_mid) {
            u = ldcg(mid + i);
            act = op.active(u, vv, rq);
            if (act) op.own(u, vv);
        }
        push(rq, u, a);
        unsigned bal = __ballot_sync(0xffffffffu, act);
        if (lane == 0) a.verts += __popc(bal);
        while (bal) {
            const int l = __ffs(bal) - 1;
            bal &= bal - 1;
            const int32_t uu = __shfl_sync(0xffffffffu, u, l);
            const int32_t uval = op.refresh(uu, __shfl_sync(0xffffffffu, vv, l));
            const uint32_t b = __ldg(row_off + uu), en = __ldg(row_off + uu + 1);
            if (lane == 0) a.edges += en - b;
            for (uint32_t eb = b; eb < en; eb += 32 * kU) {
                uint32_t e[kU];
                int32_t val[kU];
                bool in[kU];
#pragma unroll
                for (int j = 0; j < kU; j++) {
                    e[j] = eb + 32 * j + lane;
                    in[j] = e[j] < en;
                    val[j] = uval;
                }
                relax_batch(col, op, push, e, val, in, a);
            }
        }
    }
    // low-degree vertices: a thread each, edges redistributed over the warp
    for (int base = gw * 32; base < n_low; base += nw * 32) {
        int i = base + (int)lane;
        int32_t vv = 0, u = 0;
        uint32_t rb = 0, d = 0;
        bool rq = false;
        if (i < n_low) {
            u = ldcg(low + i);
            if (op.active(u, vv, rq)) {
                op.own(u, vv);
                rb = __ldg(row_off + u);
                d = __ldg(row_off + u + 1) - rb;
                a.verts++;
            }
        }
        push(rq, u, a);
        relax_rows_of_warp(col, op, push, rb, d, vv, a);
    }
}

// Load-balanced expansion of a vertex worklist to its out-edges (edge-async).
// goff(i) is item i's global edge offset (non-decreasing in i) and T the
// worklist's edge total.  The edge space [0, T) is split evenly over the
// CTAs; each CTA finds the item holding its first edge by binary search,
// stages a window of up to kBlock items' offsets, row starts and values in
// shared memory, and relaxes the window's edges in 1024-edge sub-tiles: each
// thread takes four consecutive edges, finds the first one's owner by binary
// search in the window and walks on from there.
template <class GOFF, class OP, class PUSH>
__device__ __forceinline__ void lb_expand(const Team &t, const uint32_t *__restrict__ row_off, const int32_t *__restrict__ col,
                                          const int32_t *items, int n_items, const GOFF &goff, uint32_t T,
                                          const OP &op, const PUSH &push, Acc &a) {
    __shared__ uint32_t s_goff[kBlock + 1];
    __shared__ uint32_t s_rb[kBlock];
    __shared__ int32_t s_val[kBlock];
    __shared__ int32_t s_item[kBlock];
    __shared__ int s_i0;
    const int G = t.size;
    if (T == 0 || n_items == 0) return;
    const uint64_t lo = (uint64_t)T * t.rank / G, hi = (uint64_t)T * (t.rank + 1) / G;
    if (lo >= hi) return;
    if (threadIdx.x < 32) {
        // item containing edge lo: the last item with goff <= lo, by a
        // 32-ary search of warp 0 (each step probes 32 points at once: about
        // 6 dependent loads instead of 22 for 4 M items).  goff(l) <= lo
        // holds throughout, since the first item's offset is 0.
        const unsigned lane = lane_id();
        int l = 0, r = n_items - 1;
        while (r - l > 31) {
            const int64_t span = (int64_t)(r - l);
            const bool le = goff(l + (int)(span * lane / 32)) <= (uint32_t)lo;
            const int k = __popc(__ballot_sync(0xffffffffu, le)) - 1;   // the true probes are a prefix
            const int nl = l + (int)(span * k / 32);
            r = k == 31 ? r : l + (int)(span * (k + 1) / 32);
            l = nl;
        }
        const bool le = l + (int)lane <= r && goff(l + (int)lane) <= (uint32_t)lo;
        const unsigned b = __ballot_sync(0xffffffffu, le);
        if (lane == 0) s_i0 = l + __popc(b) - 1;
    }
    __syncthreads();
    uint32_t t0 = (uint32_t)lo;
    while (t0 < (uint32_t)hi) {
        const int i0 = s_i0;
        const int cnt = min(kBlock, n_items - i0);
        bool rq = false;
        int32_t u = 0;
        if ((int)threadIdx.x < cnt) {
            int i = i0 + threadIdx.x;
            u = ldcg(items + i);
            s_goff[threadIdx.x] = goff(i);
            s_rb[threadIdx.x] = __ldg(row_off + u);
            int32_t val = 0;
            op.active(u, val, rq);
            s_val[threadIdx.x] = val;
            s_item[threadIdx.x] = u;
        }
        push(rq, u, a);
        if (threadIdx.x == 0) s_goff[cnt] = (i0 + cnt < n_items) ? goff(i0 + cnt) : T;
        __syncthreads();
        const uint32_t wend = min((uint32_t)hi, s_goff[cnt]);   // the window's edges end here
        bool first = true;
        while (t0 < wend) {
            const uint32_t t1 = min(wend, t0 + (uint32_t)(kBlock * kU));
            if (OP::kRefreshWindow && !first) {
                // in place: a source may have improved since the window was
                // staged; relax its remaining edges with its latest value
                // (SSSP: 280 M -> 207 M edges relaxed on R-MAT 22)
                __syncthreads();
                if ((int)threadIdx.x < cnt) s_val[threadIdx.x] = op.refresh(s_item[threadIdx.x], s_val[threadIdx.x]);
                __syncthreads();
            }
            first = false;
            const uint32_t x0 = t0 + kU * threadIdx.x;
            uint32_t e[kU];
            int32_t val[kU];
            bool in[kU];
            int l = 0;
            if (x0 < t1) {
                int r = cnt - 1;
                while (l < r) {
                    int mdl = (l + r + 1) >> 1;
                    if (s_goff[mdl] <= x0) l = mdl; else r = mdl - 1;
                }
            }
#pragma unroll
            for (int j = 0; j < kU; j++) {
                const uint32_t x = x0 + j;
                in[j] = x < t1;
                e[j] = 0;
                val[j] = 0;
                if (in[j]) {
                    while (l + 1 < cnt && s_goff[l + 1] <= x) l++;   // owners are consecutive
                    e[j] = s_rb[l] + (x - s_goff[l]);
                    val[j] = s_val[l];
                    a.edges++;
                }
            }
            relax_batch(col, op, push, e, val, in, a);
            t0 = t1;
        }
        if (threadIdx.x == 0) {
            // the next window starts with the item holding edge t0
            int l = 0, r = cnt;   // s_goff[cnt] may equal t0 (then item i0 + cnt)
            while (l < r) {
                int mdl = (l + r + 1) >> 1;
                if (s_goff[mdl] <= t0) l = mdl; else r = mdl - 1;
            }
            s_i0 = i0 + l;
        }
        __syncthreads();
    }
}

// ================================================================ pull rounds
// The in-neighbour iterator (innbrs): a pull round visits every vertex with
// in-edges over the transposed CSR, bucketed by in-degree like the push side
// (low: a warp's 32 vertices with their in-edges spread over its lanes and
// combined by shared-memory atomics; mid: a warp per vertex; high: a CTA per
// 2048-edge chunk).  An op reduces its in-edges' candidates by minimum:
//   skip(v)          -- nothing to pull for v (BFS: already visited)
//   weight(e)        -- in-edge e's weight (loaded with the in-neighbour id)
//   cand(u, wv, a)   -- the candidate of an in-edge from u of weight wv (kInf: none)
//   finish(v, m, a)  -- the only writer of v applies the minimum m
//   finish_part(v, m, first, a) -- one of several chunks of v applies its m
//   kEarly           -- a candidate of 0 ends v's scan (BFS: a parent found)

// SSSP / CC pull round r: next[v] = min(cur[v], min over in-edges (u, w) of
// cur[u] + w) -- Alg. 1's MIN gathered at the target, so no atomics except
// where a hub's chunks meet.  cur is the previous round's and is read through
// L1.  next may hold an older (larger) value: a single writer overwrites it,
// and the chunk holding a hub's first in-edge includes cur[v] in its MIN.
template <int ALGO>
struct PullMinOp {
    const int32_t *__restrict__ w;   // in-edge weights (SSSP)
    const int32_t *cur;
    int32_t *next;
    int32_t *snext;
    int32_t r;
    static constexpr bool kEarly = false;

    static constexpr bool kWeights = (ALGO == kSSSP);

    __device__ __forceinline__ bool skip(int32_t) const { return false; }
    __device__ __forceinline__ int32_t weight(uint32_t e) const { return kWeights ? ld_edge(w + e) : 0; }
    __device__ __forceinline__ int32_t cand(int32_t u, int32_t wv, Acc &a) const {
        const int32_t x = ldca(cur + u);
        if (ALGO != kSSSP || x == kInf) return x;
        const uint32_t y = (uint32_t)x + (uint32_t)wv;
        if (y >= (uint32_t)kInf) {
            a.overflow = 1;
            return kInf;
        }
        return (int32_t)y;
    }
    __device__ __forceinline__ void finish(int32_t v, int32_t m, Acc &a) const {
        const int32_t c = ldca(cur + v);
        stcg(next + v, min(c, m));
        if (m < c) {
            stcg(snext + v, r + 1);
            a.changed++;
            a.updates++;
        }
    }
    __device__ __forceinline__ void finish_part(int32_t v, int32_t m, bool first, Acc &a) const {
        const int32_t c = ldca(cur + v);
        if (first) red_min(next + v, min(c, m));
        else if (m < c) red_min(next + v, m);
        if (m < c) {
            stcg(snext + v, r + 1);
            a.changed++;
            a.updates++;
        }
    }
};

// BFS bottom-up step (level lev): an unvisited vertex joins level lev+1 when
// some in-neighbour is at level lev; its scan stops at the first one.
struct BfsPullOp {
    int32_t *L;
    int32_t lev;
    uint32_t *vis;     // kept in step with L for the push rounds' probes
    static constexpr bool kEarly = true;
    static constexpr bool kWeights = false;

    __device__ __forceinline__ bool skip(int32_t v) const { return ldcg(L + v) != kInf; }
    __device__ __forceinline__ int32_t weight(uint32_t) const { return 0; }
    // an in-neighbour's level was set in an earlier round (L1 is safe)
    __device__ __forceinline__ int32_t cand(int32_t u, int32_t, Acc &) const { return ldca(L + u) == lev ? 0 : kInf; }
    __device__ __forceinline__ void finish(int32_t v, int32_t m, Acc &a) const {
        if (m == 0) {
            stcg(L + v, lev + 1);
            red_or(vis + (v >> 5), 1u << (v & 31));
            a.changed++;
            a.updates++;
        }
    }
    __device__ __forceinline__ void finish_part(int32_t v, int32_t m, bool, Acc &a) const {
        if (m == 0 && atomicCAS(L + v, kInf, lev + 1) == kInf) {
            red_or(vis + (v >> 5), 1u << (v & 31));
            a.changed++;
            a.updates++;
        }
    }
};

template <class OP>
__device__ __forceinline__ void pull_vertices(const Team &t, const View &tv, const OP &op, Acc &a) {
    __shared__ int32_t s_min[kWarps][32];
    __shared__ int s_skip;
    const unsigned lane = lane_id();
    const int wid = threadIdx.x >> 5;
    const int64_t gw = (int64_t)t.rank * kWarps + wid, nw = (int64_t)t.size * kWarps;

    // high in-degree: a CTA per 2048-edge chunk
    for (int64_t ci = t.rank; ci < tv.n_high_chunks; ci += t.size) {
        const int2 hc = __ldg(tv.high + ci);
        const int32_t v = hc.x;
        if (threadIdx.x == 0) s_skip = op.skip(v);
        __syncthreads();
        const bool skip = s_skip;
        __syncthreads();
        if (skip) continue;
        const uint32_t rb = __ldg(tv.row_off + v), e0 = (uint32_t)hc.y;
        const uint32_t e1 = min(__ldg(tv.row_off + v + 1), e0 + (uint32_t)kChunk);
        int32_t m = kInf;
        for (uint32_t eb = e0 + threadIdx.x; eb < e1; eb += kBlock * kU) {
            int32_t u[kU], wv[kU];
#pragma unroll
            for (int j = 0; j < kU; j++) {
                const bool in = eb + j * kBlock < e1;
                u[j] = in ? ld_edge(tv.col + eb + j * kBlock) : -1;
                wv[j] = in ? op.weight(eb + j * kBlock) : 0;
            }
#pragma unroll
            for (int j = 0; j < kU; j++)
                if (u[j] >= 0) m = min(m, op.cand(u[j], wv[j], a));
        }
        if (threadIdx.x == 0) a.pulled += e1 - e0;
        m = block_min(m);
        if (threadIdx.x == 0) op.finish_part(v, m, e0 == rb, a);
    }

    // mid in-degree: a warp per vertex
    for (int64_t i = gw; i < tv.n_mid; i += nw) {
        const int32_t v = __ldg(tv.mid + i);
        if (__shfl_sync(0xffffffffu, lane == 0 ? (int)op.skip(v) : 0, 0)) continue;
        const uint32_t rb = __ldg(tv.row_off + v), re = __ldg(tv.row_off + v + 1);
        int32_t m = kInf;
        uint32_t seen = 0;
        for (uint32_t eb = rb + lane; eb < re; eb += 32 * kU) {
            int32_t u[kU], wv[kU];
#pragma unroll
            for (int j = 0; j < kU; j++) {
                const bool in = eb + 32 * j < re;
                u[j] = in ? ld_edge(tv.col + eb + 32 * j) : -1;
                wv[j] = in ? op.weight(eb + 32 * j) : 0;
            }
#pragma unroll
            for (int j = 0; j < kU; j++)
                if (u[j] >= 0) m = min(m, op.cand(u[j], wv[j], a));
            seen += 32 * kU;
            if (OP::kEarly && __any_sync(0xffffffffu, m == 0)) break;
        }
        if (lane == 0) a.pulled += min(seen, re - rb);
        m = warp_min(m);
        if (lane == 0) op.finish(v, m, a);
    }

    // low in-degree: a warp's 32 vertices, their in-edges spread over the lanes
    const int64_t nl = tv.n_low;
    for (int64_t i0 = gw * 32; i0 < nl; i0 += nw * 32) {
        const int64_t i = i0 + lane;
        int32_t v = -1;
        uint32_t rb = 0, d = 0;
        if (i < nl) {
            v = __ldg(tv.low + i);
            if (!op.skip(v)) {
                rb = __ldg(tv.row_off + v);
                d = __ldg(tv.row_off + v + 1) - rb;
            }
        }
        s_min[wid][lane] = kInf;
        __syncwarp();
        const uint32_t incl = warp_inclusive_scan(d);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - d;
        if (lane == 0) a.pulled += total;
        for (uint32_t k0 = 0; k0 < total; k0 += 32 * kU) {
            int32_t u[kU], wv[kU], own[kU];
            uint32_t e[kU];
#pragma unroll
            for (int j = 0; j < kU; j++) {
                const uint32_t k = k0 + 32 * j + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t pv = __shfl_sync(0xffffffffu, incl, owner + step - 1);
                    if (pv <= k) owner += step;
                }
                const uint32_t ob = __shfl_sync(0xffffffffu, rb, owner);
                const uint32_t oe = __shfl_sync(0xffffffffu, excl, owner);
                own[j] = owner;
                e[j] = ob + (k - oe);
                u[j] = k < total ? ld_edge(tv.col + e[j]) : -1;
                wv[j] = k < total ? op.weight(e[j]) : 0;
            }
#pragma unroll
            for (int j = 0; j < kU; j++)
                if (u[j] >= 0) {
                    const int32_t cnd = op.cand(u[j], wv[j], a);
                    if (cnd != kInf) atomicMin(&s_min[wid][own[j]], cnd);
                }
        }
        __syncwarp();
        if (d > 0) op.finish(v, s_min[wid][lane], a);
        __syncwarp();
    }
}

// ================================================================ sparse edge-sync rounds
// A round of the synchronous edge mode normally streams every edge.  When the
// previous round changed few vertices the round is "sparse": a flag pass
// first stamps every 128-edge warp tile that holds an out-edge of an active
// vertex, and only those tiles are streamed.  The choice is made identically
// by every CTA.

// Flag pass: a warp tests 128 consecutive vertices per step (128-bit loads of
// the activity word); each active vertex of the low and mid classes stamps
// the warp tiles of its edge range [row_off[v], row_off[v+1]) with `round`.
// The high class (>= kMidMax out-edges) is flagged from its 2048-edge chunk
// list instead, one warp per chunk over every warp of the team: graphs
// renumbered by in-degree class hold their hubs in the first few 128-vertex
// steps (on R-MAT 22 the first step alone spans 23 K of the 524 K tiles),
// which the warps owning those steps would otherwise flag alone while the
// rest of the grid waits at the barrier.
__device__ __forceinline__ void flag_edge_tiles(const Team &t, const View &g, const int32_t *actw, int32_t act_val,
                                                int32_t n, int32_t *eflag, int32_t round, Acc &a) {
    const uint32_t *__restrict__ row_off = g.row_off;
    const unsigned lane = lane_id();
    const int64_t gw = (t.rank * (int64_t)kBlock + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)t.size * kWarps;
    for (int64_t v0 = gw * 128; v0 < n; v0 += nw * 128) {
        const int64_t vb = v0 + 4 * lane;
        bool act[4] = {false, false, false, false};
        if (vb + 3 < n) {
            const int4 w4 = __ldcg(reinterpret_cast<const int4 *>(actw + vb));
            act[0] = w4.x == act_val; act[1] = w4.y == act_val; act[2] = w4.z == act_val; act[3] = w4.w == act_val;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) act[j] = vb + j < n && ldcg(actw + vb + j) == act_val;
        }
        if (lane == 0) a.scanned += (uint64_t)min((int64_t)128, (int64_t)n - v0);
        uint32_t big_t0 = 0, big_t1 = 0;
        bool big = false;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (!act[j]) continue;
            const uint32_t rb = __ldg(row_off + vb + j), re = __ldg(row_off + vb + j + 1);
            if (re <= rb || re - rb >= (uint32_t)kMidMax) continue;   // none, or high (chunk list)
            const uint32_t t0 = rb / kWTile, t1 = (re - 1) / kWTile;
            if (t1 - t0 < 8) {
                for (uint32_t k = t0; k <= t1; k++) stcg(eflag + k, round);
            } else if (!big) {
                big = true;
                big_t0 = t0;
                big_t1 = t1;
            } else {   // a second long range of the same lane (rare): alone
                for (uint32_t k = t0; k <= t1; k++) stcg(eflag + k, round);
            }
        }
        for (unsigned m = __ballot_sync(0xffffffffu, big); m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            const uint32_t t0 = __shfl_sync(0xffffffffu, big_t0, src), t1 = __shfl_sync(0xffffffffu, big_t1, src);
            for (uint32_t k = t0 + lane; k <= t1; k += 32) stcg(eflag + k, round);
        }
    }
    // high class: a chunk of at most kChunk edges spans at most
    // kChunk / kWTile + 1 = 17 tiles, one per lane
    static_assert(kChunk / kWTile + 1 <= 32, "a high chunk's tiles must fit one warp");
    for (int64_t i = gw; i < g.n_high_chunks; i += nw) {
        const int32_t u = __ldg(&g.high[i].x);
        if (ldcg(actw + u) != act_val) continue;
        const uint32_t e0 = (uint32_t)__ldg(&g.high[i].y);
        const uint32_t e1 = e0 + min((uint32_t)kChunk, __ldg(row_off + u + 1) - e0);   // e0 < row_off[u+1]
        const uint32_t k = e0 / kWTile + lane;
        if (k <= (e1 - 1) / kWTile) stcg(eflag + k, round);
    }
}

// ================================================================ staged edge stream
// The edges of a synchronous edge round are streamed through shared memory,
// each warp on its own: a 128-edge warp tile of (src, dst[, w]) arrives by
// bulk copy (TMA) into one of the warp's kWStages buffers, completed on that
// buffer's mbarrier, while the warp relaxes an earlier tile.  Each lane
// copies its four edges into registers, forms their candidates (the
// sources' values are read through L1: consecutive edges share sources), the
// warp syncs and its buffer is refilled at once, then the lane probes the
// targets and applies the updates.  No CTA-wide barrier is involved, so a
// lane waiting on a contended target line holds up only its own warp.  The
// copies carry an L2 evict-first hint so that the streamed edges do not push
// the value and stamp arrays out of L2.  Two buffers per warp keep the
// CTA's shared memory at 25 KB: on skewed graphs the targets' hot lines are
// served from L1, which shares its capacity with shared memory (a third
// buffer halved the throughput of an all-active R-MAT round).
#ifndef FG_EDGE_STAGES
#define FG_EDGE_STAGES 2
#endif
constexpr int kWStages = FG_EDGE_STAGES;   // buffers per warp; a warp tile is kWTile = 128 edges (4 per lane)

template <bool W>
struct __align__(16) WarpStage {
    int32_t src[kWTile + 4];       // src[e0-4 .. e0+cnt): src[3] is the edge before the tile
    int32_t col[kWTile];
    int32_t w[W ? kWTile : 4];
};

template <bool W>
struct __align__(16) WarpRing {
    WarpStage<W> st[kWStages];
    uint64_t full[kWStages];
};

template <bool W>
struct EdgeRings {
    WarpRing<W> warp[kWarps];
    uint64_t pol;                  // L2 policy of the copies
};

template <bool W>
__device__ __forceinline__ void rings_init(EdgeRings<W> &R) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < kWarps; i++)
            for (int j = 0; j < kWStages; j++) mbar_init(&R.warp[i].full[j], 1);
        R.pol = l2_evict_first_policy();
        mbar_init_fence();
    }
    __syncthreads();
}

// Lane 0: start the copies of warp tile `tile` into buffer `slot`.  The
// copied prefix is a multiple of 4 edges (16 bytes); the last tile's ragged
// tail (at most 3 edges) is read from global memory by its lane.  A tile
// past the end copies nothing (the arrival alone completes the phase).
template <bool W>
__device__ __forceinline__ void wring_issue(WarpRing<W> &R, uint64_t pol, int slot, int64_t tile, const View &g) {
    const int64_t e0 = tile * kWTile;
    const int64_t cnt = max((int64_t)0, min((int64_t)kWTile, g.m - e0));
    const uint32_t staged = (uint32_t)(cnt & ~3ll);
    const uint32_t lead = (e0 > 0 && cnt > 0) ? 4u : 0u;
    const uint32_t bytes = 4u * (staged + lead) + 4u * staged * (W ? 2u : 1u);
    WarpStage<W> &S = R.st[slot];
    mbar_expect_tx(&R.full[slot], bytes);
    if (staged + lead) bulk_g2s(S.src + (4 - lead), g.src + e0 - lead, 4u * (staged + lead), &R.full[slot], pol);
    if (staged) {
        bulk_g2s(S.col, g.col + e0, 4u * staged, &R.full[slot], pol);
        if (W) bulk_g2s(S.w, g.w + e0, 4u * staged, &R.full[slot], pol);
    }
}

// Bounded wait for a buffer's copies: false after timeout_ns.
__device__ __forceinline__ bool ring_wait(uint64_t *bar, uint32_t parity, unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// A lane's four edges of a tile after candidate formation: the targets, the
// candidates and which of them to apply.
struct Quad {
    int32_t vs[4], c[4];
    bool ok[4];
};

// From the warp tile in buffer S (tile starting at e0): the lane's four
// edges, their sources' activity and values, the carry of each active
// source's value into the other buffer at the source's first edge (the edge
// before it has another source, so the synchronous edge mode needs no
// separate pass over the vertices), and the candidates.  Nothing of the
// buffer is needed after.
template <bool W, class OP>
__device__ __forceinline__ void quad_form(const WarpStage<W> &S, int64_t e0, const View &g, const OP &op, Quad &q,
                                          Acc &a) {
    const int cnt = (int)max((int64_t)0, min((int64_t)kWTile, g.m - e0));
    const int staged = cnt & ~3;
    const int i4 = 4 * (int)lane_id();
    int32_t us[4] = {-1, -1, -1, -1}, ws[4] = {0, 0, 0, 0};
    int nv = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        q.vs[j] = 0;
        q.c[j] = 0;
        q.ok[j] = false;
    }
    if (i4 >= cnt) return;
    if (i4 < staged) {
        const int4 s4 = *reinterpret_cast<const int4 *>(S.src + 4 + i4);
        const int4 c4 = *reinterpret_cast<const int4 *>(S.col + i4);
        us[0] = s4.x; us[1] = s4.y; us[2] = s4.z; us[3] = s4.w;
        q.vs[0] = c4.x; q.vs[1] = c4.y; q.vs[2] = c4.z; q.vs[3] = c4.w;
        if (W) {
            const int4 w4 = *reinterpret_cast<const int4 *>(S.w + i4);
            ws[0] = w4.x; ws[1] = w4.y; ws[2] = w4.z; ws[3] = w4.w;
        }
        nv = 4;
    } else {   // ragged tail of the last tile
        nv = cnt - i4;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < nv) {
                us[j] = __ldg(g.src + e0 + i4 + j);
                q.vs[j] = __ldg(g.col + e0 + i4 + j);
                if (W) ws[j] = __ldg(g.w + e0 + i4 + j);
            }
    }
    const int32_t before = (e0 + i4 == 0) ? -1 : S.src[3 + i4];
    bool fresh[4];
    int32_t st[4], vl[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        fresh[j] = j < nv && (j == 0 || us[j] != us[j - 1]);
        st[j] = 0;
        vl[j] = 0;
        if (fresh[j]) op.load_act(us[j], st[j], vl[j]);
    }
    bool act[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (j >= nv) {
            act[j] = false;
        } else if (fresh[j]) {
            act[j] = op.is_act(st[j], vl[j]);
            if (act[j] && (j > 0 || us[0] != before)) {
                op.own(us[j], vl[j]);
                a.verts++;
            }
        } else {
            act[j] = act[j - 1];
            vl[j] = vl[j - 1];
        }
        q.ok[j] = act[j] && op.cand_w(vl[j], ws[j], q.c[j], a);
        a.edges += act[j];
    }
}

// Apply a quad: all probes of the targets, then the updates.
template <class OP>
__device__ __forceinline__ void quad_apply(const OP &op, const Quad &q, Acc &a) {
    int32_t pv[4];
#pragma unroll
    for (int j = 0; j < 4; j++) pv[j] = q.ok[j] ? op.probe(q.vs[j]) : 0;
    if constexpr (OP::kNextProbe) {
        int32_t nv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) nv[j] = (q.ok[j] && q.c[j] < pv[j]) ? op.probe_next(q.vs[j]) : 0;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (q.ok[j]) op.commit2(q.vs[j], q.c[j], pv[j], nv[j], a);
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (q.ok[j]) op.commit(q.vs[j], q.c[j], pv[j], a);
    }
}

// A warp streams `count` warp tiles, the k-th being tile_of(k), through its
// ring and relaxes them.  All lanes call it with the same arguments; `used`
// counts the tiles that went through the warp's ring so far (it fixes each
// buffer's mbarrier phase) and is kept in a register by every lane.  Returns
// false (with kStTimeout set) if a copy did not complete within timeout_ns;
// the warp then waits, again bounded, for the copies it still has in flight.
template <bool W, class TILE_OF, class OP>
__device__ __forceinline__ bool warp_stream(WarpRing<W> &R, uint64_t pol, uint32_t &used, int count,
                                            const TILE_OF &tile_of, const View &g, const OP &op, Acc &a, Ctrl *c,
                                            unsigned long long timeout_ns) {
    if (count <= 0) return true;
    const bool leader = lane_id() == 0;
    const uint32_t base = used;
    if (leader)
        for (int k = 0; k < min(count, kWStages); k++) wring_issue(R, pol, (int)((base + k) % kWStages), tile_of(k), g);
    int k = 0;
    bool ok = true;
    for (; k < count; k++) {
        const uint32_t gk = base + (uint32_t)k;
        const int slot = (int)(gk % kWStages);
        Quad q;
        const bool mine = ring_wait(&R.full[slot], (gk / kWStages) & 1u, timeout_ns);
        if (mine) quad_form(R.st[slot], tile_of(k) * kWTile, g, op, q, a);
        // past this point every lane holds its part of tile k in registers:
        // the buffer takes tile k + kWStages
        ok = __all_sync(0xffffffffu, mine);
        __syncwarp();
        if (!ok) break;
        if (leader && k + kWStages < count) wring_issue(R, pol, slot, tile_of(k + kWStages), g);
        quad_apply(op, q, a);
    }
    const int issued = min(count, kWStages + k);
    if (!ok && leader) {
        // tiles k .. issued-1 may still be in flight
        for (int j = k; j < issued; j++) {
            const uint32_t gj = base + (uint32_t)j;
            ring_wait(&R.full[gj % kWStages], (gj / kWStages) & 1u, timeout_ns);
        }
        atomicOr(&c->status, kStTimeout);
    }
    __syncwarp();
    used = base + (uint32_t)(ok ? count : issued);
    return ok;
}

// The CTA's rings; only kernels that stream edge tiles instantiate them.
template <bool W>
__device__ __forceinline__ EdgeRings<W> &edge_rings() {
    __shared__ EdgeRings<W> rings;
    return rings;
}

// Dense synchronous edge round: warp tiles dealt round-robin to the warps of
// the team.
template <bool W, class OP>
__device__ __forceinline__ bool stream_all_edges(const Team &t, uint32_t &used, const View &g, const OP &op, Acc &a,
                                                 Ctrl *c, unsigned long long timeout_ns) {
    EdgeRings<W> &R = edge_rings<W>();
    const int64_t ntiles = (g.m + kWTile - 1) / kWTile;
    const int64_t gw = (int64_t)t.rank * kWarps + (threadIdx.x >> 5), nw = (int64_t)t.size * kWarps;
    const int count = ntiles > gw ? (int)((ntiles - 1 - gw) / nw + 1) : 0;
    if (t.rank == 0 && threadIdx.x == 0) a.scanned += (uint64_t)g.m;
    const bool ok = warp_stream(R.warp[threadIdx.x >> 5], R.pol, used, count,
                                [&](int k) { return gw + (int64_t)k * nw; }, g, op, a, c, timeout_ns);
    return __syncthreads_and(ok);
}

// Sparse synchronous edge round: each warp tests its share of the warp tiles
// (tiles gw, gw + nw, ...) 128 at a time, lists the flagged ones in shared
// memory and streams them.
template <bool W, class OP>
__device__ __forceinline__ bool stream_flagged_edges(const Team &t, uint32_t &used, const View &g,
                                                     const int32_t *eflag, int32_t round, const OP &op, Acc &a,
                                                     Ctrl *c, unsigned long long timeout_ns) {
    __shared__ int32_t s_wl[kWarps][128];
    EdgeRings<W> &R = edge_rings<W>();
    const int wid = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t ntiles = (g.m + kWTile - 1) / kWTile;
    const int64_t gw = (int64_t)t.rank * kWarps + wid, nw = (int64_t)t.size * kWarps;
    bool ok = true;
    for (int64_t k0 = 0; gw + k0 * nw < ntiles && ok; k0 += 128) {
        int na = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t tile = gw + (k0 + 32 * j + lane) * nw;
            const bool f = tile < ntiles && ldcg(eflag + tile) == round;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) s_wl[wid][na + __popc(bal & lanemask_lt())] = (int32_t)tile;
            na += __popc(bal);
        }
        __syncwarp();
        if (lane == 0)
            for (int i = 0; i < na; i++) {
                const int64_t e0 = (int64_t)s_wl[wid][i] * kWTile;
                a.scanned += (uint64_t)min((int64_t)kWTile, g.m - e0);
            }
        ok = warp_stream(R.warp[wid], R.pol, used, na, [&](int i) { return (int64_t)s_wl[wid][i]; }, g, op, a, c,
                         timeout_ns);
    }
    return __syncthreads_and(ok);
}

// ================================================================ dense edge-async generations
// When a generation's worklist covers a large share of all edges, the
// edge-async mode streams the whole edge list (source-sorted COO) instead of
// expanding the worklist: the topology-driven form of the edge variant for
// dense generations, the data-driven form for sparse ones (Sec. 3.3 names
// both).  A source is in generation g's worklist iff its stamp is g: it was
// stamped g when it was queued during g - 1, and during g a stamp only moves
// on to g + 1 (the vertex is then in g + 1's worklist and is expanded there),
// so an L1 copy of a stamp, fresh since the barrier, can only err towards
// skipping a source that g + 1 expands anyway.  Each lane reads four
// consecutive edges with 16-byte streaming loads.
#ifndef FG_EA_DENSE_PCT
#define FG_EA_DENSE_PCT 25
#endif
// worklist edges, % of m, from which a generation streams.  BFS only from
// half: its frontier relaxes each edge once at most, and a quarter cost 10 %
// on R-MAT 22.
template <int ALGO>
__host__ __device__ constexpr int ea_dense_pct() { return ALGO == kBFS ? 2 * FG_EA_DENSE_PCT : FG_EA_DENSE_PCT; }

template <int ALGO>
struct AsyncStreamOp : AsyncOp<ALGO> {
    __device__ __forceinline__ void load_act(int32_t u, int32_t &st, int32_t &vl) const {
        st = ldca(this->stamp + u);
        vl = ldcg(this->D + u);
    }
    // SSSP also expands the sources lowered during this generation (stamp
    // g + 1): relaxing with a current distance is always valid, it carries
    // the new distance on at once, and a source of the worklist that was
    // lowered after its first edges keeps its remaining edges in this
    // generation.  CC keeps to the worklist: with the pointer jumps below,
    // the wider test ran slower on R-MAT 22 and the 4096^2 grid.
    static constexpr bool kAlsoLowered = (ALGO == kSSSP);
    __device__ __forceinline__ bool is_act(int32_t st, int32_t vl) const {
        return (kAlsoLowered ? st >= this->gen : st == this->gen) && vl != kInf;
    }
    // CC: the worklist expansion's pointer jumping (active()); the others
    // use the value as read
    static constexpr bool kJumps = (ALGO == kCC);
    __device__ __forceinline__ int32_t jump(int32_t u, int32_t vl, bool &rq) const {
        if (kJumps) {
            int32_t v = vl;
            this->active(u, v, rq);
            return v;
        }
        return vl;
    }
    __device__ __forceinline__ bool cand_w(int32_t vl, int32_t w, int32_t &c, Acc &a) const {
        if (ALGO == kSSSP) {
            const uint32_t x = (uint32_t)vl + (uint32_t)w;
            if (x >= (uint32_t)kInf) {
                a.overflow = 1;
                return false;
            }
            c = (int32_t)x;
        } else {
            c = vl;
        }
        return true;
    }
};

// BFS: the sources of generation g are the vertices at level g (levels are
// claimed once, by CAS, with the next generation's number)
struct BfsStreamOp : BfsAsyncOp {
    __device__ __forceinline__ void load_act(int32_t u, int32_t &st, int32_t &vl) const {
        st = ldca(this->L + u);
        vl = this->gen;
    }
    __device__ __forceinline__ bool is_act(int32_t st, int32_t) const { return st == this->gen; }
    static constexpr bool kJumps = false;
    __device__ __forceinline__ int32_t jump(int32_t, int32_t vl, bool &) const { return vl; }
    __device__ __forceinline__ bool cand_w(int32_t, int32_t, int32_t &c, Acc &) const {
        c = this->gen + 1;
        return true;
    }
};

// A lane's four consecutive edges of a warp tile, as loaded.
struct RawQuad {
    int32_t us[4], vs[4], ws[4];
    int nv;
};

template <bool W>
__device__ __forceinline__ void raw_load(const View &g, int64_t e0, RawQuad &r) {
    const int64_t e = e0 + 4 * (int64_t)lane_id();
    r.nv = (int)max((int64_t)0, min((int64_t)4, g.m - e));
#pragma unroll
    for (int j = 0; j < 4; j++) r.us[j] = r.vs[j] = r.ws[j] = 0;
    if (r.nv == 4) {   // e is a multiple of 4 and the arrays are 16-byte aligned
        const int4 s4 = __ldcs(reinterpret_cast<const int4 *>(g.src + e));
        const int4 c4 = __ldcs(reinterpret_cast<const int4 *>(g.col + e));
        r.us[0] = s4.x; r.us[1] = s4.y; r.us[2] = s4.z; r.us[3] = s4.w;
        r.vs[0] = c4.x; r.vs[1] = c4.y; r.vs[2] = c4.z; r.vs[3] = c4.w;
        if (W) {
            const int4 w4 = __ldcs(reinterpret_cast<const int4 *>(g.w + e));
            r.ws[0] = w4.x; r.ws[1] = w4.y; r.ws[2] = w4.z; r.ws[3] = w4.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < r.nv) {
                r.us[j] = __ldg(g.src + e + j);
                r.vs[j] = __ldg(g.col + e + j);
                if (W) r.ws[j] = __ldg(g.w + e + j);
            }
    }
}

// Dense edge-async generation: warp tiles dealt round-robin to the team's
// warps; targets lowered are queued for the next generation by `push`.  CC
// first shortens each active source's label by pointer jumping, as the
// worklist expansion does, and queues the source again if that lowered it;
// this happens once per source, by the lane holding its first edge (the
// edge before it has another source), and the lanes holding its other edges
// use the label as read.
// Measured and rejected: loading the next tile ahead of the current tile's
// probes (it spilled registers at the worklist kernels' budget and ran 20 %
// slower), and a contiguous range of tiles per warp instead of the
// round-robin deal (the active tiles of skewed graphs cluster; SSSP on
// R-MAT 22 ran 20 % slower, CC on the grid 2x).
template <bool W, class OP, class PUSH>
__device__ __forceinline__ void stream_edges_async(const Team &t, const View &g, const OP &op, const PUSH &push,
                                                   Acc &a) {
    const int64_t ntiles = (g.m + kWTile - 1) / kWTile;
    const int64_t gw = (int64_t)t.rank * kWarps + (threadIdx.x >> 5), nw = (int64_t)t.size * kWarps;
    if (t.rank == 0 && threadIdx.x == 0) a.scanned += (uint64_t)g.m;
    for (int64_t tile = gw; tile < ntiles; tile += nw) {   // warp-uniform
        RawQuad r;
        raw_load<W>(g, tile * kWTile, r);
        int32_t before = 0;   // source of the edge before the lane's first
        if constexpr (OP::kJumps) {
            before = __shfl_up_sync(0xffffffffu, r.us[3], 1);
            if (lane_id() == 0) before = tile > 0 ? __ldg(g.src + tile * kWTile - 1) : -1;
        }
        Quad q;
        bool fresh[4], act[4], rq[4];
        int32_t st[4], vl[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            fresh[j] = j < r.nv && (j == 0 || r.us[j] != r.us[j - 1]);
            st[j] = 0;
            vl[j] = 0;
            rq[j] = false;
            if (fresh[j]) op.load_act(r.us[j], st[j], vl[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (j >= r.nv) {
                act[j] = false;
            } else if (fresh[j]) {
                act[j] = op.is_act(st[j], vl[j]);
                if (OP::kJumps && act[j] && (j > 0 || r.us[0] != before)) vl[j] = op.jump(r.us[j], vl[j], rq[j]);
            } else {
                act[j] = act[j - 1];
                vl[j] = vl[j - 1];
            }
            q.vs[j] = r.vs[j];
            q.c[j] = 0;
            q.ok[j] = act[j] && op.cand_w(vl[j], r.ws[j], q.c[j], a);
            a.edges += act[j];
        }
        if constexpr (OP::kJumps) {
#pragma unroll
            for (int j = 0; j < 4; j++) push(rq[j], r.us[j], a);
        }
        int32_t pv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) pv[j] = q.ok[j] ? op.probe(q.vs[j]) : 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const bool rqv = q.ok[j] && op.commit(q.vs[j], q.c[j], pv[j], a);
            push(rqv, q.vs[j], a);
        }
    }
}

// ================================================================ the kernel
// Resident CTAs per SM the register budget is sized for.  The vertex-sync,
// pull and worklist kernels gain from more warps in flight (their gathers are
// latency-bound: 6 CTAs at 40 registers beat 4 at 64 by 10-30 % on R-MAT 22
// despite a few spilled registers); the edge-sync kernels keep their tile
// state in 64 registers (four CTAs; five at 48 registers spilled and ran 40 %
// slower).
#ifndef FG_SYNC_MIN_BLOCKS
#define FG_SYNC_MIN_BLOCKS 6
#endif
#ifndef FG_ASYNC_MIN_BLOCKS
#define FG_ASYNC_MIN_BLOCKS 6
#endif
#ifndef FG_PULL_SHIFT_BFS
#define FG_PULL_SHIFT_BFS 2
#endif
#ifndef FG_PULL_SHIFT_CC
#define FG_PULL_SHIFT_CC 4
#endif
#ifndef FG_PULL_SHIFT_SSSP
#define FG_PULL_SHIFT_SSSP 0
#endif
// sync modes: the running-minimum filter is used in CC's all-active first
// round and in a round whose previous round changed more than
// n / 2^FG_NEXT_PROBE_SHIFT vertices (R-MAT 22: CC 3.1 -> 2.0 ms; SSSP's
// rounds gained nothing measurable from it)
#ifndef FG_NEXT_PROBE_SHIFT
#define FG_NEXT_PROBE_SHIFT 0
#endif
// The edge-sync rounds use the filter from the first round with a few dozen
// changes on: a streamed edge tile's commits have no warp-level order, and
// the running minimum drops most repeated MINs and stamp writes on hot
// targets (R-MAT 22 SSSP edge-sync 2.83 -> 2.71 ms; vertex-sync, whose
// expansion issues the extra dependent load on its critical path, lost 2 %).
#ifndef FG_NEXT_PROBE_SHIFT_EDGE
#define FG_NEXT_PROBE_SHIFT_EDGE 16
#endif
// vertex-sync: also in a round after one that changed more than
// FG_GROW_FILTER times as many vertices as the round before it (0: never):
// R-MAT 22 SSSP vertex-sync 2.69 -> 2.58 ms, any factor from 2 to 8; pull
// rounds lost 6 % with it and keep the dense-round rule alone

#ifndef FG_GROW_FILTER
#define FG_GROW_FILTER 4
#endif
#ifndef FG_SPARSE_SHIFT
#define FG_SPARSE_SHIFT 0
#endif
// the bucketed mode runs many generations with small worklists: fewer CTAs
// pay less per barrier (4 CTAs: 10.6 ms on the 4096^2 grid, 6: 11.9 ms)
#ifndef FG_BUCKET_MIN_BLOCKS
#define FG_BUCKET_MIN_BLOCKS 4
#endif
#ifndef FG_PULL_MIN_BLOCKS
#define FG_PULL_MIN_BLOCKS 6
#endif
#ifndef FG_EDGE_SYNC_MIN_BLOCKS
#define FG_EDGE_SYNC_MIN_BLOCKS 4
#endif
// the multi-source sweep keeps two 8-value rows per edge in flight (64 registers)
#ifndef FG_MULTI_MIN_BLOCKS
#define FG_MULTI_MIN_BLOCKS 4
#endif
template <int MODE>
constexpr int min_blocks() {
    return MODE == kVertexSync ? FG_SYNC_MIN_BLOCKS
         : MODE == kEdgeSync   ? FG_EDGE_SYNC_MIN_BLOCKS
         : MODE == kPull       ? FG_PULL_MIN_BLOCKS
         : MODE == kBucket     ? FG_BUCKET_MIN_BLOCKS
         : MODE == kMulti      ? FG_MULTI_MIN_BLOCKS
                               : FG_ASYNC_MIN_BLOCKS;
}

// The whole query -- init, rounds, convergence -- run by one team of CTAs
// (the full grid for a single query, a slice of it in a batch).
// Once per kernel launch, before the first fixpoint_body: the edge-sync
// kernels initialise their CTA's tile rings (their mbarriers live for the
// whole launch; ring_used, kept by every lane, carries the phases of the
// lane's warp ring from one query of the CTA to the next).
template <int ALGO, int MODE>
__device__ __forceinline__ void fixpoint_prologue(uint32_t &ring_used) {
    ring_used = 0;
    if constexpr (MODE == kEdgeSync) rings_init(edge_rings<ALGO == kSSSP>());
}

template <int ALGO, int MODE>
__device__ __forceinline__ void fixpoint_body(const Params &p, const Team &t, uint32_t &ring_used) {
    constexpr bool SYNC = (MODE == kVertexSync || MODE == kEdgeSync || MODE == kPull);
    Ctrl *c = p.ctrl;
    const View &g = p.g;
    const int32_t n = g.n;
    const int64_t tid = t.rank * (int64_t)kBlock + threadIdx.x;
    const int64_t nth = (int64_t)t.size * kBlock;
    Acc a;
    int rounds = 0;
    int n_barriers = 0;
    bool done = false;
    // every grid barrier of the query; CTA 0 optionally timestamps each
    auto sync_ = [&]() -> bool {
        bool r = team_sync(t, c, p.timeout_ns);
        if (tid == 0) {
            if (p.trace && n_barriers < p.trace_cap) p.trace[n_barriers] = global_ns();
            n_barriers++;
        }
        return r;
    };

    // the source in internal ids (a renumbered graph takes original ones)
    const int32_t source = (ALGO != kCC && p.new_of) ? __ldg(p.new_of + p.source) : p.source;
    // ---- init: values, stamps, initial worklist (a2)
    for (int64_t v = tid; v < n; v += nth) {
        int32_t x = (ALGO == kCC) ? (int32_t)v : (v == source ? 0 : kInf);
        p.A[v] = x;
        if (SYNC && ALGO != kBFS) {
            p.B[v] = x;
            p.S1[v] = (ALGO == kCC || v == source) ? 1 : 0;   // active in round 1
            p.S0[v] = 0;
        }
        if (!SYNC && ALGO != kBFS) p.S0[v] = 0;
        if (MODE == kBucket && ALGO == kSSSP) p.far_mark[v] = 0;
        if (ALGO == kCC && p.cc_min) p.cc_min[v] = kInf;
    }
    if (ALGO == kBFS)   // visited bitmap: the source alone
        for (int64_t k = tid; k < ((int64_t)n + 31) / 32; k += nth)
            p.vis[k] = (k == (source >> 5)) ? 1u << (source & 31) : 0u;
    if (MODE == kBucket && tid == 0)
        for (int k = 0; k < 3; k++) c->far_min[k] = kInf;
    if (MODE == kEdgeSync)
        for (int64_t k = tid; k < (g.m + kWTile - 1) / kWTile; k += nth) p.eflag[k] = 0;

    if (!SYNC && ALGO != kCC && tid == 0) {
        int32_t s = source;
        uint32_t b = g.row_off[s], d = g.row_off[s + 1] - b;
        if (d > 0) {
            if (MODE == kEdgeAsync) {
                p.wl[0][0][0] = s;
                p.lb_off[0][0] = 0;
                c->wl_pack[0] = ((unsigned long long)d << 32) | 1u;
            } else if (d < (uint32_t)kLowMax) {
                p.wl[0][kWlLow][0] = s;
                c->wl_size[0][kWlLow] = 1;
            } else if (d < (uint32_t)kMidMax) {
                p.wl[0][kWlMid][0] = s;
                c->wl_size[0][kWlMid] = 1;
            } else {
                int nck = (int)((d + kChunk - 1) / kChunk);
                int2 *h = reinterpret_cast<int2 *>(p.wl[0][kWlHigh]);
                for (int k = 0; k < nck; k++) h[k] = make_int2(s, (int32_t)(b + (uint32_t)k * kChunk));
                c->wl_size[0][kWlHigh] = nck;
            }
        }
    }
    // failure-detection test: CTA 0 never arrives, the others' waits run out
    if (p.inject_missing_arrival && t.rank == 0) return;
    bool ok = sync_();

    if (SYNC && ok) {
        int pass_ctr = 0;
        int64_t ch_before = 0;   // changes of the round before the previous one (the same in every thread)
        constexpr bool kW = (ALGO == kSSSP);   // the edge rings carry weights for SSSP only
        // edge-sync: a round is sparse if the previous one accepted fewer
        // candidates than n / 2^FG_SPARSE_SHIFT (round 1: only the source is
        // active, except CC)
        // pull mode: a round pulls if the previous one changed more than
        // n / 2^shift vertices (round 1: only CC has every vertex active).
        // A pull round reads every in-edge, a push round only the active
        // vertices' out-edges; BFS pulls with an early exit per vertex.
        constexpr int kPullShift = ALGO == kBFS ? FG_PULL_SHIFT_BFS : (ALGO == kCC ? FG_PULL_SHIFT_CC : FG_PULL_SHIFT_SSSP);
        auto pull_round = [&](int r) -> bool {
            if (r == 1) return ALGO == kCC;
            const int64_t ch = __ldcg(&c->changed[(r - 1) % 3]);
            return kPullShift >= 0 ? (ch << kPullShift) > (int64_t)n : (ch >> -kPullShift) > (int64_t)n;
        };
        auto sparse_round = [&](int r) -> bool {
            if (r == 1) return ALGO != kCC;
            return ((int64_t)__ldcg(&c->changed[(r - 1) % 3]) << FG_SPARSE_SHIFT) < (int64_t)n;
        };
        for (int r = 1;; r++) {
            if (r > p.max_rounds) {
                if (tid == 0) atomicOr(&c->status, kStRoundCap);
                break;
            }
            if (tid == 0) c->changed[(r + 1) % 3] = 0;
            rounds = r;
            const bool pull = (MODE == kPull) && pull_round(r);
            if (pull && tid == 0) c->pull_rounds++;
            if constexpr (ALGO == kBFS) {
                BfsSyncOp op{p.A, r - 1, p.vis};
                if (pull) {
                    pull_vertices(t, p.tv, BfsPullOp{p.A, r - 1, p.vis}, a);
                } else if constexpr (MODE == kVertexSync || MODE == kPull) {
                    expand_vertices(t, g.row_off, g.col, g.low, 0, g.mid, g.n_mid, g.high, g.n_high_chunks, op,
                                    NoPush{}, a);
                    expand_low_dense(t, g.row_off, g.col, p.A, r - 1, n, op, a);
                } else if (sparse_round(r)) {
                    flag_edge_tiles(t, g, p.A, r - 1, n, p.eflag, r, a);
                    if (!sync_()) break;
                    if (!stream_flagged_edges<kW>(t, ring_used, g, p.eflag, r, op, a, c, p.timeout_ns)) break;
                } else {
                    if (!stream_all_edges<kW>(t, ring_used, g, op, a, c, p.timeout_ns)) break;
                }
            } else {
                const int32_t *cur = (r & 1) ? p.A : p.B;
                int32_t *next = (r & 1) ? p.B : p.A;
                const int32_t *scur = (r & 1) ? p.S1 : p.S0;
                int32_t *snext = (r & 1) ? p.S0 : p.S1;
                const int64_t ch_prev = r == 1 ? 0 : (int64_t)__ldcg(&c->changed[(r - 1) % 3]);
                // a growing frontier reaches many vertices for the first time:
                // most candidates then pass the first filter (R-MAT 22 SSSP round
                // 3: 15.7 M of 20.8 M), and the running minimum saves their MINs
                const bool growing = FG_GROW_FILTER > 0 && r > 1 &&
                                     ch_prev > (int64_t)FG_GROW_FILTER * (ch_before > 0 ? ch_before : 1);
                const bool dense_prev =
                    r == 1 ? ALGO == kCC
                           : (ch_prev << (MODE == kEdgeSync ? FG_NEXT_PROBE_SHIFT_EDGE : FG_NEXT_PROBE_SHIFT)) >
                                     (int64_t)n ||
                                 (MODE == kVertexSync && growing);
                ch_before = ch_prev;
                SyncOp<ALGO> op{g.w, cur, next, scur, snext, r, dense_prev};
                if (pull) {
                    pull_vertices(t, p.tv, PullMinOp<ALGO>{p.tv.w, cur, next, snext, r}, a);
                } else if constexpr (MODE == kVertexSync || MODE == kPull) {
                    expand_vertices(t, g.row_off, g.col, g.low, 0, g.mid, g.n_mid, g.high, g.n_high_chunks, op,
                                    NoPush{}, a);
                    expand_low_dense(t, g.row_off, g.col, scur, r, n, op, a);
                } else if (sparse_round(r)) {
                    flag_edge_tiles(t, g, scur, r, n, p.eflag, r, a);
                    if (!sync_()) break;
                    if (!stream_flagged_edges<kW>(t, ring_used, g, p.eflag, r, op, a, c, p.timeout_ns)) break;
                } else {
                    if (!stream_all_edges<kW>(t, ring_used, g, op, a, c, p.timeout_ns)) break;
                }
            }
            int ch = block_sum(a.changed);
            a.changed = 0;
            if (threadIdx.x == 0 && ch) atomicAdd(&c->changed[r % 3], ch);
            if (!sync_()) break;
            if (__ldcg(&c->changed[r % 3]) == 0) {
                done = true;
                if (tid == 0) c->result_in_b = (ALGO != kBFS) && (r & 1);
                if (ALGO == kSSSP) {
                    // A vertex without out-edges is never expanded, so no
                    // carry copies its last improvement into the other
                    // buffer: take the min of the two.
                    int32_t *res = (r & 1) ? p.B : p.A;
                    const int32_t *oth = (r & 1) ? p.A : p.B;
                    for (int64_t i = tid; i < g.n_zero; i += nth) {
                        int32_t v = __ldg(g.zero + i);
                        int32_t x = ldcg(oth + v);
                        if (x < ldcg(res + v)) stcg(res + v, x);
                    }
                }
                break;
            }
            if (ALGO == kCC) {
                // pointer jumping on next until every label is a root.  A
                // label only points to a smaller id and a root (l with
                // next[l] == l) never changes while jumping, so each vertex
                // follows its chain up to 8 steps per pass; a pass in which
                // every chain reached its root leaves labels that jumping
                // cannot change, and ends the phase without a further pass.
                int32_t *next = (r & 1) ? p.B : p.A;
                int32_t *snext = (r & 1) ? p.S0 : p.S1;
                bool jok = true;
                for (int pass = 0; pass < 16; pass++) {
                    int slot = pass_ctr % 3;
                    if (tid == 0) c->jchanged[(pass_ctr + 1) % 3] = 0;
                    pass_ctr++;
                    int jc = 0;   // chains not yet at their root
                    for (int64_t v = tid; v < n; v += nth) {
                        const int32_t l0 = ldcg(next + v);
                        if (l0 == (int32_t)v) continue;
                        int32_t l = l0;
                        bool root = false;
#pragma unroll 1
                        for (int k = 0; k < 8; k++) {
                            const int32_t ll = ldcg(next + l);
                            if (ll == l) {
                                root = true;
                                break;
                            }
                            l = ll;
                        }
                        if (!root) jc++;
                        if (l < l0) {
                            atomicMin(next + v, l);
                            stcg(snext + v, r + 1);
                        }
                    }
                    jc = block_sum(jc);
                    if (threadIdx.x == 0 && jc) atomicAdd(&c->jchanged[slot], jc);
                    if (!sync_()) { jok = false; break; }
                    if (tid == 0) c->jump_passes++;
                    if (__ldcg(&c->jchanged[slot]) == 0) break;
                }
                if (!jok) break;
            }
        }
    } else if (!SYNC && ok) {
        __shared__ WarpBuf s_buf[kWarps][2];
        if (lane_id() == 0) {
            s_buf[threadIdx.x >> 5][0].count = 0;
            s_buf[threadIdx.x >> 5][1].count = 0;
        }
        __syncwarp();
        WarpBuf *wb = s_buf[threadIdx.x >> 5];
        // bucket mode: the near threshold and the far list's epoch (epochs
        // start at 1 so that the zeroed far_mark means "in no far list")
        int32_t T = (MODE == kBucket && ALGO == kSSSP) ? p.delta : kInf;
        int epoch = 1;
        int work_gens = 0;
        for (int gen = 0;; gen++) {
            const int in_slot = gen % 3, out_slot = (gen + 1) % 3;
            const bool initial_cc = (ALGO == kCC && gen == 0);
            int n_in[3];
            for (int k = 0; k < 3; k++) n_in[k] = __ldcg(&c->wl_size[in_slot][k]);
            // edge-async: items and their edge total come packed in one word
            const unsigned long long pk = MODE == kEdgeAsync ? __ldcg(&c->wl_pack[in_slot]) : 0ull;
            if (MODE == kEdgeAsync) n_in[0] = (int)(uint32_t)pk;
            if (initial_cc) {
                if (MODE == kEdgeAsync) {
                    n_in[0] = g.n_nz; n_in[1] = n_in[2] = 0;
                } else {
                    n_in[kWlLow] = g.n_low; n_in[kWlMid] = g.n_mid; n_in[kWlHigh] = g.n_high_chunks;
                }
            }
            const bool empty = n_in[0] + n_in[1] + n_in[2] == 0;
            const bool split = empty && MODE == kBucket && ALGO == kSSSP && __ldcg(&c->far_size[epoch % 3]) > 0;
            if (empty && !split) {
                done = true;
                break;
            }
            // the cap counts worklist generations; a far-list split always
            // moves at least the far list's nearest vertex, so splits end
            if (!split && work_gens >= p.max_rounds) {
                if (tid == 0) atomicOr(&c->status, kStRoundCap);
                break;
            }
            if (!split) work_gens++;
            rounds = gen + 1;
            if (tid == 0) {
                for (int k = 0; k < 3; k++) c->wl_size[(gen + 2) % 3][k] = 0;
                c->wl_pack[(gen + 2) % 3] = 0;
            }
            const int pi = gen & 1, po = pi ^ 1;
            int *osize = c->wl_size[out_slot];
            if (split) {
                // The near worklist ran empty: the threshold moves to the far
                // list's smallest distance + delta, and the far list is split
                // into the next generation's worklist (distance below the
                // new threshold) and the next epoch's far list.  An entry
                // whose distance is now below the old threshold is stale: it
                // was lowered under that threshold later, queued as near
                // then and expanded with its current distance, so it is
                // dropped and does not hold the new threshold down.
                const int32_t T_old = T;
                const int32_t *far_in = p.far[epoch & 1];
                int32_t *far_out = p.far[(epoch + 1) & 1];
                const int fn = __ldcg(&c->far_size[epoch % 3]);
                if (tid == 0) {
                    c->far_size[(epoch + 2) % 3] = 0;
                    c->far_min[(epoch + 2) % 3] = kInf;
                    c->splits++;
                }
                int32_t fm = kInf;
                for (int64_t i = tid; i < fn; i += nth) {
                    const int32_t d = ldcg(p.A + ldcg(far_in + i));
                    if (d >= T_old) fm = min(fm, d);
                }
                fm = block_min(fm);
                if (threadIdx.x == 0 && fm < kInf) atomicMin(&c->far_min[epoch % 3], fm);
                if (!sync_()) break;
                const int32_t fmin = __ldcg(&c->far_min[epoch % 3]);
                T = fmin >= kInf - p.delta ? kInf : fmin + p.delta;
                ClassPush push{g.row_off, g.vclass, p.wl[po][kWlLow], p.wl[po][kWlMid],
                               reinterpret_cast<int2 *>(p.wl[po][kWlHigh]), osize,
                               p.wl_cap[kWlLow], p.wl_cap[kWlMid], p.wl_cap[kWlHigh] / 2, &wb[0], &wb[1], c};
                for (int64_t i0 = tid - lane_id(); i0 < fn; i0 += nth) {   // warp-uniform trip count
                    const int64_t i = i0 + lane_id();
                    bool near = false;
                    int32_t v = 0;
                    if (i < fn) {
                        v = ldcg(far_in + i);
                        const int32_t d = ldcg(p.A + v);
                        if (d < T_old) {
                            // stale: expanded in an earlier generation
                        } else if (d < T) {
                            near = atomicExch(p.S0 + v, gen + 1) != gen + 1;
                        } else if (atomicExch(p.far_mark + v, epoch + 1) != epoch + 1) {
                            const unsigned am = __activemask();
                            const int leader = __ffs(am) - 1;
                            int base = 0;
                            if ((int)lane_id() == leader) base = atomicAdd(&c->far_size[(epoch + 1) % 3], __popc(am));
                            base = __shfl_sync(am, base, leader) + __popc(am & lanemask_lt());
                            if (base < p.far_cap) far_out[base] = v;
                            else atomicOr(&c->status, kStWorklist);
                        }
                    }
                    __syncwarp();
                    push(near, v, a);
                }
                push.flush();
                epoch++;
            } else if (MODE == kVertexAsync || MODE == kBucket) {
                const int32_t *low = initial_cc ? g.low : p.wl[pi][kWlLow];
                const int32_t *mid = initial_cc ? g.mid : p.wl[pi][kWlMid];
                const int2 *high = initial_cc ? g.high : reinterpret_cast<const int2 *>(p.wl[pi][kWlHigh]);
                ClassPush push{g.row_off, g.vclass, p.wl[po][kWlLow], p.wl[po][kWlMid],
                               reinterpret_cast<int2 *>(p.wl[po][kWlHigh]), osize,
                               p.wl_cap[kWlLow], p.wl_cap[kWlMid], p.wl_cap[kWlHigh] / 2, &wb[0], &wb[1], c};
                if constexpr (ALGO == kBFS) {
                    BfsAsyncOp op{p.A, gen, p.vis};
                    expand_vertices(t, g.row_off, g.col, low, n_in[kWlLow], mid, n_in[kWlMid], high, n_in[kWlHigh],
                                    op, push, a);
                } else if constexpr (MODE == kBucket && ALGO == kSSSP) {
                    BucketOp op;
                    op.w = g.w; op.D = p.A; op.stamp = p.S0; op.gen = gen;
                    op.T = T; op.epoch = epoch; op.far = p.far[epoch & 1]; op.far_mark = p.far_mark;
                    op.far_size = &c->far_size[epoch % 3]; op.far_cap = p.far_cap; op.ctrl = c;
                    expand_vertices(t, g.row_off, g.col, low, n_in[kWlLow], mid, n_in[kWlMid], high, n_in[kWlHigh],
                                    op, push, a);
                } else {
                    const int64_t items = (int64_t)n_in[kWlLow] + n_in[kWlMid] + n_in[kWlHigh];
                    if (ALGO == kSSSP && FG_VA_DENSE_DIV > 0 && items * FG_VA_DENSE_DIV >= (int64_t)g.n_nz) {
                        AsyncScanOp op;
                        op.w = g.w; op.D = p.A; op.stamp = p.S0; op.gen = gen;
                        expand_vertices(t, g.row_off, g.col, g.low, g.n_low, g.mid, g.n_mid, g.high, g.n_high_chunks,
                                        op, push, a);
                    } else {
                        AsyncOp<ALGO> op{g.w, p.A, p.S0, gen};
                        expand_vertices(t, g.row_off, g.col, low, n_in[kWlLow], mid, n_in[kWlMid], high,
                                        n_in[kWlHigh], op, push, a);
                    }
                }
                push.flush();
            } else {
                const int32_t *items = initial_cc ? g.nz : p.wl[pi][0];
                const uint32_t *ioff = p.lb_off[pi];
                const uint32_t T = initial_cc ? (uint32_t)g.m : (uint32_t)(pk >> 32);
                // global edge offset of item i (CC's first generation: all
                // vertices with out-edges, whose offsets are their row starts)
                auto goff = [&](int i) -> uint32_t {
                    return initial_cc ? __ldg(g.row_off + __ldg(g.nz + i)) : (uint32_t)ldcg((const int32_t *)ioff + i);
                };
                LbPush push{g.row_off, g.vclass, p.wl[po][0], p.lb_off[po], &c->wl_pack[out_slot], p.wl_cap[0],
                            &wb[0], c};
                const bool dense = initial_cc || (uint64_t)T * 100u >= (uint64_t)g.m * (uint64_t)ea_dense_pct<ALGO>();
                if constexpr (ALGO == kBFS) {
                    if (dense) {
                        BfsStreamOp op;
                        op.L = p.A; op.gen = gen; op.vis = p.vis;
                        stream_edges_async<false>(t, g, op, push, a);
                    } else {
                        BfsAsyncOp op{p.A, gen, p.vis};
                        lb_expand(t, g.row_off, g.col, items, n_in[0], goff, T, op, push, a);
                    }
                } else {
                    if (dense) {
                        AsyncStreamOp<ALGO> op;
                        op.w = g.w; op.D = p.A; op.stamp = p.S0; op.gen = gen;
                        stream_edges_async<ALGO == kSSSP>(t, g, op, push, a);
                    } else {
                        AsyncOp<ALGO> op{g.w, p.A, p.S0, gen};
                        lb_expand(t, g.row_off, g.col, items, n_in[0], goff, T, op, push, a);
                    }
                }
                push.flush();
                if (tid == 0 && !dense) a.verts += (unsigned long long)n_in[0];
            }
            if (!sync_()) break;
        }
    }

    // ---- statistics
    unsigned long long ev = block_sum(a.verts), ee = block_sum(a.edges), eu = block_sum(a.updates),
                       ep = block_sum(a.pushes), es = block_sum(a.scanned), el = block_sum(a.pulled);
    int of = block_sum(a.overflow);
    if (threadIdx.x == 0) {
        if (ev) atomicAdd(&c->st_vertices, ev);
        if (ee) atomicAdd(&c->st_edges, ee);
        if (eu) atomicAdd(&c->st_updates, eu);
        if (ep) atomicAdd(&c->st_pushes, ep);
        if (es) atomicAdd(&c->st_scanned, es);
        if (el) atomicAdd(&c->st_pulled, el);
        if (of) atomicOr(&c->status, kStOverflow);
    }
    if (tid == 0) {
        c->rounds = rounds;
        c->barriers = n_barriers;
        c->done = done;
    }
    // a query of a batch with a device output: the team writes the result
    // there (both sync buffers hold values >= the fixpoint and one holds it,
    // so their minimum is the result), in original order on a renumbered
    // graph, where CC labels become each component's smallest original id
    if (done && p.out) {
        constexpr bool TWO = SYNC && ALGO != kBFS;
        auto result = [&](int64_t u) {
            int32_t x = ldcg(p.A + u);
            if (TWO) x = min(x, ldcg(p.B + u));
            return x;
        };
        if (ALGO == kCC && p.orig_of) {
            cc_min_orig_warp(tid >> 5, nth >> 5, n, result, p.orig_of, p.cc_min);
            if (sync_())
                for (int64_t v = tid; v < n; v += nth) p.out[v] = ldcg(p.cc_min + result(__ldg(p.new_of + v)));
        } else {
            for (int64_t v = tid; v < n; v += nth) p.out[v] = result(p.new_of ? __ldg(p.new_of + v) : v);
        }
    }
}


}  // namespace
}  // namespace fg
