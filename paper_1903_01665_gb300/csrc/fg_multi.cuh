// Multi-source fixpoint: up to kMsMax SSSP (or BFS) queries on one graph in
// one relaxation sweep.
//
// Independent queries on the same graph read the same edges.  Relaxing them
// together (the k-source form of Alg. 1) reads each edge's target id and
// weight once for all k sources, and keeps the k values of a vertex in one
// 32-byte row D[v][0..7] -- one L2 sector -- so that the random probe of a
// target serves all k queries at once.  The paper overlaps independent
// computations as barrier-free kernels on separate streams (Sec. 3.2) or
// parallel sections on separate devices (Sec. 3.4); on one GB300, where a
// single query on a large graph already fills the device, fusing the
// queries' sweeps is the form of that overlap that still saves work.
//
// The sweep is vertex-based over the degree buckets (as FG_VERTEX_SYNC) and
// updates D in place with atomic MIN (as the async modes), driven by a round
// stamp per vertex: a vertex lowered in round r (for any source) is stamped
// r + 1 and expanded in every round whose number is at most its stamp, i.e.
// again in r + 1 (and in r itself if the scan reaches it after the
// lowering).  Every expansion reads the vertex's values after it was last
// stamped, so every lowering is propagated; a round with no lowering ends the
// sweep.  Values only decrease, so a stale (L1) copy of a row can only let
// through a candidate that the MIN then leaves without effect -- at worst a
// spurious stamp and one more expansion, never a wrong value.  BFS has its
// own k-source sweep over source masks (multi_bfs_body, below): levels need
// no per-source distances, only which sources have reached a vertex.
#pragma once

#include "fg_device.cuh"

namespace fg {
namespace {

constexpr int kMsMax = 8;   // sources per sweep: one int32 each in a 32-byte row

__device__ __forceinline__ void ms_load_row(const int32_t *row, int32_t (&x)[kMsMax], bool fresh) {
    const int4 *r4 = reinterpret_cast<const int4 *>(row);
    const int4 a = fresh ? __ldcg(r4) : __ldca(r4);
    const int4 b = fresh ? __ldcg(r4 + 1) : __ldca(r4 + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

// The shared near-far order of the SSSP sweep.  Slots of a row at or above
// the threshold ms_T are not propagated yet; a lowering to a value at or
// above it marks the vertex far-pending (far_mark = the round) instead of
// stamping it.  ms_T = INF (no width) leaves every finite slot near.  The
// threshold sits in shared memory, one copy per CTA, written by thread 0 only
// between team barriers: it costs the hot loop no register.
struct MsNear {
    int32_t *far_mark;
};
__shared__ int32_t ms_T;

// Relaxes up to N edges per lane: all loads (targets, weights, then the
// targets' rows) are issued before any result is used.  du[j] holds the
// source values of edge j (a slot at INF, or at or above T, has no
// candidate).  A target lowered below T is stamped for the next round, one
// lowered at or above T is marked far-pending with the round.
template <int ALGO, int N>
__device__ __forceinline__ void ms_relax(const View &g, int32_t *D, int32_t *stamp, int32_t r, const MsNear &nf,
                                         const uint32_t (&e)[N], const bool (&in)[N],
                                         const int32_t (&du)[N][kMsMax], Acc &a) {
    const int32_t T = ms_T;   // read once: the atomics below would force a re-read
    int32_t v[N], wv[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        v[j] = 0;
        wv[j] = 1;
        if (in[j]) {
            v[j] = ld_edge(g.col + e[j]);
            if (ALGO == kSSSP) wv[j] = ld_edge(g.w + e[j]);
        }
    }
    int32_t pv[N][kMsMax];
#pragma unroll
    for (int j = 0; j < N; j++) {
        if (in[j]) {
            ms_load_row(D + (size_t)v[j] * kMsMax, pv[j], false);
        } else {
#pragma unroll
            for (int s = 0; s < kMsMax; s++) pv[j][s] = 0;
        }
    }
#pragma unroll
    for (int j = 0; j < N; j++) {
        if (!in[j]) continue;
        int32_t *row = D + (size_t)v[j] * kMsMax;
        bool near = false, far = false;
#pragma unroll
        for (int s = 0; s < kMsMax; s++) {
            if (du[j][s] >= T) continue;   // INF, or a far slot: not propagated yet
            const uint32_t c = (uint32_t)du[j][s] + (uint32_t)wv[j];
            if (c >= (uint32_t)kInf) {
                a.overflow = 1;
            } else if ((int32_t)c < pv[j][s]) {
                red_min(row + s, (int32_t)c);
                if ((int32_t)c < T) near = true;
                else far = true;
            }
        }
        if (near) {
            stcg(stamp + v[j], r + 1);
            a.changed++;
        }
        if (far) {
            stcg(nf.far_mark + v[j], r);
        }
        if (near || far) a.updates++;
    }
}

// Same, with one set of source values for every edge of the lane (the edges
// of one vertex).
template <int ALGO, int N>
__device__ __forceinline__ void ms_relax_one_source(const View &g, int32_t *D, int32_t *stamp, int32_t r,
                                                    const MsNear &nf, const uint32_t (&e)[N], const bool (&in)[N],
                                                    const int32_t (&du)[kMsMax], Acc &a) {
    const int32_t T = ms_T;   // read once: the atomics below would force a re-read
    int32_t v[N], wv[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        v[j] = 0;
        wv[j] = 1;
        if (in[j]) {
            v[j] = ld_edge(g.col + e[j]);
            if (ALGO == kSSSP) wv[j] = ld_edge(g.w + e[j]);
        }
    }
    int32_t pv[N][kMsMax];
#pragma unroll
    for (int j = 0; j < N; j++) {
        if (in[j]) {
            ms_load_row(D + (size_t)v[j] * kMsMax, pv[j], false);
        } else {
#pragma unroll
            for (int s = 0; s < kMsMax; s++) pv[j][s] = 0;
        }
    }
#pragma unroll
    for (int j = 0; j < N; j++) {
        if (!in[j]) continue;
        int32_t *row = D + (size_t)v[j] * kMsMax;
        bool near = false, far = false;
#pragma unroll
        for (int s = 0; s < kMsMax; s++) {
            if (du[s] >= T) continue;   // INF, or a far slot: not propagated yet
            const uint32_t c = (uint32_t)du[s] + (uint32_t)wv[j];
            if (c >= (uint32_t)kInf) {
                a.overflow = 1;
            } else if ((int32_t)c < pv[j][s]) {
                red_min(row + s, (int32_t)c);
                if ((int32_t)c < T) near = true;
                else far = true;
            }
        }
        if (near) {
            stcg(stamp + v[j], r + 1);
            a.changed++;
        }
        if (far) {
            stcg(nf.far_mark + v[j], r);
        }
        if (near || far) a.updates++;
    }
}

#ifndef FG_MULTI_EDGES_PER_LANE
#define FG_MULTI_EDGES_PER_LANE 2
#endif
constexpr int kMsU = FG_MULTI_EDGES_PER_LANE;   // edges per lane per step (each with two 16-byte row loads in flight)

// One round: every vertex stamped >= r is expanded -- high-degree chunks by
// whole CTAs, mid-degree vertices by warps, low-degree vertices found by a
// dense scan of the stamps and their edges spread over the warp's lanes.
template <int ALGO>
__device__ __forceinline__ void ms_round(const Team &t, const View &g, int32_t *D, int32_t *stamp, int32_t r,
                                         const MsNear &nf, Acc &a) {
    __shared__ int32_t s_list[kBlock];
    __shared__ int s_n;
    __shared__ uint32_t s_rb[kWarps][128];
    __shared__ uint32_t s_d[kWarps][128];
    __shared__ int32_t s_u[kWarps][128];
    const unsigned lane = lane_id();
    const int wid = threadIdx.x >> 5;
    // ---- high-degree chunks: dealt to the team's CTAs round-robin
    const int64_t G = t.size;
    for (int64_t base = t.rank; base < g.n_high_chunks; base += G * kBlock) {
        const int64_t ci = base + (int64_t)threadIdx.x * G;
        bool act = false;
        if (ci < g.n_high_chunks) {
            const int32_t cv = __ldg(&g.high[ci].x);
            act = ldcg(stamp + cv) >= r;
            if (act && (uint32_t)__ldg(&g.high[ci].y) == __ldg(g.row_off + cv)) a.verts++;
        }
        const int na = block_compact(act, (int32_t)threadIdx.x, s_list, &s_n);
        for (int i = 0; i < na; i++) {
            const int64_t cj = base + (int64_t)s_list[i] * G;
            const int32_t u = __ldg(&g.high[cj].x);
            const uint32_t e0 = (uint32_t)__ldg(&g.high[cj].y);
            const uint32_t e1 = min(e0 + (uint32_t)kChunk, __ldg(g.row_off + u + 1));
            int32_t du[kMsMax];
            ms_load_row(D + (size_t)u * kMsMax, du, true);
            if (threadIdx.x == 0) a.edges += e1 - e0;
            for (uint32_t eb = e0; eb < e1; eb += kBlock * kMsU) {
                uint32_t e[kMsU];
                bool in[kMsU];
#pragma unroll
                for (int j = 0; j < kMsU; j++) {
                    e[j] = eb + j * kBlock + threadIdx.x;
                    in[j] = e[j] < e1;
                }
                ms_relax_one_source<ALGO>(g, D, stamp, r, nf, e, in, du, a);
            }
        }
        __syncthreads();
    }
    const int gw = (int)((t.rank * (unsigned)kBlock + threadIdx.x) >> 5);
    const int nw = (int)(t.size * (unsigned)kWarps);
    // ---- mid-degree vertices: a warp tests 32 at once, expands the active ones in turn
    for (int base = gw; base < g.n_mid; base += nw * 32) {
        const int i = base + (int)lane * nw;
        int32_t u = 0;
        bool act = false;
        if (i < g.n_mid) {
            u = __ldg(g.mid + i);
            act = ldcg(stamp + u) >= r;
        }
        unsigned bal = __ballot_sync(0xffffffffu, act);
        if (lane == 0) a.verts += __popc(bal);
        while (bal) {
            const int l = __ffs(bal) - 1;
            bal &= bal - 1;
            const int32_t uu = __shfl_sync(0xffffffffu, u, l);
            int32_t du[kMsMax];
            ms_load_row(D + (size_t)uu * kMsMax, du, true);
            const uint32_t b = __ldg(g.row_off + uu), en = __ldg(g.row_off + uu + 1);
            if (lane == 0) a.edges += en - b;
            for (uint32_t eb = b; eb < en; eb += 32 * kMsU) {
                uint32_t e[kMsU];
                bool in[kMsU];
#pragma unroll
                for (int j = 0; j < kMsU; j++) {
                    e[j] = eb + 32 * j + lane;
                    in[j] = e[j] < en;
                }
                ms_relax_one_source<ALGO>(g, D, stamp, r, nf, e, in, du, a);
            }
        }
    }
    // ---- low-degree vertices (1..31 out-edges): dense scan of 128 ids per warp step
    const int32_t n = g.n;
    for (int64_t w0 = (int64_t)gw * 128; w0 < n; w0 += (int64_t)nw * 128) {
        const int64_t v0 = w0 + 4 * lane;
        if (lane == 0) a.scanned += min((int64_t)128, (int64_t)n - w0);
        int32_t st[4];
        if (v0 + 3 < n) {
            const int4 s4 = __ldcg(reinterpret_cast<const int4 *>(stamp + v0));
            st[0] = s4.x; st[1] = s4.y; st[2] = s4.z; st[3] = s4.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) st[j] = (v0 + j < n) ? ldcg(stamp + v0 + j) : 0;
        }
        bool act[4];
        uint32_t rb[4], d[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            act[j] = st[j] >= r;
            rb[j] = 0;
            d[j] = 0;
            if (act[j]) {
                rb[j] = __ldg(g.row_off + v0 + j);
                d[j] = __ldg(g.row_off + v0 + j + 1) - rb[j];
                act[j] = d[j] >= 1 && d[j] < (uint32_t)kLowMax;
            }
        }
        const unsigned cnt_lane = act[0] + act[1] + act[2] + act[3];
        if (!__ballot_sync(0xffffffffu, cnt_lane != 0)) continue;
        const unsigned incl = warp_inclusive_scan(cnt_lane);
        const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned slot = incl - cnt_lane;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (act[j]) {
                s_rb[wid][slot] = rb[j];
                s_d[wid][slot] = d[j];
                s_u[wid][slot] = (int32_t)(v0 + j);
                slot++;
            }
        }
        __syncwarp();
        if (lane == 0) a.verts += tot;
        for (unsigned g0 = 0; g0 < tot; g0 += 32) {
            // up to 32 rows, one per lane, their edges spread over the warp
            const unsigned k = g0 + lane;
            uint32_t r0 = 0, dd = 0;
            int32_t uu = 0;
            if (k < tot) {
                r0 = s_rb[wid][k];
                dd = s_d[wid][k];
                uu = s_u[wid][k];
            }
            const uint32_t inc = warp_inclusive_scan(dd);
            const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
            const uint32_t exc = inc - dd;
            if (lane == 0) a.edges += total;
            for (uint32_t k0 = 0; k0 < total; k0 += 32 * kMsU) {
                uint32_t e[kMsU];
                bool in[kMsU];
                int32_t du[kMsU][kMsMax];
#pragma unroll
                for (int j = 0; j < kMsU; j++) {
                    const uint32_t x = k0 + 32 * j + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const uint32_t pv = __shfl_sync(0xffffffffu, inc, owner + step - 1);
                        if (pv <= x) owner += step;
                    }
                    const uint32_t ob = __shfl_sync(0xffffffffu, r0, owner);
                    const uint32_t oe = __shfl_sync(0xffffffffu, exc, owner);
                    const int32_t ou = __shfl_sync(0xffffffffu, uu, owner);
                    in[j] = x < total;
                    e[j] = ob + (x - oe);
                    if (in[j]) {
                        ms_load_row(D + (size_t)ou * kMsMax, du[j], false);
                    } else {
#pragma unroll
                        for (int s = 0; s < kMsMax; s++) du[j][s] = kInf;
                    }
                }
                ms_relax<ALGO>(g, D, stamp, r, nf, e, in, du, a);
            }
        }
        __syncwarp();
    }
}

// The sweep's sources in internal ids (a renumbered graph takes original
// ones); slots beyond k get -1, which matches no vertex.
__device__ __forceinline__ void ms_internal_sources(const Params &p, int k, int32_t (&out)[kMsMax]) {
#pragma unroll
    for (int s = 0; s < kMsMax; s++)
        out[s] = s < k ? (p.new_of ? __ldg(p.new_of + p.ms_src[s]) : p.ms_src[s]) : -1;
}

// Split of the shared near-far order, when a round lowered nothing below T.
// The far-pending vertices of the epoch are those marked in one of its
// rounds (far_mark >= the epoch's first round); each may hold finite slots at
// or above T.  Pass 1 finds the smallest such slot m over all of them; none
// means the sweep is done.  Otherwise T moves to m + delta, and pass 2 stamps
// each far-pending vertex with a slot now below T for the next round, and
// marks those that still hold a slot at or above T for the next epoch.
// Every source measures distances from itself, so one threshold schedule
// serves all of them: each source's sweep is a near-far delta-stepping of
// its own.
__device__ __forceinline__ int32_t ms_far_min(const int32_t (&x)[kMsMax], int32_t T) {
    int32_t m = kInf;
#pragma unroll
    for (int s = 0; s < kMsMax; s++)
        if (x[s] >= T && x[s] < m) m = x[s];
    return m;
}

// The whole multi-source query run by one team: init, rounds until one
// lowers nothing and no vertex is far-pending, then the rows are written out
// per source (unless a candidate overflowed: the host then checks which
// sources overflowed and writes the others).
template <int ALGO>
__device__ __forceinline__ void multi_body(const Params &p, const Team &t) {
    Ctrl *c = p.ctrl;
    const View &g = p.g;
    const int32_t n = g.n;
    const int k = p.ms_k;
    int32_t *D = p.A;
    int32_t *stamp = p.S0;
    const int64_t tid = t.rank * (int64_t)kBlock + threadIdx.x;
    const int64_t nth = (int64_t)t.size * kBlock;
    Acc a;
    int rounds = 0, n_barriers = 0;
    bool done = false;
    auto sync_ = [&]() -> bool {
        const bool ok = team_sync(t, c, p.timeout_ns);
        n_barriers++;
        return ok;
    };
    // ---- init: every row INF but the sources' own slots; the sources are stamped for round 1
    int32_t msrc[kMsMax];
    ms_internal_sources(p, k, msrc);
    for (int64_t v = tid; v < n; v += nth) {
        int32_t x[kMsMax];
        bool src = false;
#pragma unroll
        for (int s = 0; s < kMsMax; s++) {
            const bool mine = msrc[s] == (int32_t)v;
            x[s] = mine ? 0 : kInf;
            src |= mine;
        }
        int4 *row = reinterpret_cast<int4 *>(D + (size_t)v * kMsMax);
        row[0] = make_int4(x[0], x[1], x[2], x[3]);
        row[1] = make_int4(x[4], x[5], x[6], x[7]);
        stamp[v] = src ? 1 : 0;
        p.far_mark[v] = 0;   // rounds start at 1
    }
    if (tid == 0)
        for (int e = 0; e < 3; e++) c->far_min[e] = kInf;
    // the epoch state lives in shared memory too, out of the round loop's registers
    __shared__ int32_t s_epoch0, s_splits;   // first round of the current epoch; splits so far
    MsNear nf{p.far_mark};
    if (threadIdx.x == 0) {
        ms_T = p.delta > 0 ? p.delta : kInf;
        s_epoch0 = 1;
        s_splits = 0;
    }
    bool ok = sync_();
    for (int r = 1; ok; r++) {
        if (r > p.max_rounds) {
            if (tid == 0) atomicOr(&c->status, kStRoundCap);
            break;
        }
        if (tid == 0) c->changed[(r + 1) % 3] = 0;
        rounds = r;
        ms_round<ALGO>(t, g, D, stamp, r, nf, a);
        const int ch = block_sum(a.changed);
        a.changed = 0;
        const int of = block_sum(a.overflow);
        if (threadIdx.x == 0) {
            if (ch) atomicAdd(&c->changed[r % 3], ch);
            if (of) atomicOr(&c->status, kStOverflow);
        }
        if (!sync_()) break;
        if (__ldcg(&c->changed[r % 3]) != 0) continue;
        const int32_t T = ms_T;
        if (T >= kInf) {   // no width: nothing is ever far
            done = true;
            break;
        }
        // ---- split, pass 1: the smallest far slot of the epoch's far-pending vertices
        const int32_t epoch0 = s_epoch0;
        const int splits = s_splits;
        int32_t fm = kInf;
        for (int64_t v = tid; v < n; v += nth) {
            if (ldcg(p.far_mark + v) < epoch0) continue;
            int32_t x[kMsMax];
            ms_load_row(D + (size_t)v * kMsMax, x, true);
            fm = min(fm, ms_far_min(x, T));
        }
        fm = block_min(fm);
        if (threadIdx.x == 0 && fm < kInf) atomicMin(&c->far_min[splits % 3], fm);
        if (!sync_()) break;
        const int32_t m = __ldcg(&c->far_min[splits % 3]);
        if (m >= kInf) {
            done = true;
            break;
        }
        // ---- pass 2: far-pending vertices that turned near run next round, the rest wait for the next epoch
        if (tid == 0) c->far_min[(splits + 1) % 3] = kInf;
        const int32_t T_old = T;
        const int32_t T_new = m >= kInf - p.delta ? kInf : m + p.delta;
        for (int64_t v = tid; v < n; v += nth) {
            if (ldcg(p.far_mark + v) < epoch0) continue;
            int32_t x[kMsMax];
            ms_load_row(D + (size_t)v * kMsMax, x, true);
            bool now = false, still = false;
#pragma unroll
            for (int s = 0; s < kMsMax; s++) {
                now |= x[s] >= T_old && x[s] < T_new;
                still |= x[s] >= T_new && x[s] < kInf;
            }
            if (now) stcg(stamp + v, r + 1);
            if (still) stcg(p.far_mark + v, r + 1);
        }
        __syncthreads();   // every thread of the CTA is done with this epoch's state
        if (threadIdx.x == 0) {
            s_epoch0 = r + 1;
            s_splits = splits + 1;
            ms_T = T_new;
        }
        if (!sync_()) break;
    }
    // ---- statistics
    const unsigned long long ev = block_sum(a.verts), ee = block_sum(a.edges), eu = block_sum(a.updates),
                             es = block_sum(a.scanned);
    if (threadIdx.x == 0) {
        if (ev) atomicAdd(&c->st_vertices, ev);
        if (ee) atomicAdd(&c->st_edges, ee);
        if (eu) atomicAdd(&c->st_updates, eu);
        if (es) atomicAdd(&c->st_scanned, es);
    }
    if (tid == 0) {
        c->rounds = rounds;
        c->barriers = n_barriers;
        c->done = done;
        c->splits = s_splits;
    }
    // ---- results: slot s of every row to source s's output, in original
    // order (the barrier above made the overflow bit visible to every CTA)
    if (done && !(__ldcg(&c->status) & kStOverflow)) {
        for (int64_t v = tid; v < n; v += nth) {
            int32_t x[kMsMax];
            ms_load_row(D + (size_t)(p.new_of ? __ldg(p.new_of + v) : v) * kMsMax, x, true);
#pragma unroll
            for (int s = 0; s < kMsMax; s++)
                if (s < k && p.ms_out[s]) p.ms_out[s][v] = x[s];
        }
    }
}

// Overflow test of a multi-source sweep: source s overflowed iff some edge
// u -> v has D[u][s] finite and D[v][s] still INF (v's true distance is
// finite but >= INT32_MAX).  Bit s of *flags is set for each such source.
__global__ void ms_overflow_check_kernel(View g, const int32_t *D, int k, int *flags) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < g.n; u += (int64_t)gridDim.x * blockDim.x) {
        int32_t du[kMsMax];
        ms_load_row(D + (size_t)u * kMsMax, du, true);
        unsigned live = 0;
        for (int s = 0; s < k; s++)
            if (du[s] != kInf) live |= 1u << s;
        if (!live) continue;
        for (uint32_t e = __ldg(g.row_off + u); e < __ldg(g.row_off + u + 1) && live; e++) {
            int32_t dv[kMsMax];
            ms_load_row(D + (size_t)__ldg(g.col + e) * kMsMax, dv, true);
            for (int s = 0; s < k; s++)
                if ((live >> s) & 1u && dv[s] == kInf) {
                    atomicOr(flags, 1 << s);
                    live &= ~(1u << s);
                }
        }
    }
}

// Writes slot s of every row to outs[s] for the sources whose output is set
// (after an overflow: the sources that did not overflow), in original order
// (new_of: a renumbered graph's internal ids, else null).
__global__ void ms_output_kernel(const int32_t *D, int32_t n, int k, MsOuts outs, const int32_t *new_of) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t x[kMsMax];
        ms_load_row(D + (size_t)(new_of ? __ldg(new_of + v) : v) * kMsMax, x, true);
#pragma unroll
        for (int s = 0; s < kMsMax; s++)
            if (s < k && outs.p[s]) outs.p[s][v] = x[s];
    }
}

// ================================================================ k-source BFS with source masks
// BFS needs no distances per source: a level is the round in which a source
// first reaches the vertex.  The k-source BFS keeps one byte per vertex, bit
// s set once source s has reached it (64 MB at 2^26 vertices: the probes stay
// in L2, where the 32-byte rows of the SSSP sweep do not), and the frontier
// of each round as byte masks (the sources that reached the vertex in the
// previous round).  An edge u -> v of a frontier vertex with mask f claims v
// for the sources in f that have not reached it, with one atomic OR on v's
// byte; each source s that newly reaches v writes level r to its output, and
// v joins the next frontier for those sources.  Three frontier buffers
// rotate: round r reads F[r % 3], fills F[(r + 1) % 3] and clears
// F[(r + 2) % 3], which held the previous round's frontier.
__device__ __forceinline__ uint32_t ldcg_u32(const uint8_t *p) {
    return (uint32_t)__ldcg(reinterpret_cast<const int32_t *>(p));
}

// Up to N edges per lane: targets first, then their mask bytes, then claims.
template <int N>
__device__ __forceinline__ void msb_relax(const View &g, const Params &p, uint8_t *vis, uint8_t *nxt, int32_t r,
                                          const uint32_t (&e)[N], const bool (&in)[N], const uint32_t (&f)[N],
                                          Acc &a) {
    int32_t v[N];
    uint32_t seen[N];
#pragma unroll
    for (int j = 0; j < N; j++) v[j] = in[j] ? ld_edge(g.col + e[j]) : 0;
#pragma unroll
    for (int j = 0; j < N; j++) seen[j] = in[j] ? (uint32_t)__ldca(vis + v[j]) : 0xffu;
#pragma unroll
    for (int j = 0; j < N; j++) {
        const uint32_t bits = in[j] ? f[j] & ~seen[j] & 0xffu : 0u;
        if (!bits) continue;
        // a stale (L1) byte misses bits set since: the OR's old value decides
        const int sh = (v[j] & 3) * 8;
        const uint32_t old = atomicOr(reinterpret_cast<uint32_t *>(vis + (v[j] & ~3)), bits << sh);
        const uint32_t newly = bits & ~(old >> sh) & 0xffu;
        if (!newly) continue;
        red_or(reinterpret_cast<uint32_t *>(nxt + (v[j] & ~3)), newly << sh);
        const int32_t ov = p.orig_of ? __ldg(p.orig_of + v[j]) : v[j];   // outputs are in original order
#pragma unroll
        for (int s = 0; s < kMsMax; s++)
            if ((newly >> s) & 1u) stcg(p.ms_out[s] + ov, r);
        a.changed++;
        a.updates++;
    }
}

__device__ __forceinline__ void msb_round(const Team &t, const View &g, const Params &p, uint8_t *vis,
                                          const uint8_t *cur, uint8_t *nxt, int32_t r, Acc &a) {
    __shared__ int32_t s_list[kBlock];
    __shared__ int s_n;
    __shared__ uint32_t s_rb[kWarps][128];
    __shared__ uint32_t s_d[kWarps][128];
    __shared__ uint32_t s_f[kWarps][128];
    const unsigned lane = lane_id();
    const int wid = threadIdx.x >> 5;
    // ---- high-degree chunks: dealt to the team's CTAs round-robin
    const int64_t G = t.size;
    for (int64_t base = t.rank; base < g.n_high_chunks; base += G * kBlock) {
        const int64_t ci = base + (int64_t)threadIdx.x * G;
        bool act = false;
        if (ci < g.n_high_chunks) {
            const int32_t cv = __ldg(&g.high[ci].x);
            act = __ldcg(cur + cv) != 0;
            if (act && (uint32_t)__ldg(&g.high[ci].y) == __ldg(g.row_off + cv)) a.verts++;
        }
        const int na = block_compact(act, (int32_t)threadIdx.x, s_list, &s_n);
        for (int i = 0; i < na; i++) {
            const int64_t cj = base + (int64_t)s_list[i] * G;
            const int32_t u = __ldg(&g.high[cj].x);
            const uint32_t e0 = (uint32_t)__ldg(&g.high[cj].y);
            const uint32_t e1 = min(e0 + (uint32_t)kChunk, __ldg(g.row_off + u + 1));
            const uint32_t fu = __ldcg(cur + u);
            if (threadIdx.x == 0) a.edges += e1 - e0;
            for (uint32_t eb = e0; eb < e1; eb += kBlock * 4) {
                uint32_t e[4], f[4];
                bool in[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    e[j] = eb + j * kBlock + threadIdx.x;
                    in[j] = e[j] < e1;
                    f[j] = fu;
                }
                msb_relax(g, p, vis, nxt, r, e, in, f, a);
            }
        }
        __syncthreads();
    }
    const int gw = (int)((t.rank * (unsigned)kBlock + threadIdx.x) >> 5);
    const int nw = (int)(t.size * (unsigned)kWarps);
    // ---- mid-degree vertices: a warp tests 32 at once, expands the active ones in turn
    for (int base = gw; base < g.n_mid; base += nw * 32) {
        const int i = base + (int)lane * nw;
        int32_t u = 0;
        uint32_t fu = 0;
        if (i < g.n_mid) {
            u = __ldg(g.mid + i);
            fu = __ldcg(cur + u);
        }
        unsigned bal = __ballot_sync(0xffffffffu, fu != 0);
        if (lane == 0) a.verts += __popc(bal);
        while (bal) {
            const int l = __ffs(bal) - 1;
            bal &= bal - 1;
            const int32_t uu = __shfl_sync(0xffffffffu, u, l);
            const uint32_t ff = __shfl_sync(0xffffffffu, fu, l);
            const uint32_t b = __ldg(g.row_off + uu), en = __ldg(g.row_off + uu + 1);
            if (lane == 0) a.edges += en - b;
            for (uint32_t eb = b; eb < en; eb += 32 * 4) {
                uint32_t e[4], f[4];
                bool in[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    e[j] = eb + 32 * j + lane;
                    in[j] = e[j] < en;
                    f[j] = ff;
                }
                msb_relax(g, p, vis, nxt, r, e, in, f, a);
            }
        }
    }
    // ---- low-degree vertices (1..31 out-edges): dense scan of the frontier bytes, 128 per warp step
    const int32_t n = g.n;
    for (int64_t w0 = (int64_t)gw * 128; w0 < n; w0 += (int64_t)nw * 128) {
        const int64_t v0 = w0 + 4 * lane;
        if (lane == 0) a.scanned += min((int64_t)128, (int64_t)n - w0);
        const uint32_t w4 = v0 < n ? ldcg_u32(cur + v0) : 0u;   // the buffers are padded to 16 bytes
        bool act[4];
        uint32_t rb[4], d[4], fm[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            fm[j] = (w4 >> (8 * j)) & 0xffu;
            act[j] = fm[j] != 0 && v0 + j < n;
            rb[j] = 0;
            d[j] = 0;
            if (act[j]) {
                rb[j] = __ldg(g.row_off + v0 + j);
                d[j] = __ldg(g.row_off + v0 + j + 1) - rb[j];
                act[j] = d[j] >= 1 && d[j] < (uint32_t)kLowMax;
            }
        }
        const unsigned cnt_lane = act[0] + act[1] + act[2] + act[3];
        if (!__ballot_sync(0xffffffffu, cnt_lane != 0)) continue;
        const unsigned incl = warp_inclusive_scan(cnt_lane);
        const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned slot = incl - cnt_lane;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (act[j]) {
                s_rb[wid][slot] = rb[j];
                s_d[wid][slot] = d[j];
                s_f[wid][slot] = fm[j];
                slot++;
            }
        }
        __syncwarp();
        if (lane == 0) a.verts += tot;
        for (unsigned g0 = 0; g0 < tot; g0 += 32) {
            const unsigned k = g0 + lane;
            uint32_t r0 = 0, dd = 0, f0 = 0;
            if (k < tot) {
                r0 = s_rb[wid][k];
                dd = s_d[wid][k];
                f0 = s_f[wid][k];
            }
            const uint32_t inc = warp_inclusive_scan(dd);
            const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
            const uint32_t exc = inc - dd;
            if (lane == 0) a.edges += total;
            for (uint32_t k0 = 0; k0 < total; k0 += 32 * 4) {
                uint32_t e[4], f[4];
                bool in[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const uint32_t x = k0 + 32 * j + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const uint32_t pv = __shfl_sync(0xffffffffu, inc, owner + step - 1);
                        if (pv <= x) owner += step;
                    }
                    const uint32_t ob = __shfl_sync(0xffffffffu, r0, owner);
                    const uint32_t oe = __shfl_sync(0xffffffffu, exc, owner);
                    f[j] = __shfl_sync(0xffffffffu, f0, owner);
                    in[j] = x < total;
                    e[j] = ob + (x - oe);
                }
                msb_relax(g, p, vis, nxt, r, e, in, f, a);
            }
        }
        __syncwarp();
    }
}

// Bytes of the k-source BFS state per mask array: n rounded up to 16.
__host__ __device__ __forceinline__ int64_t msb_pad(int32_t n) { return ((int64_t)n + 15) & ~(int64_t)15; }

// The whole k-source BFS run by one team: init (masks, frontier, outputs),
// rounds until one reaches nothing new.
__device__ __forceinline__ void multi_bfs_body(const Params &p, const Team &t) {
    Ctrl *c = p.ctrl;
    const View &g = p.g;
    const int32_t n = g.n;
    const int k = p.ms_k;
    const int64_t np = msb_pad(n);
    uint8_t *vis = reinterpret_cast<uint8_t *>(p.A);
    uint8_t *F = reinterpret_cast<uint8_t *>(p.S0);   // three frontier arrays of np bytes
    const int64_t tid = t.rank * (int64_t)kBlock + threadIdx.x;
    const int64_t nth = (int64_t)t.size * kBlock;
    Acc a;
    int rounds = 0, n_barriers = 0;
    bool done = false;
    auto sync_ = [&]() -> bool {
        const bool ok = team_sync(t, c, p.timeout_ns);
        n_barriers++;
        return ok;
    };
    // ---- init: the sources' bits (reached, and the frontier of round 1),
    // level 0 at the sources, INF elsewhere (the outputs are in original
    // order, the masks in internal ids)
    int32_t msrc[kMsMax];
    ms_internal_sources(p, k, msrc);
    for (int64_t v = tid; v < np; v += nth) {
        uint32_t bits = 0;
#pragma unroll
        for (int s = 0; s < kMsMax; s++)
            if (msrc[s] == (int32_t)v) bits |= 1u << s;
        vis[v] = (uint8_t)bits;
        F[np + v] = (uint8_t)bits;   // F[1]
        F[v] = 0;                    // F[0]
        F[2 * np + v] = 0;           // F[2]
        if (v < n)
#pragma unroll
            for (int s = 0; s < kMsMax; s++)
                if (s < k) p.ms_out[s][v] = p.ms_src[s] == (int32_t)v ? 0 : kInf;
    }
    bool ok = sync_();
    for (int r = 1; ok; r++) {
        if (r > p.max_rounds) {
            if (tid == 0) atomicOr(&c->status, kStRoundCap);
            break;
        }
        if (tid == 0) c->changed[(r + 1) % 3] = 0;
        rounds = r;
        const uint8_t *cur = F + (r % 3) * np;
        uint8_t *nxt = F + ((r + 1) % 3) * np;
        int4 *clr = reinterpret_cast<int4 *>(F + ((r + 2) % 3) * np);   // the previous round's frontier
        for (int64_t i = tid; i < np / 16; i += nth) clr[i] = make_int4(0, 0, 0, 0);
        msb_round(t, g, p, vis, cur, nxt, r, a);
        const int ch = block_sum(a.changed);
        a.changed = 0;
        if (threadIdx.x == 0 && ch) atomicAdd(&c->changed[r % 3], ch);
        if (!sync_()) break;
        if (__ldcg(&c->changed[r % 3]) == 0) {
            done = true;
            break;
        }
    }
    const unsigned long long ev = block_sum(a.verts), ee = block_sum(a.edges), eu = block_sum(a.updates),
                             es = block_sum(a.scanned);
    if (threadIdx.x == 0) {
        if (ev) atomicAdd(&c->st_vertices, ev);
        if (ee) atomicAdd(&c->st_edges, ee);
        if (eu) atomicAdd(&c->st_updates, eu);
        if (es) atomicAdd(&c->st_scanned, es);
    }
    if (tid == 0) {
        c->rounds = rounds;
        c->barriers = n_barriers;
        c->done = done;
    }
}

// A query of either kind, as the kernels run it.
template <int ALGO, int MODE>
__device__ __forceinline__ void query_body(const Params &p, const Team &t, uint32_t &ring_used) {
    if constexpr (MODE == kMulti) {
        if constexpr (ALGO == kAnyAlgo) {
            if (p.ms_bfs) multi_bfs_body(p, t);
            else multi_body<kSSSP>(p, t);
        } else if constexpr (ALGO == kBFS) {
            multi_bfs_body(p, t);
        } else if constexpr (ALGO == kSSSP) {
            multi_body<kSSSP>(p, t);
        }
    } else {
        fixpoint_body<ALGO, MODE>(p, t, ring_used);
    }
}

}  // namespace
}  // namespace fg
