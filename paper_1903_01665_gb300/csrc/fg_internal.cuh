// Internal declarations of the fg library: device graph layout, per-query
// control block and the device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/fg.h"

namespace fg {

// ---------------------------------------------------------------- constants
constexpr int kBlock = 256;            // threads per persistent CTA
constexpr int kWarps = kBlock / 32;
constexpr int kLowMax = 32;            // low bucket: 1 .. 31 out-edges (thread per vertex)
constexpr int kMidMax = 1024;          // mid bucket: 32 .. 1023 (warp per vertex)
constexpr int kChunk = 2048;           // high bucket: >= 1024, split in 2048-edge chunks (CTA each)
constexpr int32_t kInf = FG_INF;
constexpr int kMaxGrid = 152 * 8;      // persistent CTAs of one launch at most
constexpr int kWTile = 128;            // edge-sync: edges per warp tile (the streamed and flagged unit)

// device status bits (Ctrl::status)
constexpr int kStTimeout = 1;          // a grid barrier wait ran out
constexpr int kStRoundCap = 2;         // max_rounds reached
constexpr int kStOverflow = 4;         // a candidate >= INT32_MAX was formed (checked on host)
constexpr int kStWorklist = 8;         // a worklist append exceeded its capacity

// ---------------------------------------------------------------- graph
// One adjacency: the directed graph, or its symmetrised copy for CC.
struct View {
    int32_t n = 0;
    int64_t m = 0;
    const uint32_t *row_off = nullptr;  // [n+1]
    const int32_t *col = nullptr;       // [m]  CSR targets == COO dst (source-sorted)
    const int32_t *w = nullptr;         // [m]  weights (nullptr in the symmetrised view)
    const int32_t *src = nullptr;       // [m]  COO sources, non-decreasing
    const int32_t *low = nullptr;       // vertices with 1..31 out-edges, ascending
    const int32_t *mid = nullptr;       // 32..1023, ascending
    const int2 *high = nullptr;         // {vertex, first edge} per 2048-edge chunk of >= 1024
    const int32_t *nz = nullptr;        // all vertices with >= 1 out-edge, ascending
    const int32_t *zero = nullptr;      // vertices with no out-edge, ascending
    const uint8_t *vclass = nullptr;    // per vertex: 0 no out-edge, 1 low, 2 mid, 3 high
    int32_t n_low = 0, n_mid = 0, n_high = 0, n_high_chunks = 0, n_nz = 0, n_zero = 0;
    int32_t max_deg = 0;
};

}  // namespace fg

struct fg_graph {
    int device = 0;
    fg::View g;      // directed
    fg::View s;      // symmetrised
    fg::View t;      // transposed (in-neighbours), built on the first pull query
    bool t_ready = false;
    fg_graph_info_t info{};
    void *allocs[48] = {};
    int n_allocs = 0;
    // lazily computed diameter estimate and autotuned modes for fg_select_mode
    mutable std::mutex mu;
    mutable int32_t diam_est = -1;
    double w_mean = 1.0;        // mean edge weight (bucket mode's default width)
    double degree_gini = 0.0;   // Gini coefficient of the out-degrees (the selection model's skew)
    // renumbered vertices (by in-degree class), else null: every view holds
    // internal ids, the API original ones
    int32_t *new_of = nullptr;  // original id -> internal id
    int32_t *orig_of = nullptr; // internal id -> original id
    mutable int32_t tuned_mode[3] = {-1, -1, -1};
    mutable int32_t tuned_bps[3] = {0, 0, 0};   // CTAs per SM measured with the tuned mode
};

namespace fg {

// ---------------------------------------------------------------- per query
// Device control block, zeroed before each launch.
struct Ctrl {
    unsigned bar_count;
    unsigned bar_gen;
    int status;
    int rounds;                 // rounds / generations executed
    int jump_passes;
    int result_in_b;            // sync: 1 if the result is in buffer B
    int changed[3];             // per-round change counters, rotating slots
    int jchanged[3];            // per-pass pointer-jumping change counters
    int wl_size[3][4];          // async: worklist sizes per generation slot and class
    unsigned long long wl_pack[3];   // edge-async: (edges << 32 | items) per generation slot
    unsigned long long st_vertices, st_edges, st_updates, st_pushes, st_scanned;
    unsigned long long st_pulled;   // pull mode: in-edges read by pull rounds
    int barriers;
    int done;                   // the fixpoint was reached
    int pull_rounds;            // pull mode: rounds that pulled
    int far_size[3];            // bucket mode: far-list sizes, rotating by epoch
    int far_min[3];             // bucket mode: smallest distance in each epoch's far list
    int splits;                 // bucket mode: far-list splits (threshold moves)
};

// kAnyAlgo: a batch kernel of multi-source sweeps of either algorithm (the
// unit's Params.ms_bfs decides)
enum Algo { kSSSP = 0, kBFS = 1, kCC = 2, kAnyAlgo = 3 };
// kMulti: the multi-source sweep (up to 8 SSSP or BFS sources on one graph in
// one fixpoint); not a public fg_mode, it is reached through fg_run_multi
// and the fusion of same-graph queries in batches and the server
enum Mode { kVertexSync = 0, kVertexAsync = 1, kEdgeSync = 2, kEdgeAsync = 3, kPull = 5, kBucket = 6, kMulti = 7 };

// worklist classes (vertex-async): low, mid, high chunks; edge-async uses class 0 only
enum { kWlLow = 0, kWlMid = 1, kWlHigh = 2 };

struct Params {
    View g;
    View tv;                    // pull mode: the transposed view (in-neighbours; CC: the symmetrised one)
    int32_t *A = nullptr;       // values (dist / level / label); the result for async
    int32_t *B = nullptr;       // second buffer of the sync modes
    int32_t *S0 = nullptr;      // activity stamps (sync: read in odd/even rounds)
    int32_t *S1 = nullptr;      //   async: S0 = push stamp (dedup)
    int32_t *wl[2][3] = {};     // async worklists [in/out parity][class]; high as int2 pairs
    int32_t wl_cap[3] = {};     // capacity per class (in int32 slots)
    uint32_t *lb_off[2] = {};   // edge-async: global edge offset of each worklist item, by parity
    int32_t *eflag = nullptr;   // edge-sync sparse rounds: round stamp per 128-edge warp tile
    uint32_t *vis = nullptr;    // BFS: visited bitmap, bit v set once v has a level
    int32_t *far[2] = {};       // bucket mode: far lists by epoch parity
    int32_t *far_mark = nullptr; // bucket mode: epoch in whose far list a vertex is
    int32_t far_cap = 0;
    int32_t delta = 0;          // bucket mode: bucket width
    int32_t source = 0;
    int32_t max_rounds = 0;
    unsigned long long timeout_ns = 0;
    int32_t inject_missing_arrival = 0;
    int32_t *out = nullptr;                // batch: device output the team copies the result to
    int32_t ms_k = 0;                      // multi-source: sources in the sweep (A = rows of 8 values, S0 = stamps)
    int32_t ms_bfs = 0;                    // multi-source: unit weights (BFS levels)
    int32_t ms_src[8] = {};                // multi-source: source of each slot
    int32_t *ms_out[8] = {};               // multi-source: device output of each slot (null: not written)
    unsigned long long *trace = nullptr;   // optional per-barrier timestamps (CTA 0)
    int32_t trace_cap = 0;
    Ctrl *ctrl = nullptr;
    // renumbered graph (else null): sources come as original ids, device
    // outputs are written in original order, CC labels as minimum original ids
    const int32_t *new_of = nullptr;       // original id -> internal id
    const int32_t *orig_of = nullptr;      // internal id -> original id
    int32_t *cc_min = nullptr;             // batch CC: smallest original id of each internal label
};

// multi-source: one output pointer per slot, passed by value to a kernel
struct MsOuts {
    int32_t *p[8];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_i(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Arrays that other CTAs write during the current round are read through L2
// (ld.global.cg): an L1 copy could be stale.  Arrays written only before the
// current round began -- the previous round's values and activity stamps of
// the synchronous modes -- are read through L1 (ld.global.ca), where the hot
// lines of skewed graphs stay SM-local: the team barrier that separates
// rounds ends with an acquire at gpu scope on every CTA, which discards this
// SM's L1 copies of lines written in earlier rounds.
__device__ __forceinline__ int32_t ldcg(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ int32_t ldca(const int32_t *p) { return __ldca(p); }
__device__ __forceinline__ void stcg(int32_t *p, int32_t v) { __stcg(p, v); }
// atomic MIN whose result is not needed (a reduction: no round trip)
__device__ __forceinline__ void red_min(int32_t *p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.min.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// atomic OR whose result is not needed
__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// BFS visited bitmap: bit v & 31 of word v >> 5.  Bits are only ever set
// during a query, so a stale (L1) copy can only miss bits, never show one.
__device__ __forceinline__ bool vis_test(const uint32_t *vis, int32_t v) {
    return (((uint32_t)__ldca(reinterpret_cast<const int32_t *>(vis) + (v >> 5))) >> (v & 31)) & 1u;
}

// ---------------------------------------------------------------- bulk copies (TMA)
// One-dimensional bulk copies global -> shared memory, completed on an
// mbarrier with a transaction count (PTX ISA: cp.async.bulk, mbarrier).
// Both addresses must be 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the async (bulk-copy) proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// L2 policy for data read once per pass (the edge stream): evict it first so
// that the value and stamp arrays stay resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// ---------------------------------------------------------------- team barrier
// A team is the set of CTAs that run one query together: the whole grid of a
// single-query launch, or a slice of a batched launch (down to one CTA).
// rank/size replace blockIdx.x/gridDim.x in the work distribution; bar
// points at the team's {arrivals, generation} pair (unused for one CTA).
struct Team {
    int rank;
    int size;
    unsigned *bar;
};

constexpr int kStFatal = kStTimeout | kStRoundCap | kStWorklist;

// Sense-by-generation barrier over the CTAs of a team (all co-resident: the
// launch is cooperative).  The wait is bounded by timeout_ns; on expiry the
// CTA records kStTimeout in the query's status and returns false.  It also
// returns false once any fatal error bit is set, so every CTA of the team
// leaves the query at its next barrier.  A one-CTA team needs only
// __syncthreads.
__device__ __forceinline__ bool team_sync(const Team &t, Ctrl *c, unsigned long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (t.size == 1) {
        if (threadIdx.x == 0) s_ok = !(ld_acquire_i(&c->status) & kStFatal);
        __syncthreads();
        return s_ok != 0;
    }
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        unsigned *count = t.bar, *genp = t.bar + 1;
        unsigned gen = ld_acquire(genp);
        unsigned arrived = atom_add_acq_rel(count, 1u) + 1u;
        if (arrived == (unsigned)t.size) {
            *count = 0;
            st_release(genp, gen + 1u);
        } else {
            unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire(genp) == gen) {
                if (++spins > 64) {
                    __nanosleep(32);
                    if (global_ns() - t0 > timeout_ns) {
                        atomicOr(&c->status, kStTimeout);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        if (ld_acquire_i(&c->status) & kStFatal) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole grid of a cooperative launch as one team.
__device__ __forceinline__ bool grid_sync(Ctrl *c, unsigned long long timeout_ns) {
    const Team t{(int)blockIdx.x, (int)gridDim.x, &c->bar_count};
    return team_sync(t, c, timeout_ns);
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// An edge-array element (target id, weight) read once per pass over the
// edges: cached evict-first, so that the streamed edge arrays do not push
// the randomly probed values out of L1 and L2.
__device__ __forceinline__ int32_t ld_edge(const int32_t *p) { return __ldcs(p); }

// Renumbered graphs, CC: the smallest original id of each internal label,
// mn[L] = min orig_of[u] over the vertices u labelled L (mn preset to INF).
// A warp takes 32 x kRun consecutive vertices; each lane keeps the run of
// equal labels it sees (the giant component of a skewed graph is one long
// run, since its vertices come first, broken only by vertices that are their
// own label, e.g. isolated ones, which MIN their own word) and flushes a run
// with one atomic MIN; the warp's last runs are combined across lanes first.
// Without the runs, every vertex of a giant component would MIN the same word.
template <typename LabelFn>
__device__ __forceinline__ void cc_min_orig_warp(int64_t warp, int64_t nwarps, int32_t n, LabelFn lab,
                                                 const int32_t *orig_of, int32_t *mn) {
    constexpr int kRun = 64;
    const unsigned lane = lane_id();
    for (int64_t base = warp * 32 * kRun; base < n; base += nwarps * 32 * kRun) {
        int32_t cl = -1, cm = kInf;
        for (int k = 0; k < kRun; k++) {
            const int64_t u = base + (int64_t)k * 32 + lane;
            if (u >= n) break;
            const int32_t L = lab(u), o = __ldg(orig_of + u);
            if (L == cl) {
                if (o < cm) cm = o;
            } else if (L == (int32_t)u) {   // a label's own vertex (e.g. an isolated one): no run to break
                atomicMin(mn + L, o);
            } else {
                if (cl >= 0) atomicMin(mn + cl, cm);
                cl = L;
                cm = o;
            }
        }
        const unsigned act = __ballot_sync(0xffffffffu, cl >= 0);
        if (cl >= 0) {
            const unsigned peers = __match_any_sync(act, cl);
            const int32_t m = __reduce_min_sync(peers, cm);
            if ((int)lane == __ffs(peers) - 1) atomicMin(mn + cl, m);
        }
    }
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-aggregated append: every lane of `mask` calls it together; lanes with
// want != 0 get consecutive slots of list[*size]; one atomicAdd per warp.
// Returns false (and sets kStWorklist) on overflow.
__device__ __forceinline__ void warp_append(unsigned mask, bool want, int32_t value, int32_t *list,
                                            int *size, int32_t cap, Ctrl *c) {
    unsigned b = __ballot_sync(mask, want);
    if (b == 0) return;
    int leader = __ffs(b) - 1;
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(size, __popc(b));
    base = __shfl_sync(mask, base, leader);
    if (want) {
        int pos = base + __popc(b & lanemask_lt());
        if (pos < cap) list[pos] = value;
        else atomicOr(&c->status, kStWorklist);
    }
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if ((int)lane_id() >= d) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

// ---------------------------------------------------------------- host side
struct Error {
    fg_status code;
    std::string msg;
};

void set_last_error(const std::string &msg);
const char *last_error_cstr();
fg_status fail(fg_status code, const std::string &msg);
fg_status cuda_fail(cudaError_t e, const char *what);

// graph construction (fg_build.cu)
fg_status build_graph_from_coo(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                               const int32_t *w, bool src_sorted_csr, const int64_t *row_off_in, uint32_t flags,
                               fg_graph **out);

// 256-byte aligned bump allocator over one device allocation
struct Workspace {
    char *base = nullptr;
    size_t off = 0;
    template <typename T>
    T *take(int64_t count) {
        size_t bytes = need(count, sizeof(T));
        T *p = reinterpret_cast<T *>(base + off);
        off += bytes;
        return p;
    }
    static size_t need(int64_t count, size_t elem) {
        return ((size_t)(count > 1 ? count : 1) * elem + 255) & ~(size_t)255;
    }
};

struct Params;
size_t query_workspace_bytes(const View &g, Algo algo, Mode mode);
void carve_query_workspace(char *base, const View &g, Algo algo, Mode mode, Params &p);

// the transposed view for pull queries (fg_build.cu)
fg_status ensure_transpose(const fg_graph *g);

// Graphs created with FG_GRAPH_LAZY build their edge sources and symmetrised
// view on first use.  ensure_views builds what a query of `algo` in `mode`
// reads (mode < 0: whatever any mode of `algo` reads, the transposed view
// excepted); ensure_src builds the edge sources alone.  Thread-safe.
fg_status ensure_views(const fg_graph *g, Algo algo, int mode);
fg_status ensure_src(const fg_graph *g);

// queries (fg_fixpoint.cu)
int32_t default_delta(const fg_graph *G);
// renumbered graphs: an internal-order result to an output in original order
// (device or host; CC: labels to minimum original ids).  The caller has
// checked the result; res is left unchanged.
fg_status relabel_output(const fg_graph *G, Algo algo, const int32_t *res, int32_t *out, cudaStream_t st);
// fills the relabelling fields of a query's Params from its graph
void set_relabel(const fg_graph *G, Params &p);
int32_t ms_default_rounds(int32_t n, int k, bool near_far);
fg_status run_multi(const fg_graph *g, Algo algo, int32_t k, const int32_t *srcs, int32_t *const *outs,
                    const fg_options *opt, fg_status *status_out, fg_stats *stats);
fg_status run_query(const fg_graph *g, Algo algo, Mode mode, int32_t source, int32_t *out,
                    const fg_options *opt, fg_stats *stats);
fg_status run_sweep(const fg_graph *g, Mode mode, const int32_t *cur, int32_t *next,
                    cudaStream_t stream, int64_t *updates, float *kernel_ms);
void overflow_check_launch(const View &g, const int32_t *D, int *flag, cudaStream_t st);
// multi-source sweeps: bit s of *flag for each source s that overflowed; the
// rows' slots to the outputs that are set
void ms_overflow_check_launch(const View &g, const int32_t *D, int k, int *flag, cudaStream_t st);
void ms_output_launch(const int32_t *D, int32_t n, int k, const MsOuts &outs, const int32_t *new_of,
                      cudaStream_t st);

// batches (fg_batch.cu)
// One fixpoint of a batch: a plain query (its outputs all receive the one
// result: several only for CC, which has no source), or a fused multi-source
// sweep (mode kMulti: one output per slot, up to 8).
struct BatchUnit {
    const fg_graph *g = nullptr;
    Algo algo = kSSSP;
    Mode mode = kVertexSync;
    std::vector<int> q;                   // the batch query of each output / slot
};
struct BatchJob {
    int nq = 0;
    std::vector<fg_query> qs;
    std::vector<Mode> qmode;              // per query: the mode it ran in (kMulti if fused)
    std::vector<int> qunit;               // per query: its unit
    std::vector<BatchUnit> units;
    std::vector<const View *> view;       // per unit
    std::vector<Params> params;           // per unit: host copies of the device parameters
    std::vector<int32_t *> dout;          // per query: device buffer its result lands in
    std::vector<bool> staged;             // per query: host output, copied from dout
    bool host_copies_done = false;
    char *base = nullptr;                 // the batch's one device allocation
    size_t device_bytes = 0;
    cudaStream_t st = 0;
    std::vector<cudaStream_t> ks;
    std::vector<cudaEvent_t> kev;
    cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr, done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Ctrl *d_ctrls = nullptr;
    Ctrl *h_ctrls = nullptr;
    std::vector<Ctrl> own_ctrls;
    int launches = 0, teams = 0, ctas = 0;
    fg_status status = FG_OK;
    std::string msg;
};
fg_status batch_launch(const fg_query *qs, int32_t nq, const fg_batch_options *opt, double cta_fraction,
                       bool enqueue_host_copies, bool fuse, Ctrl *h_ctrls_pinned, BatchJob &job);
fg_status batch_finish(BatchJob &job, fg_status *status_out, fg_stats *stats_out, fg_batch_stats *bstats);
fg_status run_batch(const fg_query *qs, int32_t nq, const fg_batch_options *opt, fg_status *status_out,
                    fg_stats *stats_out, fg_batch_stats *bstats);

// whether a pointer is device-accessible memory of the current device
bool is_device_pointer(const void *p);
// whether a pointer is device (or managed) memory whose owning device is dev
bool is_device_pointer_on(const void *p, int dev);

// process-wide count of kernels this library has launched
void count_launch();

}  // namespace fg
