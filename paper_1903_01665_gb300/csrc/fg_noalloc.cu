// fg_sssp_csr_noalloc: shortest paths for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: their device memory is owned by
// another allocator that has already reserved the budget (a framework's
// caching pool), or they run in a latency-critical loop where an allocation
// may synchronise the device or fail at a bad moment.  This entry point
// allocates nothing.  The caller passes the graph (CSR, device memory) and
// the output; everything else the kernel needs -- the second distance
// buffer, the two activity-stamp arrays and the control block with the grid
// barrier -- lives in one file-scope device array of fixed size below, which
// every GPU that loads the library holds until the process exits.
//
// The kernel is the vertex-based synchronous fixpoint (every round relaxes
// the out-edges of the vertices whose distance changed in the previous
// round, reading one buffer and lowering the other with atomic MIN, then a
// bounded grid barrier), without the degree buckets of the main path: each
// warp takes 32 consecutive vertices, spreads the edges of its short rows
// over its lanes and walks long rows with the whole warp.
#include <algorithm>
#include <mutex>

#include "fg_internal.cuh"

namespace fg {
namespace {

constexpr int32_t kNaMaxN = FG_NOALLOC_MAX_VERTICES;
constexpr size_t kNaCtrlBytes = 256;
constexpr size_t kNaArrayBytes = (size_t)kNaMaxN * sizeof(int32_t);
// control block, then buffer B, then stamp arrays S0 and S1 (fixed offsets)
constexpr size_t kNaScratchBytes = kNaCtrlBytes + 3 * kNaArrayBytes;
static_assert(sizeof(Ctrl) <= kNaCtrlBytes, "control block must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

constexpr int kNaBadInput = 16;   // status bit: row offsets or ids out of range, or a negative weight

struct NaParams {
    int32_t n;
    int64_t m;
    const int64_t *row_off;
    const int32_t *col;
    const int32_t *w;
    int32_t source;
    int32_t max_rounds;
    unsigned long long timeout_ns;
    int32_t *A;                    // the caller's output, also the first buffer
    unsigned char *scratch;        // device address of g_noalloc_scratch
};

__device__ __forceinline__ void na_relax(const NaParams &p, const int32_t *cur, int32_t *next, int32_t *snext,
                                         int32_t r, int64_t e, int32_t val, int &changed, int &overflow) {
    int32_t v = __ldg(p.col + e);
    uint32_t c = (uint32_t)val + (uint32_t)(p.w ? __ldg(p.w + e) : 1);
    if (c >= (uint32_t)kInf) {
        overflow = 1;
        return;
    }
    int32_t cand = (int32_t)c;
    if (cand < ldcg(cur + v)) {
        if (atomicMin(next + v, cand) > cand) {
            stcg(snext + v, r + 1);
            changed++;
        }
    }
}

__global__ void __launch_bounds__(kBlock) noalloc_sssp_kernel(NaParams p) {
    Ctrl *c = reinterpret_cast<Ctrl *>(p.scratch);
    int32_t *B = reinterpret_cast<int32_t *>(p.scratch + kNaCtrlBytes);
    int32_t *S0 = reinterpret_cast<int32_t *>(p.scratch + kNaCtrlBytes + kNaArrayBytes);
    int32_t *S1 = reinterpret_cast<int32_t *>(p.scratch + kNaCtrlBytes + 2 * kNaArrayBytes);
    const int64_t tid = blockIdx.x * (int64_t)kBlock + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kBlock;
    const int32_t n = p.n;

    // validate the caller's CSR before any indexed access, and initialise
    int bad = 0;
    for (int64_t v = tid; v < n; v += nth) {
        int64_t b = p.row_off[v], e = p.row_off[v + 1];
        if (b > e || b < 0 || e > p.m) bad = 1;
        int32_t x = (v == p.source) ? 0 : kInf;
        p.A[v] = x;
        B[v] = x;
        S1[v] = (v == p.source) ? 1 : 0;
        S0[v] = 0;
    }
    if (tid == 0 && (p.row_off[0] != 0 || p.row_off[n] != p.m)) bad = 1;
    for (int64_t e = tid; e < p.m; e += nth) {
        int32_t t = p.col[e];
        if (t < 0 || t >= n || (p.w && p.w[e] < 0)) bad = 1;
    }
    if (bad) atomicOr(&c->status, kNaBadInput);
    if (!grid_sync(c, p.timeout_ns)) return;
    if (__ldcg(&c->status) & kNaBadInput) return;

    const unsigned lane = lane_id();
    const int gw = (int)(tid >> 5);
    const int nw = (int)(nth >> 5);
    int overflow = 0;
    int rounds = 0;
    int32_t *res = nullptr;
    for (int32_t r = 1;; r++) {
        if (r > p.max_rounds) {
            if (tid == 0) atomicOr(&c->status, kStRoundCap);
            break;
        }
        rounds = r;
        if (tid == 0) c->changed[(r + 1) % 3] = 0;
        const int32_t *cur = (r & 1) ? p.A : B;
        int32_t *next = (r & 1) ? B : p.A;
        const int32_t *scur = (r & 1) ? S1 : S0;
        int32_t *snext = (r & 1) ? S0 : S1;
        int changed = 0;
        for (int64_t base = (int64_t)gw * 32; base < n; base += (int64_t)nw * 32) {
            int64_t u = base + lane;
            int32_t val = 0;
            int64_t rb = 0;
            uint32_t d = 0;
            bool act = u < n && ldcg(scur + u) == r;
            if (act) {
                val = ldcg(cur + u);
                if (ldcg(next + u) > val) atomicMin(next + u, val);   // carry into the other buffer
                rb = __ldg(p.row_off + u);
                int64_t deg = __ldg(p.row_off + u + 1) - rb;
                d = deg < 32 ? (uint32_t)deg : 0u;
            }
            // long rows: the whole warp, one row at a time
            unsigned longs = __ballot_sync(0xffffffffu, act && d == 0 && __ldg(p.row_off + u + 1) - rb >= 32);
            while (longs) {
                int l = __ffs(longs) - 1;
                longs &= longs - 1;
                int64_t lb = __shfl_sync(0xffffffffu, rb, l);
                int32_t lv = __shfl_sync(0xffffffffu, val, l);
                int64_t le = __ldg(p.row_off + base + l + 1);
                for (int64_t e = lb + lane; e < le; e += 32) na_relax(p, cur, next, snext, r, e, lv, changed, overflow);
            }
            // short rows: the warp's edges spread over its lanes
            uint32_t incl = warp_inclusive_scan(d);
            uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            uint32_t excl = incl - d;
            for (uint32_t k0 = 0; k0 < total; k0 += 32) {
                uint32_t k = k0 + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    uint32_t pv = __shfl_sync(0xffffffffu, incl, owner + step - 1);
                    if (pv <= k) owner += step;
                }
                int64_t ob = __shfl_sync(0xffffffffu, rb, owner);
                uint32_t oe = __shfl_sync(0xffffffffu, excl, owner);
                int32_t ov = __shfl_sync(0xffffffffu, val, owner);
                if (k < total) na_relax(p, cur, next, snext, r, ob + (k - oe), ov, changed, overflow);
            }
        }
        changed = warp_sum(changed);
        if (lane == 0 && changed) atomicAdd(&c->changed[r % 3], changed);
        if (!grid_sync(c, p.timeout_ns)) return;
        if (__ldcg(&c->changed[r % 3]) == 0) {
            res = next;
            break;
        }
    }
    if (overflow) atomicOr(&c->status, kStOverflow);
    if (tid == 0) c->rounds = rounds;
    if (res == nullptr) return;
    if (res == B)
        for (int64_t v = tid; v < n; v += nth) p.A[v] = ldcg(B + v);
    // overflow rule: a finite vertex with an edge to a vertex left at INF
    if (!grid_sync(c, p.timeout_ns)) return;
    if (!(__ldcg(&c->status) & kStOverflow)) return;
    for (int64_t u = tid; u < n; u += nth) {
        if (ldcg(p.A + u) == kInf) continue;
        for (int64_t e = __ldg(p.row_off + u); e < __ldg(p.row_off + u + 1); e++)
            if (ldcg(p.A + __ldg(p.col + e)) == kInf) {
                atomicOr(&c->result_in_b, 1);   // reused as "overflow confirmed"
                break;
            }
    }
}

// device address of the scratch array, looked up once per device
std::mutex g_na_mu;
unsigned char *g_na_addr[64] = {};

}  // namespace
}  // namespace fg

using namespace fg;

extern "C" fg_status fg_sssp_csr_noalloc(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                                         const int32_t *w, int32_t src, int32_t *dist_out, void *stream) {
    if (n <= 0 || n > kNaMaxN)
        return fail(FG_ERR_INVALID_ARG, "fg_sssp_csr_noalloc: n must be in [1, FG_NOALLOC_MAX_VERTICES = 1048576]");
    if (m < 0 || m >= ((int64_t)1 << 31)) return fail(FG_ERR_INVALID_ARG, "fg_sssp_csr_noalloc: m must be in [0, 2^31)");
    if (!row_off || !dist_out || (m > 0 && !col)) return fail(FG_ERR_INVALID_ARG, "fg_sssp_csr_noalloc: NULL argument");
    if (src < 0 || src >= n) return fail(FG_ERR_INVALID_ARG, "fg_sssp_csr_noalloc: source vertex outside [0, n)");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return cuda_fail(e, "fg_sssp_csr_noalloc: no CUDA device");
    // every array must be memory of this device: the kernel has no peer path
    if (!is_device_pointer_on(row_off, dev) || !is_device_pointer_on(dist_out, dev) ||
        (m > 0 && !is_device_pointer_on(col, dev)) || (w && !is_device_pointer_on(w, dev)))
        return fail(FG_ERR_INVALID_ARG, "fg_sssp_csr_noalloc: inputs and output must be device memory of the current device");
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_addr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_na_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_na_addr[dev] = nullptr;
                return cuda_fail(e, "fg_sssp_csr_noalloc: scratch address lookup");
            }
        }
        scratch = g_na_addr[dev];
    }
    int sms = 0, coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(FG_ERR_CUDA, "fg_sssp_csr_noalloc: device lacks cooperative launch");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)noalloc_sssp_kernel, kBlock, 0);
    if (e != cudaSuccess) return cuda_fail(e, "fg_sssp_csr_noalloc: occupancy query");
    int grid = std::max(1, std::min(per_sm, 8) * sms);
    cudaStream_t st = (cudaStream_t)stream;
    NaParams p{n, m, row_off, col, w, src, n > INT32_MAX - 2 ? INT32_MAX : n + 2, 1000ull * 1000000ull, dist_out,
               scratch};
    Ctrl hc;
    e = cudaMemsetAsync(scratch, 0, kNaCtrlBytes, st);   // the control block must start at zero
    if (e == cudaSuccess) {
        void *args[] = {&p};
        e = cudaLaunchCooperativeKernel((const void *)noalloc_sssp_kernel, dim3(grid), dim3(kBlock), args, 0, st);
        if (e == cudaSuccess) count_launch();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, scratch, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fg_sssp_csr_noalloc");
    if (hc.status & kNaBadInput)
        return fail(FG_ERR_INVALID_ARG, "fg_sssp_csr_noalloc: invalid CSR (offsets, ids) or a negative weight");
    if (hc.status & kStTimeout) return fail(FG_ERR_TIMEOUT, "fg_sssp_csr_noalloc: a device-side wait exceeded the timeout");
    if (hc.status & kStRoundCap) return fail(FG_ERR_TIMEOUT, "fg_sssp_csr_noalloc: round cap reached");
    if (hc.result_in_b) return fail(FG_ERR_OVERFLOW, "fg_sssp_csr_noalloc: a finite shortest distance is >= INT32_MAX");
    return FG_OK;
}
