// Graph construction on the device: validation, CSR + source-sorted COO by
// counting sort, the symmetrised copy for connected components, and the
// degree buckets of the vertex kernels.
//
// Storage follows Sec. 3.1: vertex-based code reads CSR (row offsets +
// targets), edge-based code reads the edge list (source, destination,
// weight).  The COO here is the CSR's edges in CSR order, so its dst and w
// arrays are the CSR's col and w and only src is stored in addition.
#include <algorithm>
#include <vector>

#include "fg_internal.cuh"

namespace fg {

namespace {

constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

inline int grid_for(int64_t work, int per_block = kBlock) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;   // grid-stride beyond this
    return (int)b;
}

// ---------------------------------------------------------------- validation
enum { kBadId = 1, kBadWeight = 2, kBadOffsets = 4 };

__global__ void k_validate_coo(int64_t m, int32_t n, const int32_t *__restrict__ s,
                               const int32_t *__restrict__ d, const int32_t *__restrict__ w,
                               int *flags) {
    int f = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = s[e], b = d[e];
        if (a < 0 || a >= n || b < 0 || b >= n) f |= kBadId;
        if (w && w[e] < 0) f |= kBadWeight;
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if (f && lane_id() == 0) atomicOr(flags, f);
}

__global__ void k_validate_csr(int32_t n, int64_t m, const int64_t *__restrict__ ro,
                               const int32_t *__restrict__ col, const int32_t *__restrict__ w,
                               int *flags) {
    int f = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t v = t; v < n; v += stride)
        if (ro[v] > ro[v + 1]) f |= kBadOffsets;
    if (t == 0 && (ro[0] != 0 || ro[n] != m)) f |= kBadOffsets;
    for (int64_t e = t; e < m; e += stride) {
        int32_t b = col[e];
        if (b < 0 || b >= n) f |= kBadId;
        if (w && w[e] < 0) f |= kBadWeight;
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if (f && lane_id() == 0) atomicOr(flags, f);
}

// ---------------------------------------------------------------- counting sort
__global__ void k_histogram(int64_t m, const int32_t *__restrict__ keys, uint32_t *cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[keys[e]], 1u);
}

// (the source array of the result is filled afterwards from the row
// offsets, with sequential writes, by k_src_from_rows)
__global__ void k_scatter_coo(int64_t m, const int32_t *__restrict__ s, const int32_t *__restrict__ d,
                              const int32_t *__restrict__ w, uint32_t *cursor, int32_t *col, int32_t *wout) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = s[e];
        uint32_t pos = atomicAdd(&cursor[u], 1u);
        col[pos] = d[e];
        wout[pos] = w ? w[e] : 1;
    }
}

// Sum of the edge weights (for the bucket mode's default width).
__global__ void k_weight_sum(int64_t m, const int32_t *__restrict__ w, unsigned long long *sum) {
    unsigned long long x = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        x += (unsigned)w[e];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(sum, x);
}

// Out-degree histogram in power-of-two bins (bin 0: no out-edge; bin k:
// degrees in [2^(k-1), 2^k)) with each bin's degree sum: the Lorenz curve of
// the degree distribution, from which the host forms a Gini coefficient.
constexpr int kDegBins = 33;
// renumber by default above this in-degree Gini (R-MAT about 0.6-0.7, grids
// about 0.1)
constexpr double kRelabelGini = 0.5;
__device__ __forceinline__ int degree_bin(uint32_t d) { return d == 0 ? 0 : 32 - __clz(d); }

// FROM_OFFSETS: a holds row offsets (degree = a[v+1] - a[v]), else degrees.
// The lanes of a warp that fall in one bin add to it once (most vertices
// fall in a few bins).
template <bool FROM_OFFSETS>
__global__ void k_degree_bins(int32_t n, const uint32_t *__restrict__ a, unsigned long long *cnt,
                              unsigned long long *sum) {
    __shared__ unsigned long long s_cnt[kDegBins], s_sum[kDegBins];
    for (int i = threadIdx.x; i < kDegBins; i += blockDim.x) s_cnt[i] = s_sum[i] = 0;
    __syncthreads();
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        const bool valid = v < n;
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (!valid) continue;
        const uint32_t d = FROM_OFFSETS ? a[v + 1] - a[v] : a[v];
        const int b = degree_bin(d);
        const unsigned peers = __match_any_sync(act, b);
        const unsigned long long ds = __reduce_add_sync(peers, d);   // at most m < 2^31
        if ((int)lane_id() == __ffs(peers) - 1) {
            atomicAdd(&s_cnt[b], (unsigned long long)__popc(peers));
            atomicAdd(&s_sum[b], ds);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kDegBins; i += blockDim.x) {
        if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
        if (s_sum[i]) atomicAdd(&sum[i], s_sum[i]);
    }
}

// Gini coefficient of the binned degrees: 1 - twice the area under the
// Lorenz curve (vertices by increasing degree against their share of the
// edges), the curve taken as linear within a bin.
double gini_of_bins(const unsigned long long *cnt, const unsigned long long *sum) {
    double n = 0, m = 0;
    for (int i = 0; i < kDegBins; i++) {
        n += (double)cnt[i];
        m += (double)sum[i];
    }
    if (n <= 0 || m <= 0) return 0.0;
    double x0 = 0, y0 = 0, area = 0;
    for (int i = 0; i < kDegBins; i++) {
        const double x1 = x0 + (double)cnt[i] / n, y1 = y0 + (double)sum[i] / m;
        area += (x1 - x0) * (y0 + y1) / 2;
        x0 = x1;
        y0 = y1;
    }
    return 1.0 - 2.0 * area;
}

// ---------------------------------------------------------------- renumbering
// Internal ids ordered by in-degree class (the bins above), highest class
// first and original order within a class: the most probed targets then
// share cache lines.  One block per chunk of kBlock vertices; the position
// of vertex v is the exclusive prefix, over (class descending, chunk), of the
// class counts, plus v's rank among the chunk's vertices of its class.
// Counts are stored class-major: counts[(kDegBins - 1 - class) * nch + chunk].
__global__ void k_class_counts(int32_t n, const uint32_t *__restrict__ indeg, int64_t nch, uint32_t *counts) {
    __shared__ uint32_t s_cnt[kDegBins];
    for (int i = threadIdx.x; i < kDegBins; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x;
    if (v < n) atomicAdd(&s_cnt[degree_bin(indeg[v])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kDegBins; i += blockDim.x)
        counts[(int64_t)(kDegBins - 1 - i) * nch + blockIdx.x] = s_cnt[i];
}

__global__ void k_class_scatter(int32_t n, const uint32_t *__restrict__ indeg, int64_t nch,
                                const uint32_t *__restrict__ offs, int32_t *new_of, int32_t *orig_of) {
    __shared__ uint32_t s_w[kWarps][kDegBins];   // per warp: vertices of each class
    for (int i = threadIdx.x; i < kWarps * kDegBins; i += blockDim.x) (&s_w[0][0])[i] = 0;
    __syncthreads();
    const int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x;
    const int wid = threadIdx.x >> 5;
    const bool valid = v < n;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    int c = 0;
    unsigned rank = 0;
    if (valid) {
        c = degree_bin(indeg[v]);
        const unsigned peers = __match_any_sync(act, c);
        rank = __popc(peers & ((1u << lane_id()) - 1u));
        if (rank == 0) s_w[wid][c] = __popc(peers);
    }
    __syncthreads();
    if (valid) {
        uint32_t base = offs[(int64_t)(kDegBins - 1 - c) * nch + blockIdx.x] + rank;
        for (int w = 0; w < wid; w++) base += s_w[w][c];
        new_of[v] = (int32_t)base;
        orig_of[base] = (int32_t)v;
    }
}

// A renumbered graph's CSR, scattered from the original edge list: the
// cursors are indexed by original id (cursor[x] = row_off[new_of[x]]), so the
// atomics land where they would without renumbering -- spread over the ids --
// and not on the adjacent counters of the hubs, which renumbering puts first.
__global__ void k_cursor_of_orig(int32_t n, const uint32_t *__restrict__ ro, const int32_t *__restrict__ new_of,
                                 uint32_t *cursor) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        cursor[x] = ro[new_of[x]];
}
__global__ void k_scatter_coo_renum(int64_t m, const int32_t *__restrict__ s, const int32_t *__restrict__ d,
                                    const int32_t *__restrict__ w, const int32_t *__restrict__ new_of,
                                    uint32_t *cursor, int32_t *col, int32_t *wout) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pos = atomicAdd(&cursor[s[e]], 1u);
        col[pos] = new_of[d[e]];
        wout[pos] = w ? w[e] : 1;
    }
}

// out[new_of[v]] = in[v]
__global__ void k_permute_u32(int32_t n, const uint32_t *__restrict__ in, const int32_t *__restrict__ new_of,
                              uint32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[new_of[v]] = in[v];
}

// Transposed CSR: every edge u->v stored at v's in-edge list as (u, w).
__global__ void k_scatter_transpose(int64_t m, const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                    const int32_t *__restrict__ w, uint32_t *cursor, int32_t *tcol, int32_t *tw) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t pos = atomicAdd(&cursor[dst[e]], 1u);
        tcol[pos] = src[e];
        tw[pos] = w[e];
    }
}

__global__ void k_offsets_to_u32(int32_t n, const int64_t *__restrict__ ro, uint32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
         v += (int64_t)gridDim.x * blockDim.x)
        out[v] = (uint32_t)ro[v];
}

__global__ void k_fill_ones(int64_t m, int32_t *w) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        w[e] = 1;
}

// src[e] = owner row of edge e, one warp per vertex.
__global__ void k_src_from_rows(int32_t n, const uint32_t *__restrict__ ro, int32_t *src) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        uint32_t b = ro[v], e = ro[v + 1];
        for (uint32_t k = b + lane_id(); k < e; k += 32) src[k] = (int32_t)v;
    }
}

// symmetrised degree = out-degree + in-degree
__global__ void k_sym_degree(int32_t n, const uint32_t *__restrict__ ro, uint32_t *deg) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        deg[v] += ro[v + 1] - ro[v];
}

// Symmetrised adjacency of u: its out-edges first, in CSR order (their
// positions follow from the offsets, written coalesced), then its in-edges
// (placed by an atomic cursor that starts after the out-edges).
__global__ void k_sym_cursor(int32_t n, const uint32_t *__restrict__ sro, const uint32_t *__restrict__ ro,
                             uint32_t *cursor) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        cursor[v] = sro[v] + (ro[v + 1] - ro[v]);
}

// Renumbered graphs: as k_scatter_sym, but the in-edge cursors are indexed by
// original id (cursor[x] for x = orig_of[v]), so that the atomics of the
// hubs' in-edges, which renumbering makes adjacent, spread over the ids; the
// edges are still taken in CSR order, so each in-edge list stays ordered by
// source roughly as without renumbering.
__global__ void k_sym_cursor_orig(int32_t n, const uint32_t *__restrict__ sro, const uint32_t *__restrict__ ro,
                                  const int32_t *__restrict__ new_of, uint32_t *cursor) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = new_of[x];
        cursor[x] = sro[u] + (ro[u + 1] - ro[u]);
    }
}
__global__ void k_scatter_sym_renum(int64_t m, const int32_t *__restrict__ src, const int32_t *__restrict__ col,
                                    const uint32_t *__restrict__ ro, const uint32_t *__restrict__ sro,
                                    const int32_t *__restrict__ orig_of, uint32_t *cursor, int32_t *scol) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = col[e];
        scol[sro[u] + ((uint32_t)e - ro[u])] = v;
        const uint32_t q = atomicAdd(&cursor[orig_of[v]], 1u);
        scol[q] = u;
    }
}

__global__ void k_scatter_sym(int64_t m, const int32_t *__restrict__ src, const int32_t *__restrict__ col,
                              const uint32_t *__restrict__ ro, const uint32_t *__restrict__ sro, uint32_t *cursor,
                              int32_t *scol) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = col[e];
        scol[sro[u] + ((uint32_t)e - ro[u])] = v;
        const uint32_t q = atomicAdd(&cursor[v], 1u);
        scol[q] = u;
    }
}

// ---------------------------------------------------------------- scan
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *total) {
    __shared__ uint32_t warp_tot[kWarps];
    uint32_t inc = warp_inclusive_scan(x);
    int wid = threadIdx.x >> 5;
    if (lane_id() == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane_id() < kWarps ? warp_tot[lane_id()] : 0;
        uint32_t ti = warp_inclusive_scan(t);
        if (lane_id() < kWarps) warp_tot[lane_id()] = ti - t;
        if (lane_id() == kWarps - 1) *total = ti;
    }
    __syncthreads();
    uint32_t r = warp_tot[wid] + inc - x;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(int64_t len, const uint32_t *__restrict__ in, uint32_t *bsum) {
    int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * (int64_t)kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < len) s += in[base + i];
    __shared__ uint32_t tot;
    block_exclusive_scan(s, &tot);
    __syncthreads();
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(int64_t len, const uint32_t *__restrict__ in, const uint32_t *__restrict__ boff,
                             uint32_t *out) {
    int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * (int64_t)kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = (base + i < len) ? in[base + i] : 0u;
        s += v[i];
    }
    __shared__ uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + (boff ? boff[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < len) out[base + i] = run;
        run += v[i];
    }
    if (base <= len - 1 && len - 1 < base + kScanItems) out[len] = run;   // owner of the last item
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

// out[0..len] = exclusive prefix sums of in[0..len), out[len] = total (uint32).
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, int64_t len, cudaStream_t st) {
    if (len <= 0) {
        k_set_u32<<<1, 1, 0, st>>>(out, 0u);
        count_launch();
        return cudaGetLastError();
    }
    int64_t nb = (len + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_apply<<<1, kBlock, 0, st>>>(len, in, nullptr, out);
        count_launch();
        return cudaGetLastError();
    }
    uint32_t *bsum = nullptr, *boff = nullptr;
    cudaError_t e = cudaMallocAsync(&bsum, nb * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&boff, (nb + 1) * sizeof(uint32_t), st);
    if (e != cudaSuccess) { cudaFreeAsync(bsum, st); return e; }
    k_scan_reduce<<<(unsigned)nb, kBlock, 0, st>>>(len, in, bsum);
    count_launch();
    e = exclusive_scan(bsum, boff, nb, st);
    if (e == cudaSuccess) {
        k_scan_apply<<<(unsigned)nb, kBlock, 0, st>>>(len, in, boff, out);
        count_launch();
        e = cudaGetLastError();
    }
    cudaFreeAsync(bsum, st);
    cudaFreeAsync(boff, st);
    return e;
}

// ---------------------------------------------------------------- buckets
__global__ void k_bucket_counts(int32_t n, const uint32_t *__restrict__ ro, uint32_t *f_low,
                                uint32_t *f_mid, uint32_t *f_high, uint32_t *f_chunks, uint32_t *f_nz,
                                uint32_t *f_zero, int *max_deg) {
    int mx = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t d = ro[v + 1] - ro[v];
        f_low[v] = (d >= 1 && d < (uint32_t)kLowMax);
        f_mid[v] = (d >= (uint32_t)kLowMax && d < (uint32_t)kMidMax);
        f_high[v] = (d >= (uint32_t)kMidMax);
        f_chunks[v] = d >= (uint32_t)kMidMax ? (d + kChunk - 1) / kChunk : 0u;
        f_nz[v] = (d >= 1);
        f_zero[v] = (d == 0);
        mx = max(mx, (int)min(d, (uint32_t)INT32_MAX));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane_id() == 0) atomicMax(max_deg, mx);
}

__global__ void k_vertex_class(int32_t n, const uint32_t *__restrict__ ro, uint8_t *cls) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t d = ro[v + 1] - ro[v];
        cls[v] = d == 0 ? 0 : d < (uint32_t)kLowMax ? 1 : d < (uint32_t)kMidMax ? 2 : 3;
    }
}

__global__ void k_bucket_write(int32_t n, const uint32_t *__restrict__ ro, const uint32_t *p_low,
                               const uint32_t *p_mid, const uint32_t *p_chunks, const uint32_t *p_nz,
                               const uint32_t *p_zero, int32_t *low, int32_t *mid, int2 *high, int32_t *nz,
                               int32_t *zero) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = ro[v], d = ro[v + 1] - b;
        if (d == 0) {
            zero[p_zero[v]] = (int32_t)v;
            continue;
        }
        nz[p_nz[v]] = (int32_t)v;
        if (d < (uint32_t)kLowMax) {
            low[p_low[v]] = (int32_t)v;
        } else if (d < (uint32_t)kMidMax) {
            mid[p_mid[v]] = (int32_t)v;
        } else {
            uint32_t c0 = p_chunks[v];
            for (uint32_t k = 0; k * (uint32_t)kChunk < d; k++)
                high[c0 + k] = make_int2((int32_t)v, (int32_t)(b + k * (uint32_t)kChunk));
        }
    }
}

// RAII-free allocation helper recording into the graph for destroy
struct Builder {
    fg_graph *g;
    cudaStream_t st;
    fg_status status = FG_OK;
    std::string msg;

    template <typename T>
    T *alloc_graph(int64_t count) {
        if (status != FG_OK) return nullptr;
        void *p = nullptr;
        size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            status = (e == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
            msg = std::string("device allocation failed: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return nullptr;
        }
        if (g->n_allocs >= (int)(sizeof(g->allocs) / sizeof(g->allocs[0]))) {
            cudaFreeAsync(p, st);
            status = FG_ERR_CUDA;
            msg = "internal error: too many graph arrays";
            return nullptr;
        }
        g->allocs[g->n_allocs++] = p;
        g->info.device_bytes += (int64_t)bytes;
        return (T *)p;
    }
    template <typename T>
    T *alloc_tmp(int64_t count) {
        if (status != FG_OK) return nullptr;
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, (size_t)std::max<int64_t>(count, 1) * sizeof(T), st);
        if (e != cudaSuccess) {
            status = (e == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
            msg = std::string("device allocation failed: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return nullptr;
        }
        return (T *)p;
    }
    bool check(cudaError_t e, const char *what) {
        if (status != FG_OK) return false;
        if (e != cudaSuccess) {
            status = (e == cudaErrorMemoryAllocation) ? FG_ERR_OUT_OF_MEMORY : FG_ERR_CUDA;
            msg = std::string(what) + ": " + cudaGetErrorString(e);
            cudaGetLastError();
            return false;
        }
        return true;
    }
};

// Degree buckets of one view (row offsets already set).
void make_buckets(Builder &b, View &v) {
    int32_t n = v.n;
    uint32_t *f = b.alloc_tmp<uint32_t>(6 * (int64_t)n);
    uint32_t *p = b.alloc_tmp<uint32_t>(6 * ((int64_t)n + 1));
    int *mx = b.alloc_tmp<int>(1);
    if (b.status != FG_OK) return;
    b.check(cudaMemsetAsync(mx, 0, sizeof(int), b.st), "memset");
    uint32_t *f_low = f, *f_mid = f + n, *f_high = f + 2 * (int64_t)n, *f_chunks = f + 3 * (int64_t)n,
             *f_nz = f + 4 * (int64_t)n, *f_zero = f + 5 * (int64_t)n;
    int64_t pn = (int64_t)n + 1;
    uint32_t *p_low = p, *p_mid = p + pn, *p_high = p + 2 * pn, *p_chunks = p + 3 * pn, *p_nz = p + 4 * pn,
             *p_zero = p + 5 * pn;
    k_bucket_counts<<<grid_for(n), kBlock, 0, b.st>>>(n, v.row_off, f_low, f_mid, f_high, f_chunks, f_nz,
                                                      f_zero, mx);
    count_launch();
    b.check(cudaGetLastError(), "bucket counts");
    b.check(exclusive_scan(f_low, p_low, n, b.st), "scan");
    b.check(exclusive_scan(f_mid, p_mid, n, b.st), "scan");
    b.check(exclusive_scan(f_high, p_high, n, b.st), "scan");
    b.check(exclusive_scan(f_chunks, p_chunks, n, b.st), "scan");
    b.check(exclusive_scan(f_nz, p_nz, n, b.st), "scan");
    b.check(exclusive_scan(f_zero, p_zero, n, b.st), "scan");
    uint32_t tot[6];
    int mxh = 0;
    if (b.status != FG_OK) return;
    for (int i = 0; i < 6; i++)
        b.check(cudaMemcpyAsync(&tot[i], p + i * pn + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, b.st), "copy");
    b.check(cudaMemcpyAsync(&mxh, mx, sizeof(int), cudaMemcpyDeviceToHost, b.st), "copy");
    b.check(cudaStreamSynchronize(b.st), "sync");
    if (b.status != FG_OK) return;
    v.n_low = (int32_t)tot[0];
    v.n_mid = (int32_t)tot[1];
    v.n_high = (int32_t)tot[2];
    v.n_high_chunks = (int32_t)tot[3];
    v.n_nz = (int32_t)tot[4];
    v.n_zero = (int32_t)tot[5];
    v.max_deg = mxh;
    int32_t *low = b.alloc_graph<int32_t>(v.n_low);
    int32_t *mid = b.alloc_graph<int32_t>(v.n_mid);
    int2 *high = b.alloc_graph<int2>(v.n_high_chunks);
    int32_t *nz = b.alloc_graph<int32_t>(v.n_nz);
    int32_t *zero = b.alloc_graph<int32_t>(v.n_zero);
    uint8_t *vclass = b.alloc_graph<uint8_t>(n);
    if (b.status != FG_OK) return;
    k_vertex_class<<<grid_for(n), kBlock, 0, b.st>>>(n, v.row_off, vclass);
    count_launch();
    k_bucket_write<<<grid_for(n), kBlock, 0, b.st>>>(n, v.row_off, p_low, p_mid, p_chunks, p_nz, p_zero, low,
                                                     mid, high, nz, zero);
    count_launch();
    b.check(cudaGetLastError(), "bucket write");
    v.low = low;
    v.mid = mid;
    v.high = high;
    v.nz = nz;
    v.zero = zero;
    v.vclass = vclass;
    cudaFreeAsync(f, b.st);
    cudaFreeAsync(p, b.st);
    cudaFreeAsync(mx, b.st);
    // the edge stream's bulk copies need the arrays 16-byte aligned, which
    // device allocations are
    if ((((uintptr_t)v.src | (uintptr_t)v.col | (uintptr_t)v.w) & 15u) != 0) {
        b.status = FG_ERR_CUDA;
        b.msg = "internal error: edge arrays not 16-byte aligned";
    }
}

template <typename T>
const T *to_device(Builder &b, const T *p, int64_t count, T **tmp) {
    *tmp = nullptr;
    if (count == 0 || p == nullptr) return p;
    if (is_device_pointer(p)) return p;
    T *d = b.alloc_tmp<T>(count);
    if (!d) return nullptr;
    b.check(cudaMemcpyAsync(d, p, (size_t)count * sizeof(T), cudaMemcpyHostToDevice, b.st), "copy to device");
    *tmp = d;
    return d;
}

// The source of every CSR edge: with col and w it forms the source-sorted
// COO that the edge-based modes stream (Sec. 3.1); also read by the
// transposed view's build and the SSSP overflow check.
void build_src(Builder &b, View &v) {
    int32_t *esrc = b.alloc_graph<int32_t>(v.m);
    if (b.status == FG_OK && v.m > 0) {
        k_src_from_rows<<<grid_for((int64_t)v.n * 32), kBlock, 0, b.st>>>(v.n, v.row_off, esrc);
        count_launch();
        b.check(cudaGetLastError(), "edge sources");
    }
    if ((uintptr_t)esrc & 15u) {   // the edge stream's bulk copies need 16-byte alignment
        b.status = FG_ERR_CUDA;
        b.msg = "internal error: edge sources not 16-byte aligned";
    }
    v.src = esrc;
}

// The symmetrised view used by connected components: every edge u->v also
// stored as v->u (the undirected nbrs iterator, Table "foreach iterators"),
// as CSR plus edge sources.  Needs the directed view's edge sources.
// indeg: the in-degrees counted at creation (else counted here)
void build_sym(Builder &b, fg_graph *g, const uint32_t *indeg = nullptr) {
    const View &v = g->g;
    const int32_t n = v.n;
    const int64_t m = v.m;
    View &s = g->s;
    s.n = n;
    s.m = 2 * m;
    uint32_t *sro = b.alloc_graph<uint32_t>((int64_t)n + 1);
    int32_t *scol = b.alloc_graph<int32_t>(2 * m);
    int32_t *ssrc = b.alloc_graph<int32_t>(2 * m);
    if (b.status == FG_OK) {
        uint32_t *deg = b.alloc_tmp<uint32_t>(n);
        uint32_t *cursor = b.alloc_tmp<uint32_t>((int64_t)n + 1);
        if (b.status == FG_OK) {
            if (indeg) {   // the in-degrees counted at creation
                b.check(cudaMemcpyAsync(deg, indeg, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b.st),
                        "copy");
            } else {
                b.check(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(uint32_t), b.st), "memset");
                if (m > 0) { k_histogram<<<grid_for(m), kBlock, 0, b.st>>>(m, v.col, deg); count_launch(); }
            }
            k_sym_degree<<<grid_for(n), kBlock, 0, b.st>>>(n, v.row_off, deg);
            count_launch();
            b.check(exclusive_scan(deg, sro, n, b.st), "scan");
            if (g->new_of) {
                k_sym_cursor_orig<<<grid_for(n), kBlock, 0, b.st>>>(n, sro, v.row_off, g->new_of, cursor);
                count_launch();
            } else {
                k_sym_cursor<<<grid_for(n), kBlock, 0, b.st>>>(n, sro, v.row_off, cursor);
                count_launch();
            }
            if (m > 0) {
                if (g->new_of) {
                    k_scatter_sym_renum<<<grid_for(m), kBlock, 0, b.st>>>(m, v.src, v.col, v.row_off, sro,
                                                                          g->orig_of, cursor, scol);
                    count_launch();
                } else {
                    k_scatter_sym<<<grid_for(m), kBlock, 0, b.st>>>(m, v.src, v.col, v.row_off, sro, cursor, scol);
                    count_launch();
                }
                k_src_from_rows<<<grid_for((int64_t)n * 32), kBlock, 0, b.st>>>(n, sro, ssrc);
                count_launch();
            }
            b.check(cudaGetLastError(), "symmetrise");
        }
        if (deg) cudaFreeAsync(deg, b.st);
        if (cursor) cudaFreeAsync(cursor, b.st);
    }
    s.row_off = sro;
    s.col = scol;
    s.w = nullptr;
    s.src = ssrc;
    if (b.status == FG_OK) make_buckets(b, s);
    if (b.status == FG_OK) g->info.n_isolated = s.n_zero;
}

}  // namespace

// Builds a graph from COO (row_off_in == nullptr) or from CSR (row_off_in,
// with src == nullptr and dst == col).
fg_status build_graph_from_coo(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                               const int32_t *w, bool from_csr, const int64_t *row_off_in, uint32_t create_flags,
                               fg_graph **out) {
    fg_graph *g = new (std::nothrow) fg_graph();
    if (!g) return fail(FG_ERR_OUT_OF_MEMORY, "host allocation failed");
    cudaGetDevice(&g->device);
    Builder b{g, (cudaStream_t)0};
    int32_t *t_src = nullptr, *t_dst = nullptr, *t_w = nullptr;
    int64_t *t_ro = nullptr;
    const int32_t *d_src = nullptr;
    const int32_t *d_dst = to_device(b, dst, m, &t_dst);
    const int32_t *d_w = to_device(b, w, m, &t_w);
    const int64_t *d_ro = nullptr;
    if (from_csr) d_ro = to_device(b, row_off_in, (int64_t)n + 1, &t_ro);
    else d_src = to_device(b, src, m, &t_src);
    int *flags = b.alloc_tmp<int>(1);
    if (b.status == FG_OK) {
        b.check(cudaMemsetAsync(flags, 0, sizeof(int), b.st), "memset");
        if (from_csr)
            k_validate_csr<<<grid_for(std::max<int64_t>(m, n)), kBlock, 0, b.st>>>(n, m, d_ro, d_dst, d_w, flags);
        else if (m > 0)
            k_validate_coo<<<grid_for(m), kBlock, 0, b.st>>>(m, n, d_src, d_dst, d_w, flags);
        if (from_csr || m > 0) count_launch();
        b.check(cudaGetLastError(), "validate");
        int hf = 0;
        b.check(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, b.st), "copy");
        b.check(cudaStreamSynchronize(b.st), "sync");
        if (b.status == FG_OK && hf) {
            if (hf & kBadOffsets) { b.status = FG_ERR_INVALID_ARG; b.msg = "row offsets are not a valid CSR (row_off[0]=0, non-decreasing, row_off[n]=m)"; }
            else if (hf & kBadId) { b.status = FG_ERR_INVALID_ARG; b.msg = "a vertex id is outside [0, n)"; }
            else { b.status = FG_ERR_NEGATIVE_WEIGHT; b.msg = "a weight is negative"; }
        }
    }
    // ---- in-degrees (their skew decides the renumbering; the symmetrised
    // view reuses them) and the renumbering itself
    uint32_t *indeg = nullptr;     // in-degrees by internal id
    int32_t *t_csrc = nullptr;
    uint32_t *t_ro32 = nullptr;
    if (b.status == FG_OK && !(create_flags & FG_GRAPH_KEEP_IDS)) {
        indeg = b.alloc_tmp<uint32_t>(n);
        unsigned long long *bins = b.alloc_tmp<unsigned long long>(2 * kDegBins);
        unsigned long long hb[2 * kDegBins] = {};
        if (b.status == FG_OK) {
            b.check(cudaMemsetAsync(indeg, 0, (size_t)n * sizeof(uint32_t), b.st), "memset");
            b.check(cudaMemsetAsync(bins, 0, sizeof(hb), b.st), "memset");
            if (m > 0) { k_histogram<<<grid_for(m), kBlock, 0, b.st>>>(m, d_dst, indeg); count_launch(); }
            k_degree_bins<false><<<grid_for(n), kBlock, 0, b.st>>>(n, indeg, bins, bins + kDegBins);
            count_launch();
            b.check(cudaMemcpyAsync(hb, bins, sizeof(hb), cudaMemcpyDeviceToHost, b.st), "copy");
            b.check(cudaStreamSynchronize(b.st), "in-degrees");
        }
        if (bins) cudaFreeAsync(bins, b.st);
        if (b.status == FG_OK) g->info.in_degree_gini = (float)gini_of_bins(hb, hb + kDegBins);
    }
    const bool relabel = b.status == FG_OK && indeg &&
                         ((create_flags & FG_GRAPH_RELABEL) || g->info.in_degree_gini > kRelabelGini);
    if (relabel) {
        const int64_t nch = ((int64_t)n + kBlock - 1) / kBlock;
        g->new_of = b.alloc_graph<int32_t>(n);
        g->orig_of = b.alloc_graph<int32_t>(n);
        uint32_t *counts = b.alloc_tmp<uint32_t>(kDegBins * nch);
        uint32_t *offs = b.alloc_tmp<uint32_t>(kDegBins * nch + 1);
        uint32_t *pdeg = b.alloc_tmp<uint32_t>(n);
        if (from_csr) {   // the edges' sources, to renumber them as a COO
            t_ro32 = b.alloc_tmp<uint32_t>((int64_t)n + 1);
            t_csrc = b.alloc_tmp<int32_t>(m);
        }
        if (b.status == FG_OK) {
            k_class_counts<<<(unsigned)nch, kBlock, 0, b.st>>>(n, indeg, nch, counts);
            count_launch();
            b.check(exclusive_scan(counts, offs, kDegBins * nch, b.st), "scan");
            k_class_scatter<<<(unsigned)nch, kBlock, 0, b.st>>>(n, indeg, nch, offs, g->new_of, g->orig_of);
            count_launch();
            k_permute_u32<<<grid_for(n), kBlock, 0, b.st>>>(n, indeg, g->new_of, pdeg);
            count_launch();
            if (from_csr) {
                k_offsets_to_u32<<<grid_for((int64_t)n + 1), kBlock, 0, b.st>>>(n, d_ro, t_ro32);
                count_launch();
                if (m > 0) {
                    k_src_from_rows<<<grid_for((int64_t)n * 32), kBlock, 0, b.st>>>(n, t_ro32, t_csrc);
                    count_launch();
                }
                d_src = t_csrc;
                from_csr = false;   // built as a COO from here on
            }
            b.check(cudaGetLastError(), "renumbering");
            std::swap(indeg, pdeg);   // the edges stay in original ids: the scatters renumber them
        }
        if (counts) cudaFreeAsync(counts, b.st);
        if (offs) cudaFreeAsync(offs, b.st);
        if (pdeg) cudaFreeAsync(pdeg, b.st);
        g->info.relabelled = 1;
    }

    View &v = g->g;
    v.n = n;
    v.m = m;
    uint32_t *ro = b.alloc_graph<uint32_t>((int64_t)n + 1);
    int32_t *col = b.alloc_graph<int32_t>(m);
    int32_t *wt = b.alloc_graph<int32_t>(m);
    if (b.status == FG_OK) {
        if (from_csr) {
            k_offsets_to_u32<<<grid_for((int64_t)n + 1), kBlock, 0, b.st>>>(n, d_ro, ro);
            count_launch();
            if (m > 0) {
                b.check(cudaMemcpyAsync(col, d_dst, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, b.st), "copy");
                if (d_w) b.check(cudaMemcpyAsync(wt, d_w, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, b.st), "copy");
                else { k_fill_ones<<<grid_for(m), kBlock, 0, b.st>>>(m, wt); count_launch(); }
            }
        } else {
            uint32_t *cnt = b.alloc_tmp<uint32_t>(n);
            uint32_t *cursor = b.alloc_tmp<uint32_t>((int64_t)n + 1);
            uint32_t *cnt_o = g->new_of ? b.alloc_tmp<uint32_t>(n) : nullptr;
            if (b.status == FG_OK && g->new_of) {   // counted and scattered by original source id
                b.check(cudaMemsetAsync(cnt_o, 0, (size_t)n * sizeof(uint32_t), b.st), "memset");
                if (m > 0) { k_histogram<<<grid_for(m), kBlock, 0, b.st>>>(m, d_src, cnt_o); count_launch(); }
                k_permute_u32<<<grid_for(n), kBlock, 0, b.st>>>(n, cnt_o, g->new_of, cnt);
                count_launch();
                b.check(exclusive_scan(cnt, ro, n, b.st), "scan");
                k_cursor_of_orig<<<grid_for(n), kBlock, 0, b.st>>>(n, ro, g->new_of, cursor);
                count_launch();
                if (m > 0) {
                    k_scatter_coo_renum<<<grid_for(m), kBlock, 0, b.st>>>(m, d_src, d_dst, d_w, g->new_of, cursor,
                                                                          col, wt);
                    count_launch();
                }
                b.check(cudaGetLastError(), "scatter");
            } else if (b.status == FG_OK) {
                b.check(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(uint32_t), b.st), "memset");
                if (m > 0) { k_histogram<<<grid_for(m), kBlock, 0, b.st>>>(m, d_src, cnt); count_launch(); }
                b.check(exclusive_scan(cnt, ro, n, b.st), "scan");
                b.check(cudaMemcpyAsync(cursor, ro, ((size_t)n + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b.st), "copy");
                if (m > 0) {
                    k_scatter_coo<<<grid_for(m), kBlock, 0, b.st>>>(m, d_src, d_dst, d_w, cursor, col, wt);
                    count_launch();
                }
                b.check(cudaGetLastError(), "scatter");
            }
            if (cnt) cudaFreeAsync(cnt, b.st);
            if (cnt_o) cudaFreeAsync(cnt_o, b.st);
            if (cursor) cudaFreeAsync(cursor, b.st);
        }
        b.check(cudaGetLastError(), "csr");
    }
    v.row_off = ro;
    v.col = col;
    v.w = wt;
    v.src = nullptr;
    if (b.status == FG_OK) make_buckets(b, v);
    g->s.n = n;
    g->s.m = 2 * m;
    g->info.n_isolated = -1;
    if (!(create_flags & FG_GRAPH_LAZY)) {
        build_src(b, v);
        build_sym(b, g, indeg);
    }

    if (indeg) cudaFreeAsync(indeg, b.st);
    if (t_csrc) cudaFreeAsync(t_csrc, b.st);
    if (t_ro32) cudaFreeAsync(t_ro32, b.st);
    if (t_src) cudaFreeAsync(t_src, b.st);
    if (t_dst) cudaFreeAsync(t_dst, b.st);
    if (t_w) cudaFreeAsync(t_w, b.st);
    if (t_ro) cudaFreeAsync(t_ro, b.st);
    if (flags) cudaFreeAsync(flags, b.st);
    b.check(cudaStreamSynchronize(b.st), "graph build");
    if (b.status != FG_OK) {
        fg_status st = b.status;
        std::string msg = b.msg;
        for (int i = 0; i < g->n_allocs; i++) cudaFree(g->allocs[i]);
        delete g;
        return fail(st, msg);
    }
    {   // mean weight (the bucket mode's default width) and the degree bins
        // (the selection model's skew measure), in one small allocation
        unsigned long long *d_sum = nullptr, h[1 + 2 * kDegBins] = {};
        cudaError_t e = cudaMalloc(&d_sum, sizeof(h));
        if (e == cudaSuccess) e = cudaMemset(d_sum, 0, sizeof(h));
        if (e == cudaSuccess && m > 0) {
            k_weight_sum<<<grid_for(m), kBlock>>>(m, v.w, d_sum);
            count_launch();
        }
        if (e == cudaSuccess) {
            k_degree_bins<true><<<grid_for(n), kBlock>>>(n, v.row_off, d_sum + 1, d_sum + 1 + kDegBins);
            count_launch();
            e = cudaMemcpy(h, d_sum, sizeof(h), cudaMemcpyDeviceToHost);
        }
        if (d_sum) cudaFree(d_sum);
        if (e != cudaSuccess) {
            for (int i = 0; i < g->n_allocs; i++) cudaFree(g->allocs[i]);
            delete g;
            return cuda_fail(e, "graph statistics");
        }
        if (m > 0) g->w_mean = (double)h[0] / (double)m;
        g->degree_gini = gini_of_bins(h + 1, h + 1 + kDegBins);
    }
    fg_graph_info_t &I = g->info;
    I.n = n;
    I.m = m;
    I.m_sym = 2 * m;
    I.max_out_degree = v.max_deg;
    I.n_zero_out = n - v.n_nz;
    I.n_low = v.n_low;
    I.n_mid = v.n_mid;
    I.n_high = v.n_high;
    I.n_high_chunks = v.n_high_chunks;
    *out = g;
    return FG_OK;
}

// The transposed view of the directed graph (in-neighbours with their
// weights, bucketed by in-degree), built once on the first pull query and
// kept with the graph.  Thread-safe: callers hold no lock.
namespace {

// Lazily built parts of a graph created with FG_GRAPH_LAZY; the caller holds
// the graph's lock.  Arrays of a failed build stay with the graph (freed by
// fg_graph_destroy) and the part is built again on the next use.
fg_status ensure_src_locked(fg_graph *g) {
    if (g->g.src) return FG_OK;
    Builder b{g, (cudaStream_t)0};
    View v = g->g;
    build_src(b, v);
    b.check(cudaStreamSynchronize(b.st), "edge sources");
    if (b.status != FG_OK) return fail(b.status, b.msg);
    g->g.src = v.src;
    return FG_OK;
}

fg_status ensure_sym_locked(fg_graph *g) {
    if (g->s.row_off) return FG_OK;
    fg_status st = ensure_src_locked(g);
    if (st != FG_OK) return st;
    Builder b{g, (cudaStream_t)0};
    build_sym(b, g);
    b.check(cudaStreamSynchronize(b.st), "symmetrised view");
    if (b.status != FG_OK) {
        g->s.row_off = nullptr;   // built again on the next use
        return fail(b.status, b.msg);
    }
    return FG_OK;
}

}  // namespace

fg_status ensure_views(const fg_graph *cg, Algo algo, int mode) {
    fg_graph *g = const_cast<fg_graph *>(cg);
    if (algo != kCC && mode == kPull) return ensure_transpose(cg);
    std::lock_guard<std::mutex> lk(g->mu);
    if (algo == kCC) return ensure_sym_locked(g);
    if (mode == kEdgeSync || mode == kEdgeAsync || mode < 0) return ensure_src_locked(g);
    return FG_OK;
}

fg_status ensure_src(const fg_graph *cg) {
    fg_graph *g = const_cast<fg_graph *>(cg);
    std::lock_guard<std::mutex> lk(g->mu);
    return ensure_src_locked(g);
}

fg_status ensure_transpose(const fg_graph *cg) {
    fg_graph *g = const_cast<fg_graph *>(cg);
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->t_ready) return FG_OK;
    fg_status sst = ensure_src_locked(g);
    if (sst != FG_OK) return sst;
    const View &v = g->g;
    const int32_t n = v.n;
    const int64_t m = v.m;
    Builder b{g, (cudaStream_t)0};
    uint32_t *tro = b.alloc_graph<uint32_t>((int64_t)n + 1);
    int32_t *tcol = b.alloc_graph<int32_t>(m);
    int32_t *tw = b.alloc_graph<int32_t>(m);
    uint32_t *cnt = b.alloc_tmp<uint32_t>(n);
    uint32_t *cursor = b.alloc_tmp<uint32_t>((int64_t)n + 1);
    if (b.status == FG_OK) {
        b.check(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(uint32_t), b.st), "memset");
        if (m > 0) { k_histogram<<<grid_for(m), kBlock, 0, b.st>>>(m, v.col, cnt); count_launch(); }
        b.check(exclusive_scan(cnt, tro, n, b.st), "scan");
        b.check(cudaMemcpyAsync(cursor, tro, ((size_t)n + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b.st), "copy");
        if (m > 0) { k_scatter_transpose<<<grid_for(m), kBlock, 0, b.st>>>(m, v.src, v.col, v.w, cursor, tcol, tw); count_launch(); }
        b.check(cudaGetLastError(), "transpose");
    }
    if (cnt) cudaFreeAsync(cnt, b.st);
    if (cursor) cudaFreeAsync(cursor, b.st);
    View t;
    t.n = n;
    t.m = m;
    t.row_off = tro;
    t.col = tcol;
    t.w = tw;
    if (b.status == FG_OK) make_buckets(b, t);
    b.check(cudaStreamSynchronize(b.st), "transpose build");
    if (b.status != FG_OK) return fail(b.status, b.msg);
    g->t = t;
    g->t_ready = true;
    return FG_OK;
}

}  // namespace fg
