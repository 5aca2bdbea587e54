/*
 * Seeded synthetic graph generators shared by the tests, the benchmark and
 * the oracle runs.  They hold none of the relaxation arithmetic: they only
 * draw edge lists, weights and source vertices.
 *
 * Every random number is a pure function of (seed, stream, counter): the
 * i-th output of the splitmix64 sequence started at seed + stream salt
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014; constants as published by Vigna).  The arrays are therefore
 * identical on every machine and for every thread count.
 *
 * Shapes (they stand in for the paper's graph classes, Table "Benchmark
 * characteristics", Sec. 4.1):
 *   - G(n,m) Erdos-Renyi: directed, no self-loops, no duplicates ("rand").
 *   - R-MAT: recursive quadrant choice with (a,b,c,d) per bit, no noise,
 *     self-loops and duplicates kept ("rmat" and the social graphs).
 *   - 2-D grid, 4-neighbour, symmetric, with random pair deletions and
 *     random long-range shortcut pairs ("USA road": low degree, high
 *     diameter).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

/* i-th output (i = 0, 1, ...) of the splitmix64 stream whose state starts at s. */
static inline uint64_t gg_draw(uint64_t s, uint64_t i) {
    uint64_t z = s + (i + 1) * GG_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Stream salts: one independent stream per purpose. */
static inline uint64_t gg_stream(uint64_t seed, uint64_t salt) {
    return gg_draw(seed, salt) ^ (salt * 0xD1B54A32D192ED03ULL);
}

/* Uniform integer in [lo, hi] (hi - lo < 2^32) by multiply-high. */
static inline int32_t gg_uniform_int(uint64_t x, int64_t lo, int64_t hi) {
    uint64_t range = (uint64_t)(hi - lo + 1);
    return (int32_t)(lo + (int64_t)(((x >> 32) * range) >> 32));
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double gg_unit(uint64_t x) {
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

enum { SALT_ER_PAIR = 1, SALT_ER_W = 2, SALT_RMAT = 3, SALT_GRID_DEL = 4,
       SALT_GRID_W = 5, SALT_GRID_SC = 6, SALT_GRID_SCW = 7, SALT_SRC = 8,
       SALT_PERM = 9 };

/*
 * G(n, m): draw (u, v) uniformly and independently; reject u == v and pairs
 * already drawn, and draw again.  Weights uniform in [wlo, whi].
 * Returns the number of draws made, or -1 if m is impossible.
 */
int64_t gg_er(int32_t n, int64_t m, uint64_t seed, int32_t wlo, int32_t whi,
              int32_t *src, int32_t *dst, int32_t *w) {
    if (n < 2 || m < 0 || (double)m > (double)n * (double)(n - 1)) return -1;
    uint64_t sp = gg_stream(seed, SALT_ER_PAIR), sw = gg_stream(seed, SALT_ER_W);
    uint64_t cap = 1;
    while (cap < 2 * (uint64_t)m + 16) cap <<= 1;
    uint64_t *table = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!table) return -1;
    memset(table, 0xff, cap * sizeof(uint64_t));
    int64_t k = 0;
    uint64_t i = 0;
    while (k < m) {
        int32_t u = gg_uniform_int(gg_draw(sp, 2 * i), 0, n - 1);
        int32_t v = gg_uniform_int(gg_draw(sp, 2 * i + 1), 0, n - 1);
        i++;
        if (u == v) continue;
        uint64_t key = (uint64_t)u * (uint64_t)n + (uint64_t)v;
        uint64_t h = (key * GG_GAMMA) & (cap - 1);
        int dup = 0;
        while (table[h] != ~0ULL) {
            if (table[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        table[h] = key;
        src[k] = u;
        dst[k] = v;
        w[k] = gg_uniform_int(gg_draw(sw, (uint64_t)k), wlo, whi);
        k++;
    }
    free(table);
    return (int64_t)i;
}

/*
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each edge picks one of
 * four quadrants per bit of the vertex id, most significant bit first, with
 * probabilities a, b, c and d = 1 - a - b - c.  No noise.  Self-loops and
 * duplicates are kept.  Draw counter e*64 + level for edge e; the weight
 * uses counter e*64 + 63.  If perm_seed != 0, vertex ids are relabelled by
 * a seeded Fisher-Yates permutation (Graph500-style).
 */
void gg_rmat(int32_t scale, int64_t m, double a, double b, double c, uint64_t seed,
             int32_t wlo, int32_t whi, uint64_t perm_seed,
             int32_t *src, int32_t *dst, int32_t *w) {
    uint64_t s = gg_stream(seed, SALT_RMAT);
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint32_t u = 0, v = 0;
        uint64_t base = (uint64_t)e * 64;
        for (int l = 0; l < scale; l++) {
            double r = gg_unit(gg_draw(s, base + (uint64_t)l));
            uint32_t row = 0, col = 0;
            if (r < a) { row = 0; col = 0; }
            else if (r < ab) { row = 0; col = 1; }
            else if (r < abc) { row = 1; col = 0; }
            else { row = 1; col = 1; }
            u = (u << 1) | row;
            v = (v << 1) | col;
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
        w[e] = gg_uniform_int(gg_draw(s, base + 63), wlo, whi);
    }
    if (perm_seed) {
        int64_t n = (int64_t)1 << scale;
        int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        if (!perm) return;
        uint64_t sp = gg_stream(perm_seed, SALT_PERM);
        for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
        for (int64_t i = n - 1; i > 0; i--) {
            int64_t j = gg_uniform_int(gg_draw(sp, (uint64_t)i), 0, i);
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < m; e++) {
            src[e] = perm[src[e]];
            dst[e] = perm[dst[e]];
        }
        free(perm);
    }
}

/*
 * side x side grid, vertex id = r*side + c.  Undirected neighbour pairs are
 * numbered: horizontal (r,c)-(r,c+1) as r*(side-1)+c, then vertical
 * (r,c)-(r+1,c) as side*(side-1) + r*side + c.  Each pair is deleted with
 * probability p_del (both directions go).  Then n_short undirected shortcut
 * pairs (u, v), u uniform, v uniform among the other vertices, are added.
 * Every directed edge gets its own weight in [wlo, whi].
 * Output: kept pairs in pair order, each as (lo->hi, hi->lo), then the
 * shortcut pairs the same way.  Returns the number of directed edges, or -1
 * if the buffers (capacity cap) are too small.
 */
int64_t gg_grid(int32_t side, double p_del, int64_t n_short, uint64_t seed,
                int32_t wlo, int32_t whi, int64_t cap,
                int32_t *src, int32_t *dst, int32_t *w) {
    uint64_t sd = gg_stream(seed, SALT_GRID_DEL), sw = gg_stream(seed, SALT_GRID_W);
    uint64_t ss = gg_stream(seed, SALT_GRID_SC), ssw = gg_stream(seed, SALT_GRID_SCW);
    int64_t n = (int64_t)side * side;
    int64_t hpairs = (int64_t)side * (side - 1);
    int64_t npairs = 2 * hpairs;
    int64_t k = 0;
    for (int64_t p = 0; p < npairs; p++) {
        if (p_del > 0.0 && gg_unit(gg_draw(sd, (uint64_t)p)) < p_del) continue;
        int64_t u, v;
        if (p < hpairs) {
            int64_t r = p / (side - 1), c = p % (side - 1);
            u = r * side + c;
            v = u + 1;
        } else {
            int64_t q = p - hpairs;
            u = q;            /* (r, c) with r < side-1 */
            v = q + side;
        }
        if (k + 2 > cap) return -1;
        src[k] = (int32_t)u; dst[k] = (int32_t)v;
        w[k] = gg_uniform_int(gg_draw(sw, 2 * (uint64_t)p), wlo, whi);
        k++;
        src[k] = (int32_t)v; dst[k] = (int32_t)u;
        w[k] = gg_uniform_int(gg_draw(sw, 2 * (uint64_t)p + 1), wlo, whi);
        k++;
    }
    for (int64_t s = 0; s < n_short; s++) {
        int64_t u = gg_uniform_int(gg_draw(ss, 2 * (uint64_t)s), 0, n - 1);
        int64_t d = gg_uniform_int(gg_draw(ss, 2 * (uint64_t)s + 1), 1, n - 1);
        int64_t v = (u + d) % n;
        if (k + 2 > cap) return -1;
        src[k] = (int32_t)u; dst[k] = (int32_t)v;
        w[k] = gg_uniform_int(gg_draw(ssw, 2 * (uint64_t)s), wlo, whi);
        k++;
        src[k] = (int32_t)v; dst[k] = (int32_t)u;
        w[k] = gg_uniform_int(gg_draw(ssw, 2 * (uint64_t)s + 1), wlo, whi);
        k++;
    }
    return k;
}

/*
 * k distinct source vertices drawn uniformly from the vertices with
 * out-degree > 0 (draw, reject zero out-degree and repeats).  Returns the
 * number found (< k only if fewer such vertices exist).
 */
int32_t gg_sources(int32_t n, int64_t m, const int32_t *src, int32_t k, uint64_t seed,
                   int32_t *out) {
    uint8_t *has_out = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
    if (!has_out || !taken) { free(has_out); free(taken); return -1; }
    int64_t avail = 0;
    for (int64_t e = 0; e < m; e++) {
        if (src[e] >= 0 && src[e] < n && !has_out[src[e]]) { has_out[src[e]] = 1; avail++; }
    }
    if (avail < k) k = (int32_t)avail;
    uint64_t s = gg_stream(seed, SALT_SRC);
    int32_t got = 0;
    for (uint64_t i = 0; got < k; i++) {
        int32_t v = gg_uniform_int(gg_draw(s, i), 0, n - 1);
        if (!has_out[v] || taken[v]) continue;
        taken[v] = 1;
        out[got++] = v;
    }
    free(has_out);
    free(taken);
    return got;
}

/* Raw stream access, for tests of the generator itself. */
uint64_t gg_splitmix64(uint64_t state, uint64_t i) { return gg_draw(state, i); }
