/*
 * Seeded synthetic graph generators for the BGPC / D2GC workloads.
 *
 * This module builds inputs only: it holds none of the coloring method's
 * arithmetic and is shared by the CPU oracle's tests, the GPU tests and the
 * benchmark.  Every random draw comes from a counter-based generator, so a
 * graph depends only on (generator, parameters, seed) and not on the number
 * of OpenMP threads that built it.
 *
 * Counter-based generator: the SplitMix64 finaliser (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014; constants
 * as published by Vigna for splitmix64) applied to seed + counter * golden
 * gamma.  Integer-only generators (random bipartite, stencil, R-MAT) give the
 * same graph on every platform; the Chung-Lu weights and the batch sizes go
 * through libm (pow/exp/log), whose last bit may differ between platforms.
 *
 * Output format: int32 CSR over V_A (a_ptr, a_idx = nets(u)) and int32 CSC
 * over V_B (b_ptr, b_idx = vtxs(v)); both sorted by id, no duplicates.  The
 * undirected generators return a symmetric CSR without self loops in a_*,
 * and b_* aliases it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int64_t n_a, n_b, nnz;
    int32_t *a_ptr, *a_idx, *b_ptr, *b_idx;
    int undirected;
} gg_graph;

/* ---------------------------------------------------------------- PRNG -- */

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Value number `ctr` of stream `stream` under `seed`. */
static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t s = sm64_mix(seed * 0x9E3779B97F4A7C15ULL + stream + 1ULL);
    return sm64_mix(s + (ctr + 1ULL) * 0x9E3779B97F4A7C15ULL);
}

/* Uniform integer in [0, n) by the multiply-high method. */
static inline uint64_t below(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unif(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------- radix sort u64 -- */

static void radix_sort_u64(uint64_t *a, int64_t n, int key_bits) {
    if (n <= 1) return;
    uint64_t *tmp = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    const int RB = 11, R = 1 << RB;
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * R);
    uint64_t *src = a, *dst = tmp;
    for (int shift = 0; shift < key_bits; shift += RB) {
        memset(cnt, 0, sizeof(int64_t) * R);
        for (int64_t i = 0; i < n; i++) cnt[(src[i] >> shift) & (R - 1)]++;
        int64_t s = 0;
        for (int b = 0; b < R; b++) { int64_t c = cnt[b]; cnt[b] = s; s += c; }
        for (int64_t i = 0; i < n; i++) dst[cnt[(src[i] >> shift) & (R - 1)]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
    free(tmp);
    free(cnt);
}

static int64_t dedup_sorted(uint64_t *a, int64_t n) {
    if (n == 0) return 0;
    int64_t m = 1;
    for (int64_t i = 1; i < n; i++)
        if (a[i] != a[m - 1]) a[m++] = a[i];
    return m;
}

static int bits_for(int64_t n) {
    int b = 1;
    while (((int64_t)1 << b) < n) b++;
    return b;
}

/* Build CSR (by a) and CSC (by b) from sorted unique keys (a << sh) | b. */
static gg_graph *from_pairs(uint64_t *keys, int64_t m, int64_t n_a, int64_t n_b, int sh) {
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    g->n_a = n_a; g->n_b = n_b; g->nnz = m;
    g->a_ptr = (int32_t *)calloc((size_t)n_a + 1, sizeof(int32_t));
    g->a_idx = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    g->b_ptr = (int32_t *)calloc((size_t)n_b + 1, sizeof(int32_t));
    g->b_idx = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    uint64_t mask = (sh == 64) ? ~0ULL : ((1ULL << sh) - 1ULL);
    for (int64_t i = 0; i < m; i++) {
        int64_t u = (int64_t)(keys[i] >> sh), v = (int64_t)(keys[i] & mask);
        g->a_ptr[u + 1]++;
        g->b_ptr[v + 1]++;
        g->a_idx[i] = (int32_t)v;
    }
    for (int64_t u = 0; u < n_a; u++) g->a_ptr[u + 1] += g->a_ptr[u];
    for (int64_t v = 0; v < n_b; v++) g->b_ptr[v + 1] += g->b_ptr[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_b ? n_b : 1));
    for (int64_t v = 0; v < n_b; v++) fill[v] = g->b_ptr[v];
    /* keys are sorted by (a, b): scanning in order keeps each vtxs list sorted */
    for (int64_t i = 0; i < m; i++) {
        int64_t u = (int64_t)(keys[i] >> sh), v = (int64_t)(keys[i] & mask);
        g->b_idx[fill[v]++] = (int32_t)u;
    }
    free(fill);
    return g;
}

/* ------------------------------------------------------------ generators -- */

/* Each V_A vertex joins `deg` distinct V_B nets drawn uniformly. */
void *gg_random_bipartite(int32_t n_a, int32_t n_b, int32_t deg, uint64_t seed) {
    if (deg > n_b) deg = n_b;
    int sh = bits_for(n_b);
    int64_t m = (int64_t)n_a * deg;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n_a; u++) {
        int32_t nets[64 * 4];
        int32_t *buf = deg <= 256 ? nets : (int32_t *)malloc(sizeof(int32_t) * deg);
        int got = 0;
        uint64_t ctr = 0;
        while (got < deg) {
            int32_t v = (int32_t)below(rnd(seed, (uint64_t)u, ctr++), (uint64_t)n_b);
            int dup = 0;
            for (int k = 0; k < got; k++) dup |= (buf[k] == v);
            if (!dup) buf[got++] = v;
        }
        for (int k = 0; k < deg; k++) keys[u * deg + k] = ((uint64_t)u << sh) | (uint64_t)buf[k];
        if (buf != nets) free(buf);
    }
    radix_sort_u64(keys, m, sh + bits_for(n_a));
    gg_graph *g = from_pairs(keys, m, n_a, n_b, sh);
    free(keys);
    return g;
}

/* Jacobian pattern of a 9-point stencil on an n x n grid: net (row) r=(i,j)
 * holds the columns (i+di, j+dj), di,dj in {-1,0,1}, inside the grid; ids are
 * row-major (id = i*n + j) on both sides. */
void *gg_stencil9(int32_t n) {
    int64_t N = (int64_t)n * n;
    int sh = bits_for(N);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(N * 9 + 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            for (int di = -1; di <= 1; di++)
                for (int dj = -1; dj <= 1; dj++) {
                    int64_t ii = i + di, jj = j + dj;
                    if (ii < 0 || jj < 0 || ii >= n || jj >= n) continue;
                    keys[m++] = ((uint64_t)(i * n + j) << sh) | (uint64_t)(ii * n + jj);
                }
    /* generated in (column, row) order already */
    gg_graph *g = from_pairs(keys, m, N, N, sh);
    free(keys);
    return g;
}

/* Chung-Lu bipartite graph, n x n.  Both sides carry the weight profile
 * w_i = wmax * (1 + i/i0)^(-1/(beta-1)) (heaviest at id 0), with i0 set so
 * that the mean weight is `mean`; round(mean*n) endpoint pairs are drawn with
 * both endpoints proportional to w, then duplicates are removed. */
static double cl_mean(double i0, double wmax, double ex, double n) {
    /* continuous approximation of (1/n) * sum_i w_i */
    double e1 = 1.0 - ex;
    return wmax * i0 / (n * e1) * (pow(1.0 + n / i0, e1) - 1.0);
}

void *gg_chung_lu(int32_t n, double mean, double wmax, double beta, uint64_t seed) {
    double ex = 1.0 / (beta - 1.0);
    double lo = 1e-6, hi = (double)n;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (cl_mean(mid, wmax, ex, (double)n) < mean) lo = mid; else hi = mid;
    }
    double i0 = 0.5 * (lo + hi);
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    cum[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        double w = wmax * pow(1.0 + (double)i / i0, -ex);
        uint64_t wi = (uint64_t)(w * 1048576.0);
        if (wi == 0) wi = 1;
        cum[i + 1] = cum[i] + wi;
    }
    uint64_t total = cum[n];
    int64_t m = (int64_t)llround(mean * (double)n);
    int sh = bits_for(n);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint64_t end[2];
        for (int s = 0; s < 2; s++) {
            uint64_t r = below(rnd(seed, (uint64_t)s, (uint64_t)e), total);
            /* largest i with cum[i] <= r */
            int64_t a = 0, b = n;
            while (b - a > 1) {
                int64_t mid = (a + b) >> 1;
                if (cum[mid] <= r) a = mid; else b = mid;
            }
            end[s] = (uint64_t)a;
        }
        keys[e] = (end[0] << sh) | end[1];
    }
    free(cum);
    radix_sort_u64(keys, m, 2 * sh);
    m = dedup_sorted(keys, m);
    gg_graph *g = from_pairs(keys, m, n, n, sh);
    free(keys);
    return g;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with 2^scale vertices and
 * edge_factor * 2^scale directed edges, quadrant probabilities (a, b, c, d);
 * no label permutation; self loops dropped; symmetrised; deduplicated.
 * Returns an undirected graph (a_* = symmetric CSR; b_* aliases it). */
void *gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed) {
    int64_t n = (int64_t)1 << scale;
    int64_t m = (int64_t)edge_factor * n;
    const double two64 = 18446744073709551616.0;
    uint64_t ta = (uint64_t)(a * two64), tb = (uint64_t)((a + b) * two64);
    uint64_t tc = (uint64_t)((a + b + c) * two64);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint64_t u = 0, v = 0;
        for (int l = 0; l < scale; l++) {
            uint64_t r = rnd(seed, (uint64_t)l, (uint64_t)e);
            uint64_t ub, vb;
            if (r < ta) { ub = 0; vb = 0; }
            else if (r < tb) { ub = 0; vb = 1; }
            else if (r < tc) { ub = 1; vb = 0; }
            else { ub = 1; vb = 1; }
            u = (u << 1) | ub;
            v = (v << 1) | vb;
        }
        if (u == v) { keys[2 * e] = ~0ULL; keys[2 * e + 1] = ~0ULL; }
        else { keys[2 * e] = (u << scale) | v; keys[2 * e + 1] = (v << scale) | u; }
    }
    int64_t mm = 0;
    for (int64_t i = 0; i < 2 * m; i++)
        if (keys[i] != ~0ULL) keys[mm++] = keys[i];
    radix_sort_u64(keys, mm, 2 * scale);
    mm = dedup_sorted(keys, mm);
    gg_graph *g = from_pairs(keys, mm, n, n, scale);
    free(keys);
    /* symmetric: CSC equals CSR; keep one copy */
    free(g->b_ptr); free(g->b_idx);
    g->b_ptr = g->a_ptr; g->b_idx = g->a_idx;
    g->undirected = 1;
    return g;
}

/* Undirected graph from an explicit edge list (for small hand-made cases):
 * symmetrised, deduplicated, self loops dropped. */
void *gg_from_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    int sh = bits_for(n);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    int64_t k = 0;
    for (int64_t e = 0; e < m; e++) {
        if (src[e] == dst[e]) continue;
        keys[k++] = ((uint64_t)src[e] << sh) | (uint64_t)dst[e];
        keys[k++] = ((uint64_t)dst[e] << sh) | (uint64_t)src[e];
    }
    radix_sort_u64(keys, k, 2 * sh);
    k = dedup_sorted(keys, k);
    gg_graph *g = from_pairs(keys, k, n, n, sh);
    free(keys);
    free(g->b_ptr); free(g->b_idx);
    g->b_ptr = g->a_ptr; g->b_idx = g->a_idx;
    g->undirected = 1;
    return g;
}

/* Bipartite graph from an explicit incidence list (u in V_A, v in V_B),
 * deduplicated. */
void *gg_from_pairs(int32_t n_a, int32_t n_b, int64_t m, const int32_t *u, const int32_t *v) {
    int sh = bits_for(n_b);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m + 1));
    for (int64_t e = 0; e < m; e++) keys[e] = ((uint64_t)u[e] << sh) | (uint64_t)v[e];
    radix_sort_u64(keys, m, sh + bits_for(n_a));
    m = dedup_sorted(keys, m);
    gg_graph *g = from_pairs(keys, m, n_a, n_b, sh);
    free(keys);
    return g;
}

/* One graph of the batched workload: |V_A| log-uniform in [lo, hi],
 * |V_B| = |V_A| * U[0.5, 2], per-vertex degree Poisson(lambda) clipped to
 * [1, maxdeg], distinct uniform nets.  Graph `index` of a batch under `seed`. */
void gg_batch_sizes(uint64_t seed, int32_t index, double lo, double hi, int32_t *n_a, int32_t *n_b) {
    double u1 = unif(rnd(seed, 0xB47C0000ULL + (uint64_t)index, 0));
    double u2 = unif(rnd(seed, 0xB47C0000ULL + (uint64_t)index, 1));
    double na = exp(log(lo) + u1 * (log(hi) - log(lo)));
    int32_t a = (int32_t)na;
    if (a < 1) a = 1;
    int32_t b = (int32_t)((double)a * (0.5 + 1.5 * u2));
    if (b < 1) b = 1;
    *n_a = a;
    *n_b = b;
}

void *gg_batch_graph(uint64_t seed, int32_t index, double lo, double hi, double lambda, int32_t maxdeg) {
    int32_t n_a, n_b;
    gg_batch_sizes(seed, index, lo, hi, &n_a, &n_b);
    if (maxdeg > n_b) maxdeg = n_b;
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_a);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n_a + 1));
    double L = exp(-lambda);
    uint64_t gstream = ((uint64_t)index + 1ULL) << 32;
    for (int64_t u = 0; u < n_a; u++) {
        /* Knuth's multiplication method for Poisson sampling */
        int32_t k = 0;
        double p = 1.0;
        uint64_t ctr = 0;
        do {
            k++;
            p *= unif(rnd(seed, gstream | 0x1ULL, (uint64_t)u * 64ULL + ctr++));
        } while (p > L && ctr < 1000);
        int32_t d = k - 1;
        if (d < 1) d = 1;
        if (d > maxdeg) d = maxdeg;
        deg[u] = d;
    }
    off[0] = 0;
    for (int64_t u = 0; u < n_a; u++) off[u + 1] = off[u] + deg[u];
    int64_t m = off[n_a];
    int sh = bits_for(n_b);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n_a; u++) {
        int32_t buf[256];
        int got = 0;
        uint64_t ctr = 0;
        while (got < deg[u]) {
            int32_t v = (int32_t)below(rnd(seed, gstream | 0x2ULL, (uint64_t)u * 4096ULL + ctr++), (uint64_t)n_b);
            int dup = 0;
            for (int k = 0; k < got; k++) dup |= (buf[k] == v);
            if (!dup) buf[got++] = v;
        }
        for (int k = 0; k < got; k++) keys[off[u] + k] = ((uint64_t)u << sh) | (uint64_t)buf[k];
    }
    radix_sort_u64(keys, m, sh + bits_for(n_a));
    gg_graph *g = from_pairs(keys, m, n_a, n_b, sh);
    free(keys);
    free(deg);
    free(off);
    return g;
}

/* --------------------------------------------------------------- access -- */

int64_t gg_n_a(void *h) { return ((gg_graph *)h)->n_a; }
int64_t gg_n_b(void *h) { return ((gg_graph *)h)->n_b; }
int64_t gg_nnz(void *h) { return ((gg_graph *)h)->nnz; }
int gg_undirected(void *h) { return ((gg_graph *)h)->undirected; }

void gg_copy(void *h, int32_t *a_ptr, int32_t *a_idx, int32_t *b_ptr, int32_t *b_idx) {
    gg_graph *g = (gg_graph *)h;
    memcpy(a_ptr, g->a_ptr, sizeof(int32_t) * ((size_t)g->n_a + 1));
    memcpy(a_idx, g->a_idx, sizeof(int32_t) * (size_t)g->nnz);
    if (b_ptr) memcpy(b_ptr, g->b_ptr, sizeof(int32_t) * ((size_t)g->n_b + 1));
    if (b_idx) memcpy(b_idx, g->b_idx, sizeof(int32_t) * (size_t)g->nnz);
}

void gg_free(void *h) {
    gg_graph *g = (gg_graph *)h;
    if (!g) return;
    if (g->b_ptr != g->a_ptr) free(g->b_ptr);
    if (g->b_idx != g->a_idx) free(g->b_idx);
    free(g->a_ptr);
    free(g->a_idx);
    free(g);
}
