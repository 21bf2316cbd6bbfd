/*
 * CPU oracle for BGPC / D2GC, after Tas, Kaya, Saule, "Greed is Good"
 * (arXiv 1701.02628).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; shares no code with the CUDA
 * path.  Plain, slow and written to be checked against the paper by eye.
 *
 * Parity pins (what fixes each function independently of itself) are listed
 * in tests/test_oracle_pins.py.  Every function here is pinned; none is
 * "parity unpinned".
 */
#include "bgpc_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define UNSET INT32_MIN

/* ------------------------------------------------------------------------
 * Forbidden color set F.  Section III, "Implementation details": F is a
 * plain array that is never reset; membership is "mark[col] == stamp" and a
 * new vertex just takes a new stamp.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t *mark;
    int32_t size;
    int32_t stamp;
} fset;

static int fs_init(fset *F, int32_t size) {
    F->size = size;
    F->stamp = 0;
    F->mark = (int32_t *)calloc((size_t)size, sizeof(int32_t));
    return F->mark ? 0 : -1;
}
static void fs_free(fset *F) { free(F->mark); }
static void fs_clear(fset *F) {
    if (F->stamp == INT32_MAX) {
        memset(F->mark, 0, sizeof(int32_t) * (size_t)F->size);
        F->stamp = 0;
    }
    F->stamp++;
}
static void fs_add(fset *F, int32_t col) {
    if (col >= 0 && col < F->size) F->mark[col] = F->stamp;
}
static int fs_has(const fset *F, int32_t col) {
    return col >= 0 && col < F->size && F->mark[col] == F->stamp;
}

/* ------------------------------------------------------------------------
 * Coloring policies.
 *   FF: first fit, Alg. 2 lines 6-9.
 *   B1: Alg. ColorWorkQueue-B1 (Section V): even vertex ids search down from
 *       col_max, and if nothing below is free, up from col_max + 1; odd ids
 *       use first fit; then col_max = max(col_max, col).
 *   B2: Alg. ColorWorkQueue-B2: search up from col_next; if the color found
 *       exceeds col_max, use first fit; then col_max = max(col_max, col) and
 *       col_next = min(col + 1, col_max / 3 + 1)  (box, integer division).
 *   B2X: the prose's reading of the last line, col_next = max(...), so that
 *       the search starts at least at col_max / 3 + 1.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t col_max;
    int32_t col_next;
} pstate;

static int32_t first_fit(const fset *F) {
    int32_t col = 0;
    while (fs_has(F, col)) col++;
    return col;
}

static int32_t policy_color(int32_t policy, const fset *F, int32_t w, const pstate *st) {
    int32_t col;
    if (policy == ORC_B1) {
        if (w % 2 == 0) {
            col = st->col_max;
            while (col >= 0 && fs_has(F, col)) col--;
            if (col == -1) {
                col = st->col_max + 1;
                while (fs_has(F, col)) col++;
            }
        } else {
            col = first_fit(F);
        }
    } else if (policy == ORC_B2 || policy == ORC_B2X) {
        col = st->col_next;
        while (fs_has(F, col)) col++;
        if (col > st->col_max) col = first_fit(F);
    } else {
        col = first_fit(F);
    }
    return col;
}

static void policy_update(int32_t policy, int32_t col, pstate *st) {
    if (col > st->col_max) st->col_max = col;
    if (policy == ORC_B2 || policy == ORC_B2X) {
        int32_t a = col + 1, b = st->col_max / 3 + 1;
        st->col_next = (policy == ORC_B2) ? (a < b ? a : b) : (a > b ? a : b);
    }
}

static int valid_policy(int32_t p) { return p >= ORC_FF && p <= ORC_B2X; }

/* Processing order: vertices by increasing rank (a permutation), else ids. */
static int make_order(int32_t n, const int32_t *rank, int32_t *order) {
    if (!rank) {
        for (int32_t i = 0; i < n; i++) order[i] = i;
        return 0;
    }
    for (int32_t i = 0; i < n; i++) order[i] = -1;
    for (int32_t w = 0; w < n; w++) {
        int32_t r = rank[w];
        if (r < 0 || r >= n || order[r] != -1) return -1;
        order[r] = w;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * O-1: sequential greedy (Alg. 1 with one thread; ColorWorkQueue is Alg. 4,
 * the vertex-based two-hop gather; no conflicts can arise).
 * ---------------------------------------------------------------------- */
int orc_seq_color(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                  const int32_t *b_ptr, const int32_t *b_idx, const int32_t *rank,
                  int32_t policy, int32_t *c) {
    (void)n_b;
    if (n_a < 0 || !valid_policy(policy)) return ORC_EINVAL;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_a + 1));
    fset F;
    if (!order || fs_init(&F, n_a + 2)) { free(order); return ORC_ENOMEM; }
    if (make_order(n_a, rank, order)) { free(order); fs_free(&F); return ORC_EINVAL; }
    for (int32_t w = 0; w < n_a; w++) c[w] = -1;
    pstate st = {0, 0};
    for (int32_t i = 0; i < n_a; i++) {
        int32_t w = order[i];
        fs_clear(&F);
        for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++) {
            int32_t v = a_idx[e];
            for (int32_t f = b_ptr[v]; f < b_ptr[v + 1]; f++) {
                int32_t u = b_idx[f];
                if (u != w && c[u] != -1) fs_add(&F, c[u]);
            }
        }
        int32_t col = policy_color(policy, &F, w, &st);
        c[w] = col;
        policy_update(policy, col, &st);
    }
    free(order);
    fs_free(&F);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * O-2: round-synchronous speculative coloring RS(C, Q, T, policy, rank).
 *
 * Round r works on W_r (rank order, m = |W_r|).  Chunk j is W_r[jC, jC+C),
 * j < nch = ceil(m/C).  Chunk j belongs to wave q(j) = floor(frac(j*phi)*Q),
 * phi = (sqrt(5)-1)/2, evaluated in 32-bit fixed point (wave_of below), so
 * that the chunks of a wave are spread evenly over W_r and chunks close in
 * rank order run in different waves, as in the paper's runs where only a
 * handful of consecutive OpenMP chunks are in flight at any time.
 * All chunks of a wave read the same snapshot S; a chunk colors its vertices
 * one after the other like one of the paper's threads (chunk 64 of V-V-64,
 * Section VI), seeing its own earlier colors through an overlay; after the
 * wave its colors are published into S.
 *
 * Owner net own(w) = the largest net of w (ties: larger net id); if
 * s = |vtxs(own(w))| > T, w uses the reverse first fit of Alg. 8 rendered per
 * vertex: with k = number of vertices before w in vtxs(own(w)) that are in
 * W_r and own the same net, w takes the k-th (0-based) color not in F
 * counting down from s - 1; if there are not k + 1 of them, the policy color.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t n_a;
    const int32_t *a_ptr, *a_idx, *b_ptr, *b_idx;
    int32_t policy, C;
    int64_t T;
    const int32_t *S, *W;
    int32_t m;
    const int32_t *s_own;  /* |vtxs(own(w))|, 0 if w has no net */
    const int32_t *k;      /* by W position */
    int32_t col_max0;      /* max(S), at least 0 */
    int32_t *out;          /* by W position */
} rs_ctx;

static void rs_color_chunk(const rs_ctx *x, int64_t j, fset *F, int32_t *ovl) {
    int64_t lo = j * (int64_t)x->C, hi = lo + x->C;
    if (hi > x->m) hi = x->m;
    pstate st = {x->col_max0, 0};
    for (int64_t p = lo; p < hi; p++) {
        int32_t w = x->W[p];
        fs_clear(F);
        for (int32_t e = x->a_ptr[w]; e < x->a_ptr[w + 1]; e++) {
            int32_t v = x->a_idx[e];
            for (int32_t f = x->b_ptr[v]; f < x->b_ptr[v + 1]; f++) {
                int32_t u = x->b_idx[f];
                if (u == w) continue;
                int32_t cu = (ovl[u] != UNSET) ? ovl[u] : x->S[u];
                if (cu >= 0) fs_add(F, cu);
            }
        }
        int32_t col = -1;
        if ((int64_t)x->s_own[w] > x->T) {
            int32_t cnt = 0;
            for (int32_t cc = x->s_own[w] - 1; cc >= 0; cc--) {
                if (fs_has(F, cc)) continue;
                if (cnt == x->k[p]) { col = cc; break; }
                cnt++;
            }
        }
        if (col < 0) col = policy_color(x->policy, F, w, &st);
        policy_update(x->policy, col, &st);
        ovl[w] = col;
        x->out[p] = col;
    }
    for (int64_t p = lo; p < hi; p++) ovl[x->W[p]] = UNSET;
}

typedef struct {
    const rs_ctx *x;
    const int64_t *chunks;  /* explicit list, or NULL for [jlo, jhi) */
    int64_t jlo, jhi;
    fset F;
    int32_t *ovl;
} rs_worker;

static void *rs_worker_run(void *arg) {
    rs_worker *wk = (rs_worker *)arg;
    for (int64_t t = wk->jlo; t < wk->jhi; t++)
        rs_color_chunk(wk->x, wk->chunks ? wk->chunks[t] : t, &wk->F, wk->ovl);
    return NULL;
}

static int alloc_workers(rs_worker *wk, int32_t nthreads, int32_t n_a) {
    for (int32_t t = 0; t < nthreads; t++) {
        if (fs_init(&wk[t].F, n_a + 2)) return -1;
        wk[t].ovl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_a + 1));
        if (!wk[t].ovl) return -1;
        for (int32_t u = 0; u < n_a; u++) wk[t].ovl[u] = UNSET;
    }
    return 0;
}

static void free_workers(rs_worker *wk, int32_t nthreads) {
    for (int32_t t = 0; t < nthreads; t++) {
        fs_free(&wk[t].F);
        free(wk[t].ovl);
    }
}

/* Color chunks [jlo, jhi) (or chunks[jlo..jhi) if given) on nthreads threads. */
static void rs_run_chunks(const rs_ctx *x, const int64_t *chunks, int64_t jlo, int64_t jhi,
                          rs_worker *wk, int32_t nthreads) {
    int64_t n = jhi - jlo;
    if (n <= 0) return;
    int32_t nt = nthreads;
    if (n < nt) nt = (int32_t)n;
    if (nt <= 1) {
        wk[0].x = x; wk[0].chunks = chunks; wk[0].jlo = jlo; wk[0].jhi = jhi;
        rs_worker_run(&wk[0]);
        return;
    }
    pthread_t th[256];
    for (int32_t t = 0; t < nt; t++) {
        wk[t].x = x;
        wk[t].chunks = chunks;
        wk[t].jlo = jlo + n * t / nt;
        wk[t].jhi = jlo + n * (t + 1) / nt;
        pthread_create(&th[t], NULL, rs_worker_run, &wk[t]);
    }
    for (int32_t t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

/* own(w) and |vtxs(own(w))|. */
static void owners(int32_t n_a, const int32_t *a_ptr, const int32_t *a_idx, const int32_t *b_ptr,
                   int32_t *own, int32_t *s_own) {
    for (int32_t w = 0; w < n_a; w++) {
        int32_t best = -1, bs = 0;
        for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++) {
            int32_t v = a_idx[e], s = b_ptr[v + 1] - b_ptr[v];
            if (best < 0 || s > bs || (s == bs && v > best)) { best = v; bs = s; }
        }
        own[w] = best;
        s_own[w] = best < 0 ? 0 : bs;
    }
}

/* k for every big vertex of W: prefix count along vtxs(own) of the members
 * that are in W and own this net. inW[u] = position of u in W or -1. */
static void reverse_offsets(int32_t n_b, const int32_t *b_ptr, const int32_t *b_idx,
                            const int32_t *own, const int32_t *inW, int64_t T, int32_t *k) {
    for (int32_t v = 0; v < n_b; v++) {
        if ((int64_t)(b_ptr[v + 1] - b_ptr[v]) <= T) continue;
        int32_t cnt = 0;
        for (int32_t f = b_ptr[v]; f < b_ptr[v + 1]; f++) {
            int32_t u = b_idx[f];
            if (inW[u] >= 0 && own[u] == v) k[inW[u]] = cnt++;
        }
    }
}

/* Wave of chunk j: ((j * 0x9E3779B9 mod 2^32) * Q) >> 32, i.e. the Weyl
 * sequence frac(j * phi) with phi = 0x9E3779B9 / 2^32, scaled to Q waves. */
static int32_t wave_of(int64_t j, int32_t Q) {
    uint32_t x = (uint32_t)((uint64_t)j * 0x9E3779B9ull);
    return (int32_t)(((uint64_t)x * (uint64_t)Q) >> 32);
}

/* Chunks of every wave, in increasing chunk order: list[off[q] .. off[q+1]). */
static void wave_lists(int64_t nch, int32_t Q, int64_t *off, int64_t *list) {
    for (int32_t q = 0; q <= Q; q++) off[q] = 0;
    for (int64_t j = 0; j < nch; j++) off[wave_of(j, Q) + 1]++;
    for (int32_t q = 0; q < Q; q++) off[q + 1] += off[q];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)Q + 1));
    for (int32_t q = 0; q <= Q; q++) fill[q] = off[q];
    for (int64_t j = 0; j < nch; j++) list[fill[wave_of(j, Q)]++] = j;
    free(fill);
}

static int32_t max_color(const int32_t *S, int32_t n) {
    int32_t mx = -1;
    for (int32_t u = 0; u < n; u++)
        if (S[u] > mx) mx = S[u];
    return mx;
}

/* Conflict rule for one W position p: 1 if w loses, 0 if it keeps its color.
 * A vertex outside W sharing w's color: after a vertex-based round this
 * cannot happen (F held that color), so it returns ORC_EFIXED unless
 * fixed_wins is set (after a net-based round, where a net only sees its own
 * members), in which case the fixed vertex keeps its color and w loses.  An
 * uncolored w (no net proposed a color for it) always stays in the queue. */
static int rs_lose_one(const int32_t *a_ptr, const int32_t *a_idx, const int32_t *b_ptr,
                       const int32_t *b_idx, const int32_t *c, const int32_t *inW,
                       const int32_t *W, int32_t p, int fixed_wins) {
    int32_t w = W[p];
    if (c[w] < 0) return 1;
    int lose = 0;
    for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++) {
        int32_t v = a_idx[e];
        for (int32_t f = b_ptr[v]; f < b_ptr[v + 1]; f++) {
            int32_t u = b_idx[f];
            if (u == w || c[u] != c[w]) continue;
            if (inW[u] < 0) {
                if (!fixed_wins) return ORC_EFIXED;
                lose = 1;
            } else if (inW[u] < p) {
                lose = 1;
            }
        }
    }
    return lose;
}

/* ------------------------------------------------------------------------
 * Net-based coloring round: Alg. 8 (BGPC-ColorWorkQueue-Net), and Alg. 9
 * (D2GC-ColorWorkQueue-Net) when center_first is set, as one deterministic
 * round.  Every net v reads the snapshot S of the round start:
 *   F = colors of the members that are colored and not yet in F;
 *   W_local = the other members (uncolored, or colored with a color already
 *             in F), in adjacency order; for D2GC (nets are the closed
 *             neighbourhoods N[v]) the center v is visited first, as Alg. 9
 *             does before the loop over nbor(v);
 *   reverse first fit: col starts at |vtxs(v)| - 1 (= |nbor(v)| for D2GC);
 *   every W_local member takes the largest col not in F, then col drops by
 *   one.
 * In the paper every net writes its W_local members and the last writer
 * wins; here vertex w of W takes the color proposed by its owner net own(w)
 * (the largest net of w, ties to the larger id), the same owner as the
 * per-vertex reverse first fit of the vertex-based rounds.  A member colored
 * with a color already in F would be a conflict left in S, which the
 * conflict removal never leaves: it returns ORC_EFIXED.  A W vertex without
 * nets gets no proposal and stays uncolored.
 * ---------------------------------------------------------------------- */
static int rs_net_round(int32_t n_b, const int32_t *b_ptr, const int32_t *b_idx,
                        const int32_t *own, const int32_t *inW, int center_first,
                        const int32_t *S, fset *F, int32_t *Wl, int32_t *c) {
    for (int32_t v = 0; v < n_b; v++) {
        int32_t beg = b_ptr[v], end = b_ptr[v + 1], s = end - beg, nl = 0;
        fs_clear(F);
        int has_center = 0;
        if (center_first)
            for (int32_t f = beg; f < end; f++)
                if (b_idx[f] == v) has_center = 1;
        for (int32_t t = -1; t < s; t++) {
            int32_t u;
            if (t < 0) {
                if (!has_center) continue;
                u = v;
            } else {
                u = b_idx[beg + t];
                if (has_center && u == v) continue;
            }
            if (S[u] != -1 && !fs_has(F, S[u])) {
                fs_add(F, S[u]);
            } else {
                if (S[u] != -1) return ORC_EFIXED;
                Wl[nl++] = u;
            }
        }
        int32_t col = s - 1;
        for (int32_t i = 0; i < nl; i++) {
            while (fs_has(F, col)) col--;
            if (col < 0) return ORC_EINVAL;  /* at least |W_local| colors are free */
            int32_t u = Wl[i];
            if (inW[u] >= 0 && own[u] == v) c[u] = col;
            col--;
        }
    }
    return ORC_OK;
}

int orc_rs_color(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                 const int32_t *b_ptr, const int32_t *b_idx, const int32_t *rank,
                 int32_t policy, int32_t C, int32_t Q, int64_t T, int32_t max_rounds,
                 int32_t net_rounds, int32_t center_first, int64_t stop_after_waves,
                 int32_t stop_before_removal, int32_t nthreads, int32_t *c,
                 int32_t *rounds_out, int64_t *w_per_round, int64_t *trav_per_round,
                 int32_t max_report, int32_t *W_out, int32_t *m_out, int32_t *wave_out) {
    if (n_a < 0 || C < 1 || Q < 1 || net_rounds < 0 || !valid_policy(policy)) return ORC_EINVAL;
    if (center_first && n_a != n_b) return ORC_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    size_t na = (size_t)n_a + 1;
    int32_t *W = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *Wn = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *inW = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *s_own = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *k = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * na);
    uint8_t *lose = (uint8_t *)malloc(na);
    int64_t *woff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)Q + 1));
    int64_t *wlist = (int64_t *)malloc(sizeof(int64_t) * na);
    rs_worker *wk = (rs_worker *)calloc((size_t)nthreads, sizeof(rs_worker));
    int rc = ORC_OK;
    int32_t *Wl = (int32_t *)malloc(sizeof(int32_t) * na);
    if (!W || !Wn || !inW || !own || !s_own || !k || !S || !out || !lose || !wk || !woff || !wlist ||
        !Wl || alloc_workers(wk, nthreads, n_a)) {
        rc = ORC_ENOMEM;
        goto done;
    }
    if (make_order(n_a, rank, W)) { rc = ORC_EINVAL; goto done; }
    owners(n_a, a_ptr, a_idx, b_ptr, own, s_own);
    for (int32_t u = 0; u < n_a; u++) { c[u] = -1; inW[u] = -1; }

    int32_t m = n_a, r = 0;
    int64_t waves_done = 0;
    while (m > 0) {
        if (r >= max_rounds) { rc = ORC_EROUNDS; break; }
        const int net = r < net_rounds;
        for (int32_t p = 0; p < m; p++) inW[W[p]] = p;
        if (r < max_report) {
            /* vertex round: the two-hop entries the vertices of W read;
             * net round: the members of the nets touching W, read once */
            int64_t trav = 0;
            if (net) {
                for (int32_t v = 0; v < n_b; v++) {
                    int touch = 0;
                    for (int32_t f = b_ptr[v]; f < b_ptr[v + 1] && !touch; f++)
                        touch = inW[b_idx[f]] >= 0;
                    if (touch) trav += b_ptr[v + 1] - b_ptr[v];
                }
            } else {
                for (int32_t p = 0; p < m; p++) {
                    int32_t w = W[p];
                    for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++) {
                        int32_t v = a_idx[e];
                        trav += b_ptr[v + 1] - b_ptr[v] - 1;
                    }
                }
            }
            if (w_per_round) w_per_round[r] = m;
            if (trav_per_round) trav_per_round[r] = trav;
        }
        r++;
        memcpy(S, c, sizeof(int32_t) * (size_t)n_a);
        if (net) {
            /* a net round counts as one wave for stop_after_waves */
            if (stop_after_waves > 0 && waves_done == stop_after_waves) {
                if (W_out) memcpy(W_out, W, sizeof(int32_t) * (size_t)m);
                if (m_out) *m_out = m;
                if (wave_out) *wave_out = 0;
                if (rounds_out) *rounds_out = r;
                rc = ORC_STOPPED;
                goto done;
            }
            if ((rc = rs_net_round(n_b, b_ptr, b_idx, own, inW, center_first, S, &wk[0].F, Wl,
                                   c)) != ORC_OK)
                goto done;
            waves_done++;
        } else {
        reverse_offsets(n_b, b_ptr, b_idx, own, inW, T, k);

        rs_ctx x;
        x.n_a = n_a; x.a_ptr = a_ptr; x.a_idx = a_idx; x.b_ptr = b_ptr; x.b_idx = b_idx;
        x.policy = policy; x.C = C; x.T = T; x.S = S; x.W = W; x.m = m;
        x.s_own = s_own; x.k = k; x.out = out;
        int64_t nch = ((int64_t)m + C - 1) / C;
        wave_lists(nch, Q, woff, wlist);
        for (int32_t q = 0; q < Q; q++) {
            if (stop_after_waves > 0 && waves_done == stop_after_waves) {
                memcpy(c, S, sizeof(int32_t) * (size_t)n_a);
                if (W_out) memcpy(W_out, W, sizeof(int32_t) * (size_t)m);
                if (m_out) *m_out = m;
                if (wave_out) *wave_out = q;
                if (rounds_out) *rounds_out = r;
                rc = ORC_STOPPED;
                goto done;
            }
            int32_t mx = max_color(S, n_a);
            x.col_max0 = mx < 0 ? 0 : mx;
            rs_run_chunks(&x, wlist, woff[q], woff[q + 1], wk, nthreads);
            for (int64_t t = woff[q]; t < woff[q + 1]; t++) {
                int64_t plo = wlist[t] * C, phi = plo + C;
                if (phi > m) phi = m;
                for (int64_t p = plo; p < phi; p++) S[W[p]] = out[p];
            }
            waves_done++;
        }
        memcpy(c, S, sizeof(int32_t) * (size_t)n_a);
        }
        if (stop_before_removal && stop_after_waves > 0 && waves_done == stop_after_waves) {
            if (W_out) memcpy(W_out, W, sizeof(int32_t) * (size_t)m);
            if (m_out) *m_out = m;
            if (wave_out) *wave_out = net ? 1 : Q;
            if (rounds_out) *rounds_out = r;
            rc = ORC_STOPPED;
            goto done;
        }

        /* RemoveConflicts (Alg. 3/5 rule, lower rank wins; after a net round
         * a fixed vertex also wins) */
        int32_t mn = 0;
        for (int32_t p = 0; p < m; p++) {
            int l = rs_lose_one(a_ptr, a_idx, b_ptr, b_idx, c, inW, W, p, net);
            if (l == ORC_EFIXED) { rc = ORC_EFIXED; goto done; }
            lose[p] = (uint8_t)l;
        }
        for (int32_t p = 0; p < m; p++) {
            if (lose[p]) Wn[mn++] = W[p];
        }
        for (int32_t p = 0; p < m; p++) inW[W[p]] = -1;
        for (int32_t i = 0; i < mn; i++) c[Wn[i]] = -1;
        int32_t *t = W; W = Wn; Wn = t;
        m = mn;
    }
    if (rounds_out) *rounds_out = r;
    if (m_out) *m_out = m;
    if (W_out && m > 0) memcpy(W_out, W, sizeof(int32_t) * (size_t)m);
done:
    if (wk) free_workers(wk, nthreads);
    free(wk); free(W); free(Wn); free(inW); free(own); free(s_own); free(k);
    free(S); free(out); free(lose); free(woff); free(wlist); free(Wl);
    return rc;
}

int orc_rs_chunks(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                  const int32_t *b_ptr, const int32_t *b_idx, const int32_t *S,
                  const int32_t *W, int32_t m, int32_t policy, int32_t C, int64_t T,
                  const int32_t *chunks, int32_t nchunks, int32_t nthreads, int32_t *out) {
    if (n_a < 0 || C < 1 || m < 0 || m > n_a || !valid_policy(policy)) return ORC_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    size_t na = (size_t)n_a + 1;
    int32_t *inW = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *s_own = (int32_t *)malloc(sizeof(int32_t) * na);
    int32_t *k = (int32_t *)malloc(sizeof(int32_t) * na);
    int64_t *ch = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nchunks + 1));
    rs_worker *wk = (rs_worker *)calloc((size_t)nthreads, sizeof(rs_worker));
    int rc = ORC_OK;
    if (!inW || !own || !s_own || !k || !ch || !wk || alloc_workers(wk, nthreads, n_a)) {
        rc = ORC_ENOMEM;
        goto done;
    }
    for (int32_t u = 0; u < n_a; u++) inW[u] = -1;
    for (int32_t p = 0; p < m; p++) {
        if (W[p] < 0 || W[p] >= n_a || inW[W[p]] >= 0) { rc = ORC_EINVAL; goto done; }
        inW[W[p]] = p;
    }
    owners(n_a, a_ptr, a_idx, b_ptr, own, s_own);
    reverse_offsets(n_b, b_ptr, b_idx, own, inW, T, k);
    int64_t nch = ((int64_t)m + C - 1) / C;
    for (int32_t i = 0; i < nchunks; i++) {
        if (chunks[i] < 0 || chunks[i] >= nch) { rc = ORC_EINVAL; goto done; }
        ch[i] = chunks[i];
    }
    rs_ctx x;
    x.n_a = n_a; x.a_ptr = a_ptr; x.a_idx = a_idx; x.b_ptr = b_ptr; x.b_idx = b_idx;
    x.policy = policy; x.C = C; x.T = T; x.S = S; x.W = W; x.m = m;
    x.s_own = s_own; x.k = k; x.out = out;
    int32_t mx = max_color(S, n_a);
    x.col_max0 = mx < 0 ? 0 : mx;
    rs_run_chunks(&x, ch, 0, nchunks, wk, nthreads);
done:
    if (wk) free_workers(wk, nthreads);
    free(wk);
    free(inW); free(own); free(s_own); free(k); free(ch);
    return rc;
}

int orc_rs_losers(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                  const int32_t *b_ptr, const int32_t *b_idx, const int32_t *c,
                  const int32_t *W, int32_t m, const int32_t *which, int32_t nwhich,
                  uint8_t *lose) {
    (void)n_b;
    int32_t *inW = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_a + 1));
    if (!inW) return ORC_ENOMEM;
    for (int32_t u = 0; u < n_a; u++) inW[u] = -1;
    for (int32_t p = 0; p < m; p++) inW[W[p]] = p;
    int rc = ORC_OK;
    for (int32_t i = 0; i < nwhich; i++) {
        int l = rs_lose_one(a_ptr, a_idx, b_ptr, b_idx, c, inW, W, which[i], 0);
        if (l == ORC_EFIXED) { rc = ORC_EFIXED; l = 1; }
        lose[i] = (uint8_t)l;
    }
    free(inW);
    return rc;
}

/* ------------------------------------------------------------------------
 * Checks and statistics.
 * ---------------------------------------------------------------------- */
int64_t orc_conflicts(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                      const int32_t *b_ptr, const int32_t *b_idx, const int32_t *c) {
    (void)n_b;
    int64_t bad = 0;
    for (int32_t w = 0; w < n_a; w++) {
        if (c[w] < 0) { bad++; continue; }
        int hit = 0;
        for (int32_t e = a_ptr[w]; e < a_ptr[w + 1] && !hit; e++) {
            int32_t v = a_idx[e];
            for (int32_t f = b_ptr[v]; f < b_ptr[v + 1]; f++) {
                int32_t u = b_idx[f];
                if (u != w && c[u] == c[w]) { hit = 1; break; }
            }
        }
        bad += hit;
    }
    return bad;
}

int32_t orc_max_nbor(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                     const int32_t *b_ptr, const int32_t *b_idx, int32_t *nbor_size) {
    (void)n_b;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_a + 1));
    if (!mark) return -1;
    for (int32_t u = 0; u < n_a; u++) mark[u] = -1;
    int32_t best = 0;
    for (int32_t w = 0; w < n_a; w++) {
        int32_t cnt = 0;
        for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++) {
            int32_t v = a_idx[e];
            for (int32_t f = b_ptr[v]; f < b_ptr[v + 1]; f++) {
                int32_t u = b_idx[f];
                if (u != w && mark[u] != w) { mark[u] = w; cnt++; }
            }
        }
        if (nbor_size) nbor_size[w] = cnt;
        if (cnt > best) best = cnt;
    }
    free(mark);
    return best;
}

/* Exhaustive minimum coloring of the conflict graph (u ~ w iff they share a
 * net): try k = 0, 1, ... colors with backtracking in id order. */
static int bf_try(int32_t w, int32_t n, const uint32_t *adj, int32_t k, int32_t *col) {
    if (w == n) return 1;
    for (int32_t c = 0; c < k; c++) {
        int ok = 1;
        for (int32_t u = 0; u < w && ok; u++)
            if (((adj[w] >> u) & 1u) && col[u] == c) ok = 0;
        if (!ok) continue;
        col[w] = c;
        if (bf_try(w + 1, n, adj, k, col)) return 1;
    }
    return 0;
}

int32_t orc_bruteforce_min(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                           const int32_t *b_ptr, const int32_t *b_idx) {
    (void)n_b;
    if (n_a > 20) return -1;
    if (n_a == 0) return 0;
    uint32_t adj[20] = {0};
    int32_t col[20];
    for (int32_t w = 0; w < n_a; w++)
        for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++)
            for (int32_t f = b_ptr[a_idx[e]]; f < b_ptr[a_idx[e] + 1]; f++)
                if (b_idx[f] != w) adj[w] |= 1u << b_idx[f];
    for (int32_t k = 1; k <= n_a; k++)
        if (bf_try(0, n_a, adj, k, col)) return k;
    return n_a;
}

int orc_closed_nbhd(int32_t n, const int32_t *ptr, const int32_t *idx, int32_t *cptr, int32_t *cidx) {
    int32_t o = 0;
    cptr[0] = 0;
    for (int32_t u = 0; u < n; u++) {
        int placed = 0;
        for (int32_t e = ptr[u]; e < ptr[u + 1]; e++) {
            if (!placed && idx[e] > u) { cidx[o++] = u; placed = 1; }
            cidx[o++] = idx[e];
        }
        if (!placed) cidx[o++] = u;
        cptr[u + 1] = o;
    }
    return ORC_OK;
}

int64_t orc_d2_conflicts(int32_t n, const int32_t *ptr, const int32_t *idx, const int32_t *c) {
    int64_t bad = 0;
    for (int32_t u = 0; u < n; u++) {
        if (c[u] < 0) { bad++; continue; }
        int hit = 0;
        for (int32_t e = ptr[u]; e < ptr[u + 1] && !hit; e++) {
            int32_t v = idx[e];
            if (c[v] == c[u]) { hit = 1; break; }
            for (int32_t f = ptr[v]; f < ptr[v + 1]; f++) {
                int32_t x = idx[f];
                if (x != u && c[x] == c[u]) { hit = 1; break; }
            }
        }
        bad += hit;
    }
    return bad;
}

int32_t orc_color_sets(int32_t n, const int32_t *c, int32_t *n_sets, int64_t *card) {
    int32_t mx = -1;
    for (int32_t u = 0; u < n; u++)
        if (c[u] > mx) mx = c[u];
    if (card) {
        for (int32_t k = 0; k <= mx; k++) card[k] = 0;
        for (int32_t u = 0; u < n; u++)
            if (c[u] >= 0) card[c[u]]++;
    }
    if (n_sets) {
        int64_t *tmp = card;
        if (!tmp) {
            tmp = (int64_t *)calloc((size_t)mx + 2, sizeof(int64_t));
            for (int32_t u = 0; u < n; u++)
                if (c[u] >= 0) tmp[c[u]]++;
        }
        int32_t K = 0;
        for (int32_t k = 0; k <= mx; k++) K += tmp[k] > 0;
        *n_sets = K;
        if (!card) free(tmp);
    }
    return mx;
}

/* ------------------------------------------------------------------------
 * Smallest-last order (the static order of Table II and Table IV, Sec. VI)
 * on the conflict graph of BGPC: u ~ w iff they share a net.  Repeatedly
 * remove, among the vertices not yet removed, one of smallest degree in the
 * remaining conflict graph (ties: the smallest id); the coloring order is the
 * reverse of the removal order, rank[w] = its position in the coloring order.
 * Plain O(n^2 + E2) version for small graphs: degrees are distinct two-hop
 * neighbour counts, the minimum is found by a scan.  *degeneracy (if not
 * NULL) = the largest degree a vertex had when it was removed.
 * ---------------------------------------------------------------------- */
int orc_sl_rank(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                const int32_t *b_ptr, const int32_t *b_idx, int32_t *rank,
                int32_t *degeneracy) {
    (void)n_b;
    if (n_a < 0) return ORC_EINVAL;
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_a + 1));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_a + 1));
    uint8_t *gone = (uint8_t *)calloc((size_t)n_a + 1, 1);
    if (!deg || !mark || !gone) { free(deg); free(mark); free(gone); return ORC_ENOMEM; }
    for (int32_t u = 0; u < n_a; u++) mark[u] = -1;
    for (int32_t w = 0; w < n_a; w++) {
        int32_t cnt = 0;
        for (int32_t e = a_ptr[w]; e < a_ptr[w + 1]; e++)
            for (int32_t f = b_ptr[a_idx[e]]; f < b_ptr[a_idx[e] + 1]; f++) {
                int32_t u = b_idx[f];
                if (u != w && mark[u] != w) { mark[u] = w; cnt++; }
            }
        deg[w] = cnt;
    }
    int32_t dg = 0;
    for (int32_t step = 0; step < n_a; step++) {
        int32_t best = -1;
        for (int32_t w = 0; w < n_a; w++)
            if (!gone[w] && (best < 0 || deg[w] < deg[best])) best = w;
        if (deg[best] > dg) dg = deg[best];
        gone[best] = 1;
        rank[best] = n_a - 1 - step;
        /* every remaining distinct neighbour loses one degree */
        for (int32_t e = a_ptr[best]; e < a_ptr[best + 1]; e++)
            for (int32_t f = b_ptr[a_idx[e]]; f < b_ptr[a_idx[e] + 1]; f++) {
                int32_t u = b_idx[f];
                if (u != best && !gone[u] && mark[u] != n_a + best) {
                    mark[u] = n_a + best;
                    deg[u]--;
                }
            }
    }
    if (degeneracy) *degeneracy = dg;
    free(deg); free(mark); free(gone);
    return ORC_OK;
}
