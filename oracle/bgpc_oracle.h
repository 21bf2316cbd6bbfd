/*
 * CPU oracle for optimistic bipartite-graph partial coloring (BGPC) and
 * distance-2 coloring (D2GC), after Tas, Kaya, Saule, "Greed is Good"
 * (arXiv 1701.02628).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path and must never be used by it.
 *
 * Notation follows the paper (Section II): V_A vertices are colored, V_B
 * vertices are nets; nets(u) = a_idx[a_ptr[u] .. a_ptr[u+1]), vtxs(v) =
 * b_idx[b_ptr[v] .. b_ptr[v+1]) (sorted, unique);
 * nbor(w) = (U_{v in nets(w)} vtxs(v)) \ {w}; colors are non-negative and -1
 * means uncolored.
 */
#ifndef BGPC_ORACLE_H
#define BGPC_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EROUNDS (-4)
#define ORC_EFIXED (-7)   /* a W vertex took the color of a fixed neighbour */
#define ORC_STOPPED 1     /* stopped after the requested number of waves */

#define ORC_FF 0   /* first fit (Alg. 2) */
#define ORC_B1 1   /* balancing heuristic B1 (Alg. ColorWorkQueue-B1) */
#define ORC_B2 2   /* B2 with the algorithm box's update col_next = min(...) */
#define ORC_B2X 3  /* B2 with the prose's reading: start at least at col_max/3+1 */

/* O-1: sequential greedy coloring (Alg. 1 + Alg. 2/4 on one thread, so no
 * conflicts), vertices taken in increasing rank (rank == NULL: id order).
 * rank must be a permutation of 0..n_a-1.  Writes c[0..n_a). */
int orc_seq_color(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                  const int32_t *b_ptr, const int32_t *b_idx, const int32_t *rank,
                  int32_t policy, int32_t *c);

/* O-2: round-synchronous speculative coloring RS(C, Q, T, policy, rank).
 * Deterministic replay of Alg. 1 with chunked, wave-published coloring and
 * lower-rank-wins conflict removal.  Chunk j (C consecutive work-queue
 * entries) belongs to wave ((j * 0x9E3779B9 mod 2^32) * Q) >> 32.  nthreads > 1 colors the chunks of a wave
 * on several host threads (results do not depend on it).
 * The first net_rounds rounds are net-based instead (Alg. 8 as one
 * round-synchronous round: every net reads the round's snapshot and proposes
 * reverse first-fit colors for its uncolored members, every vertex takes its
 * owner net's proposal, and a vertex outside W wins a clash; center_first:
 * Alg. 9's order for D2GC, where net v is N[v] and v is visited first).
 * stop_after_waves > 0 stops after that many waves (counted over all rounds;
 * a net round counts as one wave) and returns ORC_STOPPED with c = the
 * snapshot at that point, W_out (if not NULL) = the current round's work
 * queue in rank order, *m_out = its length and *wave_out = the index, within
 * its round, of the next wave; with stop_before_removal, a stop that lands on
 * the end of a round comes before its conflict removal (c = the tentative
 * colors, *wave_out = the round's wave count).
 * Per-round |W_r| and traversed two-hop entries go to w_per_round /
 * trav_per_round (first max_report rounds; NULL to skip). */
int orc_rs_color(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                 const int32_t *b_ptr, const int32_t *b_idx, const int32_t *rank,
                 int32_t policy, int32_t C, int32_t Q, int64_t T, int32_t max_rounds,
                 int32_t net_rounds, int32_t center_first, int64_t stop_after_waves,
                 int32_t stop_before_removal, int32_t nthreads, int32_t *c,
                 int32_t *rounds, int64_t *w_per_round, int64_t *trav_per_round,
                 int32_t max_report, int32_t *W_out, int32_t *m_out, int32_t *wave_out);

/* One wave step of O-2 on given state: S = colors at the start of the wave
 * (uncolored W vertices hold -1), W = the round's work queue in rank order
 * (length m).  Colors the chunks listed in `chunks` and writes each chunk
 * vertex's color to out[its position in W] (other entries untouched). */
int orc_rs_chunks(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                  const int32_t *b_ptr, const int32_t *b_idx, const int32_t *S,
                  const int32_t *W, int32_t m, int32_t policy, int32_t C, int64_t T,
                  const int32_t *chunks, int32_t nchunks, int32_t nthreads, int32_t *out);

/* Conflict rule of O-2 (Alg. 3 line "c[u] = c[w] and w > u", with rank in
 * place of id): for each listed W position p, lose[p] = 1 iff some
 * u in nbor(W[p]) has c[u] == c[W[p]] and is either outside W or earlier in
 * W.  Returns ORC_EFIXED if the "outside W" clause fires. */
int orc_rs_losers(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                  const int32_t *b_ptr, const int32_t *b_idx, const int32_t *c,
                  const int32_t *W, int32_t m, const int32_t *which, int32_t nwhich,
                  uint8_t *lose);

/* Number of V_A vertices that are uncolored or share a color with some
 * vertex of nbor(.) (0 means a valid complete BGPC coloring, Section II). */
int64_t orc_conflicts(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                      const int32_t *b_ptr, const int32_t *b_idx, const int32_t *c);

/* max_w |nbor(w)| (distinct two-hop neighbours), the greedy bound. */
int32_t orc_max_nbor(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                     const int32_t *b_ptr, const int32_t *b_idx, int32_t *nbor_size);

/* Minimum number of colors of a valid BGPC coloring, by exhaustive search
 * (n_a <= 20).  Returns -1 if n_a is too large. */
int32_t orc_bruteforce_min(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                           const int32_t *b_ptr, const int32_t *b_idx);

/* D2GC as BGPC on closed neighbourhoods N[u] = {u} u adj(u) (Section IV):
 * writes the CSR of N[.] (cptr[n+1], cidx[nnz+n]) for a symmetric graph. */
int orc_closed_nbhd(int32_t n, const int32_t *ptr, const int32_t *idx,
                    int32_t *cptr, int32_t *cidx);

/* Number of vertices of an undirected graph that are uncolored or share a
 * color with a vertex at shortest-path distance 1 or 2 (direct definition). */
int64_t orc_d2_conflicts(int32_t n, const int32_t *ptr, const int32_t *idx, const int32_t *c);

/* Color-set statistics (Table VI): number of non-empty color sets K, and the
 * cardinality of each color 0..max (card must hold max+1 entries; pass NULL
 * to only get K).  Returns the largest color, or -1. */
int32_t orc_color_sets(int32_t n, const int32_t *c, int32_t *n_sets, int64_t *card);

/* Smallest-last order (Sec. VI, Tables II and IV) on the conflict graph
 * (u ~ w iff they share a net): remove, one at a time, a remaining vertex of
 * smallest remaining degree (ties: smallest id); rank[w] = position of w in
 * the reverse of the removal order (the coloring order).  *degeneracy (may be
 * NULL) = the largest degree at removal.  O(n^2 + E2): small graphs only. */
int orc_sl_rank(int32_t n_a, int32_t n_b, const int32_t *a_ptr, const int32_t *a_idx,
                const int32_t *b_ptr, const int32_t *b_idx, int32_t *rank,
                int32_t *degeneracy);

#endif
