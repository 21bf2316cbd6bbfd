/*
 * bgpc.h -- C ABI of the GB300 (sm_103a) library for optimistic bipartite-graph
 * partial coloring (BGPC) and distance-2 graph coloring (D2GC), after Tas,
 * Kaya, Saule, "Greed is Good: Optimistic Algorithms for Bipartite-Graph
 * Partial Coloring on Multicore Architectures" (arXiv 1701.02628).
 *
 * Problem (Sec. II): G = (V_A u V_B, E).  Color every V_A vertex with a
 * non-negative int32 so that two V_A vertices that share a V_B vertex ("net")
 * get different colors.  D2GC (Sec. II, IV): color every vertex of an
 * undirected graph so that vertices within shortest-path distance 2 differ.
 *
 * Conventions for every call
 *  - Graph, color, rank and work-queue arrays are DEVICE pointers owned by the
 *    caller; the library never frees or retains them after the call returns.
 *    Host pointers are marked "(host)".
 *  - `stream` is a cudaStream_t (passed as void* so that this header needs no
 *    CUDA include); every device operation of a call is ordered on it.  NULL
 *    means the legacy default stream.
 *  - Every call returns an int status: BGPC_OK (0), BGPC_STOPPED (1, only when
 *    requested), or a negative BGPC_E* code.  Output arrays are fully written
 *    only on BGPC_OK.  The calls that return statistics synchronise `stream`.
 *  - A context owns the library's scratch memory (grown on demand, freed by
 *    bgpc_ctx_destroy).  A context may be used by one host thread at a time;
 *    different contexts are independent.  The library keeps no other state.
 *  - Colors are in [0, n_a); -1 never appears in a successful result.
 */
#ifndef BGPC_H
#define BGPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BGPC_OK 0
#define BGPC_STOPPED 1        /* stopped after opts.stop_after_waves waves (debug) */
#define BGPC_EINVAL (-1)      /* bad argument, size or option */
#define BGPC_ENOMEM (-2)      /* device allocation failed */
#define BGPC_ECUDA (-3)       /* a CUDA runtime call failed */
#define BGPC_EROUNDS (-4)     /* more than opts.max_rounds rounds */
#define BGPC_ETIMEOUT (-5)    /* opts.timeout_us exceeded */
#define BGPC_EUNSORTED (-6)   /* adjacency not sorted / not unique / CSR and CSC disagree */
#define BGPC_EINTERNAL (-7)   /* a device-side consistency check failed */

/* ---- coloring policies (Sec. V) -------------------------------------- */
#define BGPC_FF 0   /* first fit (Alg. 2, lines 6-9) */
#define BGPC_B1 1   /* balancing heuristic B1 (Alg. ColorWorkQueue-B1) */
#define BGPC_B2 2   /* B2, update col_next = min(col+1, col_max/3+1) as in the algorithm box */
#define BGPC_B2X 3  /* B2, prose reading: start at least at col_max/3+1, i.e. max(...) */

#define BGPC_MAX_REPORT 64   /* rounds reported in bgpc_stats_t */

typedef struct bgpc_ctx bgpc_ctx_t;

/* Bipartite graph (Sec. II): nets(u) = a_idx[a_ptr[u] .. a_ptr[u+1]) for
 * u in V_A = [0, n_a), vtxs(v) = b_idx[b_ptr[v] .. b_ptr[v+1]) for v in
 * V_B = [0, n_b).  int32, sorted ascending, no duplicates, the two sides
 * describe the same edge set, nnz = a_ptr[n_a] = b_ptr[n_b] < 2^31. */
typedef struct {
    int32_t n_a, n_b, nnz;
    const int32_t *a_ptr, *a_idx;
    const int32_t *b_ptr, *b_idx;
} bgpc_graph_t;

/* Undirected graph for D2GC: adj(u) = idx[ptr[u] .. ptr[u+1]), symmetric,
 * sorted, unique, no self loops; nnz + n < 2^31. */
typedef struct {
    int32_t n, nnz;
    const int32_t *ptr, *idx;
} bgpc_ugraph_t;

/* Options.  The semantic parameters (policy, chunk, waves, big_net, rank)
 * fix the result bit for bit; nothing else (block sizes, autotuned mapping)
 * changes it.  Round-synchronous semantics RS(C, Q, T, policy, rank):
 *   round r colors W_r (rank order) in chunks of C consecutive entries, the
 *   chunks split into Q waves; every chunk of a wave reads the colors
 *   published by the earlier waves and colors its own vertices one after the
 *   other, as one of the paper's threads with OpenMP chunk C would (V-V-64,
 *   Sec. VI); vertices whose largest net has more than T members take the
 *   reverse first-fit color of Alg. 8 (k-th free color below |vtxs(v)|);
 *   then conflicts are removed per net, the lower rank keeping its color
 *   (Alg. 3 rule, Alg. 7 traversal), and the losers form W_{r+1}. */
typedef struct {
    int32_t policy;          /* BGPC_FF, BGPC_B1, BGPC_B2, BGPC_B2X */
    int32_t chunk;           /* C in [1, 64]; default 64 */
    int32_t waves;           /* Q >= 1; default 16 */
    int32_t big_net;         /* T >= 0; default 64; INT32_MAX disables Alg. 8's rule */
    const int32_t *rank;     /* device, permutation of [0, n_a), or NULL for id order */
    int32_t max_rounds;      /* BGPC_EROUNDS beyond this; default 1000 */
    int32_t validate;        /* 1: check sortedness, ranges, CSR/CSC agreement, rank
                                (0: the graph is trusted as given) */
    int64_t stop_after_waves;/* debug: > 0 stops after that many waves (all rounds
                                counted, empty waves too) and returns BGPC_STOPPED */
    int32_t *W_out;          /* debug, device [n_a] or NULL: work queue when stopped */
    int32_t want_balance;    /* 1: fill the color-set statistics of bgpc_stats_t */
    int32_t profile;         /* 1: time each phase with CUDA events on `stream`
                                (the ms_* fields of bgpc_stats_t) */
    int32_t stop_before_removal; /* debug: when stop_after_waves lands on the end
                                of a round, stop before its conflict removal
                                (colors = every vertex's tentative color,
                                stopped_wave = waves) */
    int32_t batch_streams;   /* bgpc_color_batched only: graphs colored concurrently
                                (0 = 8); a mapping parameter, results do not change */
    int32_t detect;          /* conflict detection of rounds after the first:
                                BGPC_DETECT_AUTO (0), BGPC_DETECT_NETS (every net
                                scanned) or BGPC_DETECT_PAIRS (only the (W member,
                                net) pairs, through a hash table); a mapping
                                parameter, results do not change */
    int32_t gather;          /* large-vertex gather: BGPC_GATHER_AUTO (0: one warp per
                                piece with its own bitmap when eight bitmaps fit in
                                a CTA's shared memory, else one CTA per piece) or
                                BGPC_GATHER_CTA (1: always one CTA per piece); a
                                mapping parameter, results do not change */
    int32_t net_rounds;      /* semantic: 1 colors the first round net by net (Alg. 8;
                                Alg. 9's order for D2GC) instead of by vertex waves,
                                the N1-* schedules of Sec. VI; 0 (default) = V-*.
                                A net round counts as one wave for stop_after_waves.
                                Other values: BGPC_EINVAL (see bgpc_color) */
    int64_t timeout_us;      /* > 0: wall-clock limit of the call in microseconds,
                                checked each time the host waits for the device (after
                                the setup and after every round); when exceeded the
                                call returns BGPC_ETIMEOUT (outputs undefined).
                                0 = no limit */
    int32_t batch_engine;    /* bgpc_color_batched only, a mapping parameter (results do
                                not change): BGPC_BATCH_PERSISTENT (0, default: one
                                persistent launch with a device task queue, captured
                                in a CUDA graph) or BGPC_BATCH_STREAMS (1: the
                                single-graph engine on batch_streams host workers) */
    int32_t batch_mapping;   /* BGPC_BATCH_PERSISTENT: 0 = the mapping the autotuner
                                measured fastest for this batch (tuned on the first
                                call, then cached in the context); k in
                                [1, BGPC_BATCH_MAPPINGS] = candidate k - 1 */
    int32_t reserved[2];
} bgpc_opts_t;

enum { BGPC_BATCH_PERSISTENT = 0, BGPC_BATCH_STREAMS = 1 };
#define BGPC_BATCH_MAPPINGS 12   /* autotuner candidates of the persistent engine */

enum { BGPC_DETECT_AUTO = 0, BGPC_DETECT_NETS = 1, BGPC_DETECT_PAIRS = 2 };
enum { BGPC_GATHER_AUTO = 0, BGPC_GATHER_CTA = 1 };

/* Statistics of one call (host struct). */
typedef struct {
    int32_t rounds;                       /* rounds run */
    int32_t colors;                       /* max color + 1 */
    int64_t w_per_round[BGPC_MAX_REPORT]; /* |W_r| */
    int64_t trav_per_round[BGPC_MAX_REPORT]; /* sum over W_r of sum over nets(w) (|vtxs|-1) */
    int64_t trav_total;                   /* all rounds */
    int32_t stopped_m;                    /* when BGPC_STOPPED: |W_r| of the current round */
    int32_t stopped_wave;                 /* when BGPC_STOPPED: index of the next wave */
    int32_t n_sets;                       /* non-empty color sets (want_balance) */
    int32_t max_card;                     /* largest color set (want_balance) */
    double mean_card, std_card;           /* over non-empty sets (want_balance) */
    int64_t incid_total;                  /* all rounds: sum over W_r of |nets(w)| */
    int64_t w_total;                      /* all rounds: sum of |W_r| */
    int64_t trav_large, incid_large, w_large; /* the same three over the vertices taking
                                                 the multi-CTA gather path */
    int64_t pieces_total;                 /* gather work items, all rounds */
    int64_t kernel_launches;              /* kernels this call launched */
    int64_t color_launches;               /* wave-coloring kernel launches */
    double ms_setup, ms_color, ms_publish, ms_detect, ms_gather; /* device time per phase (profile) */
    int64_t trav_hub;    /* all rounds: the part of trav_large in hub nets (more than
                            hub_threshold members), read from per-net color bitmaps instead
                            of streamed */
    int64_t hub_pairs;   /* all rounds: (vertex, hub net) pairs so read */
    int64_t hub_words;   /* all rounds: bitmap words so read (under first fit a one-piece
                            vertex reads only the words its summary needs) */
    double ms_total;     /* host wall-clock time of the whole call (it synchronises its
                            stream, so this covers all of its device work) */
    int32_t hub_threshold; /* nets with more members are hubs: the smallest of 512 * 2^(k/2)
                              whose hubs' first-round bitmaps fit in half the L2 cache
                              (INT32_MAX: no net qualifies); batched calls: the
                              smallest over the graphs */
    int32_t hubs;        /* hub nets (batched calls: summed over the graphs) */
} bgpc_stats_t;

/* Fill `opts` with the defaults: FF, C=64, Q=16, T=64, id order,
 * max_rounds=1000, no validation, no stop, no balance statistics. */
void bgpc_opts_default(bgpc_opts_t *opts);

/* Create a context on CUDA device `device` (made current for the call). */
int bgpc_ctx_create(bgpc_ctx_t **ctx, int device);
int bgpc_ctx_destroy(bgpc_ctx_t *ctx);

/* BGPC (Sec. III; Alg. 1 round loop, Alg. 4 vertex-based two-hop gather,
 * Alg. 8 reverse first fit for big nets, Alg. 7 net-based conflict removal
 * with the Alg. 3 lower-rank-wins rule, Sec. V balancing).
 * With opts.net_rounds = 1 the first round is Alg. 8's net-based coloring:
 * every net proposes the colors |vtxs(v)| - 1, |vtxs(v)| - 2, ... to its
 * members in adjacency order (all are uncolored, so F is empty), every
 * vertex keeps the proposal of its owner net (its largest net, ties to the
 * larger id, standing for the paper's last writer) and a vertex without nets
 * stays uncolored for the next round; the conflict removal and the later
 * vertex-based rounds are unchanged.  The net round reads nnz entries instead
 * of the two-hop volume; it uses reverse first fit whatever opts.policy.
 * colors: device int32 [n_a], written on BGPC_OK (or the snapshot on
 * BGPC_STOPPED).  stats (host) may be NULL.  Synchronises `stream`. */
int bgpc_color(bgpc_ctx_t *ctx, const bgpc_graph_t *g, const bgpc_opts_t *opts,
               int32_t *colors, bgpc_stats_t *stats, void *stream);

/* Batched BGPC: colors n_graphs independent bipartite graphs with one call
 * (no counterpart in the paper, which colors one graph at a time).  Every
 * graph gets exactly the coloring that bgpc_color gives it with the same
 * opts (id order).  By default (opts.batch_engine = BGPC_BATCH_PERSISTENT)
 * one persistent kernel colors all graphs: per graph a device ticket hands
 * out the tasks of its current phase (waves, publication, detection,
 * compaction) to whichever CTA is free, and the launch sequence is captured
 * in a CUDA graph that later calls on the same batch replay; a graph whose
 * colors outgrow the engine's shared-memory window is then colored by the
 * single-graph engine.  graphs: host array [n_graphs] of graphs with device
 * arrays; colors: host array [n_graphs] of device int32 pointers ([n_a]
 * each).  stats (host, may be NULL): the whole batch (rounds and colors =
 * the largest over the graphs; the per-round and total counters summed).
 * rounds_out / ncolors_out: host [n_graphs] or NULL, per graph.  opts.rank
 * must be NULL, opts.stop_after_waves and opts.net_rounds 0 (else
 * BGPC_EINVAL); n_graphs in [1, 65535].  BGPC_ETIMEOUT if the persistent
 * launch made no progress for opts.timeout_us (default 10 s).  Synchronises
 * `stream`. */
int bgpc_color_batched(bgpc_ctx_t *ctx, int32_t n_graphs, const bgpc_graph_t *graphs,
                       const bgpc_opts_t *opts, int32_t *const *colors, bgpc_stats_t *stats,
                       int32_t *rounds_out, int32_t *ncolors_out, void *stream);

/* D2GC (Sec. IV, Alg. 9-10): BGPC on the closed neighbourhoods
 * nets(u) = vtxs(u) = N[u] = {u} u adj(u), built on the device; the reverse
 * first fit starts at |N[v]| - 1 = |nbor(v)| as in Alg. 9.
 * colors: device int32 [n]. */
int d2gc_color(bgpc_ctx_t *ctx, const bgpc_ugraph_t *g, const bgpc_opts_t *opts,
               int32_t *colors, bgpc_stats_t *stats, void *stream);

/* Validity check (Sec. II definition): *n_bad (host) = number of V_A vertices
 * that are uncolored or share a color with a vertex of a common net. */
int bgpc_validate(bgpc_ctx_t *ctx, const bgpc_graph_t *g, const int32_t *colors,
                  int64_t *n_bad, void *stream);

/* Color-set statistics (Sec. VI-C, Table VI): card (device int64 [max_colors])
 * receives the cardinality of every color 0..max_colors-1 (colors >= max_colors
 * are an error); *n_sets, *max_card (host) and *mean_card, *std_card (host,
 * over non-empty sets) may each be NULL. */
int bgpc_color_sets(bgpc_ctx_t *ctx, const int32_t *colors, int32_t n, int64_t *card,
                    int32_t max_colors, int32_t *n_sets, int32_t *max_card,
                    double *mean_card, double *std_card, void *stream);

/* Color-set statistics that allocate nothing (no counterpart in the paper:
 * this is a calling convention, not a step of the method).  For callers that
 * cannot allocate device memory: code under an allocator that owns the whole
 * device memory budget (a framework's caching allocator, a fixed budget), and
 * latency-critical loops that must not enter the driver's allocator, whose
 * cudaMalloc / cudaFree can synchronise the device.  Same results as
 * bgpc_color_sets without the cardinality array and without a context: the
 * histogram lives in a fixed device array of BGPC_NOALLOC_MAX_COLORS 64-bit
 * counters (8 MiB, held by every GPU that loads the library until exit).
 * colors: device int32 [n] on the current device, each in [0, max_colors);
 * max_colors in [1, BGPC_NOALLOC_MAX_COLORS], else BGPC_EINVAL (also for a
 * color out of range, and for a colors array on another device or in
 * unregistered host memory).  Outputs are host pointers (each may be NULL).
 * The first call on a device looks up the array's device address (make it
 * before any stream capture; after cudaDeviceReset the cached address is
 * stale, so do not call it again in that process).  All calls share the
 * array: calls that overlap on the GPU race.  Copies the accumulators to the
 * host and synchronises `stream`. */
#define BGPC_NOALLOC_MAX_COLORS (1 << 20)
int bgpc_color_sets_noalloc(const int32_t *colors, int32_t n, int32_t max_colors,
                            int32_t *n_sets, int32_t *max_card, double *mean_card,
                            double *std_card, void *stream);

/* ---- learned vertex order ---------------------------------------------
 * The paper colors in a given vertex order and discusses how static orders
 * (natural, smallest-last) change the number of colors (Sec. VI, Table II).
 * These calls build an order from a small regression model instead: per
 * vertex features -> MLP 8 -> 64 -> 64 -> 1 (ReLU, bfloat16 weights, float32
 * arithmetic) -> score -> rank (decreasing score first); the rank is then
 * passed as bgpc_opts_t.rank.  The model itself is not in the paper.
 *
 * Parameter packing (float, 4801 values): W1[64][8] at 0, b1[64] at 512,
 * W2[64][64] at 576, b2[64] at 4672, W3[64] at 4736, b3 at 4800 (row-major,
 * row = output unit).  z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2,
 * h2 = relu(z2), score = W3 . h2 + b3, computed with the bfloat16 values of
 * the weights (w_bf16). */
#define BGPC_MLP_IN 8
#define BGPC_MLP_HIDDEN 64
#define BGPC_MLP_PARAMS 4801

typedef struct {
    float *w;           /* device [4801]: float32 master parameters, caller-initialised */
    uint16_t *w_bf16;   /* device [4801]: their bfloat16 values (bgpc_mlp_sync) */
    float *adam_m;      /* device [4801]: Adam first moments, caller-zeroed */
    float *adam_v;      /* device [4801]: Adam second moments, caller-zeroed */
    int64_t step;       /* (host) Adam steps taken so far, caller-zeroed */
} bgpc_mlp_t;

/* Features X (device float [n_a][8]) of every V_A vertex w, from the sizes
 * s_v = |vtxs(v)| of its nets: log1p of |nets(w)|, mean s, max s, sum s,
 * sum (s - 1) (the two-hop volume of Sec. III), min s, #{v : s_v > big_net},
 * sum s^2 / sum s.  A vertex with no nets gets zeros.  big_net >= 0. */
int bgpc_features(bgpc_ctx_t *ctx, const bgpc_graph_t *g, int32_t big_net, float *X,
                  void *stream);

/* w_bf16 <- bfloat16(w), round to nearest even (call after writing w). */
int bgpc_mlp_sync(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, void *stream);

/* score (device float [n]) of the rows of X (device float [n][8]). */
int bgpc_mlp_forward(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, const float *X, int32_t n,
                     float *score, void *stream);

/* Gradient (device float [4801]) of L = mean_i (score_i - y_i)^2 with respect
 * to the (bfloat16-valued) parameters, and *loss = L (host, may be NULL).
 * Deterministic: the reduction order does not depend on timing.  n >= 1.
 * Synchronises `stream` when loss is not NULL. */
int bgpc_mlp_grad(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, const float *X, const float *y,
                  int32_t n, float *grad, float *loss, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on w with
 * the gradient grad (device float [4801]); increments mlp->step, refreshes
 * w_bf16. */
int bgpc_mlp_adam(bgpc_ctx_t *ctx, bgpc_mlp_t *mlp, const float *grad, float lr, void *stream);

/* bgpc_mlp_grad followed by bgpc_mlp_adam (the gradient in context scratch);
 * *loss (host, may be NULL) is the loss before the step. */
int bgpc_mlp_train_step(bgpc_ctx_t *ctx, bgpc_mlp_t *mlp, const float *X, const float *y,
                        int32_t n, float lr, float *loss, void *stream);

/* rank (device int32 [n]) = position of every index in the order of
 * decreasing score (device float [n]), equal scores by increasing index;
 * -0.0 and +0.0 are equal; a NaN score is BGPC_EINVAL.  A stable LSD radix
 * sort on order-preserving 32-bit keys.  Synchronises `stream`. */
int bgpc_rank_from_scores(bgpc_ctx_t *ctx, const float *score, int32_t n, int32_t *rank,
                          void *stream);

/* Smallest-last order (the static order of Sec. VI, Tables II and IV) as a
 * rank for bgpc_color: on the conflict graph (u ~ w iff they share a net) the
 * vertices are removed one at a time, always a remaining vertex of smallest
 * remaining degree (ties: the smallest id), and rank[w] = the position of w in
 * the reverse removal order.  Each removal depends on all the earlier ones,
 * so the order is built by one host thread (the graph is copied from the
 * device; O(E2 log n) time); the coloring in that order runs on the GPU.
 * rank: device int32 [n_a]; *degeneracy (host, may be NULL) = the largest
 * degree at removal (first fit in this order uses at most degeneracy + 1
 * colors).  BGPC_ENOMEM if the conflict graph has more than max_pairs
 * (distinct ordered) neighbour pairs.  Synchronises `stream`. */
int bgpc_rank_smallest_last(bgpc_ctx_t *ctx, const bgpc_graph_t *g, int64_t max_pairs,
                            int32_t *rank, int32_t *degeneracy, void *stream);

/* Human-readable text of a status code (static storage). */
const char *bgpc_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* BGPC_H */
