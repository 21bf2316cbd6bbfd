// Internal declarations of the GB300 BGPC/D2GC library (not part of the ABI).
//
// Device data layout (all int32 unless noted; sizes for the power-law 4M x 4M
// graph in brackets):
//   graph (caller)  a_ptr[n_a+1] a_idx[nnz] b_ptr[n_b+1] b_idx[nnz]    [~0.55 GB]
//   tpos[nnz]       CSR entry -> CSC position of the same edge (static)
//   nc[nnz]         net-major color mirror: nc[f] for CSC entry f of net v is
//                   the published color of b_idx[f], or -2 - pos if b_idx[f]
//                   is in the current work queue W at position pos and not yet
//                   published.  The two-hop gather of Alg. 4 streams nc
//                   contiguously per net instead of gathering c[b_idx[f]].
//   npos[nnz]       net-major W position (-1 when not in W), for detection
//   nown[nnz] (u8)  1 if b_idx[f] owns net v (largest net, ties larger id)
//   s_own, d2tot [n_a]   |vtxs(own(w))| and sum over nets(w) of |vtxs(v)|
//   W0/W1, kofs, stage, newpos [n_a], lose [n_a] (u8)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bgpc.h"

namespace bgpc {

// ---------------------------------------------------------------- errors
enum : int32_t {
  ERR_RANGE = 1,      // index out of range / bad pointer array
  ERR_UNSORTED = 2,   // adjacency not sorted or has duplicates
  ERR_MISMATCH = 4,   // CSR and CSC disagree
  ERR_RANK = 8,       // rank is not a permutation
  ERR_INTERNAL = 16,  // a device consistency check failed
  ERR_COLOR = 32,     // a color outside the bound the kernels were sized for
};

constexpr int kMaxChunk = 64;       // C <= 64: adjacency masks are 64-bit
constexpr int kSmallWindow = 512;   // bits of the per-vertex small-path window
constexpr int kSmallD2 = 448;       // small path: sum of net sizes <= this
constexpr int kSmallMaxDeg = 16;    // small path: at most this many nets
constexpr int kPairCap = kMaxChunk * kSmallMaxDeg;  // (vertex, net) pairs per chunk
constexpr int kPiece = 32;          // gather work item: up to this many nets of one vertex
constexpr int kDetectWarpMax = 32;  // nets up to this size use the warp tier
// First-fit summary of a large vertex's forbidden set F_S (written by the
// gather, read by the resolve): the kSumCand smallest free colors, the free
// colors from the k-th below the owner-net top on (reverse first fit), their
// count, and the 64-bit chunk-mate mask.  A chunk adds at most C - 1 <= 63
// colors to F_S, so 64 candidates always leave one free.
constexpr int kSumCand = 64;
constexpr int kSumInts = 2 * kSumCand + 4;  // cand | rcand | rcnt, pad | adj (u64)

// Hub nets (colors kept as bitmaps) have more members than a threshold taken
// per call from the ladder kHubMin * 2^(k/2), k < kHubLadder: the smallest
// one whose hubs' first-round bitmaps fit in half the L2 cache (bitmaps read
// from L2 cost less than streaming the members' mirror words; once they spill
// to DRAM they cost more).
constexpr int32_t kHubMin = 512;
constexpr int kHubLadder = 24;
__host__ __device__ inline int32_t hub_ladder(int k) { return ((k & 1) ? 724 : 512) << (k >> 1); }

// Device scalars shared by the kernels of one call.
struct DevScalars {
  int32_t err;
  int32_t gmax;      // largest color currently in c
  int32_t m_next;    // |W_{r+1}|
  int32_t nbig_t;    // nets with |vtxs| > T
  int32_t nbig_d;    // nets with |vtxs| > kDetectWarpMax
  int32_t maxnet;    // largest net
  int32_t maxcolor;  // for validation / statistics
  int32_t nseg;      // gather pieces of the round
  int32_t nhub;      // hub nets of the round (their colors kept as bitmaps)
  int32_t pad;
  unsigned long long trav;   // traversed two-hop entries of the round
  unsigned long long incid;  // incidences sum over W_r of |nets(w)| of the round
  unsigned long long trav_large, incid_large, w_large;  // the same over gathered (large) vertices
  unsigned long long trav_hub;   // two-hop entries of hub nets, read as bitmaps instead
  unsigned long long hub_pairs;  // (vertex, hub net) pairs gathered from bitmaps
  unsigned long long hub_words;  // hub bitmap words ORed by those pairs
  unsigned long long acc[4]; // reductions (statistics)
  unsigned long long incid_next;  // sum over W_{r+1} of |nets(w)| (set by the compaction)
  int32_t hub_hist[kHubLadder];   // nets with hub_ladder(k) < size <= hub_ladder(k + 1)
  int32_t hub_H;                  // the hub threshold of the call
  int32_t pad2;
};
constexpr int kRoundCounters = 8;  // trav .. hub_words, zeroed at the start of a round
template <typename T>
struct Buf {
  T *p = nullptr;
  size_t cap = 0;
};

// Batched coloring in one persistent launch (bgpc_batch.cu).
constexpr int kBatchReport = 64;  // rounds reported per graph
enum : int32_t {
  kBatchRunning = 0,
  kBatchDone = 1,
  kBatchWindow = 2,   // colors outgrew the shared-memory window: single-graph engine
  kBatchRounds = 3,   // more than max_rounds rounds
  kBatchFailed = 4,   // internal error
};
struct BatchDesc {    // one graph of the batch (read-only during the launch)
  const int32_t *a_ptr, *a_idx, *b_ptr, *b_idx;
  int32_t *colors;
  int32_t n_a, n_b, nnz, pad;
  int64_t voff;       // offset of the graph's vertex scratch (n_a entries per pool)
  int64_t noff;       // offset of its net scratch (n_b entries)
  int64_t toff;       // offset of its tile scratch (tiles of W + 1)
};
struct __align__(128) BatchState {  // one graph's progress (zeroed but for the ticket)
  unsigned long long ticket;  // sequence:16 | tasks of the phase:24 | next task:24
  int32_t done;               // finished tasks of the current phase
  int32_t ntasks;
  int32_t seq;
  int32_t phase, q, r, m, nch, cur;
  int32_t col_max0;           // chunk-private col_max at the start of a wave: max color published
  int32_t gmax_fixed;         // largest color of the vertices outside W_r
  int32_t gmax_wave;          // largest color published in this round so far
  int32_t gmax_win;           // largest color kept by this round's winners
  int32_t m_next, ntiles, nbig, status;
  int32_t tagged;             // this round's detection visits only nets tagged r + 1
  int32_t tag_next;           // the scatter tags the nets of W_{r+1} with r + 2
};
struct BatchStat {    // one graph's statistics (zeroed before the launch)
  int32_t rounds, colors, status, pad;
  int64_t w_per_round[kBatchReport];
  int64_t trav_per_round[kBatchReport];
  int64_t trav_total, w_total, incid_total;
};
constexpr int kBatchPosts = 1024;  // ring of recently posted graphs (a power of two)
struct BatchGlobal {
  int32_t finished;              // graphs done (or handed back)
  int32_t err;                   // 1: a CTA saw no progress for timeout_ns
  unsigned long long progress;   // phase advances so far
  uint32_t posts;                // phases posted so far ...
  int32_t post[kBatchPosts];     // ... and the graph of each, by post count mod the ring
};
struct BatchMapping {  // mapping parameters: they never change a result
  int32_t ww;          // forbidden-window words per vertex: 16, 32 or 64
  int32_t ctas_per_sm; // 0 = as many as fit
  int32_t cpt;         // a wave task covers cpt * Q chunk indices
  int32_t tile;        // vertices / queue positions / nets per task
  int32_t small_nch;   // a round of at most this many chunks runs as one task
};
}  // namespace bgpc

struct bgpc_ctx {
  int device = 0;
  // bgpc_color_batched: one sub-context (own scratch) and one stream per
  // concurrent worker, created on first use and kept with the context
  std::vector<bgpc_ctx *> subs;
  std::vector<cudaStream_t> sub_streams;
  int num_sms = 0;
  int smem_optin = 0;  // max dynamic shared memory per block (bytes)
  int l2_bytes = 0;    // L2 cache size
  bgpc::Buf<int32_t> tpos, nc, npos;
  bgpc::Buf<uint8_t> nown;
  bgpc::Buf<int32_t> s_own, d2tot, W0, W1, kofs, stage, newpos;
  bgpc::Buf<int32_t> netc;             // net-based first round: proposal of the owner net
  bgpc::Buf<int32_t> ihub;             // per CSR entry: hub slot of its net, or -1
  bgpc::Buf<int32_t> brow;             // setup scratch (nnz ints)
  bgpc::Buf<int32_t> thist, tsums;     // setup: digit counts of the tpos sort, scan scratch
  bgpc::Buf<int32_t> ownid;            // owner net of each vertex (-1: none)
  bgpc::Buf<int32_t> ksc[4], kgstart;  // kofs sort: scratch [n_a] x 4, group starts [n_b]
  bgpc::Buf<uint8_t> lose;
  bgpc::Buf<int32_t> blocksum, bigt, bigd;
  bgpc::Buf<int32_t> wlist;            // chunks of the round ordered by wave
  bgpc::Buf<int32_t> segoff;           // gather pieces: exclusive prefix in wave order
  bgpc::Buf<int4> segmap;              // gather piece -> {slot, vertex, first incidence,
                                       //   nets | pieces of the vertex << 6}
  bgpc::Buf<uint32_t> gbm;             // per-slot forbidden bitmaps of large vertices
  bgpc::Buf<int32_t> hub_id, hub_net;  // net -> hub slot (-1: not a hub), slot -> net
  bgpc::Buf<uint32_t> nbm;             // hub color bitmaps [nhub][words]
  bgpc::Buf<unsigned long long> gadj;  // per-slot chunk-mate adjacency of large vertices
  bgpc::Buf<int32_t> gcnt;             // per-slot count of merged pieces (first fit)
  bgpc::Buf<int32_t> gsum;             // per-slot first-fit summaries [kSumInts]
  bgpc::Buf<uint32_t> lbm;             // per-slot bitmaps kept for the reverse first fit
  size_t gbm_zeroed = 0;               // words of gbm (and slots of gadj, gcnt) known zero
  int32_t *h_wlist = nullptr;          // pinned host staging of wlist
  size_t h_wlist_cap = 0;
  bgpc::Buf<int32_t> cptr, cidx;       // D2GC closed neighbourhoods
  bgpc::Buf<int32_t> dtab;             // per-slot color tables (detection)
  bgpc::Buf<unsigned long long> pkeys; // pair-tier detection: slots of (net, color) key and
                                       // smallest position, 16 bytes each
  bgpc::Buf<int32_t> vtab;             // per-slot color counts (validation)
  size_t dtab_filled = 0;              // entries of dtab already set to INT_MAX
  bgpc::Buf<unsigned long long> card;  // color-set cardinalities
  bgpc::Buf<uint8_t> bad;              // validation flags
  bgpc::Buf<uint32_t> rkey0, rkey1;    // rank_from_scores: radix-sort keys (ping-pong)
  bgpc::Buf<int32_t> rval0, rval1;     // ... and the indices they carry
  bgpc::Buf<int32_t> rhist;            // ... per-tile digit counts, then their offsets
  bgpc::Buf<int32_t> rsum;             // ... scan block sums
  bgpc::Buf<float> mpart;              // MLP gradient: per-block partial sums
  bgpc::Buf<float> mgrad;              // MLP gradient (train step)
  // bgpc_color_batched, persistent engine: scratch pools over the whole batch
  bgpc::Buf<int32_t> bW0, bW1, bstage, bown, bsown, bd2, bkofs, bbig, btcnt, btofs, bntag;
  bgpc::Buf<uint8_t> blose, binW;
  bgpc::Buf<bgpc::BatchDesc> bdesc;
  bgpc::Buf<bgpc::BatchState> bst;
  bgpc::Buf<bgpc::BatchStat> bstat;
  bgpc::Buf<bgpc::BatchGlobal> bglob;
  void *h_batch = nullptr;             // pinned staging: descriptors, state, global, statistics
  size_t h_batch_cap = 0;
  cudaStream_t bstream = nullptr;      // private stream (capturable) of the persistent launch
  cudaEvent_t bev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t bexec = nullptr;     // captured launch of the last batch ...
  unsigned long long bkey = 0;         // ... and the batch it belongs to
  std::vector<std::pair<unsigned long long, int>> btuned;  // autotuned mapping per batch
  bgpc::DevScalars *dev = nullptr;     // device scalars
  std::vector<cudaEvent_t> events;     // phase timing (opts.profile)
  bgpc::DevScalars *host = nullptr;    // pinned mirror
};

namespace bgpc {

// Grow a device buffer to at least n elements (contents not preserved).
template <typename T>
inline cudaError_t grow(Buf<T> &b, size_t n) {
  if (n <= b.cap) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = n + n / 8 + 64;
  cudaError_t e = cudaMalloc((void **)&b.p, want * sizeof(T));
  if (e != cudaSuccess) return e;
  b.cap = want;
  return cudaSuccess;
}

template <typename T>
inline void release(Buf<T> &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------ launchers
// Setup (bgpc_setup.cu)
int launch_check_ptr(const int32_t *ptr, int32_t n, int32_t nnz, int32_t *err, cudaStream_t s);
int launch_check_rows(const int32_t *ptr, const int32_t *idx, int32_t n, int32_t bound,
                       int32_t *err, int sms, cudaStream_t s);
// tpos by a stable radix sort of the CSC indices by member id (scratch: four
// arrays of nnz ints; hist: tpos_hist_len(nnz) ints; sums: its scan scratch);
// validate: also check that CSR and CSC hold the same pairs.
int64_t tpos_hist_len(int64_t nnz);
int launch_tpos(const bgpc_graph_t &g, int32_t *tpos, int32_t *const scratch[4], int32_t *hist,
                int32_t *sums, int32_t validate, int32_t *err, const int32_t *hub_id,
                int32_t *ihub, int sms, cudaStream_t s);
// Exclusive scan of a[0, len) in place (sums: ceil(len / 4096) scratch ints).
int launch_excl_scan(int32_t *a, int64_t len, int32_t *sums, cudaStream_t s);
int launch_vertex_static(const bgpc_graph_t &g, const int32_t *tpos, int32_t *s_own,
                          int32_t *d2tot, uint8_t *nown, int32_t *netc, int32_t center_first,
                          int32_t *ownid, int sms, cudaStream_t s);
// kofs for W in id order, by a stable sort of the W positions by owner net
// (scratch: four arrays of m ints; hist: tpos_hist_len(m); gstart: n_b ints)
int launch_kofs_sorted(const int32_t *W, int32_t m, const int32_t *ownid, const int32_t *s_own,
                       int32_t T, int32_t n_b, int32_t *const scratch[4], int32_t *hist,
                       int32_t *sums, int32_t *gstart, int32_t *kofs, int sms, cudaStream_t s);
// The net-based first round (Alg. 8 / Alg. 9): its colors, computed by
// launch_vertex_static into netc, published into c and the mirror.
int launch_net_publish(const bgpc_graph_t &g, const int32_t *netc, const int32_t *rank,
                       int32_t *nc, int32_t *colors, uint8_t *lose, int sms, cudaStream_t s);
int launch_net_static(const bgpc_graph_t &g, int32_t T, int32_t *bigt, int32_t *bigd,
                       DevScalars *dev, cudaStream_t s);
int launch_init_queue(const int32_t *rank, int32_t n_a, int32_t *W, int32_t *err, cudaStream_t s);
int launch_init_mirror(const bgpc_graph_t &g, const int32_t *rank, int32_t *nc, int32_t *npos,
                       int32_t *colors, int sms, cudaStream_t s);
int launch_closed_nbhd(const bgpc_ugraph_t &g, int32_t *cptr, int32_t *cidx, int sms,
                        cudaStream_t s);

// Coloring (bgpc_color.cu)
struct WaveArgs {
  const int32_t *a_ptr, *a_idx, *b_ptr;
  const int32_t *nc;
  const int32_t *W;
  const int32_t *kofs;
  const int32_t *s_own;
  const int32_t *d2tot;
  int32_t *stage;
  const DevScalars *dev;
  int32_t *err;
  int32_t m, C, T;
  const int32_t *chunks;       // chunk indices of this wave
  int32_t nchunks;
  int32_t maxnet;
  int32_t words;               // forbidden-bitmap words per vertex (multiple of 4)
  int32_t small_ok;            // the small path is usable this round
  uint32_t *gbm;               // per-slot bitmaps of large vertices (slot = list index*C + i)
  unsigned long long *gadj;    // per-slot chunk-mate masks of large vertices
  const int32_t *gsum;         // first fit: per-slot summaries written by the gather
  const uint32_t *lbm;         // first fit: per-slot bitmaps of reverse first-fit vertices
};
struct GatherArgs {
  const int32_t *a_ptr, *a_idx, *b_ptr;
  const int32_t *nc;
  const int32_t *W;
  const int32_t *wlist;        // the round's chunks in wave order
  const int4 *segmap;          // piece -> {slot, vertex, first incidence, nets | pieces << 6}
  const int32_t *segoff;       // exclusive prefix of pieces over wave-order slots
  int32_t m, C;
  int32_t slot_lo, slot_hi;    // wave-order slots of this wave
  int32_t words;
  uint32_t *gbm;
  unsigned long long *gadj;
  const int32_t *b_idx;        // vtxs lists (chunk-mate search in hub nets)
  const int32_t *tpos;         // CSR entry (w, v) -> CSC index of w in vtxs(v)
  const int32_t *hub_id;       // net -> hub slot or -1
  const uint32_t *nbm;         // hub color bitmaps [nhub][words] (the wave snapshot)
  DevScalars *dev;             // hub counters
  int32_t id_order;            // W is in vertex-id order (no rank): a chunk's ids increase
  // first fit only (summ != 0): the gather ends with each large vertex's
  // summary (kSumInts per slot) instead of leaving its bitmap for the resolve
  int32_t summ;
  int32_t T;                   // reverse first fit for owners of nets larger than T
  const int32_t *s_own;        // vertex -> size of its owner net
  const int32_t *kofs;         // queue position -> reverse first-fit offset k
  int32_t *gcnt;               // per-slot merged-piece counts (zero at rest)
  int32_t *gsum;               // per-slot summaries
  uint32_t *lbm;               // per-slot bitmaps for the resolve's overlay tests
};
// Largest bitmap (in words) the wave kernels can hold in shared memory.
int32_t wave_max_words(int smem_optin);
cudaError_t launch_color_wave(int policy, const WaveArgs &a, int sms, cudaStream_t s);
cudaError_t launch_gather(const GatherArgs &a, bool cta_only, int sms, cudaStream_t s);
// Per round: pieces per wave-order slot, their prefix and the piece map.
int launch_pieces(const int32_t *a_ptr, const int32_t *d2tot, const int32_t *W,
                  const int32_t *wlist, int32_t nch, int32_t C, int32_t m, int32_t small_ok,
                  int32_t *segoff, int32_t *blocksum, int4 *segmap, DevScalars *dev,
                  cudaStream_t s);
int launch_publish(const int32_t *a_ptr, const int32_t *d2tot, const int32_t *ihub,
                   const int32_t *tpos, const int32_t *W, const int32_t *stage,
                   const int32_t *wlist, int32_t C, int32_t m, int32_t small_ok,
                   int32_t slot_lo, int32_t slot_hi, const int32_t *segoff, const int4 *segmap,
                   int32_t *nc, int32_t *colors, uint32_t *nbm, int32_t words, DevScalars *dev,
                   int sms, cudaStream_t s);
// Per round: hub nets (more than H members) get a slot (hub_id, -1 otherwise)
// and a color bitmap of their published members.
int launch_hub_select(const int32_t *b_ptr, int32_t n_b, int32_t C, int32_t Q,
                      int64_t budget_words, int32_t *hub_id, int32_t *hub_net, DevScalars *dev,
                      int sms, cudaStream_t s);
int launch_hub_build(const int32_t *b_ptr, const int32_t *nc, const int32_t *hub_net,
                     int32_t nhub, int32_t words, uint32_t *nbm, int sms, cudaStream_t s);

struct BatchLaunch {
  const BatchDesc *desc;
  BatchState *st;
  BatchStat *stat;
  BatchGlobal *glob;
  int32_t G, C, Q, T, max_rounds, policy, sms;
  int64_t timeout_ns;
  BatchMapping map;
  int32_t *W0, *W1, *stage, *own, *s_own, *d2, *kofs, *big, *tcnt, *tofs, *ntag;
  uint8_t *lose, *inW;
};
cudaError_t launch_batch(const BatchLaunch &L, cudaStream_t s);

// Wave of chunk j under Q waves: the Weyl sequence frac(j * phi), phi =
// 0x9E3779B9 / 2^32, scaled to [0, Q).
inline int32_t wave_of(int64_t j, int32_t Q) {
  uint32_t x = (uint32_t)((uint64_t)j * 0x9E3779B9ull);
  return (int32_t)(((uint64_t)x * (uint64_t)Q) >> 32);
}

// Detection, compaction, per-round bookkeeping (bgpc_detect.cu)
int launch_kofs(const int32_t *b_ptr, const int32_t *nc_unused, const int32_t *npos,
                 const uint8_t *nown, const int32_t *bigt, int32_t nbig, int32_t *kofs,
                 int sms, cudaStream_t s);
int launch_trav(const int32_t *a_ptr, const int32_t *W, const int32_t *d2tot, int32_t m,
                int32_t small_ok, DevScalars *dev, cudaStream_t s);
int launch_detect(const int32_t *b_ptr, int32_t n_b, const int32_t *nc, const int32_t *npos,
                   const int32_t *bigd, int32_t nbigd, int32_t *dtab, int32_t tabcap,
                   int32_t nslots, int32_t id_order, uint8_t *lose, int sms, cudaStream_t s);
int launch_detect_pairs(const int32_t *a_ptr, const int32_t *a_idx, const int32_t *W, int32_t m,
                        const int32_t *colors, unsigned long long *kv, uint32_t mask,
                        uint8_t *lose, int32_t *err, int sms, cudaStream_t s);
int launch_compact(const uint8_t *lose, const int32_t *W, int32_t m, int32_t *newpos,
                    int32_t *Wn, int32_t *blocksum, const int32_t *a_ptr, DevScalars *dev,
                    cudaStream_t s);
int launch_relabel_csc(int64_t nnz, const int32_t *W, int32_t m, uint8_t *lose,
                       const int32_t *newpos, int32_t *nc, int32_t *npos, int32_t *colors,
                       int sms, cudaStream_t s);
int launch_relabel(const int32_t *a_ptr, const int32_t *tpos, const int32_t *W, int32_t m,
                    uint8_t *lose, const int32_t *newpos, int32_t *nc, int32_t *npos,
                    int32_t *colors, int sms, cudaStream_t s);
int launch_gmax(const int32_t *colors, int32_t n, DevScalars *dev, cudaStream_t s);
int launch_fill(int32_t *p, size_t n, int32_t v, cudaStream_t s);

// Statistics and validation (bgpc_metrics.cu)
int launch_card(const int32_t *colors, int32_t n, unsigned long long *card, int32_t ncard,
                 int32_t *err, cudaStream_t s);
int launch_card_stats(const unsigned long long *card, int32_t ncard, DevScalars *dev,
                       cudaStream_t s);
int launch_validate(const bgpc_graph_t &g, const int32_t *colors, const int32_t *bigd,
                     int32_t nbigd, int32_t *tab, int32_t tabcap, int32_t nslots,
                     uint8_t *bad, DevScalars *dev, int sms, cudaStream_t s);

}  // namespace bgpc
