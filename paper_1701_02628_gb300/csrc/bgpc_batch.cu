// Batched coloring: many independent graphs in one persistent launch with a
// device task queue (bgpc_color_batched).  No counterpart in the paper, which
// colors one graph at a time.
//
// Every graph is colored exactly as bgpc_color colors it alone, under the
// round-synchronous semantics RS(C, Q, T, policy) in id order: the same
// chunks, waves, policies, reverse first fit (Alg. 8 per vertex) and conflict
// rule (Alg. 3, lower id wins).  Only the execution differs.  The
// single-graph engine issues a few launches per wave and per round, which
// leaves a batch of small graphs launch-bound; here one kernel runs the whole
// batch:
//
//  * Every graph walks through phases (analysis, then per round: reverse
//    first-fit offsets, Q x (color wave q, publish wave q), conflict
//    detection, loser count, scan, scatter).  A phase is a set of tasks.
//  * The task queue is one 64-bit ticket per graph: sequence (16 bits), task
//    count of the current phase (24 bits) and next task index (24 bits).  A
//    CTA claims a task with one atomicAdd and knows from the returned word
//    which phase it claimed and whether the index is valid; the CTA that
//    finishes a phase's last task sets up the next phase (its parameters
//    first, a fence, then a fresh ticket).  A task never waits for another:
//    it is only created once the tasks it depends on are done, so the launch
//    cannot deadlock however many CTAs are resident.
//  * A CTA that finds no task sleeps and retries; if the batch makes no
//    progress for `timeout_ns` it records an error and returns (bounded
//    wait), and every CTA returns once any CTA has recorded one.
//  * Data that other CTAs write during the launch (colors, work queues,
//    staged colors, flags, per-graph state) is read through L2 (ld.global.cg),
//    never from a possibly stale L1 line; writes are followed by a fence
//    before the completion count.
//  * The per-chunk coloring is done by one CTA: the two-hop colors of all the
//    chunk's vertices are gathered at once (flattened over (vertex, net,
//    member)) into one forbidden window per vertex in shared memory (WW
//    words), earlier chunk-mates that are neighbours into a 64-bit mask; then
//    the vertices are resolved in chunk order (under first fit, those with no
//    earlier neighbour all at once).  Colors are read from c[] directly (the
//    batch's graphs are small; their color arrays stay in L2).
//  * A graph whose colors do not fit the window (a search that would have to
//    look at a color >= 32 * WW) stops and is marked for the single-graph
//    engine, which the host runs on it afterwards: same result, other mapping.
#include "bgpc_internal.cuh"

namespace bgpc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBT = 256;          // threads per CTA
constexpr int kBW = kBT / 32;     // warps per CTA
constexpr int kPairBatch = 1024;  // (vertex, net) pairs gathered at once
constexpr int kThreadNet = 32;    // nets up to this size are walked by one thread

enum : int32_t {
  BP_ANALYZE = 0,
  BP_KOFS = 1,
  BP_WAVE = 2,
  BP_PUBLISH = 3,
  BP_DETECT = 4,
  BP_COUNT = 5,
  BP_SCAN = 6,
  BP_SCATTER = 7,
  BP_ROUND = 8,    // a small graph's whole round in one task
};

__device__ __forceinline__ int32_t ldcg(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldcg8(const uint8_t *p) {
  return (uint8_t)__ldcg(reinterpret_cast<const unsigned char *>(p));
}

__device__ __forceinline__ int32_t wave_of_dev(int64_t j, int32_t Q) {
  const uint32_t x = (uint32_t)((uint64_t)j * 0x9E3779B9ull);
  return (int32_t)(((uint64_t)x * (uint64_t)Q) >> 32);
}

__device__ __forceinline__ unsigned long long make_ticket(uint32_t seq, int32_t ntasks) {
  return ((unsigned long long)(seq & 0xffffu) << 48) |
         ((unsigned long long)(uint32_t)ntasks << 24);
}

__device__ __forceinline__ int32_t warp_incl_scan(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan over the CTA's threads; *total = sum (two barriers).
__device__ __forceinline__ int32_t cta_excl_scan(int32_t v, int32_t *red, int32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t inc = warp_incl_scan(v);
  if (lane == 31) red[warp] = inc;
  __syncthreads();
  int32_t before = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kBW; i++) {
    const int32_t r = red[i];
    before += (i < warp) ? r : 0;
    tot += r;
  }
  __syncthreads();
  *total = tot;
  return before + inc - v;
}

// ---------------------------------------- window searches (one warp, smem)
// bm: WW words, bit x set = color x forbidden.  Lane l owns words l and l+32.
// Each returns -1 when the answer is not inside the window.

template <int WW>
__device__ __forceinline__ int32_t win_first_free(const uint32_t *bm, int32_t p) {
  const int lane = threadIdx.x & 31;
  if (p < 0) p = 0;
#pragma unroll
  for (int h = 0; h < (WW + 31) / 32; h++) {
    const int32_t wi = lane + 32 * h;
    uint32_t fr = 0u;
    if (wi < WW) {
      fr = ~bm[wi];
      const int32_t lo = wi * 32;
      if (p >= lo + 32) fr = 0u;
      else if (p > lo) fr &= kFull << (p - lo);
    }
    const unsigned b = __ballot_sync(kFull, fr != 0u);
    if (b) {
      const int fl = __ffs(b) - 1;
      const uint32_t fw = __shfl_sync(kFull, fr, fl);
      return (fl + 32 * h) * 32 + __ffs(fw) - 1;
    }
  }
  return -1;
}

template <int WW>
__device__ __forceinline__ int32_t win_last_free(const uint32_t *bm, int32_t p) {
  const int lane = threadIdx.x & 31;
  if (p < 0) return -1;
  if (p >= WW * 32) return -2;  // the search would start outside the window
#pragma unroll
  for (int h = (WW + 31) / 32 - 1; h >= 0; h--) {
    const int32_t wi = lane + 32 * h;
    uint32_t fr = 0u;
    if (wi < WW) {
      fr = ~bm[wi];
      const int32_t lo = wi * 32;
      if (p < lo) fr = 0u;
      else if (p < lo + 31) fr &= kFull >> (31 - (p - lo));
    }
    const unsigned b = __ballot_sync(kFull, fr != 0u);
    if (b) {
      const int fl = 31 - __clz(b);
      const uint32_t fw = __shfl_sync(kFull, fr, fl);
      return (fl + 32 * h) * 32 + 31 - __clz(fw);
    }
  }
  return -1;
}

// k-th (0-based) free color counting down from top (top < 32 * WW), or -1.
template <int WW>
__device__ __forceinline__ int32_t win_kth_free_down(const uint32_t *bm, int32_t top, int32_t k) {
  const int lane = threadIdx.x & 31;
  int32_t remaining = k;
#pragma unroll
  for (int h = (WW + 31) / 32 - 1; h >= 0; h--) {
    const int32_t wi = lane + 32 * h;
    uint32_t fr = 0u;
    if (wi < WW) {
      fr = ~bm[wi];
      const int32_t lo = wi * 32;
      if (top < lo) fr = 0u;
      else if (top < lo + 31) fr &= kFull >> (31 - (top - lo));
    }
    const int32_t cnt = __popc(fr);
    int32_t suf = cnt;  // free colors in this lane and the lanes above it
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_down_sync(kFull, suf, o);
      if (lane + o < 32) suf += y;
    }
    const int32_t total = __shfl_sync(kFull, suf, 0);
    if (remaining < total) {
      const int32_t above = suf - cnt;
      const bool mine = above <= remaining && remaining < above + cnt;
      int32_t res = -1;
      if (mine) {
        int32_t r = remaining - above;
        uint32_t f = fr;
        while (true) {
          const int32_t x = 31 - __clz(f);
          if (r == 0) {
            res = wi * 32 + x;
            break;
          }
          f &= ~(1u << x);
          r--;
        }
      }
      const unsigned b = __ballot_sync(kFull, mine);
      return __shfl_sync(kFull, res, __ffs(b) - 1);
    }
    remaining -= total;
  }
  return -1;
}

struct BArgs {
  const BatchDesc *desc;
  BatchState *st;
  BatchStat *stat;
  BatchGlobal *glob;
  int32_t G, C, Q, T, max_rounds;
  int32_t tile;          // vertices / positions / nets per task
  int32_t cpt;           // chunk indices per wave task = cpt * Q
  int32_t small_nch;     // rounds of at most this many chunks run as one task
  int64_t timeout_ns;
  int32_t *W0, *W1, *stage, *own, *s_own, *d2, *kofs, *big, *tcnt, *tofs, *ntag;
  uint8_t *lose, *inW;
};

// ------------------------------------------------------------- the phases

// The parameters of the phase a task belongs to, read once through L2 when
// the task starts (they stay fixed until every task of the phase is done).
struct PhaseView {
  int32_t phase, q, m, nch, cur, col_max0, r, nbig, ntiles, tagged, tag_next;
};

__device__ __forceinline__ PhaseView view_of(const BatchState *S) {
  const volatile BatchState *V = S;
  PhaseView p;
  p.phase = V->phase;
  p.q = V->q;
  p.m = V->m;
  p.nch = V->nch;
  p.cur = V->cur;
  p.col_max0 = V->col_max0;
  p.r = V->r;
  p.nbig = V->nbig;
  p.ntiles = V->ntiles;
  p.tagged = V->tagged;
  p.tag_next = V->tag_next;
  return p;
}

template <int WW>
struct ChunkSmem {
  int32_t w[kMaxChunk], ab[kMaxChunk], deg[kMaxChunk], so[kMaxChunk], k[kMaxChunk];
  int32_t col[kMaxChunk], pinc[kMaxChunk];
  unsigned long long adj[kMaxChunk];
  uint32_t bm[kMaxChunk][WW];
  int32_t pstart[kPairBatch], psize[kPairBatch];  // queued large pairs
  uint8_t pv[kPairBatch];
  int32_t red[kBW];
  int32_t nbigp;
};

// Color chunk j of the graph's current round (RS semantics): writes the
// tentative colors of its positions into stage[].  Returns false (and marks
// the graph for the single-graph engine) if a search left the window.
template <int POLICY, int WW>
__device__ void color_chunk(const BArgs &A, const BatchDesc &D, const PhaseView &S,
                            const int32_t *Wc, int32_t j, ChunkSmem<WW> &sm, int32_t *flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t C = A.C, m = S.m;
  const int32_t p0 = j * C, n = min(C, m - p0);
  const int64_t vo = D.voff;
  if (tid < n) {
    const int32_t w = ldcg(Wc + p0 + tid);
    const int32_t ab = D.a_ptr[w];
    const int32_t so = ldcg(A.s_own + vo + w);
    sm.w[tid] = w;
    sm.ab[tid] = ab;
    sm.deg[tid] = D.a_ptr[w + 1] - ab;
    sm.so[tid] = so;
    sm.k[tid] = (so > A.T) ? ldcg(A.kofs + vo + w) : 0;
    sm.adj[tid] = 0ull;
  }
  for (int x = tid; x < kMaxChunk * WW; x += kBT) (&sm.bm[0][0])[x] = 0u;
  __syncthreads();
  // inclusive prefix of the degrees (pair index -> vertex)
  if (warp == 0) {
    const int32_t d0 = lane < n ? sm.deg[lane] : 0;
    const int32_t d1 = lane + 32 < n ? sm.deg[lane + 32] : 0;
    const int32_t i0 = warp_incl_scan(d0);
    const int32_t t0 = __shfl_sync(kFull, i0, 31);
    const int32_t i1 = warp_incl_scan(d1) + t0;
    sm.pinc[lane] = i0;
    sm.pinc[lane + 32] = i1;
  }
  __syncthreads();
  const int32_t P = sm.pinc[n - 1];
  const int32_t wlo = sm.w[0];
  // one member u of a net of vertex i: a published color joins i's window,
  // an uncolored earlier chunk-mate joins its adjacency mask
  auto take = [&](int32_t i, int32_t u, int32_t c) {
    const int32_t wi = sm.w[i];
    if (u == wi) return;
    if (c >= 0) {
      if (c < WW * 32) atomicOr(&sm.bm[i][c >> 5], 1u << (c & 31));
    } else if (u >= wlo && u < wi) {
      // uncolored in the snapshot: an earlier chunk-mate if it is in the
      // chunk (the chunk's ids increase)
      int32_t a = 0, b = i - 1;
      while (a < b) {
        const int32_t mid = (a + b) >> 1;
        if (sm.w[mid] < u) a = mid + 1; else b = mid;
      }
      if (i > 0 && sm.w[a] == u) atomicOr(&sm.adj[i], 1ull << a);
    }
  };
  for (int32_t pb = 0; pb < P; pb += kPairBatch) {
    const int32_t np = min(kPairBatch, P - pb);
    if (tid == 0) sm.nbigp = 0;
    __syncthreads();
    // thread per (vertex, net) pair: nets of up to kThreadNet members are
    // walked by their thread (four members' loads in flight), larger ones
    // are queued for whole warps
    for (int32_t t = tid; t < np; t += kBT) {
      const int32_t pt = pb + t;
      int32_t lo = 0, hi = n - 1;  // smallest i with pinc[i] > pt
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (sm.pinc[mid] > pt) hi = mid; else lo = mid + 1;
      }
      const int32_t before = sm.pinc[lo] - sm.deg[lo];
      const int32_t v = D.a_idx[sm.ab[lo] + (pt - before)];
      const int32_t bp = D.b_ptr[v], sz = D.b_ptr[v + 1] - bp;
      if (sz > kThreadNet) {
        const int32_t k = atomicAdd(&sm.nbigp, 1);
        sm.pstart[k] = bp;
        sm.psize[k] = sz;
        sm.pv[k] = (uint8_t)lo;
        continue;
      }
      for (int32_t k0 = 0; k0 < sz; k0 += 4) {
        int32_t u[4], c[4];
#pragma unroll
        for (int q = 0; q < 4; q++) u[q] = k0 + q < sz ? D.b_idx[bp + k0 + q] : -1;
#pragma unroll
        for (int q = 0; q < 4; q++) c[q] = u[q] >= 0 ? ldcg(D.colors + u[q]) : 0;
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (u[q] >= 0) take(lo, u[q], c[q]);
      }
    }
    __syncthreads();
    // warp per large pair, lanes over its members
    const int32_t nbp = sm.nbigp;
    for (int32_t k = warp; k < nbp; k += kBW) {
      const int32_t bp = sm.pstart[k], sz = sm.psize[k], i = sm.pv[k];
      for (int32_t f = lane; f < sz; f += 64) {
        const int32_t u0 = D.b_idx[bp + f];
        const int32_t u1 = f + 32 < sz ? D.b_idx[bp + f + 32] : -1;
        const int32_t c0 = ldcg(D.colors + u0);
        const int32_t c1 = u1 >= 0 ? ldcg(D.colors + u1) : 0;
        take(i, u0, c0);
        if (u1 >= 0) take(i, u1, c1);
      }
    }
    __syncthreads();
  }

  // ---- resolve.  First fit: vertices without an earlier neighbour in the
  // chunk see no overlay and are resolved all at once.
  if (POLICY == BGPC_FF) {
    for (int32_t i = warp; i < n; i += kBW) {
      if (sm.adj[i] != 0ull) continue;
      int32_t x = -1;
      const int32_t so = sm.so[i];
      if (so > A.T) {
        if (so - 1 >= WW * 32) x = -2;
        else x = win_kth_free_down<WW>(sm.bm[i], so - 1, sm.k[i]);
      }
      if (x == -1) x = win_first_free<WW>(sm.bm[i], 0);
      if (x < 0 && lane == 0) *flag = 1;
      if (lane == 0) sm.col[i] = x < 0 ? 0 : x;
    }
    __syncthreads();
  }
  if (warp == 0) {
    int32_t col_max = max(S.col_max0, 0), col_next = 0;
    for (int32_t i = 0; i < n; i++) {
      const unsigned long long am = sm.adj[i];
      if (POLICY == BGPC_FF && am == 0ull) continue;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int32_t jj = lane + 32 * h;
        if (jj < i && ((am >> jj) & 1ull)) {
          const int32_t c = sm.col[jj];
          if (c < WW * 32) atomicOr(&sm.bm[i][c >> 5], 1u << (c & 31));
        }
      }
      __syncwarp();
      int32_t x = -1;
      const int32_t so = sm.so[i];
      if (so > A.T) {
        if (so - 1 >= WW * 32) x = -2;
        else x = win_kth_free_down<WW>(sm.bm[i], so - 1, sm.k[i]);
      }
      if (x == -1) {
        if (POLICY == BGPC_B1) {
          if ((sm.w[i] & 1) == 0) {
            x = win_last_free<WW>(sm.bm[i], col_max);
            if (x == -1) x = win_first_free<WW>(sm.bm[i], col_max + 1);
          } else {
            x = win_first_free<WW>(sm.bm[i], 0);
          }
        } else if (POLICY == BGPC_B2 || POLICY == BGPC_B2X) {
          // the first free color from col_next on; beyond col_max (every
          // color of the graph, col_max included, lies inside the window, so
          // "none inside" means beyond col_max as well) first fit instead
          x = win_first_free<WW>(sm.bm[i], col_next);
          if (x < 0 || x > col_max) x = win_first_free<WW>(sm.bm[i], 0);
        } else {
          x = win_first_free<WW>(sm.bm[i], 0);
        }
      }
      if (x < 0) {
        if (lane == 0) *flag = 1;
        x = 0;
      }
      col_max = max(col_max, x);
      if (POLICY == BGPC_B2) col_next = min(x + 1, col_max / 3 + 1);
      if (POLICY == BGPC_B2X) col_next = max(x + 1, col_max / 3 + 1);
      if (lane == 0) sm.col[i] = x;
      __syncwarp();
    }
  }
  __syncthreads();
  if (tid < n) A.stage[D.voff + p0 + tid] = sm.col[tid];
  __syncthreads();
}

template <int WW>
union TaskSmem {
  ChunkSmem<WW> chunk;
  uint32_t detect[kBW][WW];
  int32_t red[kBW + 8];
};

// Start of round S.r (S.m > 0): reverse offsets if the graph has big nets,
// else wave 0.  Called by the advancer.
__device__ void begin_round(const BArgs &A, int32_t g, volatile BatchState &S,
                            volatile BatchStat &X) {
  S.ntiles = (S.m + A.tile - 1) / A.tile;
  S.nch = (S.m + A.C - 1) / A.C;
  S.gmax_wave = -1;
  S.gmax_win = -1;
  S.col_max0 = S.gmax_fixed;  // the snapshot at the round start: the fixed colors
  S.tagged = S.tag_next;      // the previous scatter tagged the nets of this W
  S.tag_next = 0;
  if (S.r < kBatchReport) X.w_per_round[S.r] = S.m;
  X.w_total = X.w_total + S.m;
  if (S.nch <= A.small_nch && A.desc[g].n_b <= 64 * A.tile) {
    S.phase = BP_ROUND;
    S.ntasks = 1;
  } else if (S.nbig > 0) {
    S.phase = BP_KOFS;
    S.ntasks = (S.nbig + kBW - 1) / kBW;
  } else {
    S.phase = BP_WAVE;
    S.q = 0;
    S.col_max0 = S.gmax_fixed;
    const int32_t span = A.cpt * A.Q;
    S.ntasks = (S.nch + span - 1) / span;
  }
}

// The CTA that completed the last task of graph g's phase sets up the next
// phase (thread 0 only).
// The per-graph state and statistics are read and written through L2
// (volatile): the advancer of the next phase may run on another SM.
__device__ void advance(const BArgs &A, int32_t g) {
  volatile BatchState &S = A.st[g];
  volatile BatchStat &X = A.stat[g];
  const BatchDesc &D = A.desc[g];
  if (S.status != kBatchRunning) {  // the graph left the window or failed
    X.status = S.status;
    atomicAdd(&A.glob->finished, 1);
    return;
  }
  const int32_t span = A.cpt * A.Q;
  switch (S.phase) {
    case BP_ANALYZE:
      S.m = D.n_a;
      S.r = 0;
      S.cur = 0;
      S.gmax_fixed = -1;
      begin_round(A, g, S, X);
      break;
    case BP_KOFS:
      S.phase = BP_WAVE;
      S.q = 0;
      S.col_max0 = S.gmax_fixed;
      S.ntasks = (S.nch + span - 1) / span;
      break;
    case BP_WAVE:
      S.phase = BP_PUBLISH;  // same task ranges
      break;
    case BP_PUBLISH:
      if (S.q + 1 < A.Q) {
        S.phase = BP_WAVE;
        S.q++;
        S.col_max0 = max(S.gmax_fixed, S.gmax_wave);
        S.ntasks = (S.nch + span - 1) / span;
      } else {
        S.phase = BP_DETECT;
        S.ntasks = D.n_b > 0 ? (D.n_b + A.tile - 1) / A.tile : 1;
      }
      break;
    case BP_DETECT:
      S.phase = BP_COUNT;
      S.ntasks = S.ntiles;
      break;
    case BP_COUNT:
      S.phase = BP_SCAN;
      S.ntasks = 1;
      break;
    case BP_SCAN:
      S.phase = BP_SCATTER;
      S.ntasks = S.ntiles;
      break;
    case BP_ROUND:
    case BP_SCATTER: {
      S.gmax_fixed = max(S.gmax_fixed, S.gmax_win);
      S.r = S.r + 1;
      X.rounds = S.r;
      X.colors = S.gmax_fixed + 1;
      S.m = S.m_next;
      S.cur = S.cur ^ 1;
      if (S.m == 0) {
        X.status = kBatchDone;
        S.status = kBatchDone;
        atomicAdd(&A.glob->finished, 1);
        return;
      }
      if (S.r >= A.max_rounds) {
        X.status = kBatchRounds;
        S.status = kBatchRounds;
        atomicAdd(&A.glob->finished, 1);
        return;
      }
      begin_round(A, g, S, X);
      break;
    }
    default:
      X.status = kBatchFailed;
      S.status = kBatchFailed;
      atomicAdd(&A.glob->finished, 1);
      return;
  }
  S.done = 0;
  S.seq = S.seq + 1;
  __threadfence();
  atomicExch(&A.st[g].ticket, make_ticket((uint32_t)S.seq, S.ntasks));
  atomicAdd(&A.glob->progress, 1ull);
  // announce the graph to idle CTAs (a stale slot only costs a look)
  const uint32_t slot = atomicAdd(&A.glob->posts, 1u);
  volatile int32_t *ring = A.glob->post;
  ring[slot & (kBatchPosts - 1)] = g;
}

// Claim a task of graph g if its current phase has one left: one atomicAdd
// on the ticket, whose returned word says which phase and index were taken.
__device__ __forceinline__ bool try_claim(const BArgs &A, int32_t g, int32_t *task) {
  BatchState &S = A.st[g];
  const unsigned long long tk = __ldcg(&S.ticket);
  if ((int32_t)(tk & 0xffffffull) >= (int32_t)((tk >> 24) & 0xffffffull)) return false;
  const unsigned long long old = atomicAdd(&S.ticket, 1ull);
  const int32_t ont = (int32_t)((old >> 24) & 0xffffffull);
  const int32_t onx = (int32_t)(old & 0xffffffull);
  if (onx >= ont) return false;
  *task = onx;
  return true;
}

// One warp, big net number b of the graph: k of every member that is in W
// and owns the net = the number of such members before it (the order of
// Alg. 8's W_local), for the reverse first fit.
__device__ __forceinline__ void kofs_net(const BArgs &A, const BatchDesc &D, int32_t b) {
  const int lane = threadIdx.x & 31;
  const int64_t vo = D.voff;
  const int32_t v = ldcg(A.big + D.noff + b);
  const int32_t beg = D.b_ptr[v], end = D.b_ptr[v + 1];
  int32_t base = 0;
  for (int32_t f0 = beg; f0 < end; f0 += 32) {
    const int32_t f = f0 + lane;
    int32_t u = -1;
    bool mine = false;
    if (f < end) {
      u = D.b_idx[f];
      mine = ldcg8(A.inW + vo + u) && ldcg(A.own + vo + u) == v;
    }
    const unsigned bal = __ballot_sync(kFull, mine);
    if (mine) A.kofs[vo + u] = base + __popc(bal & ((1u << lane) - 1u));
    base += __popc(bal);
  }
}

// Conflict detection (Alg. 7's per-net traversal with Alg. 3's rule) on
// nets [v0, v1): in id order a member loses when an earlier member of the
// net has its color (after a vertex-based round only members of W can
// clash).  Each warp takes four nets at a time, one per group of 8 lanes
// (four nets' loads in flight); a net of more than 8 members is done after
// that by the whole warp, 32 members at a time, with a window of seen
// colors.  bm: the warp's window of WW words (zero on entry and on exit).
template <int WW>
__device__ void detect_nets(const BArgs &A, const BatchDesc &D, int32_t v0, int32_t v1,
                            int32_t want, uint32_t *bm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane >> 3, sl = lane & 7;
  const int64_t vo = D.voff;
  for (int x = lane; x < WW; x += 32) bm[x] = 0u;
  __syncwarp();
  for (int32_t vb = v0 + warp * 4; vb < v1; vb += kBW * 4) {
    // group `sub` takes net vb + sub when it has at most 8 members (and,
    // when the round tagged the nets of W, only a tagged net: no other net
    // has a member in W)
    const int32_t v = vb + sub;
    int32_t beg = 0, size = 0;
    if (v < v1 && (want == 0 || ldcg(A.ntag + D.noff + v) == want)) {
      beg = D.b_ptr[v];
      size = D.b_ptr[v + 1] - beg;
    }
    int32_t u = -1, c = -1 - lane;  // unique dummy colors for idle lanes
    if (size >= 2 && size <= 8 && sl < size) {
      u = D.b_idx[beg + sl];
      c = ldcg(D.colors + u);
    }
    // the key keeps the groups apart: colors are below 2^24 (the window)
    const unsigned grp = __match_any_sync(kFull, c >= 0 ? (c << 2) | sub : c);
    const unsigned below = ((1u << sl) - 1u) << (sub * 8);
    if (c >= 0 && (grp & below)) A.lose[vo + u] = 1;
    // larger nets: the whole warp
    const unsigned big = __ballot_sync(kFull, sl == 0 && size > 8);
    for (unsigned bb = big; bb; bb &= bb - 1u) {
      const int src = __ffs(bb) - 1;
      const int32_t nb = __shfl_sync(kFull, beg, src);
      const int32_t ne = nb + __shfl_sync(kFull, size, src);
      for (int32_t f0 = nb; f0 < ne; f0 += 32) {
        const int32_t f = f0 + lane;
        int32_t uu = -1, cc = -1 - lane;
        if (f < ne) {
          uu = D.b_idx[f];
          cc = ldcg(D.colors + uu);
        }
        const unsigned g2 = __match_any_sync(kFull, cc);
        bool l = (g2 & ((1u << lane) - 1u)) != 0u;
        if (f < ne && cc >= 0 && cc < WW * 32) l = l || ((bm[cc >> 5] >> (cc & 31)) & 1u);
        __syncwarp();
        if (f < ne && cc >= 0 && cc < WW * 32) atomicOr(&bm[cc >> 5], 1u << (cc & 31));
        if (l) A.lose[vo + uu] = 1;
        __syncwarp();
      }
      for (int x = lane; x < WW; x += 32) bm[x] = 0u;
      __syncwarp();
    }
  }
}

// One task of graph g: phase parameters were fixed before the ticket that
// handed it out.
template <int POLICY, int WW>
__device__ void run_task(const BArgs &A, int32_t g, int32_t t, TaskSmem<WW> &sm,
                         int32_t *s_flag) {
  const BatchDesc &D = A.desc[g];
  BatchState &S = A.st[g];
  BatchStat &X = A.stat[g];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t vo = D.voff;
  const PhaseView V = view_of(&S);
  const int32_t phase = V.phase;
  const int32_t *Wc = (V.cur ? A.W1 : A.W0) + vo;
  int32_t *Wn = (V.cur ? A.W0 : A.W1) + vo;
  const int32_t tile = A.tile;

  if (phase == BP_ANALYZE) {
    const int32_t nvt = (D.n_a + tile - 1) / tile;
    if (t < nvt) {
      // per vertex (one thread each): owner net (largest, ties to the
      // larger id), its size, the sum of its net sizes; W_0 = V_A in id order
      const int32_t w0 = t * tile, w1 = min(D.n_a, w0 + tile);
      for (int32_t w = w0 + tid; w < w1; w += kBT) {
        const int32_t beg = D.a_ptr[w], end = D.a_ptr[w + 1];
        long long sum = 0;
        unsigned long long best = 0ull;
        for (int32_t i = beg; i < end; i++) {
          const int32_t v = D.a_idx[i];
          const int32_t sz = D.b_ptr[v + 1] - D.b_ptr[v];
          sum += sz;
          const unsigned long long key = ((unsigned long long)(uint32_t)sz << 32) | (uint32_t)v;
          best = key > best ? key : best;
        }
        const bool has = end > beg;
        A.own[vo + w] = has ? (int32_t)(best & 0xffffffffull) : -1;
        A.s_own[vo + w] = has ? (int32_t)(best >> 32) : 0;
        A.d2[vo + w] = (int32_t)sum;
        A.kofs[vo + w] = 0;
        A.W0[vo + w] = w;
        A.inW[vo + w] = 1;
        A.lose[vo + w] = 0;
        D.colors[w] = -1;
      }
    } else {
      // per net: nets above T (the reverse first fit's owners count along them)
      const int32_t v0 = (t - nvt) * tile, v1 = min(D.n_b, v0 + tile);
      for (int32_t v = v0 + tid; v < v1; v += kBT) {
        const int32_t s = D.b_ptr[v + 1] - D.b_ptr[v];
        if (s > A.T) A.big[D.noff + atomicAdd(&S.nbig, 1)] = v;
      }
    }
    return;
  }

  if (phase == BP_KOFS) {
    const int32_t b = t * kBW + warp;
    if (b < V.nbig) kofs_net(A, D, b);
    return;
  }

  if (phase == BP_WAVE || phase == BP_PUBLISH) {
    const int32_t span = A.cpt * A.Q;
    const int32_t j0 = t * span, j1 = min(V.nch, j0 + span);
    const int32_t q = V.q;
    if (phase == BP_WAVE) {
      for (int32_t j = j0; j < j1; j++) {
        if (wave_of_dev(j, A.Q) != q) continue;
        color_chunk<POLICY, WW>(A, D, V, Wc, j, sm.chunk, s_flag);
      }
      return;
    }
    int32_t mx = -1;
    for (int32_t j = j0; j < j1; j++) {
      if (wave_of_dev(j, A.Q) != q) continue;
      const int32_t p0 = j * A.C, n = min(A.C, V.m - p0);
      if (tid < n) {
        const int32_t w = ldcg(Wc + p0 + tid);
        const int32_t c = ldcg(A.stage + vo + p0 + tid);
        D.colors[w] = c;
        mx = max(mx, c);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if (lane == 0 && mx >= 0) atomicMax(&S.gmax_wave, mx);
    return;
  }

  if (phase == BP_DETECT) {
    const int32_t v0 = t * tile, v1 = min(D.n_b, v0 + tile);
    detect_nets<WW>(A, D, v0, v1, V.tagged ? V.r + 1 : 0, sm.detect[warp]);
    return;
  }

  if (phase == BP_ROUND) {
    // a small graph's whole round in this CTA: reverse offsets, the Q waves
    // (each published before the next), conflict detection, compaction
    for (int32_t b = warp; b < V.nbig; b += kBW) kofs_net(A, D, b);
    __syncthreads();
    PhaseView W = V;
    int32_t gm = V.col_max0;  // largest color of the snapshot
    for (int32_t q = 0; q < A.Q; q++) {
      W.col_max0 = gm;
      for (int32_t j = 0; j < V.nch; j++)
        if (wave_of_dev(j, A.Q) == q) color_chunk<POLICY, WW>(A, D, W, Wc, j, sm.chunk, s_flag);
      int32_t mx = -1;
      for (int32_t j = 0; j < V.nch; j++) {
        if (wave_of_dev(j, A.Q) != q) continue;
        const int32_t p0 = j * A.C, n = min(A.C, V.m - p0);
        if (tid < n) {
          const int32_t w = ldcg(Wc + p0 + tid);
          const int32_t c = ldcg(A.stage + vo + p0 + tid);
          D.colors[w] = c;
          mx = max(mx, c);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
      if (lane == 0) sm.red[warp] = mx;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kBW; i++) gm = max(gm, sm.red[i]);
      __syncthreads();
    }
    detect_nets<WW>(A, D, 0, D.n_b, 0, sm.detect[warp]);
    __syncthreads();
    // losers in queue order form the next queue; winners leave W
    int32_t carry = 0, mxw = -1;
    long long trav = 0, incid = 0;
    for (int32_t b0 = 0; b0 < V.m; b0 += kBT) {
      const int32_t p = b0 + tid;
      int32_t w = -1, l = 0;
      if (p < V.m) {
        w = ldcg(Wc + p);
        l = ldcg8(A.lose + vo + w);
        const int32_t deg = D.a_ptr[w + 1] - D.a_ptr[w];
        trav += ldcg(A.d2 + vo + w) - deg;
        incid += deg;
      }
      int32_t total;
      const int32_t ex = cta_excl_scan(l, sm.red, &total);
      if (p < V.m) {
        if (l) {
          Wn[carry + ex] = w;
          D.colors[w] = -1;
          A.lose[vo + w] = 0;
        } else {
          A.inW[vo + w] = 0;
          mxw = max(mxw, ldcg(D.colors + w));
        }
      }
      carry += total;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mxw = max(mxw, __shfl_xor_sync(kFull, mxw, o));
      trav += __shfl_xor_sync(kFull, trav, o);
      incid += __shfl_xor_sync(kFull, incid, o);
    }
    if (lane == 0) {
      if (mxw >= 0) atomicMax(&S.gmax_win, mxw);
      if (trav) {
        if (V.r < kBatchReport)
          atomicAdd(reinterpret_cast<unsigned long long *>(&X.trav_per_round[V.r]),
                    (unsigned long long)trav);
        atomicAdd(reinterpret_cast<unsigned long long *>(&X.trav_total), (unsigned long long)trav);
      }
      if (incid)
        atomicAdd(reinterpret_cast<unsigned long long *>(&X.incid_total), (unsigned long long)incid);
    }
    if (tid == 0) {
      volatile int32_t *mn = &S.m_next;
      *mn = carry;
    }
    return;
  }

  if (phase == BP_COUNT) {
    // losers of this tile of W_r; traversed two-hop entries; winners' max color
    const int32_t p0 = t * tile, p1 = min(V.m, p0 + tile);
    int32_t cnt = 0, mx = -1;
    long long trav = 0, incid = 0;
    for (int32_t p = p0 + tid; p < p1; p += kBT) {
      const int32_t w = ldcg(Wc + p);
      const int32_t deg = D.a_ptr[w + 1] - D.a_ptr[w];
      trav += ldcg(A.d2 + vo + w) - deg;
      incid += deg;
      if (ldcg8(A.lose + vo + w)) cnt++;
      else mx = max(mx, ldcg(D.colors + w));
    }
    int32_t total;
    cta_excl_scan(cnt, sm.red, &total);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(kFull, mx, o));
      trav += __shfl_xor_sync(kFull, trav, o);
      incid += __shfl_xor_sync(kFull, incid, o);
    }
    if (tid == 0) A.tcnt[D.toff + t] = total;
    if (lane == 0) {
      if (mx >= 0) atomicMax(&S.gmax_win, mx);
      if (trav) {
        if (V.r < kBatchReport)
          atomicAdd(reinterpret_cast<unsigned long long *>(&X.trav_per_round[V.r]),
                    (unsigned long long)trav);
        atomicAdd(reinterpret_cast<unsigned long long *>(&X.trav_total), (unsigned long long)trav);
      }
      if (incid)
        atomicAdd(reinterpret_cast<unsigned long long *>(&X.incid_total), (unsigned long long)incid);
    }
    return;
  }

  if (phase == BP_SCAN) {
    const int32_t nt = V.ntiles;
    int32_t carry = 0;
    for (int32_t b0 = 0; b0 < nt; b0 += kBT) {
      const int32_t b = b0 + tid;
      const int32_t x = b < nt ? ldcg(A.tcnt + D.toff + b) : 0;
      int32_t total;
      const int32_t ex = cta_excl_scan(x, sm.red, &total);
      if (b < nt) A.tofs[D.toff + b] = carry + ex;
      carry += total;
    }
    if (tid == 0) {
      volatile BatchState &VS = S;
      VS.m_next = carry;
      // a small next queue: tag its nets so that the next detection skips
      // the others (the tags cost one write per incidence of W_{r+1})
      VS.tag_next = (int64_t)carry * 8 < (int64_t)D.n_a ? 1 : 0;
    }
    return;
  }

  if (phase == BP_SCATTER) {
    // W_{r+1} = the losers in queue order; losers uncolored, winners leave W
    const int32_t p0 = t * tile, p1 = min(V.m, p0 + tile);
    int32_t carry = ldcg(A.tofs + D.toff + t);
    for (int32_t b0 = p0; b0 < p1; b0 += kBT) {
      const int32_t p = b0 + tid;
      int32_t w = -1;
      int32_t l = 0;
      if (p < p1) {
        w = ldcg(Wc + p);
        l = ldcg8(A.lose + vo + w);
      }
      int32_t total;
      const int32_t ex = cta_excl_scan(l, sm.red, &total);
      if (p < p1) {
        if (l) {
          Wn[carry + ex] = w;
          D.colors[w] = -1;
          A.lose[vo + w] = 0;
          if (V.tag_next)
            for (int32_t i = D.a_ptr[w]; i < D.a_ptr[w + 1]; i++)
              A.ntag[D.noff + D.a_idx[i]] = V.r + 2;
        } else {
          A.inW[vo + w] = 0;
        }
      }
      carry += total;
    }
    return;
  }
}

template <int POLICY, int WW>
__global__ void __launch_bounds__(kBT, 8) k_batch(BArgs A) {
  __shared__ TaskSmem<WW> sm;
  __shared__ int32_t s_g, s_t, s_flag, s_cmd;
  __shared__ unsigned long long s_seen;
  __shared__ long long s_idle0;
  __shared__ int32_t s_backoff;
  const int tid = threadIdx.x;
  int32_t cursor = (int32_t)(blockIdx.x % (unsigned)max(A.G, 1));
  if (tid == 0) {
    s_seen = ~0ull;
    s_idle0 = 0;
    s_backoff = 0;
  }
  for (;;) {
    if (tid == 0) {
      s_cmd = 0;  // 0 idle, 1 task, -1 exit
      const volatile BatchGlobal *gl = A.glob;
      if (gl->err != 0 || gl->finished >= A.G) {
        s_cmd = -1;
      } else {
        // the graph this CTA worked on last, then the most recently posted
        // phases, then up to kScan graphs from the cursor onwards: idle CTAs
        // find new phases at once and poll little
        constexpr int32_t kScan = 64, kRecent = 32;
        int32_t tk = 0;
        if (try_claim(A, cursor, &tk)) {
          s_g = cursor;
          s_t = tk;
          s_cmd = 1;
        }
        const uint32_t np = __ldcg(&A.glob->posts);
        for (uint32_t k = 1; k <= (uint32_t)kRecent && k <= np && s_cmd == 0; k++) {
          const int32_t g = __ldcg(&A.glob->post[(np - k) & (kBatchPosts - 1)]);
          if (g >= 0 && g < A.G && try_claim(A, g, &tk)) {
            s_g = g;
            s_t = tk;
            s_cmd = 1;
            cursor = g;
          }
        }
        const int32_t nscan = A.G < kScan ? A.G : kScan;
        for (int32_t i = 0; i < nscan && s_cmd == 0; i++) {
          const int32_t g = cursor + i < A.G ? cursor + i : cursor + i - A.G;
          if (try_claim(A, g, &tk)) {
            s_g = g;
            s_t = tk;
            s_cmd = 1;
            cursor = g;
          }
        }
        if (s_cmd == 0) {
          cursor = cursor + nscan < A.G ? cursor + nscan : cursor + nscan - A.G;
          // no task: wait for progress elsewhere, within a time limit
          const unsigned long long pr = __ldcg(&A.glob->progress);
          long long now;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
          if (pr != s_seen) {
            s_seen = pr;
            s_idle0 = now;
          } else if (now - s_idle0 > A.timeout_ns) {
            atomicExch(&A.glob->err, 1);
            s_cmd = -1;
          }
        }
      }
      s_flag = 0;
    }
    __syncthreads();
    const int32_t cmd = s_cmd;
    if (cmd < 0) return;
    if (cmd == 0) {
      // back off while idle: 0.5, 1, 2, 4 us
      if (tid == 0) {
        __nanosleep(500u << s_backoff);
        if (s_backoff < 3) s_backoff++;
      }
      __syncthreads();
      continue;
    }
    if (tid == 0) s_backoff = 0;
    const int32_t g = s_g, t = s_t;
    __threadfence();
    run_task<POLICY, WW>(A, g, t, sm, &s_flag);
    __syncthreads();
    if (tid == 0) {
      if (s_flag) atomicCAS(&A.st[g].status, kBatchRunning, kBatchWindow);
      __threadfence();
      const int32_t nt = __ldcg(&A.st[g].ntasks);
      if (atomicAdd(&A.st[g].done, 1) + 1 == nt) {
        __threadfence();
        advance(A, g);
      }
    }
  }
}

template <int POLICY, int WW>
cudaError_t launch_one(const BArgs &A, int ctas_per_sm, int sms, cudaStream_t s) {
  auto kern = k_batch<POLICY, WW>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  kern<<<per_sm * sms, kBT, 0, s>>>(A);
  return cudaGetLastError();
}

template <int POLICY>
cudaError_t launch_window(const BArgs &A, int ww, int ctas_per_sm, int sms, cudaStream_t s) {
  switch (ww) {
    case 16: return launch_one<POLICY, 16>(A, ctas_per_sm, sms, s);
    case 64: return launch_one<POLICY, 64>(A, ctas_per_sm, sms, s);
    default: return launch_one<POLICY, 32>(A, ctas_per_sm, sms, s);
  }
}

}  // namespace

cudaError_t launch_batch(const BatchLaunch &L, cudaStream_t s) {
  BArgs A;
  A.desc = L.desc;
  A.st = L.st;
  A.stat = L.stat;
  A.glob = L.glob;
  A.G = L.G;
  A.C = L.C;
  A.Q = L.Q;
  A.T = L.T;
  A.max_rounds = L.max_rounds;
  A.tile = L.map.tile;
  A.cpt = L.map.cpt;
  A.small_nch = L.map.small_nch;
  A.timeout_ns = L.timeout_ns;
  A.W0 = L.W0;
  A.W1 = L.W1;
  A.stage = L.stage;
  A.own = L.own;
  A.s_own = L.s_own;
  A.d2 = L.d2;
  A.kofs = L.kofs;
  A.big = L.big;
  A.tcnt = L.tcnt;
  A.tofs = L.tofs;
  A.ntag = L.ntag;
  A.lose = L.lose;
  A.inW = L.inW;
  switch (L.policy) {
    case BGPC_B1: return launch_window<BGPC_B1>(A, L.map.ww, L.map.ctas_per_sm, L.sms, s);
    case BGPC_B2: return launch_window<BGPC_B2>(A, L.map.ww, L.map.ctas_per_sm, L.sms, s);
    case BGPC_B2X: return launch_window<BGPC_B2X>(A, L.map.ww, L.map.ctas_per_sm, L.sms, s);
    default: return launch_window<BGPC_FF>(A, L.map.ww, L.map.ctas_per_sm, L.sms, s);
  }
}

}  // namespace bgpc
