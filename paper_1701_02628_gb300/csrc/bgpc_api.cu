// C ABI of the library (include/bgpc.h): argument checks, context scratch,
// setup and the round loop of Alg. 1 (ColorWorkQueue in Q waves, then
// RemoveConflicts, until the work queue is empty).
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "bgpc_internal.cuh"

using namespace bgpc;

namespace {

struct Guard {  // restores the caller's current device
  int prev = -1;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Wall-clock limit of one call (opts.timeout_us), checked where the host
// waits for the device anyway; the round loop itself has no device-side wait.
struct Deadline {
  using clk = std::chrono::steady_clock;
  clk::time_point t0 = clk::now();
  int64_t limit_us;
  explicit Deadline(int64_t us) : limit_us(us) {}
  double ms() const {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  }
  bool passed() const { return limit_us > 0 && ms() * 1000.0 > (double)limit_us; }
};

int err_to_status(int32_t err) {
  if (err & (ERR_UNSORTED | ERR_MISMATCH)) return BGPC_EUNSORTED;
  if (err & (ERR_RANGE | ERR_RANK)) return BGPC_EINVAL;
  if (err) return BGPC_EINTERNAL;
  return BGPC_OK;
}

#define CU(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return e_ == cudaErrorMemoryAllocation ? BGPC_ENOMEM : BGPC_ECUDA; \
    }                                              \
  } while (0)

int sync_scalars(bgpc_ctx_t *ctx, cudaStream_t s) {
  CU(cudaMemcpyAsync(ctx->host, ctx->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return BGPC_OK;
}

int check_graph_args(const bgpc_graph_t *g) {
  if (!g || g->n_a < 0 || g->n_b < 0 || g->nnz < 0) return BGPC_EINVAL;
  if (g->n_a > 0 && (!g->a_ptr || !g->b_ptr)) return BGPC_EINVAL;
  if (g->nnz > 0 && (!g->a_idx || !g->b_idx || !g->a_ptr || !g->b_ptr)) return BGPC_EINVAL;
  if (g->n_b > 0 && !g->b_ptr) return BGPC_EINVAL;
  return BGPC_OK;
}

int check_opts(const bgpc_opts_t *o) {
  if (!o) return BGPC_EINVAL;
  if (o->policy < BGPC_FF || o->policy > BGPC_B2X) return BGPC_EINVAL;
  if (o->detect < BGPC_DETECT_AUTO || o->detect > BGPC_DETECT_PAIRS) return BGPC_EINVAL;
  if (o->gather < BGPC_GATHER_AUTO || o->gather > BGPC_GATHER_CTA) return BGPC_EINVAL;
  if (o->chunk < 1 || o->chunk > kMaxChunk) return BGPC_EINVAL;
  if (o->waves < 1 || o->big_net < 0 || o->max_rounds < 1 || o->stop_after_waves < 0)
    return BGPC_EINVAL;
  // net-based coloring is built for the first round (N1-*), where every
  // vertex is uncolored; later net rounds (N2-*) are not
  if (o->net_rounds < 0 || o->net_rounds > 1 || o->timeout_us < 0) return BGPC_EINVAL;
  return BGPC_OK;
}

// Validate a CSR: pointer array first (so that row checks stay in bounds).
int validate_csr(bgpc_ctx_t *ctx, const int32_t *ptr, const int32_t *idx, int32_t n,
                 int32_t nnz, int32_t bound, cudaStream_t s) {
  CU(cudaMemsetAsync(&ctx->dev->err, 0, sizeof(int32_t), s));
  launch_check_ptr(ptr, n, nnz, &ctx->dev->err, s);
  int rc = sync_scalars(ctx, s);
  if (rc) return rc;
  if (ctx->host->err) return err_to_status(ctx->host->err);
  launch_check_rows(ptr, idx, n, bound, &ctx->dev->err, ctx->num_sms, s);
  rc = sync_scalars(ctx, s);
  if (rc) return rc;
  return err_to_status(ctx->host->err);
}

// Phase timing with CUDA events recorded on the launch stream (opts.profile).
enum Phase { PH_SETUP = 0, PH_COLOR = 1, PH_PUBLISH = 2, PH_DETECT = 3, PH_GATHER = 4 };
struct PhaseTimer {
  bgpc_ctx_t *ctx;
  cudaStream_t s;
  bool on;
  int used = 0;
  std::vector<int> phase;
  double ms[5] = {0, 0, 0, 0, 0};
  PhaseTimer(bgpc_ctx_t *c, cudaStream_t st, bool enabled) : ctx(c), s(st), on(enabled) {}
  cudaEvent_t ev(int i) {
    while ((int)ctx->events.size() <= i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ctx->events.push_back(e);
    }
    return ctx->events[i];
  }
  int begin() {
    if (!on) return -1;
    int i = used;
    cudaEventRecord(ev(i), s);
    used += 2;
    return i;
  }
  void end(int i, int ph) {
    if (!on || i < 0) return;
    cudaEventRecord(ev(i + 1), s);
    if ((int)phase.size() <= i / 2) phase.resize(i / 2 + 1);
    phase[i / 2] = ph;
  }
  // after the stream has been synchronised
  void collect() {
    if (!on) return;
    for (int k = 0; k < used / 2; k++) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ctx->events[2 * k], ctx->events[2 * k + 1]) == cudaSuccess)
        ms[phase[k]] += t;
      else
        cudaGetLastError();
    }
    used = 0;
  }
};

int ensure_table(bgpc_ctx_t *ctx, size_t entries, cudaStream_t s, int64_t *nk) {
  if (entries > ctx->dtab.cap) {
    CU(grow(ctx->dtab, entries));
    ctx->dtab_filled = 0;
  }
  if (entries > ctx->dtab_filled) {
    *nk += launch_fill(ctx->dtab.p, ctx->dtab.cap, INT32_MAX, s);
    ctx->dtab_filled = ctx->dtab.cap;
  }
  return BGPC_OK;
}

// center_first: the nets are D2GC's closed neighbourhoods (net v = N[v]),
// and a net-based round visits the center v first (Alg. 9).
int color_impl(bgpc_ctx_t *ctx, const bgpc_graph_t &g, const bgpc_opts_t &o, int32_t *colors,
               bgpc_stats_t *stats, cudaStream_t s, const Deadline &dl,
               int32_t center_first = 0) {
  bgpc_stats_t st;
  memset(&st, 0, sizeof(st));
  st.hub_threshold = INT32_MAX;
  const int32_t n_a = g.n_a, n_b = g.n_b, nnz = g.nnz;
  const int sms = ctx->num_sms;
  if (n_a == 0) {
    if (stats) *stats = st;
    return BGPC_OK;
  }
  int rc;
  if (o.validate) {
    if ((rc = validate_csr(ctx, g.a_ptr, g.a_idx, n_a, nnz, n_b, s))) return rc;
    if ((rc = validate_csr(ctx, g.b_ptr, g.b_idx, n_b, nnz, n_a, s))) return rc;
  }
  const size_t nz = (size_t)(nnz > 0 ? nnz : 1);
  CU(grow(ctx->tpos, nz));
  CU(grow(ctx->nc, nz));
  CU(grow(ctx->npos, nz));
  CU(grow(ctx->nown, nz));
  CU(grow(ctx->s_own, (size_t)n_a));
  CU(grow(ctx->ownid, (size_t)n_a));
  for (int q = 0; q < 4; q++) CU(grow(ctx->ksc[q], (size_t)n_a));
  CU(grow(ctx->kgstart, (size_t)(n_b > 0 ? n_b : 1)));
  CU(grow(ctx->d2tot, (size_t)n_a));
  CU(grow(ctx->W0, (size_t)n_a));
  CU(grow(ctx->W1, (size_t)n_a));
  CU(grow(ctx->kofs, (size_t)n_a));
  CU(grow(ctx->stage, (size_t)n_a));
  CU(grow(ctx->newpos, (size_t)n_a));
  CU(grow(ctx->lose, (size_t)n_a));
  CU(grow(ctx->blocksum, (size_t)div_up((long long)n_a + kMaxChunk, 4096) + 1));
  CU(grow(ctx->segoff, (size_t)n_a + kMaxChunk + 1));
  CU(grow(ctx->segmap, (size_t)n_a + (size_t)nnz / kPiece + 16));
  CU(grow(ctx->bigt, (size_t)(n_b > 0 ? n_b : 1)));
  CU(grow(ctx->bigd, (size_t)(n_b > 0 ? n_b : 1)));
  CU(grow(ctx->hub_id, (size_t)(n_b > 0 ? n_b : 1)));
  CU(grow(ctx->hub_net, (size_t)nnz / (kHubMin + 1) + 1));
  if (o.net_rounds > 0) CU(grow(ctx->netc, (size_t)n_a));
  CU(grow(ctx->ihub, nz));
  CU(grow(ctx->brow, nz));

  // ---- setup (Alg. 1: W <- V_color, c <- -1), static graph analysis
  PhaseTimer tm(ctx, s, o.profile != 0);
  int64_t nk = 0;
  int ev = tm.begin();
  CU(cudaMemsetAsync(ctx->dev, 0, sizeof(DevScalars), s));
  CU(cudaMemsetAsync(&ctx->dev->gmax, 0xff, sizeof(int32_t), s));
  CU(cudaMemsetAsync(ctx->lose.p, 0, (size_t)n_a, s));
  nk += launch_net_static(g, o.big_net, ctx->bigt.p, ctx->bigd.p, ctx->dev, s);
  // hub bitmaps: at most half the L2 cache in the first round
  nk += launch_hub_select(g.b_ptr, n_b, o.chunk, o.waves, (int64_t)ctx->l2_bytes / 8,
                          ctx->hub_id.p, ctx->hub_net.p, ctx->dev, sms, s);
  {
    // the sort's scratch: buffers that are written only later in the setup
    int32_t *const scratch[4] = {ctx->nc.p, ctx->npos.p, ctx->ihub.p, ctx->brow.p};
    const int64_t hlen = tpos_hist_len(nnz);
    CU(grow(ctx->thist, (size_t)(hlen > 0 ? hlen : 1)));
    CU(grow(ctx->tsums, (size_t)(hlen / 4096 + 1)));
    nk += launch_tpos(g, ctx->tpos.p, scratch, ctx->thist.p, ctx->tsums.p, o.validate,
                      &ctx->dev->err, ctx->hub_id.p, n_b > 0 ? ctx->ihub.p : nullptr, sms, s);
  }
  // the owner flags serve the reverse offsets' net scan, used for caller ranks only
  nk += launch_vertex_static(g, ctx->tpos.p, ctx->s_own.p, ctx->d2tot.p,
                             o.rank ? ctx->nown.p : nullptr,
                             o.net_rounds > 0 ? ctx->netc.p : nullptr, center_first,
                             ctx->ownid.p, sms, s);
  nk += launch_init_queue(o.rank, n_a, ctx->W0.p, &ctx->dev->err, s);
  nk += launch_init_mirror(g, o.rank, ctx->nc.p, ctx->npos.p, colors, sms, s);
  tm.end(ev, PH_SETUP);
  CU(cudaGetLastError());
  if ((rc = sync_scalars(ctx, s))) return rc;
  tm.collect();
  if (ctx->host->err) return err_to_status(ctx->host->err);
  if (dl.passed()) return BGPC_ETIMEOUT;
  const int32_t nbig_t = ctx->host->nbig_t, nbig_d = ctx->host->nbig_d;
  const int32_t nhub = ctx->host->nhub;
  const int32_t maxnet = ctx->host->maxnet;
  if (n_b > 0) st.hub_threshold = ctx->host->hub_H;
  st.hubs = nhub;
  const int32_t max_words = wave_max_words(ctx->smem_optin);

  int32_t *W = ctx->W0.p, *Wn = ctx->W1.p;
  int32_t m = n_a, gmax = -1, r = 0;
  int64_t incid_w = -1;  // sum over W of |nets(w)| (known from the second round on)
  int64_t waves_done = 0;
  const int32_t C = o.chunk, Q = o.waves;
  while (m > 0) {
    if (r >= o.max_rounds) return BGPC_EROUNDS;
    // every color of this round is <= max(gmax, maxnet - 1, 0) + C * Q (each
    // color is at most one above the largest one its chunk can see)
    const int64_t b0 = (int64_t)(gmax > maxnet - 1 ? gmax : maxnet - 1);
    const int64_t ncol64 = (b0 > 0 ? b0 : 0) + (int64_t)C * Q + C + 2;
    const int64_t words64 = ((ncol64 + 31) / 32 + 3) & ~(int64_t)3;
    if (words64 > max_words) return BGPC_ENOMEM;
    const int32_t words = (int32_t)words64;
    const int32_t cbw = words * 32;  // color capacity of bitmaps and tables
    const int32_t small_ok = (o.policy == BGPC_FF || cbw <= kSmallWindow) ? 1 : 0;
    const int32_t nslots = nbig_d < 2 * sms ? (nbig_d > 0 ? nbig_d : 1) : 2 * sms;
    if ((rc = ensure_table(ctx, (size_t)nslots * (size_t)cbw, s, &nk))) return rc;

    const bool net = r < o.net_rounds;
    if (net) {
      // ---- net-based coloring round (Alg. 8 / Alg. 9): every vertex takes
      // its owner net's reverse first-fit proposal, computed in the setup;
      // it counts as one wave
      if (o.stop_after_waves > 0 && waves_done == o.stop_after_waves) {
        if (o.W_out) CU(cudaMemcpyAsync(o.W_out, W, sizeof(int32_t) * (size_t)m,
                                        cudaMemcpyDeviceToDevice, s));
        CU(cudaStreamSynchronize(s));
        tm.collect();
        st.rounds = r + 1;
        st.stopped_m = m;
        st.stopped_wave = 0;
        st.colors = gmax + 1;
        if (stats) *stats = st;
        return BGPC_STOPPED;
      }
      CU(cudaMemsetAsync(&ctx->dev->trav, 0, kRoundCounters * sizeof(unsigned long long), s));
      ev = tm.begin();
      nk += launch_net_publish(g, ctx->netc.p, o.rank, ctx->nc.p, colors, ctx->lose.p, sms, s);
      tm.end(ev, PH_COLOR);
      waves_done++;
    } else {
    ev = tm.begin();
    if (nbig_t > 0 && !o.rank) {
      // W in id order: k by a sort of the W positions by owner net (work in |W|)
      int32_t *const sc[4] = {ctx->ksc[0].p, ctx->ksc[1].p, ctx->ksc[2].p, ctx->ksc[3].p};
      const int64_t hlen = tpos_hist_len(m);
      CU(grow(ctx->thist, (size_t)(hlen > 0 ? hlen : 1)));
      CU(grow(ctx->tsums, (size_t)(hlen / 4096 + 1)));
      nk += launch_kofs_sorted(W, m, ctx->ownid.p, ctx->s_own.p, o.big_net, n_b, sc,
                               ctx->thist.p, ctx->tsums.p, ctx->kgstart.p, ctx->kofs.p, sms, s);
    } else if (nbig_t > 0) {
      nk += launch_kofs(g.b_ptr, ctx->nc.p, ctx->npos.p, ctx->nown.p, ctx->bigt.p, nbig_t,
                        ctx->kofs.p, sms, s);
    }
    CU(cudaMemsetAsync(&ctx->dev->trav, 0, kRoundCounters * sizeof(unsigned long long), s));
    nk += launch_trav(g.a_ptr, W, ctx->d2tot.p, m, small_ok, ctx->dev, s);
    tm.end(ev, PH_DETECT);

    // chunks of every wave (a pure function of nch and Q), uploaded once per round
    const int64_t nch = ((int64_t)m + C - 1) / C;
    std::vector<int64_t> woff((size_t)Q + 1, 0);
    {
      if ((size_t)nch > ctx->h_wlist_cap) {
        if (ctx->h_wlist) cudaFreeHost(ctx->h_wlist);
        ctx->h_wlist = nullptr;
        ctx->h_wlist_cap = 0;
        CU(cudaMallocHost((void **)&ctx->h_wlist, sizeof(int32_t) * (size_t)nch));
        ctx->h_wlist_cap = (size_t)nch;
      }
      CU(grow(ctx->wlist, (size_t)nch));
      for (int64_t j = 0; j < nch; j++) woff[(size_t)wave_of(j, Q) + 1]++;
      for (int32_t q = 0; q < Q; q++) woff[q + 1] += woff[q];
      std::vector<int64_t> fill(woff.begin(), woff.end());
      for (int64_t j = 0; j < nch; j++) ctx->h_wlist[fill[(size_t)wave_of(j, Q)]++] = (int32_t)j;
      CU(cudaMemcpyAsync(ctx->wlist.p, ctx->h_wlist, sizeof(int32_t) * (size_t)nch,
                         cudaMemcpyHostToDevice, s));
    }
    // per-slot forbidden bitmaps of the large vertices of one wave (zero at rest)
    int64_t maxwave = 0;
    for (int32_t q = 0; q < Q; q++)
      maxwave = woff[q + 1] - woff[q] > maxwave ? woff[q + 1] - woff[q] : maxwave;
    {
      const size_t gw = (size_t)maxwave * C * (size_t)words;
      const size_t slots = (size_t)maxwave * C;
      if (gw > ctx->gbm.cap || gw > ctx->gbm_zeroed || slots > ctx->gadj.cap ||
          slots > ctx->gcnt.cap) {
        CU(grow(ctx->gbm, gw));
        CU(grow(ctx->gadj, slots));
        CU(grow(ctx->gcnt, slots));
        CU(cudaMemsetAsync(ctx->gbm.p, 0, ctx->gbm.cap * sizeof(uint32_t), s));
        CU(cudaMemsetAsync(ctx->gadj.p, 0, ctx->gadj.cap * sizeof(unsigned long long), s));
        CU(cudaMemsetAsync(ctx->gcnt.p, 0, ctx->gcnt.cap * sizeof(int32_t), s));
        ctx->gbm_zeroed = ctx->gbm.cap;
      }
      // first fit: the gather's per-slot summaries and the bitmaps kept for
      // the reverse first fit (both written before they are read)
      if (o.policy == BGPC_FF) {
        CU(grow(ctx->gsum, slots * kSumInts));
        CU(grow(ctx->lbm, gw));
      }
    }
    // the colors published so far, per hub net, at this round's bitmap width
    if (nhub > 0) CU(grow(ctx->nbm, (size_t)nhub * (size_t)words));
    ev = tm.begin();
    nk += launch_hub_build(g.b_ptr, ctx->nc.p, ctx->hub_net.p, nhub, words, ctx->nbm.p, sms, s);
    nk += launch_pieces(g.a_ptr, ctx->d2tot.p, W, ctx->wlist.p, (int32_t)nch, C, m, small_ok,
                        ctx->segoff.p, ctx->blocksum.p, ctx->segmap.p, ctx->dev, s);
    tm.end(ev, PH_DETECT);
    for (int32_t q = 0; q < Q; q++) {
      if (o.stop_after_waves > 0 && waves_done == o.stop_after_waves) {
        if (o.W_out) CU(cudaMemcpyAsync(o.W_out, W, sizeof(int32_t) * (size_t)m,
                                        cudaMemcpyDeviceToDevice, s));
        CU(cudaStreamSynchronize(s));
        tm.collect();
        st.rounds = r + 1;
        st.stopped_m = m;
        st.stopped_wave = q;
        st.colors = gmax + 1;
        if (stats) *stats = st;
        return BGPC_STOPPED;
      }
      const int32_t *wchunks = ctx->wlist.p + woff[q];
      const int32_t nwave = (int32_t)(woff[q + 1] - woff[q]);
      if (nwave > 0) {
        GatherArgs ga;
        ga.a_ptr = g.a_ptr;
        ga.a_idx = g.a_idx;
        ga.b_ptr = g.b_ptr;
        ga.nc = ctx->nc.p;
        ga.W = W;
        ga.wlist = ctx->wlist.p;
        ga.segmap = ctx->segmap.p;
        ga.segoff = ctx->segoff.p;
        ga.m = m;
        ga.C = C;
        ga.slot_lo = (int32_t)(woff[q] * C);
        ga.slot_hi = (int32_t)(woff[q + 1] * C);
        ga.words = words;
        ga.gbm = ctx->gbm.p;
        ga.gadj = ctx->gadj.p;
        ga.b_idx = g.b_idx;
        ga.tpos = ctx->tpos.p;
        ga.hub_id = nhub > 0 ? ctx->hub_id.p : nullptr;
        ga.nbm = ctx->nbm.p;
        ga.dev = ctx->dev;
        ga.id_order = o.rank ? 0 : 1;
        ga.summ = o.policy == BGPC_FF;
        ga.T = o.big_net;
        ga.s_own = ctx->s_own.p;
        ga.kofs = ctx->kofs.p;
        ga.gcnt = ctx->gcnt.p;
        ga.gsum = ctx->gsum.p;
        ga.lbm = ctx->lbm.p;
        ev = tm.begin();
        CU(launch_gather(ga, o.gather == BGPC_GATHER_CTA, sms, s));
        tm.end(ev, PH_GATHER);
        nk++;
        WaveArgs a;
        a.a_ptr = g.a_ptr;
        a.a_idx = g.a_idx;
        a.b_ptr = g.b_ptr;
        a.nc = ctx->nc.p;
        a.W = W;
        a.kofs = ctx->kofs.p;
        a.s_own = ctx->s_own.p;
        a.d2tot = ctx->d2tot.p;
        a.stage = ctx->stage.p;
        a.dev = ctx->dev;
        a.err = &ctx->dev->err;
        a.m = m;
        a.C = C;
        a.T = o.big_net;
        a.chunks = wchunks;
        a.nchunks = nwave;
        a.maxnet = maxnet;
        a.words = words;
        a.small_ok = small_ok;
        a.gbm = ctx->gbm.p;
        a.gadj = ctx->gadj.p;
        a.gsum = ctx->gsum.p;
        a.lbm = ctx->lbm.p;
        ev = tm.begin();
        CU(launch_color_wave(o.policy, a, sms, s));
        tm.end(ev, PH_COLOR);
        nk++;
        st.color_launches++;
        ev = tm.begin();
        nk += launch_publish(g.a_ptr, ctx->d2tot.p, nhub > 0 ? ctx->ihub.p : nullptr,
                             ctx->tpos.p, W, ctx->stage.p, ctx->wlist.p, C, m, small_ok,
                             ga.slot_lo, ga.slot_hi, ctx->segoff.p, ctx->segmap.p, ctx->nc.p,
                             colors, ctx->nbm.p, words, ctx->dev, sms, s);
        tm.end(ev, PH_PUBLISH);
      }
      waves_done++;
    }
    }  // vertex-based round
    if (o.stop_before_removal && o.stop_after_waves > 0 && waves_done == o.stop_after_waves) {
      if (o.W_out) CU(cudaMemcpyAsync(o.W_out, W, sizeof(int32_t) * (size_t)m,
                                      cudaMemcpyDeviceToDevice, s));
      CU(cudaStreamSynchronize(s));
      tm.collect();
      st.rounds = r + 1;
      st.stopped_m = m;
      st.stopped_wave = net ? 1 : Q;
      if (stats) *stats = st;
      return BGPC_STOPPED;
    }
    // ---- RemoveConflicts and the next work queue
    ev = tm.begin();
    // after the first round W is usually a small part of the graph: then
    // only its (member, net) pairs are examined instead of every net
    int64_t cap = 1024;  // hash table at load <= 1/2
    while (incid_w >= 0 && cap < 2 * incid_w) cap <<= 1;
    const bool pairs = incid_w >= 0 && cap <= ((int64_t)1 << 31) &&
                       o.detect != BGPC_DETECT_NETS &&
                       (o.detect == BGPC_DETECT_PAIRS || incid_w * 4 <= (int64_t)nnz);
    if (pairs) {
      CU(grow(ctx->pkeys, 2 * (size_t)cap));
      nk += launch_detect_pairs(g.a_ptr, g.a_idx, W, m, colors, ctx->pkeys.p,
                                (uint32_t)(cap - 1), ctx->lose.p, &ctx->dev->err, sms, s);
    } else {
      nk += launch_detect(g.b_ptr, n_b, ctx->nc.p, ctx->npos.p, ctx->bigd.p, nbig_d,
                          ctx->dtab.p, cbw, nslots, o.rank ? 0 : 1, ctx->lose.p, sms, s);
    }
    nk += launch_compact(ctx->lose.p, W, m, ctx->newpos.p, Wn, ctx->blocksum.p, g.a_ptr,
                         ctx->dev, s);
    // W large against the graph (the first round): relabel in CSC order
    if (incid_w < 0 || incid_w * 4 > (int64_t)nnz)
      nk += launch_relabel_csc(nnz, W, m, ctx->lose.p, ctx->newpos.p, ctx->nc.p, ctx->npos.p,
                               colors, sms, s);
    else
      nk += launch_relabel(g.a_ptr, ctx->tpos.p, W, m, ctx->lose.p, ctx->newpos.p, ctx->nc.p,
                           ctx->npos.p, colors, sms, s);
    nk += launch_gmax(colors, n_a, ctx->dev, s);
    tm.end(ev, PH_DETECT);
    CU(cudaGetLastError());
    if ((rc = sync_scalars(ctx, s))) return rc;
    tm.collect();
    if (ctx->host->err) {
      ctx->gbm_zeroed = 0;  // a kernel may have stopped before clearing its slots
      return err_to_status(ctx->host->err);
    }
    if (dl.passed()) return BGPC_ETIMEOUT;
    // a net round reads every net touching W once: all of them in the
    // first round, sum of |vtxs(v)| = nnz entries and incidences
    const int64_t trav_r = net ? (int64_t)nnz : (int64_t)ctx->host->trav;
    if (r < BGPC_MAX_REPORT) {
      st.w_per_round[r] = m;
      st.trav_per_round[r] = trav_r;
    }
    st.trav_total += trav_r;
    st.incid_total += net ? (int64_t)nnz : (int64_t)ctx->host->incid;
    st.trav_large += (int64_t)ctx->host->trav_large;
    st.incid_large += (int64_t)ctx->host->incid_large;
    st.w_large += (int64_t)ctx->host->w_large;
    st.trav_hub += (int64_t)ctx->host->trav_hub;
    st.hub_pairs += (int64_t)ctx->host->hub_pairs;
    st.hub_words += (int64_t)ctx->host->hub_words;
    st.pieces_total += ctx->host->nseg;
    st.w_total += m;
    r++;
    const int32_t mn = ctx->host->m_next;
    incid_w = (int64_t)ctx->host->incid_next;
    if (mn < 0 || mn > m) return BGPC_EINTERNAL;
    int32_t *t = W;
    W = Wn;
    Wn = t;
    m = mn;
    gmax = ctx->host->gmax;
  }
  st.rounds = r;
  st.colors = gmax + 1;
  if (o.want_balance && gmax >= 0) {
    CU(grow(ctx->card, (size_t)gmax + 1));
    nk += launch_card(colors, n_a, ctx->card.p, gmax + 1, &ctx->dev->err, s);
    nk += launch_card_stats(ctx->card.p, gmax + 1, ctx->dev, s);
    if ((rc = sync_scalars(ctx, s))) return rc;
    if (ctx->host->err) return err_to_status(ctx->host->err);
    const double sets = (double)ctx->host->acc[0];
    st.n_sets = (int32_t)ctx->host->acc[0];
    st.max_card = (int32_t)ctx->host->acc[1];
    st.mean_card = sets > 0 ? (double)ctx->host->acc[2] / sets : 0.0;
    const double ex2 = sets > 0 ? (double)ctx->host->acc[3] / sets : 0.0;
    const double var = ex2 - st.mean_card * st.mean_card;
    st.std_card = var > 0 ? sqrt(var) : 0.0;
  }
  st.kernel_launches = nk;
  st.ms_setup = tm.ms[PH_SETUP];
  st.ms_color = tm.ms[PH_COLOR];
  st.ms_publish = tm.ms[PH_PUBLISH];
  st.ms_detect = tm.ms[PH_DETECT];
  st.ms_gather = tm.ms[PH_GATHER];
  st.ms_total = dl.ms();
  if (stats) *stats = st;
  return BGPC_OK;
}


// ------------------------------------------------ batched, persistent engine

// Mapping candidates of the persistent engine: forbidden-window words per
// vertex, CTAs per SM (0 = as many as fit), chunk indices per wave task
// (times Q), vertices / positions / nets per task, and the largest round (in
// chunks) that one CTA runs as a single task.  None changes a result.
const BatchMapping kBatchMaps[BGPC_BATCH_MAPPINGS] = {
    {32, 0, 1, 2048, 32}, {32, 0, 4, 2048, 32}, {16, 0, 1, 2048, 32}, {16, 0, 4, 2048, 32},
    {64, 0, 1, 2048, 32}, {64, 0, 4, 2048, 32}, {32, 0, 1, 2048, 0},  {32, 0, 1, 2048, 128},
    {16, 0, 1, 2048, 128}, {32, 4, 1, 2048, 32}, {64, 4, 4, 2048, 0},  {16, 4, 4, 2048, 128}};

unsigned long long fnv(unsigned long long h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Identity of a batch: its graphs (pointers and sizes), outputs and the
// semantic options.  Equal keys color the same arrays the same way.
unsigned long long batch_key(int32_t G, const bgpc_graph_t *graphs, int32_t *const *colors,
                             const bgpc_opts_t &o) {
  unsigned long long h = 1469598103934665603ull;
  h = fnv(h, &G, sizeof(G));
  h = fnv(h, graphs, sizeof(bgpc_graph_t) * (size_t)G);
  h = fnv(h, colors, sizeof(int32_t *) * (size_t)G);
  const int32_t sem[5] = {o.policy, o.chunk, o.waves, o.big_net, o.max_rounds};
  return fnv(h, sem, sizeof(sem));
}

struct BatchHost {  // views into the pinned staging block
  BatchDesc *desc;
  BatchState *st;
  BatchGlobal *glob;
  BatchStat *stat;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int batch_host_views(bgpc_ctx_t *ctx, int32_t G, BatchHost *h) {
  const size_t o1 = align_up(sizeof(BatchDesc) * (size_t)G, 128);
  const size_t o2 = o1 + align_up(sizeof(BatchState) * (size_t)G, 128);
  const size_t o3 = o2 + align_up(sizeof(BatchGlobal), 128);
  const size_t need = o3 + sizeof(BatchStat) * (size_t)G;
  if (need > ctx->h_batch_cap) {
    if (ctx->h_batch) cudaFreeHost(ctx->h_batch);
    ctx->h_batch = nullptr;
    ctx->h_batch_cap = 0;
    if (ctx->bexec) {  // the captured launch copies from the old block
      cudaGraphExecDestroy(ctx->bexec);
      ctx->bexec = nullptr;
    }
    CU(cudaMallocHost(&ctx->h_batch, need));
    ctx->h_batch_cap = need;
  }
  char *b = static_cast<char *>(ctx->h_batch);
  h->desc = reinterpret_cast<BatchDesc *>(b);
  h->st = reinterpret_cast<BatchState *>(b + o1);
  h->glob = reinterpret_cast<BatchGlobal *>(b + o2);
  h->stat = reinterpret_cast<BatchStat *>(b + o3);
  return BGPC_OK;
}

// One run of the persistent engine with mapping `map` on ctx->bstream
// (ordered after everything already on `s`, and `s` after it).  With
// use_graph, the launch sequence is captured in a CUDA graph, cached in the
// context with the batch key and replayed by later calls on the same batch.
// Per-graph results land in the pinned statistics (h->stat).
int batch_once(bgpc_ctx_t *ctx, int32_t G, const bgpc_graph_t *graphs, int32_t *const *colors,
               const bgpc_opts_t &o, const BatchMapping &map, int map_id, cudaStream_t s,
               bool use_graph, BatchHost *h, float *ms_kernel) {
  int64_t voff = 0, noff = 0, toff = 0;
  int32_t empty = 0;
  const int32_t tile = map.tile;
  for (int32_t k = 0; k < G; k++) {
    const bgpc_graph_t &gk = graphs[k];
    BatchDesc &d = h->desc[k];
    d.a_ptr = gk.a_ptr;
    d.a_idx = gk.a_idx;
    d.b_ptr = gk.b_ptr;
    d.b_idx = gk.b_idx;
    d.colors = colors[k];
    d.n_a = gk.n_a;
    d.n_b = gk.n_b;
    d.nnz = gk.nnz;
    d.pad = 0;
    d.voff = voff;
    d.noff = noff;
    d.toff = toff;
    voff += gk.n_a;
    noff += gk.n_b;
    toff += (gk.n_a + tile - 1) / tile + 1;
    BatchState &st = h->st[k];
    memset(&st, 0, sizeof(st));
    const int32_t nt = gk.n_a > 0 ? (gk.n_a + tile - 1) / tile + (gk.n_b + tile - 1) / tile : 0;
    st.ticket = (unsigned long long)(uint32_t)nt << 24;
    st.ntasks = nt;
    st.phase = 0;  // analysis
    st.gmax_fixed = -1;
    st.status = gk.n_a > 0 ? kBatchRunning : kBatchDone;
    empty += gk.n_a > 0 ? 0 : 1;
  }
  memset(h->glob, 0, sizeof(BatchGlobal));
  h->glob->finished = empty;
  const size_t nv = (size_t)(voff > 0 ? voff : 1), nn = (size_t)(noff > 0 ? noff : 1);
  CU(grow(ctx->bW0, nv));
  CU(grow(ctx->bW1, nv));
  CU(grow(ctx->bstage, nv));
  CU(grow(ctx->bown, nv));
  CU(grow(ctx->bsown, nv));
  CU(grow(ctx->bd2, nv));
  CU(grow(ctx->bkofs, nv));
  CU(grow(ctx->blose, nv));
  CU(grow(ctx->binW, nv));
  CU(grow(ctx->bbig, nn));
  CU(grow(ctx->bntag, nn));
  CU(grow(ctx->btcnt, (size_t)toff + 1));
  CU(grow(ctx->btofs, (size_t)toff + 1));
  CU(grow(ctx->bdesc, (size_t)G));
  CU(grow(ctx->bst, (size_t)G));
  CU(grow(ctx->bstat, (size_t)G));
  CU(grow(ctx->bglob, 1));
  if (!ctx->bstream) CU(cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking));
  for (int i = 0; i < 4; i++)
    if (!ctx->bev[i]) CU(cudaEventCreate(&ctx->bev[i]));
  cudaStream_t bs = ctx->bstream;
  CU(cudaEventRecord(ctx->bev[0], s));
  CU(cudaStreamWaitEvent(bs, ctx->bev[0], 0));

  BatchLaunch L;
  L.desc = ctx->bdesc.p;
  L.st = ctx->bst.p;
  L.stat = ctx->bstat.p;
  L.glob = ctx->bglob.p;
  L.G = G;
  L.C = o.chunk;
  L.Q = o.waves;
  L.T = o.big_net;
  L.max_rounds = o.max_rounds;
  L.policy = o.policy;
  L.sms = ctx->num_sms;
  L.timeout_ns = o.timeout_us > 0 ? o.timeout_us * 1000 : 10000000000ll;
  L.map = map;
  L.W0 = ctx->bW0.p;
  L.W1 = ctx->bW1.p;
  L.stage = ctx->bstage.p;
  L.own = ctx->bown.p;
  L.s_own = ctx->bsown.p;
  L.d2 = ctx->bd2.p;
  L.kofs = ctx->bkofs.p;
  L.big = ctx->bbig.p;
  L.tcnt = ctx->btcnt.p;
  L.tofs = ctx->btofs.p;
  L.ntag = ctx->bntag.p;
  L.lose = ctx->blose.p;
  L.inW = ctx->binW.p;

  auto enqueue = [&](cudaStream_t st) -> int {
    CU(cudaMemcpyAsync(ctx->bdesc.p, h->desc, sizeof(BatchDesc) * (size_t)G,
                       cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(ctx->bst.p, h->st, sizeof(BatchState) * (size_t)G, cudaMemcpyHostToDevice,
                       st));
    CU(cudaMemcpyAsync(ctx->bglob.p, h->glob, sizeof(BatchGlobal), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(ctx->bstat.p, 0, sizeof(BatchStat) * (size_t)G, st));
    CU(launch_batch(L, st));
    CU(cudaMemcpyAsync(h->stat, ctx->bstat.p, sizeof(BatchStat) * (size_t)G,
                       cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(h->glob, ctx->bglob.p, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, st));
    return BGPC_OK;
  };
  int rc;
  unsigned long long key = batch_key(G, graphs, colors, o);
  key = fnv(key, &map_id, sizeof(map_id));
  // the launch sequence (descriptor uploads, the persistent kernel, the
  // statistics download) is timed from outside any capture
  CU(cudaEventRecord(ctx->bev[2], bs));
  if (use_graph && ctx->bexec && ctx->bkey == key) {
    CU(cudaGraphLaunch(ctx->bexec, bs));
  } else if (use_graph &&
             cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    rc = enqueue(bs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(bs, &graph);
    if (rc != BGPC_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != BGPC_OK ? rc : BGPC_ECUDA;
    }
    if (ctx->bexec) cudaGraphExecDestroy(ctx->bexec);
    ctx->bexec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ctx->bexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      ctx->bexec = nullptr;
      return BGPC_ECUDA;
    }
    ctx->bkey = key;
    CU(cudaGraphLaunch(ctx->bexec, bs));
  } else {
    cudaGetLastError();
    if ((rc = enqueue(bs))) return rc;
  }
  CU(cudaEventRecord(ctx->bev[3], bs));
  CU(cudaEventRecord(ctx->bev[1], bs));
  CU(cudaStreamWaitEvent(s, ctx->bev[1], 0));
  CU(cudaStreamSynchronize(bs));
  if (ms_kernel) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->bev[2], ctx->bev[3]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    *ms_kernel = t;
  }
  if (h->glob->err) return BGPC_ETIMEOUT;
  return BGPC_OK;
}

int batch_persistent(bgpc_ctx_t *ctx, int32_t G, const bgpc_graph_t *graphs,
                     int32_t *const *colors, const bgpc_opts_t &o, bgpc_stats_t *stats,
                     int32_t *rounds_out, int32_t *ncolors_out, cudaStream_t s,
                     const Deadline &dl) {
  BatchHost h;
  int rc = batch_host_views(ctx, G, &h);
  if (rc) return rc;
  int map_id = o.batch_mapping > 0 ? o.batch_mapping - 1 : -1;
  const unsigned long long key = batch_key(G, graphs, colors, o);
  if (map_id < 0) {
    for (const auto &e : ctx->btuned)
      if (e.first == key) map_id = e.second;
  }
  if (map_id < 0) {
    // autotune: one timed run of every candidate on this batch; the fastest
    // is kept for later calls on it (the results are the same for all)
    float best = -1.f;
    for (int c = 0; c < BGPC_BATCH_MAPPINGS; c++) {
      float ms = 0.f;
      if ((rc = batch_once(ctx, G, graphs, colors, o, kBatchMaps[c], c, s, false, &h, &ms)))
        return rc;
      int32_t nfall = 0;
      for (int32_t k = 0; k < G; k++) nfall += h.stat[k].status == kBatchWindow;
      ms += 1000.f * (float)nfall;  // graphs handed back cost a single-graph coloring each
      if (best < 0.f || ms < best) {
        best = ms;
        map_id = c;
      }
    }
    if (ctx->btuned.size() > 64) ctx->btuned.erase(ctx->btuned.begin());
    ctx->btuned.emplace_back(key, map_id);
  }
  float ms_k = 0.f;
  if ((rc = batch_once(ctx, G, graphs, colors, o, kBatchMaps[map_id], map_id, s, true, &h,
                       &ms_k)))
    return rc;
  // per-graph outcome: done, or handed to the single-graph engine
  bgpc_stats_t tot;
  memset(&tot, 0, sizeof(tot));
  tot.hub_threshold = INT32_MAX;  // the persistent kernel keeps no hub bitmaps
  tot.kernel_launches = 1;
  tot.color_launches = 1;
  tot.ms_color = o.profile ? ms_k : 0.0;
  for (int32_t k = 0; k < G; k++) {
    const BatchStat &x = h.stat[k];
    const int32_t status = graphs[k].n_a > 0 ? x.status : kBatchDone;
    int32_t rounds = x.rounds, ncol = x.colors;
    if (status == kBatchRounds) return BGPC_EROUNDS;
    if (status == kBatchWindow) {
      bgpc_stats_t one;
      memset(&one, 0, sizeof(one));
      if ((rc = color_impl(ctx, graphs[k], o, colors[k], &one, s, dl))) return rc;
      rounds = one.rounds;
      ncol = one.colors;
      for (int r = 0; r < BGPC_MAX_REPORT && r < one.rounds; r++) {
        tot.w_per_round[r] += one.w_per_round[r];
        tot.trav_per_round[r] += one.trav_per_round[r];
      }
      tot.trav_total += one.trav_total;
      tot.incid_total += one.incid_total;
      tot.w_total += one.w_total;
      tot.kernel_launches += one.kernel_launches;
      tot.hub_threshold = one.hub_threshold < tot.hub_threshold ? one.hub_threshold
                                                                : tot.hub_threshold;
      tot.hubs += one.hubs;
      tot.pieces_total++;  // graphs handed to the single-graph engine
    } else if (status != kBatchDone) {
      return BGPC_EINTERNAL;
    } else {
      for (int r = 0; r < BGPC_MAX_REPORT && r < kBatchReport && r < x.rounds; r++) {
        tot.w_per_round[r] += x.w_per_round[r];
        tot.trav_per_round[r] += x.trav_per_round[r];
      }
      tot.trav_total += x.trav_total;
      tot.incid_total += x.incid_total;
      tot.w_total += x.w_total;
    }
    if (graphs[k].n_a == 0) {
      rounds = 0;
      ncol = 0;
    }
    if (rounds_out) rounds_out[k] = rounds;
    if (ncolors_out) ncolors_out[k] = ncol;
    tot.rounds = rounds > tot.rounds ? rounds : tot.rounds;
    tot.colors = ncol > tot.colors ? ncol : tot.colors;
  }
  tot.ms_total = dl.ms();
  if (stats) *stats = tot;
  return BGPC_OK;
}

}  // namespace

extern "C" {

void bgpc_opts_default(bgpc_opts_t *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->policy = BGPC_FF;
  o->chunk = 64;
  o->waves = 16;
  o->big_net = 64;
  o->rank = nullptr;
  o->max_rounds = 1000;
  o->validate = 0;
  o->stop_after_waves = 0;
  o->W_out = nullptr;
  o->want_balance = 0;
}

int bgpc_ctx_create(bgpc_ctx_t **out, int device) {
  if (!out) return BGPC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BGPC_EINVAL;
  }
  Guard guard(device);
  bgpc_ctx_t *ctx = new bgpc_ctx_t();
  ctx->device = device;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                             device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, device) != cudaSuccess ||
      cudaMalloc((void **)&ctx->dev, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost((void **)&ctx->host, sizeof(DevScalars)) != cudaSuccess) {
    cudaGetLastError();
    bgpc_ctx_destroy(ctx);
    return BGPC_ECUDA;
  }
  *out = ctx;
  return BGPC_OK;
}

int bgpc_ctx_destroy(bgpc_ctx_t *ctx) {
  if (!ctx) return BGPC_OK;
  Guard guard(ctx->device);
  cudaDeviceSynchronize();
  release(ctx->tpos); release(ctx->nc); release(ctx->npos); release(ctx->nown);
  release(ctx->s_own); release(ctx->d2tot); release(ctx->W0); release(ctx->W1);
  release(ctx->kofs); release(ctx->stage); release(ctx->newpos); release(ctx->lose);
  release(ctx->netc); release(ctx->ihub); release(ctx->brow);
  release(ctx->thist); release(ctx->tsums); release(ctx->ownid); release(ctx->kgstart);
  for (int q = 0; q < 4; q++) release(ctx->ksc[q]);
  release(ctx->blocksum); release(ctx->bigt); release(ctx->bigd);
  release(ctx->hub_id); release(ctx->hub_net); release(ctx->nbm);
  release(ctx->cptr); release(ctx->cidx); release(ctx->dtab); release(ctx->vtab);
  release(ctx->wlist); release(ctx->segoff); release(ctx->segmap); release(ctx->gbm);
  release(ctx->gcnt); release(ctx->gsum); release(ctx->lbm); release(ctx->pkeys);
  release(ctx->gadj);
  if (ctx->h_wlist) cudaFreeHost(ctx->h_wlist);
  for (bgpc_ctx_t *sub : ctx->subs) bgpc_ctx_destroy(sub);
  for (cudaStream_t st : ctx->sub_streams) cudaStreamDestroy(st);
  ctx->subs.clear();
  ctx->sub_streams.clear();
  release(ctx->card); release(ctx->bad);
  release(ctx->bW0); release(ctx->bW1); release(ctx->bstage); release(ctx->bown);
  release(ctx->bsown); release(ctx->bd2); release(ctx->bkofs); release(ctx->bbig);
  release(ctx->btcnt); release(ctx->btofs); release(ctx->blose); release(ctx->binW);
  release(ctx->bntag);
  release(ctx->bdesc); release(ctx->bst); release(ctx->bstat); release(ctx->bglob);
  if (ctx->bexec) cudaGraphExecDestroy(ctx->bexec);
  if (ctx->h_batch) cudaFreeHost(ctx->h_batch);
  if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
  for (cudaEvent_t e : ctx->bev)
    if (e) cudaEventDestroy(e);
  release(ctx->rkey0); release(ctx->rkey1); release(ctx->rval0); release(ctx->rval1);
  release(ctx->rhist); release(ctx->rsum); release(ctx->mpart); release(ctx->mgrad);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  ctx->events.clear();
  if (ctx->dev) cudaFree(ctx->dev);
  if (ctx->host) cudaFreeHost(ctx->host);
  delete ctx;
  return BGPC_OK;
}

int bgpc_color(bgpc_ctx_t *ctx, const bgpc_graph_t *g, const bgpc_opts_t *opts, int32_t *colors,
               bgpc_stats_t *stats, void *stream) {
  if (!ctx) return BGPC_EINVAL;
  int rc = check_graph_args(g);
  if (rc) return rc;
  if ((rc = check_opts(opts))) return rc;
  if (g->n_a > 0 && !colors) return BGPC_EINVAL;
  Guard guard(ctx->device);
  Deadline dl(opts->timeout_us);
  return color_impl(ctx, *g, *opts, colors, stats, (cudaStream_t)stream, dl);
}

int bgpc_color_batched(bgpc_ctx_t *ctx, int32_t n_graphs, const bgpc_graph_t *graphs,
                       const bgpc_opts_t *opts, int32_t *const *colors, bgpc_stats_t *stats,
                       int32_t *rounds_out, int32_t *ncolors_out, void *stream) {
  if (!ctx || n_graphs < 1 || n_graphs > 65535 || !graphs || !colors) return BGPC_EINVAL;
  int rc = check_opts(opts);
  if (rc) return rc;
  if (opts->rank || opts->stop_after_waves || opts->batch_streams < 0 ||
      opts->batch_streams > 64)
    return BGPC_EINVAL;
  for (int32_t k = 0; k < n_graphs; k++) {
    if ((rc = check_graph_args(&graphs[k]))) return rc;
    if (graphs[k].n_a > 0 && !colors[k]) return BGPC_EINVAL;
  }
  if (opts->net_rounds != 0 || opts->batch_engine < BGPC_BATCH_PERSISTENT ||
      opts->batch_engine > BGPC_BATCH_STREAMS || opts->batch_mapping < 0 ||
      opts->batch_mapping > BGPC_BATCH_MAPPINGS)
    return BGPC_EINVAL;
  Guard guard(ctx->device);
  Deadline dl(opts->timeout_us);
  cudaStream_t s = (cudaStream_t)stream;
  if (opts->validate) {
    for (int32_t k = 0; k < n_graphs; k++) {
      const bgpc_graph_t &gk = graphs[k];
      if (gk.n_a > 0 && (rc = validate_csr(ctx, gk.a_ptr, gk.a_idx, gk.n_a, gk.nnz, gk.n_b, s)))
        return rc;
      if (gk.n_b > 0 && (rc = validate_csr(ctx, gk.b_ptr, gk.b_idx, gk.n_b, gk.nnz, gk.n_a, s)))
        return rc;
    }
  }
  // the persistent engine's task counters hold up to 2^23 tasks per phase
  bool fits = true;
  for (int32_t k = 0; k < n_graphs; k++) {
    const int64_t na = graphs[k].n_a, nb = graphs[k].n_b;
    const int64_t nch = (na + opts->chunk - 1) / opts->chunk;
    if ((na + 1023) / 1024 + (nb + 1023) / 1024 >= (1 << 23) || nch / opts->waves >= (1 << 23))
      fits = false;
  }
  if (opts->batch_engine == BGPC_BATCH_PERSISTENT && fits) {
    bgpc_opts_t o = *opts;
    o.validate = 0;
    return batch_persistent(ctx, n_graphs, graphs, colors, o, stats, rounds_out, ncolors_out, s,
                            dl);
  }
  int K = opts->batch_streams > 0 ? opts->batch_streams : 8;
  if (K > n_graphs) K = n_graphs;
  while ((int)ctx->subs.size() < K) {
    bgpc_ctx_t *sub = nullptr;
    if ((rc = bgpc_ctx_create(&sub, ctx->device))) return rc;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      bgpc_ctx_destroy(sub);
      return BGPC_ECUDA;
    }
    ctx->subs.push_back(sub);
    ctx->sub_streams.push_back(st);
  }
  // the workers' streams start after everything already queued on `stream`
  cudaEvent_t ev = nullptr;
  CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CU(cudaEventRecord(ev, s));
  for (int w = 0; w < K; w++) CU(cudaStreamWaitEvent(ctx->sub_streams[(size_t)w], ev, 0));
  std::vector<bgpc_stats_t> per((size_t)n_graphs);
  std::atomic<int32_t> next(0);
  std::atomic<int> err(0);
  auto work = [&](int w) {
    cudaSetDevice(ctx->device);
    for (;;) {
      if (err.load() != 0) return;
      const int32_t k = next.fetch_add(1);
      if (k >= n_graphs) return;
      memset(&per[(size_t)k], 0, sizeof(bgpc_stats_t));
      const int r = color_impl(ctx->subs[(size_t)w], graphs[k], *opts, colors[k],
                               &per[(size_t)k], ctx->sub_streams[(size_t)w], dl);
      if (r != BGPC_OK) {
        int zero = 0;
        err.compare_exchange_strong(zero, r);
        return;
      }
    }
  };
  if (K == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    th.reserve((size_t)K);
    for (int w = 0; w < K; w++) th.emplace_back(work, w);
    for (auto &t : th) t.join();
  }
  for (int w = 0; w < K; w++) cudaStreamSynchronize(ctx->sub_streams[(size_t)w]);
  cudaEventDestroy(ev);
  if (err.load() != 0) return err.load();
  bgpc_stats_t tot;
  memset(&tot, 0, sizeof(tot));
  tot.hub_threshold = INT32_MAX;
  for (int32_t k = 0; k < n_graphs; k++) {
    const bgpc_stats_t &st = per[(size_t)k];
    tot.hub_threshold = st.hub_threshold < tot.hub_threshold ? st.hub_threshold
                                                             : tot.hub_threshold;
    tot.hubs += st.hubs;
    if (rounds_out) rounds_out[k] = st.rounds;
    if (ncolors_out) ncolors_out[k] = st.colors;
    tot.rounds = st.rounds > tot.rounds ? st.rounds : tot.rounds;
    tot.colors = st.colors > tot.colors ? st.colors : tot.colors;
    for (int r = 0; r < BGPC_MAX_REPORT && r < st.rounds; r++) {
      tot.w_per_round[r] += st.w_per_round[r];
      tot.trav_per_round[r] += st.trav_per_round[r];
    }
    tot.trav_total += st.trav_total;
    tot.incid_total += st.incid_total;
    tot.w_total += st.w_total;
    tot.trav_large += st.trav_large;
    tot.incid_large += st.incid_large;
    tot.w_large += st.w_large;
    tot.trav_hub += st.trav_hub;
    tot.hub_pairs += st.hub_pairs;
    tot.hub_words += st.hub_words;
    tot.pieces_total += st.pieces_total;
    tot.kernel_launches += st.kernel_launches;
    tot.color_launches += st.color_launches;
    tot.ms_setup += st.ms_setup;
    tot.ms_color += st.ms_color;
    tot.ms_publish += st.ms_publish;
    tot.ms_detect += st.ms_detect;
    tot.ms_gather += st.ms_gather;
  }
  tot.ms_total = dl.ms();
  if (stats) *stats = tot;
  return BGPC_OK;
}

int d2gc_color(bgpc_ctx_t *ctx, const bgpc_ugraph_t *g, const bgpc_opts_t *opts, int32_t *colors,
               bgpc_stats_t *stats, void *stream) {
  if (!ctx || !g || g->n < 0 || g->nnz < 0) return BGPC_EINVAL;
  if (g->n > 0 && (!g->ptr || !colors)) return BGPC_EINVAL;
  if (g->nnz > 0 && !g->idx) return BGPC_EINVAL;
  if ((int64_t)g->nnz + g->n >= INT32_MAX) return BGPC_EINVAL;
  int rc = check_opts(opts);
  if (rc) return rc;
  Guard guard(ctx->device);
  Deadline dl(opts->timeout_us);
  cudaStream_t s = (cudaStream_t)stream;
  if (opts->validate && g->n > 0) {
    if ((rc = validate_csr(ctx, g->ptr, g->idx, g->n, g->nnz, g->n, s))) return rc;
  }
  const int32_t cn = g->nnz + g->n;
  CU(grow(ctx->cptr, (size_t)g->n + 1));
  CU(grow(ctx->cidx, (size_t)(cn > 0 ? cn : 1)));
  launch_closed_nbhd(*g, ctx->cptr.p, ctx->cidx.p, ctx->num_sms, s);
  CU(cudaGetLastError());
  bgpc_graph_t bg;
  bg.n_a = g->n;
  bg.n_b = g->n;
  bg.nnz = cn;
  bg.a_ptr = ctx->cptr.p;
  bg.a_idx = ctx->cidx.p;
  bg.b_ptr = ctx->cptr.p;
  bg.b_idx = ctx->cidx.p;
  bgpc_opts_t o = *opts;
  return color_impl(ctx, bg, o, colors, stats, s, dl, 1);
}

int bgpc_validate(bgpc_ctx_t *ctx, const bgpc_graph_t *g, const int32_t *colors, int64_t *n_bad,
                  void *stream) {
  if (!ctx || !n_bad) return BGPC_EINVAL;
  int rc = check_graph_args(g);
  if (rc) return rc;
  if (g->n_a > 0 && !colors) return BGPC_EINVAL;
  Guard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  *n_bad = 0;
  if (g->n_a == 0) return BGPC_OK;
  CU(grow(ctx->bigt, (size_t)(g->n_b > 0 ? g->n_b : 1)));
  CU(grow(ctx->bigd, (size_t)(g->n_b > 0 ? g->n_b : 1)));
  CU(grow(ctx->bad, (size_t)g->n_a));
  CU(cudaMemsetAsync(ctx->dev, 0, sizeof(DevScalars), s));
  launch_net_static(*g, INT32_MAX, ctx->bigt.p, ctx->bigd.p, ctx->dev, s);
  launch_gmax(colors, g->n_a, ctx->dev, s);
  if ((rc = sync_scalars(ctx, s))) return rc;
  const int32_t tabcap = ctx->host->gmax + 1 > 0 ? ctx->host->gmax + 1 : 1;
  const int32_t nbig_d = ctx->host->nbig_d;
  const int32_t nslots = nbig_d < 2 * ctx->num_sms ? (nbig_d > 0 ? nbig_d : 1) : 2 * ctx->num_sms;
  const size_t need = (size_t)nslots * (size_t)tabcap;
  if (need > ctx->vtab.cap) {
    CU(grow(ctx->vtab, need));
    CU(cudaMemsetAsync(ctx->vtab.p, 0, ctx->vtab.cap * sizeof(int32_t), s));
  }
  launch_validate(*g, colors, ctx->bigd.p, nbig_d, ctx->vtab.p, tabcap, nslots, ctx->bad.p,
                  ctx->dev, ctx->num_sms, s);
  CU(cudaGetLastError());
  if ((rc = sync_scalars(ctx, s))) return rc;
  *n_bad = (int64_t)ctx->host->acc[0];
  return BGPC_OK;
}

int bgpc_color_sets(bgpc_ctx_t *ctx, const int32_t *colors, int32_t n, int64_t *card,
                    int32_t max_colors, int32_t *n_sets, int32_t *max_card, double *mean_card,
                    double *std_card, void *stream) {
  if (!ctx || n < 0 || max_colors < 1 || !card || (n > 0 && !colors)) return BGPC_EINVAL;
  Guard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaMemsetAsync(&ctx->dev->err, 0, sizeof(int32_t), s));
  launch_card(colors, n, (unsigned long long *)card, max_colors, &ctx->dev->err, s);
  launch_card_stats((const unsigned long long *)card, max_colors, ctx->dev, s);
  CU(cudaGetLastError());
  int rc = sync_scalars(ctx, s);
  if (rc) return rc;
  if (ctx->host->err) return BGPC_EINVAL;
  const double sets = (double)ctx->host->acc[0];
  const double mean = sets > 0 ? (double)ctx->host->acc[2] / sets : 0.0;
  const double var = sets > 0 ? (double)ctx->host->acc[3] / sets - mean * mean : 0.0;
  if (n_sets) *n_sets = (int32_t)ctx->host->acc[0];
  if (max_card) *max_card = (int32_t)ctx->host->acc[1];
  if (mean_card) *mean_card = mean;
  if (std_card) *std_card = var > 0 ? sqrt(var) : 0.0;
  return BGPC_OK;
}

const char *bgpc_strerror(int status) {
  switch (status) {
    case BGPC_OK: return "ok";
    case BGPC_STOPPED: return "stopped after the requested number of waves";
    case BGPC_EINVAL: return "invalid argument";
    case BGPC_ENOMEM: return "out of device memory or on-chip capacity";
    case BGPC_ECUDA: return "CUDA runtime error";
    case BGPC_EROUNDS: return "round limit exceeded";
    case BGPC_ETIMEOUT: return "a bounded device wait timed out";
    case BGPC_EUNSORTED: return "adjacency not sorted/unique or CSR and CSC disagree";
    case BGPC_EINTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

}  // extern "C"
