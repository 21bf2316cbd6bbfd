// Setup of one coloring call: input validation, the static per-graph
// analysis (CSR->CSC edge map, owner nets, two-hop volumes) and the initial
// work queue and net-major mirrors (Alg. 1, first two lines: W <- V_color,
// c <- -1).  Also the D2GC front end: closed neighbourhoods N[u] (Sec. IV).
#include "bgpc_internal.cuh"

namespace bgpc {
namespace {

constexpr int kNT = 256;
constexpr unsigned kFull = 0xffffffffu;

__global__ void k_check_ptr(const int32_t *__restrict__ ptr, int32_t n, int32_t nnz,
                            int32_t *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  int32_t x = ptr[i];
  bool bad = (x < 0 || x > nnz);
  if (i == 0) bad |= (x != 0);
  if (i == n) bad |= (x != nnz);
  if (i < n) bad |= (ptr[i + 1] < x);
  if (bad) atomicOr(err, ERR_RANGE);
}

// One warp per row: indices in [0, bound), strictly increasing.
__global__ void k_check_rows(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                             int32_t n, int32_t bound, int32_t *err) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    int32_t beg = ptr[r], end = ptr[r + 1];
    int flags = 0;
    for (int32_t e = beg + lane; e < end; e += 32) {
      int32_t x = idx[e];
      if (x < 0 || x >= bound) flags |= ERR_RANGE;
      if (e + 1 < end && idx[e + 1] <= x) flags |= ERR_UNSORTED;
    }
    if (flags) atomicOr(err, flags);
  }
}

// ---- tpos: the CSC entry of every CSR entry.  CSR entry i of vertex w is
// the pair (w, v); the CSC lists each net's members in increasing order, so
// the CSC indices f of w's pairs, in increasing f, are in increasing v: tpos
// restricted to row w is exactly the CSC indices whose member is w, in
// order.  tpos is therefore the stable sort of the CSC indices by member id
// (an LSD radix sort, 8-bit digits, tiles of 4096 entries).
constexpr int kSortPer = 16;
constexpr int kSortTile = kNT * kSortPer;
static_assert(kNT == 256, "one thread per digit");

// Digit counts of one tile: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kNT) k_tsort_hist(const int32_t *__restrict__ key, int64_t n,
                                                    int shift, int32_t ntiles,
                                                    int32_t *__restrict__ hist) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x;
  int32_t d[kSortPer];
#pragma unroll
  for (int q = 0; q < kSortPer; q++) {
    const int64_t i = base + (int64_t)q * kNT;
    d[q] = i < n ? (int32_t)(((uint32_t)key[i] >> shift) & 255u) : -1;
  }
#pragma unroll
  for (int q = 0; q < kSortPer; q++)
    if (d[q] >= 0) atomicAdd(&cnt[d[q]], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile, in 16 batches of 256: an entry goes to its
// digit's start for this tile (scanned counts) plus the entries of that digit
// in earlier batches, earlier warps and earlier lanes.  vin == nullptr: the
// value is the index; kout == nullptr: keys are not written (last pass).
__global__ void __launch_bounds__(kNT) k_tsort_scatter(const int32_t *__restrict__ kin,
                                                       const int32_t *__restrict__ vin, int64_t n,
                                                       int shift, int32_t ntiles,
                                                       const int32_t *__restrict__ off,
                                                       int32_t *__restrict__ kout,
                                                       int32_t *__restrict__ vout) {
  constexpr int NW = kNT / 32;
  __shared__ int32_t wc[NW][256];
  __shared__ int32_t run[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = off[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x;
  // the tile's keys and values, all loaded before the batches are ranked
  int32_t kq[kSortPer], vq[kSortPer];
#pragma unroll
  for (int q = 0; q < kSortPer; q++) {
    const int64_t i = base + (int64_t)q * kNT;
    kq[q] = i < n ? kin[i] : 0;
    vq[q] = i < n ? (vin ? vin[i] : (int32_t)i) : 0;
  }
#pragma unroll
  for (int q = 0; q < kSortPer; q++) {
    for (int x = threadIdx.x; x < NW * 256; x += kNT) (&wc[0][0])[x] = 0;
    __syncthreads();
    const int64_t i = base + (int64_t)q * kNT;
    const bool live = i < n;
    const int32_t k = kq[q], val = vq[q];
    const int d = live ? (int)(((uint32_t)k >> shift) & 255u) : -1 - lane;  // dummies differ
    const unsigned peers = __match_any_sync(kFull, d);
    const int before = __popc(peers & ((1u << lane) - 1u));
    if (live && before == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    {  // this batch's start of each digit per warp, and the next batch's start
      int32_t r = run[threadIdx.x];
      for (int w = 0; w < NW; w++) {
        const int32_t t = wc[w][threadIdx.x];
        wc[w][threadIdx.x] = r;
        r += t;
      }
      run[threadIdx.x] = r;
    }
    __syncthreads();
    if (live) {
      const int32_t pos = wc[warp][d] + before;
      if (kout) kout[pos] = k;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

// ihub[i] = the hub slot of the net of CSR entry i, or -1.
__global__ void k_ihub(const int32_t *__restrict__ a_idx, int64_t nnz,
                       const int32_t *__restrict__ hub_id, int32_t *__restrict__ ihub) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x)
    ihub[i] = hub_id[a_idx[i]];
}

// ---- kofs in id order (W in increasing id): a vertex's k is the number of
// earlier W vertices with the same owner net (of more than T members), i.e.
// its index within its owner's group after a stable sort of the W positions
// by owner net.  Keys: the owner net, or n_b for the vertices without one.
__global__ void k_kofs_keys(const int32_t *__restrict__ W, int32_t m,
                            const int32_t *__restrict__ ownid, const int32_t *__restrict__ s_own,
                            int32_t T, int32_t n_b, int32_t *__restrict__ key) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = W[p];
    key[p] = s_own[w] > T ? ownid[w] : n_b;
  }
}

// gstart[v] = the first sorted index of group v.
__global__ void k_kofs_heads(const int32_t *__restrict__ ks, int32_t m, int32_t n_b,
                             int32_t *__restrict__ gstart) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = ks[j];
    if (k < n_b && (j == 0 || ks[j - 1] != k)) gstart[k] = (int32_t)j;
  }
}

__global__ void k_kofs_write(const int32_t *__restrict__ ks, const int32_t *__restrict__ vs,
                             int32_t m, int32_t n_b, const int32_t *__restrict__ gstart,
                             int32_t *__restrict__ kofs) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = ks[j];
    if (k < n_b) kofs[vs[j]] = (int32_t)j - gstart[k];
  }
}

// Validation: CSR entry i = (w, v) and CSC entry tpos[i] are the same pair
// (member w, in net v); otherwise CSR and CSC differ.
__global__ void k_tpos_check(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ a_idx,
                             const int32_t *__restrict__ b_ptr, const int32_t *__restrict__ b_idx,
                             int32_t n_a, const int32_t *__restrict__ tpos, int32_t *err) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < n_a; w += nwarps) {
    const int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    bool bad = false;
    for (int32_t i = beg + lane; i < end; i += 32) {
      const int32_t f = tpos[i], v = a_idx[i];
      bad |= b_idx[f] != (int32_t)w || f < b_ptr[v] || f >= b_ptr[v + 1];
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, ERR_MISMATCH);
  }
}

// Per vertex: owner net (largest, ties -> larger id), its size, the sum of
// its net sizes (two-hop volume incl. w itself), and the owner flag nown[]
// of every CSC entry.
// With netc != NULL also the color the net-based first round (Alg. 8) gives
// w: in that round every vertex is uncolored, so F is empty in every net and
// the i-th visited member of net v is proposed |vtxs(v)| - 1 - i; w keeps
// the proposal of its owner net, where it sits at CSC position tpos of its
// owner entry (i = that position within the net; with center_first, Alg. 9's
// order for D2GC, the center v is visited first and the others follow in
// adjacency order).  A vertex without nets gets -1.
__global__ void k_vertex_static(const int32_t *__restrict__ a_ptr,
                                const int32_t *__restrict__ a_idx,
                                const int32_t *__restrict__ b_ptr,
                                const int32_t *__restrict__ tpos, int32_t n_a,
                                int32_t *__restrict__ s_own, int32_t *__restrict__ d2tot,
                                uint8_t *__restrict__ nown, int32_t *__restrict__ netc,
                                int32_t center_first, int32_t *__restrict__ ownid) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < n_a; w += nwarps) {
    int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    long long sum = 0;
    // pack (size, net) so that max() breaks ties towards the larger net id
    unsigned long long best = 0;
    for (int32_t i = beg + lane; i < end; i += 32) {
      int32_t v = a_idx[i];
      int32_t s = b_ptr[v + 1] - b_ptr[v];
      sum += s;
      unsigned long long key = ((unsigned long long)(uint32_t)s << 32) | (uint32_t)v;
      if (key > best) best = key;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
      unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      if (ob > best) best = ob;
    }
    int32_t own = (end > beg) ? (int32_t)(best & 0xffffffffu) : -1;
    const int32_t so = (end > beg) ? (int32_t)(best >> 32) : 0;
    if (lane == 0) {
      s_own[w] = so;
      ownid[w] = own;
      d2tot[w] = (int32_t)sum;
      if (netc && end == beg) netc[w] = -1;
    }
    // the owner flags per CSC entry (nown may be NULL: not needed in id
    // order) and the N1 proposal from the owner entry's CSC position
    for (int32_t i = beg + lane; i < end && (nown || netc); i += 32) {
      const bool mine = a_idx[i] == own;
      if (!nown && !mine) continue;
      const int32_t f = tpos[i];
      if (nown) nown[f] = mine ? 1 : 0;
      if (netc && mine) {
        int32_t k = f - b_ptr[own];
        if (center_first) k = ((int32_t)w == own) ? 0 : k + 1 - (own < (int32_t)w ? 1 : 0);
        // in [0, so) for consistent CSR and CSC (kept there for any input)
        netc[w] = so - 1 - min(max(k, 0), max(so - 1, 0));
      }
    }
  }
}

// Largest net, the lists of nets above T (reverse first fit) and above the
// warp-detection size, and the histogram of net sizes over the hub ladder.
// List order does not affect any result.
__global__ void k_net_static(const int32_t *__restrict__ b_ptr, int32_t n_b, int32_t T,
                             int32_t *__restrict__ bigt, int32_t *__restrict__ bigd,
                             DevScalars *dev) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int32_t s = 0;
  if (v < n_b) {
    s = b_ptr[v + 1] - b_ptr[v];
    if (s > T) bigt[atomicAdd(&dev->nbig_t, 1)] = (int32_t)v;
    if (s > kDetectWarpMax) bigd[atomicAdd(&dev->nbig_d, 1)] = (int32_t)v;
    if (s > kHubMin) {
      int k = 0;
      while (k + 1 < kHubLadder && hub_ladder(k + 1) < s) k++;
      atomicAdd(&dev->hub_hist[k], 1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s = max(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0 && s > 0) atomicMax(&dev->maxnet, s);
}

// W_0 = V_A in rank order: W[rank[w]] = w, and a check that rank is a
// permutation (every slot written exactly once).
__global__ void k_queue_scatter(const int32_t *__restrict__ rank, int32_t n, int32_t *W,
                                int32_t *err) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  if (!rank) { W[w] = (int32_t)w; return; }
  int32_t r = rank[w];
  if (r < 0 || r >= n) { atomicOr(err, ERR_RANK); return; }
  W[r] = (int32_t)w;
}

__global__ void k_queue_check(const int32_t *__restrict__ rank, int32_t n,
                              const int32_t *__restrict__ W, int32_t *err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !rank) return;
  int32_t w = W[p];
  if (w < 0 || w >= n || rank[w] != (int32_t)p) atomicOr(err, ERR_RANK);
}

// The net-major mirrors at the start: every member is uncolored and in W_0
// at position pos(u) = rank[u] (or u), so nc[f] = -2 - pos and npos[f] = pos
// for the CSC entry f of member u.  Written in CSC order (coalesced; only
// rank is read at random), and c <- -1.
__global__ void k_init_mirror(const int32_t *__restrict__ b_idx, int64_t nnz,
                              const int32_t *__restrict__ rank, int32_t n_a,
                              int32_t *__restrict__ nc, int32_t *__restrict__ npos,
                              int32_t *__restrict__ colors) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nnz; f += stride) {
    const int32_t u = b_idx[f];
    const int32_t pos = rank ? rank[u] : u;
    nc[f] = -2 - pos;
    npos[f] = pos;
  }
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_a; w += stride)
    colors[w] = -1;
}

// N[u] = adj(u) with u inserted at its sorted place: cptr[u] = ptr[u] + u.
__global__ void k_closed_nbhd(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                              int32_t n, int32_t *__restrict__ cptr, int32_t *__restrict__ cidx) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    int32_t beg = ptr[u], end = ptr[u + 1];
    int32_t obase = beg + (int32_t)u;
    if (lane == 0) {
      cptr[u] = obase;
      if (u == n - 1) cptr[n] = end + n;
    }
    int32_t below = 0;  // neighbours smaller than u seen so far
    for (int32_t e0 = beg; e0 < end; e0 += 32) {
      int32_t e = e0 + lane;
      int32_t x = (e < end) ? idx[e] : INT32_MAX;
      unsigned lt = __ballot_sync(0xffffffffu, e < end && x < (int32_t)u);
      if (e < end) {
        int32_t o = (x < (int32_t)u) ? (e - beg) : (e - beg + 1);
        cidx[obase + o] = x;
      }
      below += __popc(lt);
    }
    if (lane == 0) cidx[obase + below] = (int32_t)u;
  }
}

inline int grid_warps(long long items, int sms) {
  long long g = div_up(items * 32, kNT);
  long long cap = (long long)sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int launch_check_ptr(const int32_t *ptr, int32_t n, int32_t nnz, int32_t *err, cudaStream_t s) {
  k_check_ptr<<<div_up((long long)n + 1, kNT), kNT, 0, s>>>(ptr, n, nnz, err);
  return 1;
}

int launch_check_rows(const int32_t *ptr, const int32_t *idx, int32_t n, int32_t bound,
                       int32_t *err, int sms, cudaStream_t s) {
  if (n <= 0) return 0;
  k_check_rows<<<grid_warps(n, sms), kNT, 0, s>>>(ptr, idx, n, bound, err);
  return 1;
}

int64_t tpos_hist_len(int64_t nnz) { return div_up(nnz, (long long)kSortTile) * 256; }

int launch_tpos(const bgpc_graph_t &g, int32_t *tpos, int32_t *const scratch[4], int32_t *hist,
                int32_t *sums, int32_t validate, int32_t *err, const int32_t *hub_id,
                int32_t *ihub, int sms, cudaStream_t s) {
  if (g.n_a <= 0 || g.nnz <= 0) return 0;
  const int64_t n = g.nnz;
  const int32_t ntiles = (int32_t)div_up(n, (long long)kSortTile);
  const int64_t hlen = (int64_t)ntiles * 256;
  const uint32_t top = g.n_a > 1 ? (uint32_t)(g.n_a - 1) : 1u;
  const int passes = (32 - __builtin_clz(top) + 7) / 8;  // 8-bit digits of the member ids
  int nk = 0;
  const int32_t *kin = g.b_idx, *vin = nullptr;
  for (int p = 0; p < passes; p++) {
    const bool last = p == passes - 1;
    int32_t *kout = last ? nullptr : scratch[2 * (p & 1)];
    int32_t *vout = last ? tpos : scratch[2 * (p & 1) + 1];
    k_tsort_hist<<<ntiles, kNT, 0, s>>>(kin, n, 8 * p, ntiles, hist);
    nk += 1 + launch_excl_scan(hist, hlen, sums, s);
    k_tsort_scatter<<<ntiles, kNT, 0, s>>>(kin, vin, n, 8 * p, ntiles, hist, kout, vout);
    nk++;
    kin = kout;
    vin = vout;
  }
  if (validate) {
    k_tpos_check<<<grid_warps(g.n_a, sms), kNT, 0, s>>>(g.a_ptr, g.a_idx, g.b_ptr, g.b_idx, g.n_a,
                                                        tpos, err);
    nk++;
  }
  if (ihub) {
    long long grid = div_up(n, (long long)kNT);
    if (grid > (long long)sms * 16) grid = (long long)sms * 16;
    k_ihub<<<(int)grid, kNT, 0, s>>>(g.a_idx, n, hub_id, ihub);
    nk++;
  }
  return nk;
}

int launch_kofs_sorted(const int32_t *W, int32_t m, const int32_t *ownid, const int32_t *s_own,
                       int32_t T, int32_t n_b, int32_t *const scratch[4], int32_t *hist,
                       int32_t *sums, int32_t *gstart, int32_t *kofs, int sms, cudaStream_t s) {
  if (m <= 0) return 0;
  const int32_t ntiles = (int32_t)div_up((long long)m, (long long)kSortTile);
  const int64_t hlen = (int64_t)ntiles * 256;
  long long grid = div_up((long long)m, (long long)kNT);
  if (grid > (long long)sms * 16) grid = (long long)sms * 16;
  int nk = 0;
  k_kofs_keys<<<(int)grid, kNT, 0, s>>>(W, m, ownid, s_own, T, n_b, scratch[0]);
  nk++;
  const int passes = (32 - __builtin_clz((uint32_t)(n_b > 0 ? n_b : 1)) + 7) / 8;
  // pass p reads the pair (p & 1) (pass 0: the keys alone) and writes the other
  const int32_t *kin = scratch[0], *vin = nullptr;
  for (int p = 0; p < passes; p++) {
    int32_t *kout = scratch[2 * ((p + 1) & 1)];
    int32_t *vout = scratch[2 * ((p + 1) & 1) + 1];
    k_tsort_hist<<<ntiles, kNT, 0, s>>>(kin, m, 8 * p, ntiles, hist);
    nk += 1 + launch_excl_scan(hist, hlen, sums, s);
    k_tsort_scatter<<<ntiles, kNT, 0, s>>>(kin, vin, m, 8 * p, ntiles, hist, kout, vout);
    nk++;
    kin = kout;
    vin = vout;
  }
  k_kofs_heads<<<(int)grid, kNT, 0, s>>>(kin, m, n_b, gstart);
  k_kofs_write<<<(int)grid, kNT, 0, s>>>(kin, vin, m, n_b, gstart, kofs);
  return nk + 2;
}

int launch_vertex_static(const bgpc_graph_t &g, const int32_t *tpos, int32_t *s_own,
                          int32_t *d2tot, uint8_t *nown, int32_t *netc, int32_t center_first,
                          int32_t *ownid, int sms, cudaStream_t s) {
  if (g.n_a <= 0) return 0;
  k_vertex_static<<<grid_warps(g.n_a, sms), kNT, 0, s>>>(g.a_ptr, g.a_idx, g.b_ptr, tpos,
                                                          g.n_a, s_own, d2tot, nown, netc,
                                                          center_first, ownid);
  return 1;
}

// The net-based first round's colors (netc, from k_vertex_static) become the
// round's tentative coloring: c[w] = netc[w], mirrored into every CSC entry
// (nc[f] = netc[b_idx[f]], written in CSC order); a vertex without nets got
// no proposal and is flagged to stay in the work queue (it has no CSC entry,
// so the conflict removal never sees it).
__global__ void k_net_publish(const int32_t *__restrict__ b_idx, int64_t nnz,
                              const int32_t *__restrict__ netc, const int32_t *__restrict__ rank,
                              int32_t n_a, int32_t *__restrict__ nc,
                              int32_t *__restrict__ colors, uint8_t *__restrict__ lose) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nnz; f += stride)
    nc[f] = netc[b_idx[f]];
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_a; w += stride) {
    const int32_t c = netc[w];
    colors[w] = c;
    if (c < 0) lose[rank ? rank[w] : (int32_t)w] = 1;
  }
}

int launch_net_publish(const bgpc_graph_t &g, const int32_t *netc, const int32_t *rank,
                       int32_t *nc, int32_t *colors, uint8_t *lose, int sms, cudaStream_t s) {
  if (g.n_a <= 0) return 0;
  const int64_t n = (int64_t)g.nnz > (int64_t)g.n_a ? (int64_t)g.nnz : (int64_t)g.n_a;
  const int64_t cap = (int64_t)sms * 8;
  const int64_t grid = div_up(n, (int64_t)kNT) < cap ? div_up(n, (int64_t)kNT) : cap;
  k_net_publish<<<(int)grid, kNT, 0, s>>>(g.b_idx, g.nnz, netc, rank, g.n_a, nc, colors, lose);
  return 1;
}

int launch_net_static(const bgpc_graph_t &g, int32_t T, int32_t *bigt, int32_t *bigd,
                       DevScalars *dev, cudaStream_t s) {
  if (g.n_b <= 0) return 0;
  k_net_static<<<div_up(g.n_b, kNT), kNT, 0, s>>>(g.b_ptr, g.n_b, T, bigt, bigd, dev);
  return 1;
}

int launch_init_queue(const int32_t *rank, int32_t n_a, int32_t *W, int32_t *err,
                       cudaStream_t s) {
  if (n_a <= 0) return 0;
  if (rank) cudaMemsetAsync(W, 0xff, sizeof(int32_t) * (size_t)n_a, s);
  k_queue_scatter<<<div_up(n_a, kNT), kNT, 0, s>>>(rank, n_a, W, err);
  if (rank) k_queue_check<<<div_up(n_a, kNT), kNT, 0, s>>>(rank, n_a, W, err);
  return rank ? 2 : 1;
}

int launch_init_mirror(const bgpc_graph_t &g, const int32_t *rank, int32_t *nc, int32_t *npos,
                        int32_t *colors, int sms, cudaStream_t s) {
  if (g.n_a <= 0) return 0;
  const int64_t n = (int64_t)g.nnz > (int64_t)g.n_a ? (int64_t)g.nnz : (int64_t)g.n_a;
  const int64_t cap = (int64_t)sms * 8;
  const int64_t grid = div_up(n, (int64_t)kNT) < cap ? div_up(n, (int64_t)kNT) : cap;
  k_init_mirror<<<(int)grid, kNT, 0, s>>>(g.b_idx, g.nnz, rank, g.n_a, nc, npos, colors);
  return 1;
}

int launch_closed_nbhd(const bgpc_ugraph_t &g, int32_t *cptr, int32_t *cidx, int sms,
                        cudaStream_t s) {
  if (g.n <= 0) return 0;
  k_closed_nbhd<<<grid_warps(g.n, sms), kNT, 0, s>>>(g.ptr, g.idx, g.n, cptr, cidx);
  return 1;
}

}  // namespace bgpc
