// RemoveConflicts and the per-round bookkeeping of Alg. 1:
//  * reverse first-fit offsets k for the owners of big nets (Alg. 8's W_local
//    order, restricted to vertices still in W that own the net),
//  * per-net conflict detection (Alg. 7's traversal) with the lower-rank-wins
//    rule of Alg. 3: among members of W_r sharing a color in a net, all but
//    the lowest position lose,
//  * rank-ordered compaction of the losers into W_{r+1} (prefix sums, no
//    order-dependent atomics) and the relabelling of the net-major mirrors.
#include "bgpc_internal.cuh"

namespace bgpc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNT = 256;
constexpr int kScanNT = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanNT * kScanPer;

template <int NT>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *red, int32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) red[warp] = inc;
  __syncthreads();
  int32_t before = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < NT / 32; i++) {
    int32_t r = red[i];
    before += (i < warp) ? r : 0;
    tot += r;
  }
  __syncthreads();
  *total = tot;
  return before + inc - v;
}

// k for each owner of a net with |vtxs| > T that is in W: the number of
// members before it in vtxs order that are in W and own the same net.  Used
// when W follows a caller's rank; in id order the same k comes from a sort
// of the W positions by owner net (launch_kofs_sorted), in work |W|.
__global__ void __launch_bounds__(kNT) k_kofs(const int32_t *__restrict__ b_ptr,
                                              const int32_t *__restrict__ npos,
                                              const uint8_t *__restrict__ nown,
                                              const int32_t *__restrict__ bigt, int32_t nbig,
                                              int32_t *__restrict__ kofs) {
  __shared__ int32_t red[kNT / 32];
  for (int32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const int32_t v = bigt[b];
    const int32_t beg = b_ptr[v], end = b_ptr[v + 1];
    int32_t carry = 0;
    for (int32_t t0 = beg; t0 < end; t0 += kNT) {
      const int32_t f = t0 + (int32_t)threadIdx.x;
      int32_t pos = -1, flag = 0;
      if (f < end) {
        pos = npos[f];
        flag = (pos >= 0 && nown[f]) ? 1 : 0;
      }
      // after the first round most tiles hold no owner in W: one barrier
      if (__syncthreads_count(flag) == 0) continue;
      int32_t total;
      int32_t ex = block_excl_scan<kNT>(flag, red, &total);
      if (flag) kofs[pos] = carry + ex;
      carry += total;
    }
  }
}

__global__ void k_trav(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ W,
                       const int32_t *__restrict__ d2tot, int32_t m, int32_t small_ok,
                       DevScalars *dev) {
  unsigned long long acc = 0, inc = 0, accl = 0, incl = 0, wl = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = W[p];
    const int32_t deg = a_ptr[w + 1] - a_ptr[w];
    const int32_t d2 = d2tot[w];
    acc += (unsigned long long)(d2 - deg);
    inc += (unsigned long long)deg;
    if (!(small_ok && d2 <= kSmallD2 && deg <= kSmallMaxDeg)) {
      accl += (unsigned long long)(d2 - deg);
      incl += (unsigned long long)deg;
      wl++;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(kFull, acc, o);
    inc += __shfl_xor_sync(kFull, inc, o);
    accl += __shfl_xor_sync(kFull, accl, o);
    incl += __shfl_xor_sync(kFull, incl, o);
    wl += __shfl_xor_sync(kFull, wl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (acc) atomicAdd(&dev->trav, acc);
    if (inc) atomicAdd(&dev->incid, inc);
    if (accl) atomicAdd(&dev->trav_large, accl);
    if (incl) atomicAdd(&dev->incid_large, incl);
    if (wl) atomicAdd(&dev->w_large, wl);
  }
}

// Warp tier: one warp per net with at most 32 members.  Members outside W
// never share a color with a W member (their colors were forbidden), so
// only W members take part; a member loses when a member of its color
// class has a smaller position.  In id order (W sorted by id, and a net's
// members too) the W positions grow along the member list, so that member
// is simply an earlier lane of the class.
__global__ void k_detect_warp(const int32_t *__restrict__ b_ptr, int32_t n_b,
                              const int32_t *__restrict__ nc, const int32_t *__restrict__ npos,
                              int32_t id_order, uint8_t *__restrict__ lose) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n_b; v += nwarps) {
    const int32_t beg = b_ptr[v], size = b_ptr[v + 1] - beg;
    if (size < 2 || size > kDetectWarpMax) continue;
    int32_t pos = -1, col = -1 - lane;  // unique dummies for inactive lanes
    if (lane < size) {
      pos = npos[beg + lane];
      if (pos >= 0) col = nc[beg + lane];
    }
    const unsigned grp = __match_any_sync(kFull, col);
    if (id_order) {
      if (pos >= 0 && (grp & ((1u << lane) - 1u))) lose[pos] = 1;
      continue;
    }
    int32_t minpos = (pos >= 0) ? pos : INT32_MAX;
#pragma unroll
    for (int k = 0; k < 32; k++) {
      int32_t pk = __shfl_sync(kFull, pos, k);
      if (((grp >> k) & 1u) && pk >= 0 && pk < minpos) minpos = pk;
    }
    if (pos >= 0 && minpos < pos) lose[pos] = 1;
  }
}

// Table tier: one CTA per net with more than 32 members; a per-CTA table
// indexed by color holds the smallest W position of that color in the net
// (all entries INT32_MAX between nets).
__global__ void __launch_bounds__(kNT) k_detect_table(const int32_t *__restrict__ b_ptr,
                                                      const int32_t *__restrict__ nc,
                                                      const int32_t *__restrict__ npos,
                                                      const int32_t *__restrict__ bigd,
                                                      int32_t nbig, int32_t min_size,
                                                      int32_t *__restrict__ dtab,
                                                      int32_t tabcap, uint8_t *__restrict__ lose) {
  int32_t *tab = dtab + (size_t)blockIdx.x * (size_t)tabcap;
  for (int32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const int32_t v = bigd[b];
    const int32_t beg = b_ptr[v], end = b_ptr[v + 1];
    if (end - beg <= min_size) continue;  // taken by the mid tier
    for (int32_t f = beg + threadIdx.x; f < end; f += kNT) {
      const int32_t pos = npos[f];
      if (pos >= 0) {
        const int32_t c = nc[f];
        if (c >= 0 && c < tabcap) atomicMin(&tab[c], pos);
      }
    }
    __syncthreads();
    for (int32_t f = beg + threadIdx.x; f < end; f += kNT) {
      const int32_t pos = npos[f];
      if (pos >= 0) {
        const int32_t c = nc[f];
        if (c >= 0 && c < tabcap && tab[c] < pos) lose[pos] = 1;
      }
    }
    __syncthreads();
    for (int32_t f = beg + threadIdx.x; f < end; f += kNT) {
      const int32_t pos = npos[f];
      if (pos >= 0) {
        const int32_t c = nc[f];
        if (c >= 0 && c < tabcap) tab[c] = INT32_MAX;
      }
    }
    __syncthreads();
  }
}

// Mid tier, id order: one warp per net of 33 to kMidMax members.  The W
// positions grow along the member list, so a W member loses when an earlier
// member of the net has its color: chunks of 32 members in order, the
// earlier lanes of a color class from __match_any_sync, the earlier chunks
// from a per-warp set of the colors seen (open addressing in shared memory,
// load <= 1/2, emptied after each net).
constexpr int kMidMax = 256;
constexpr int kMidSlots = 512;
__global__ void __launch_bounds__(kNT) k_detect_mid(const int32_t *__restrict__ b_ptr,
                                                    const int32_t *__restrict__ nc,
                                                    const int32_t *__restrict__ npos,
                                                    const int32_t *__restrict__ bigd, int32_t nbig,
                                                    uint8_t *__restrict__ lose) {
  constexpr int NW = kNT / 32;
  __shared__ int32_t tabs[NW][kMidSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t *tab = tabs[warp];
  for (int x = lane; x < kMidSlots; x += 32) tab[x] = -1;
  __syncwarp();
  const unsigned below = (1u << lane) - 1u;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = gw; b < nbig; b += nw) {
    const int32_t v = bigd[b];
    const int32_t beg = b_ptr[v], size = b_ptr[v + 1] - beg;
    if (size > kMidMax) continue;
    int32_t used[kMidMax / 32];  // the slot this lane filled in each chunk, or -1
#pragma unroll
    for (int c = 0; c < kMidMax / 32; c++) {
      used[c] = -1;
      const int32_t k = c * 32 + lane;
      if (c * 32 >= size) continue;  // warp-uniform
      int32_t pos = -1, col = -1 - lane;  // distinct dummies outside W and past the end
      if (k < size) {
        pos = npos[beg + k];
        if (pos >= 0) col = nc[beg + k];
      }
      const unsigned grp = __match_any_sync(kFull, col);
      const bool first = (grp & below) == 0u;  // the class's first lane in this chunk
      bool seen = false;
      if (pos >= 0 && first) {
        uint32_t h = ((uint32_t)col * 0x9E3779B1u) >> 23;  // 9 bits: kMidSlots
        for (;;) {
          const int32_t t = tab[h];
          if (t == col) { seen = true; break; }
          if (t == -1) {
            const int32_t o = atomicCAS(&tab[h], -1, col);
            if (o == -1) { used[c] = (int32_t)h; break; }
            if (o == col) { seen = true; break; }
          }
          h = (h + 1) & (kMidSlots - 1);
        }
      }
      const bool seen_g = __shfl_sync(kFull, seen, __ffs(grp) - 1);
      if (pos >= 0 && (!first || seen_g)) lose[pos] = 1;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < kMidMax / 32; c++)
      if (used[c] >= 0) tab[used[c]] = -1;
    __syncwarp();
  }
}

// Pair tier, for rounds whose W is small against the graph: the net tiers
// read every net, while only the (W member, net) pairs can conflict.  Every
// pair inserts the key (net, color) with its position into an open-addressing
// hash table that keeps the smallest position per key; then every pair looks
// its key up, and a member loses when a smaller position holds one of its
// keys.  The same lose flags as the net tiers, at a cost proportional to the
// sum over W of |nets(w)|.  Keys never leave the table within a round (it is
// cleared before the next use), so a probe sequence never breaks.
constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ unsigned long long pair_key(int32_t v, int32_t c) {
  return ((unsigned long long)(uint32_t)v << 32) | (uint32_t)c;  // v, c >= 0: never empty
}

// The splitmix64 output function (a 64-bit mixer with full avalanche).
__device__ __forceinline__ uint32_t pair_hash(unsigned long long k) {
  k ^= k >> 30;
  k *= 0xbf58476d1ce4e5b9ull;
  k ^= k >> 27;
  k *= 0x94d049bb133111ebull;
  k ^= k >> 31;
  return (uint32_t)k;
}

__global__ void k_pairs_insert(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ a_idx,
                               const int32_t *__restrict__ W, int32_t m,
                               const int32_t *__restrict__ colors, unsigned long long *kv,
                               uint32_t mask, int32_t *err) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < m; p += nwarps) {
    const int32_t w = W[p];
    const int32_t c = colors[w];
    const int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    for (int32_t i = beg + lane; i < end; i += 32) {
      const unsigned long long key = pair_key(a_idx[i], c);
      uint32_t slot = pair_hash(key) & mask;
      for (uint32_t probe = 0;; probe++) {
        if (probe > mask) {  // full table: cannot happen at load <= 1/2
          atomicOr(err, ERR_INTERNAL);
          break;
        }
        unsigned long long k = __ldcg(kv + 2 * (size_t)slot);
        if (k == kEmptyKey) k = atomicCAS(kv + 2 * (size_t)slot, kEmptyKey, key);
        if (k == kEmptyKey || k == key) {
          atomicMin(reinterpret_cast<uint32_t *>(kv + 2 * (size_t)slot + 1), (uint32_t)p);
          break;
        }
        slot = (slot + 1) & mask;
      }
    }
  }
}

__global__ void k_pairs_lookup(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ a_idx,
                               const int32_t *__restrict__ W, int32_t m,
                               const int32_t *__restrict__ colors,
                               const unsigned long long *__restrict__ kv, uint32_t mask,
                               uint8_t *__restrict__ lose, int32_t *err) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < m; p += nwarps) {
    const int32_t w = W[p];
    const int32_t c = colors[w];
    const int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    bool l = false;
    for (int32_t i = beg + lane; i < end && !l; i += 32) {
      const unsigned long long key = pair_key(a_idx[i], c);
      uint32_t slot = pair_hash(key) & mask;
      for (uint32_t probe = 0;; probe++) {
        const unsigned long long k = kv[2 * (size_t)slot];
        if (k == key) {
          l = reinterpret_cast<const uint32_t *>(kv + 2 * (size_t)slot + 1)[0] < (uint32_t)p;
          break;
        }
        if (k == kEmptyKey || probe > mask) {  // every pair inserted its key
          atomicOr(err, ERR_INTERNAL);
          break;
        }
        slot = (slot + 1) & mask;
      }
    }
    if (__any_sync(kFull, l) && lane == 0) lose[p] = 1;
  }
}

// ----------------------------------------------------------- compaction
__global__ void __launch_bounds__(kScanNT) k_scan_count(const uint8_t *__restrict__ lose,
                                                        int32_t m, int32_t *__restrict__ blocksum) {
  __shared__ int32_t red[kScanNT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t c = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; q++) c += (base + q < m) ? lose[base + q] : 0;
  int32_t total;
  block_excl_scan<kScanNT>(c, red, &total);
  if (threadIdx.x == 0) blocksum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanNT) k_scan_blocks(int32_t *__restrict__ blocksum,
                                                         int32_t nblocks, DevScalars *dev) {
  __shared__ int32_t red[kScanNT / 32];
  int32_t carry = 0;
  for (int32_t b0 = 0; b0 < nblocks; b0 += kScanNT) {
    const int32_t b = b0 + (int32_t)threadIdx.x;
    const int32_t x = (b < nblocks) ? blocksum[b] : 0;
    int32_t total;
    const int32_t ex = block_excl_scan<kScanNT>(x, red, &total);
    if (b < nblocks) blocksum[b] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) dev->m_next = carry;
}

__global__ void __launch_bounds__(kScanNT) k_scan_scatter(const uint8_t *__restrict__ lose,
                                                          const int32_t *__restrict__ W,
                                                          int32_t m,
                                                          const int32_t *__restrict__ blocksum,
                                                          int32_t *__restrict__ newpos,
                                                          int32_t *__restrict__ Wn,
                                                          const int32_t *__restrict__ a_ptr,
                                                          DevScalars *dev) {
  __shared__ int32_t red[kScanNT / 32];
  __shared__ unsigned long long s_inc;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t f[kScanPer];
  int32_t c = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    f[q] = (base + q < m) ? lose[base + q] : 0;
    c += f[q];
  }
  if (threadIdx.x == 0) s_inc = 0ull;
  int32_t total;
  int32_t ex = block_excl_scan<kScanNT>(c, red, &total) + blocksum[blockIdx.x];
  unsigned long long inc = 0ull;  // incidences of the next round's W
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    if (f[q]) {
      const int32_t w = W[base + q];
      newpos[base + q] = ex;
      Wn[ex] = w;
      inc += (unsigned long long)(a_ptr[w + 1] - a_ptr[w]);
      ex++;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) inc += __shfl_xor_sync(kFull, inc, o);
  if ((threadIdx.x & 31) == 0 && inc) atomicAdd(&s_inc, inc);
  __syncthreads();
  if (threadIdx.x == 0 && s_inc) atomicAdd(&dev->incid_next, s_inc);
}

// Losers: uncolored again, and their nc / npos entries carry the new
// position; winners leave W (npos = -1).  Clears the lose flags.
__global__ void k_relabel(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ tpos,
                          const int32_t *__restrict__ W, int32_t m, uint8_t *__restrict__ lose,
                          const int32_t *__restrict__ newpos, int32_t *__restrict__ nc,
                          int32_t *__restrict__ npos, int32_t *__restrict__ colors) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < m; p += nwarps) {
    const int32_t w = W[p];
    const bool l = lose[p] != 0;
    const int32_t np = l ? newpos[p] : -1;
    const int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    // four CSR->CSC entries per lane and step, their loads issued together
    for (int32_t i0 = beg + lane; i0 < end; i0 += 128) {
      int32_t f[4];
#pragma unroll
      for (int q = 0; q < 4; q++) f[q] = i0 + 32 * q < end ? tpos[i0 + 32 * q] : -1;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (f[q] < 0) continue;
        npos[f[q]] = np;
        if (l) nc[f[q]] = -2 - np;
      }
    }
    __syncwarp();
    if (lane == 0) {
      if (l) colors[w] = -1;
      lose[p] = 0;
    }
  }
}

// The same relabelling in CSC order, for rounds whose W covers much of the
// graph: every mirror entry of a W member (npos >= 0) is rewritten in place
// (coalesced; lose and newpos are read at random but are n_a-sized), then
// k_relabel_tail resets the losers' colors and all lose flags.
__global__ void k_relabel_csc(int64_t nnz, uint8_t const *__restrict__ lose,
                              const int32_t *__restrict__ newpos, int32_t *__restrict__ nc,
                              int32_t *__restrict__ npos) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nnz;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = npos[f];
    if (p < 0) continue;
    if (lose[p]) {
      const int32_t np = newpos[p];
      npos[f] = np;
      nc[f] = -2 - np;
    } else {
      npos[f] = -1;
    }
  }
}

__global__ void k_relabel_tail(const int32_t *__restrict__ W, int32_t m,
                               uint8_t *__restrict__ lose, int32_t *__restrict__ colors) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (lose[p]) {
      colors[W[p]] = -1;
      lose[p] = 0;
    }
  }
}

__global__ void k_gmax(const int32_t *__restrict__ colors, int32_t n, DevScalars *dev) {
  int32_t mx = -1;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, colors[u]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if ((threadIdx.x & 31) == 0 && mx >= 0) atomicMax(&dev->gmax, mx);
}

__global__ void k_fill(int32_t *p, size_t n, int32_t v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

inline int warps_grid(long long items, int sms) {
  long long g = div_up(items * 32, kNT);
  // one resident set of CTAs (8 of 256 threads per SM): every warp's share
  // of the grid-stride loop starts at once, with no second set as a tail
  long long cap = (long long)sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int launch_kofs(const int32_t *b_ptr, const int32_t *, const int32_t *npos, const uint8_t *nown,
                 const int32_t *bigt, int32_t nbig, int32_t *kofs, int sms, cudaStream_t s) {
  if (nbig <= 0) return 0;
  int grid = nbig < sms * 8 ? nbig : sms * 8;
  k_kofs<<<grid, kNT, 0, s>>>(b_ptr, npos, nown, bigt, nbig, kofs);
  return 1;
}

int launch_trav(const int32_t *a_ptr, const int32_t *W, const int32_t *d2tot, int32_t m,
                int32_t small_ok, DevScalars *dev, cudaStream_t s) {
  if (m <= 0) return 0;
  int grid = div_up(m, kNT);
  if (grid > 1184) grid = 1184;
  k_trav<<<grid, kNT, 0, s>>>(a_ptr, W, d2tot, m, small_ok, dev);
  return 1;
}

int launch_detect(const int32_t *b_ptr, int32_t n_b, const int32_t *nc, const int32_t *npos,
                   const int32_t *bigd, int32_t nbigd, int32_t *dtab, int32_t tabcap,
                   int32_t nslots, int32_t id_order, uint8_t *lose, int sms, cudaStream_t s) {
  int n = 0;
  if (n_b > 0) {
    k_detect_warp<<<warps_grid(n_b, sms), kNT, 0, s>>>(b_ptr, n_b, nc, npos, id_order, lose);
    n++;
  }
  if (nbigd > 0 && id_order) {
    k_detect_mid<<<warps_grid(nbigd, sms), kNT, 0, s>>>(b_ptr, nc, npos, bigd, nbigd, lose);
    n++;
  }
  if (nbigd > 0) {
    int grid = nbigd < nslots ? nbigd : nslots;
    k_detect_table<<<grid, kNT, 0, s>>>(b_ptr, nc, npos, bigd, nbigd, id_order ? kMidMax : 0,
                                        dtab, tabcap, lose);
    n++;
  }
  return n;
}

int launch_detect_pairs(const int32_t *a_ptr, const int32_t *a_idx, const int32_t *W, int32_t m,
                        const int32_t *colors, unsigned long long *kv, uint32_t mask,
                        uint8_t *lose, int32_t *err, int sms, cudaStream_t s) {
  if (m <= 0) return 0;
  const size_t cap = (size_t)mask + 1;
  // slot i: the key at kv[2i], the smallest position in the low word of
  // kv[2i + 1] (both in one 32-byte sector); all ones = empty / no position
  cudaMemsetAsync(kv, 0xff, 2 * sizeof(unsigned long long) * cap, s);
  const int grid = warps_grid(m, sms);
  k_pairs_insert<<<grid, kNT, 0, s>>>(a_ptr, a_idx, W, m, colors, kv, mask, err);
  k_pairs_lookup<<<grid, kNT, 0, s>>>(a_ptr, a_idx, W, m, colors, kv, mask, lose, err);
  return 2;
}

int launch_compact(const uint8_t *lose, const int32_t *W, int32_t m, int32_t *newpos,
                    int32_t *Wn, int32_t *blocksum, const int32_t *a_ptr, DevScalars *dev,
                    cudaStream_t s) {
  const int nblocks = div_up(m, kScanTile);
  cudaMemsetAsync(&dev->incid_next, 0, sizeof(unsigned long long), s);
  if (m <= 0) {
    cudaMemsetAsync(&dev->m_next, 0, sizeof(int32_t), s);
    return 0;
  }
  k_scan_count<<<nblocks, kScanNT, 0, s>>>(lose, m, blocksum);
  k_scan_blocks<<<1, kScanNT, 0, s>>>(blocksum, nblocks, dev);
  k_scan_scatter<<<nblocks, kScanNT, 0, s>>>(lose, W, m, blocksum, newpos, Wn, a_ptr, dev);
  return 3;
}

int launch_relabel_csc(int64_t nnz, const int32_t *W, int32_t m, uint8_t *lose,
                       const int32_t *newpos, int32_t *nc, int32_t *npos, int32_t *colors,
                       int sms, cudaStream_t s) {
  if (m <= 0) return 0;
  const long long cap = (long long)sms * 8;
  long long g1 = div_up(nnz, kNT);
  if (g1 > cap) g1 = cap;
  if (g1 < 1) g1 = 1;
  k_relabel_csc<<<(int)g1, kNT, 0, s>>>(nnz, lose, newpos, nc, npos);
  long long g2 = div_up(m, kNT);
  if (g2 > cap) g2 = cap;
  k_relabel_tail<<<(int)g2, kNT, 0, s>>>(W, m, lose, colors);
  return 2;
}

int launch_relabel(const int32_t *a_ptr, const int32_t *tpos, const int32_t *W, int32_t m,
                    uint8_t *lose, const int32_t *newpos, int32_t *nc, int32_t *npos,
                    int32_t *colors, int sms, cudaStream_t s) {
  if (m <= 0) return 0;
  k_relabel<<<warps_grid(m, sms), kNT, 0, s>>>(a_ptr, tpos, W, m, lose, newpos, nc, npos, colors);
  return 1;
}

int launch_gmax(const int32_t *colors, int32_t n, DevScalars *dev, cudaStream_t s) {
  cudaMemsetAsync(&dev->gmax, 0xff, sizeof(int32_t), s);  // -1
  if (n <= 0) return 0;
  int grid = div_up(n, kNT);
  if (grid > 1184) grid = 1184;
  k_gmax<<<grid, kNT, 0, s>>>(colors, n, dev);
  return 1;
}

int launch_fill(int32_t *p, size_t n, int32_t v, cudaStream_t s) {
  if (n == 0) return 0;
  long long grid = div_up((long long)n, kNT);
  if (grid > 4096) grid = 4096;
  k_fill<<<(int)grid, kNT, 0, s>>>(p, n, v);
  return 1;
}

}  // namespace bgpc
