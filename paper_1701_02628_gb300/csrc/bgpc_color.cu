// Wave coloring kernel: the ColorWorkQueue phase (Alg. 2 / Alg. 4, with the
// reverse first fit of Alg. 8 for owners of big nets and the B1/B2 policies
// of Sec. V) for the chunks of one wave, and the publish step that makes the
// wave's colors visible to the next wave.
//
// One CTA colors one chunk of C <= 64 consecutive work-queue entries at a
// time (persistent grid, chunk-stride loop).  The chunk's vertices are
// colored one after the other, exactly like one thread of the paper's
// OpenMP loop with chunk C, but the memory traffic is not serialised:
//
//  * small vertices (sum of net sizes <= 448): phase A gathers the two-hop
//    colors of ALL small vertices of the chunk at once, flattened over
//    (vertex, net, member) triples so every thread streams contiguous net
//    ranges of the net-major mirror nc[], into a 512-bit forbidden window per
//    vertex in shared memory; phase B (one warp) then resolves the vertices
//    in order with ballot/ffs searches, adding the colors of earlier chunk
//    mates that are neighbours (64-bit adjacency mask) before each search.
//  * large vertices: the whole CTA gathers that vertex's two-hop colors into
//    a byte map over the wave's color range (one byte per color, plain
//    stores, no atomics) and searches it with block-wide reductions.
//
// Colors are never read through c[]: nc[f] already holds, for every CSC entry
// f, the member's published color, or -2 - pos for a member that is still in
// the work queue at position pos (which identifies chunk mates and w itself).
#include "bgpc_internal.cuh"

namespace bgpc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWords = kSmallWindow / 32;  // 16

__device__ __forceinline__ int32_t warp_incl_scan(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <int NT>
__device__ __forceinline__ int32_t block_min(int32_t v, int32_t *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int32_t r = red[0];
#pragma unroll
  for (int i = 1; i < NT / 32; i++) r = min(r, red[i]);
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ int32_t block_max(int32_t v, int32_t *red) {
  return -block_min<NT>(-v, red);
}

// Exclusive scan over the threads of the block (thread order); *total gets
// the sum.  Contains two __syncthreads.
template <int NT>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *red, int32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = warp_incl_scan(v);
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

// ------------------------------------------- bitmap searches (CTA, smem)
// bm[x >> 5] bit (x & 31) set means color x is forbidden; `words` is a multiple
// of 4 and every color >= 32 * words is free.  Thread t of a tile covers the
// 128 colors of one uint4.

__device__ __forceinline__ uint32_t mask_from(int32_t lo, int32_t p) {
  // bits of the word starting at color lo that are >= p
  if (p <= lo) return 0xffffffffu;
  if (p >= lo + 32) return 0u;
  return 0xffffffffu << (p - lo);
}

__device__ __forceinline__ uint32_t mask_upto(int32_t lo, int32_t p) {
  // bits of the word starting at color lo that are <= p
  if (p >= lo + 31) return 0xffffffffu;
  if (p < lo) return 0u;
  return 0xffffffffu >> (31 - (p - lo));
}

// Smallest free x >= p, or 32 * words if every color up to there is taken.
template <int NT>
__device__ int32_t bm_first_free_up(const uint32_t *bm, int32_t words, int32_t p, int32_t *red) {
  const int32_t lim = words * 32;
  for (int32_t base = (p >> 7) << 7; base < lim; base += NT * 128) {
    const int32_t x0 = base + (int32_t)threadIdx.x * 128;
    int32_t found = INT32_MAX;
    if (x0 < lim) {
      const uint4 v = *reinterpret_cast<const uint4 *>(bm + (x0 >> 5));
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const uint32_t fr = ~wv[q] & mask_from(x0 + 32 * q, p);
        if (fr && found == INT32_MAX) found = x0 + 32 * q + __ffs(fr) - 1;
      }
    }
    found = block_min<NT>(found, red);
    if (found != INT32_MAX) return found;
  }
  return lim;
}

// Largest free x with 0 <= x <= p, or -1.
template <int NT>
__device__ int32_t bm_last_free_down(const uint32_t *bm, int32_t p, int32_t *red) {
  for (int32_t top = ((p >> 7) << 7) + 127; top >= 0; top -= NT * 128) {
    const int32_t x0 = top - 127 - (int32_t)threadIdx.x * 128;  // multiple of 128
    int32_t found = -1;
    if (x0 >= 0 && x0 <= p) {
      const uint4 v = *reinterpret_cast<const uint4 *>(bm + (x0 >> 5));
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 3; q >= 0; q--) {
        const uint32_t fr = ~wv[q] & mask_upto(x0 + 32 * q, p);
        if (fr && found < 0) found = x0 + 32 * q + 31 - __clz(fr);
      }
    }
    found = block_max<NT>(found, red);
    if (found >= 0) return found;
  }
  return -1;
}

// The k-th (0-based) free color counting down from top, or -1.
template <int NT>
__device__ int32_t bm_kth_free_down(const uint32_t *bm, int32_t top, int32_t k, int32_t *red) {
  int32_t remaining = k;
  for (int32_t t0 = ((top >> 7) << 7) + 127; t0 >= 0; t0 -= NT * 128) {
    const int32_t x0 = t0 - 127 - (int32_t)threadIdx.x * 128;
    uint32_t fr[4] = {0u, 0u, 0u, 0u};
    int32_t cnt = 0;
    if (x0 >= 0 && x0 <= top) {
      const uint4 v = *reinterpret_cast<const uint4 *>(bm + (x0 >> 5));
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        fr[q] = ~wv[q] & mask_upto(x0 + 32 * q, top);
        cnt += __popc(fr[q]);
      }
    }
    int32_t total;
    const int32_t excl = block_excl_scan<NT>(cnt, red, &total);
    if (remaining < total) {
      int32_t res = -1;
      if (cnt > 0 && excl <= remaining && remaining < excl + cnt) {
        int32_t r = remaining - excl;
        for (int q = 3; q >= 0 && res < 0; q--) {
          uint32_t f = fr[q];
          const int32_t c = __popc(f);
          if (r >= c) { r -= c; continue; }
          while (true) {
            const int32_t b = 31 - __clz(f);
            if (r == 0) { res = x0 + 32 * q + b; break; }
            f &= ~(1u << b);
            r--;
          }
        }
      }
      return block_max<NT>(res, red);
    }
    remaining -= total;
  }
  return -1;
}

// ---------------------------------------------- 512-bit window searches (warp)
// `word` is lane l's 32 bits of the window (l < 16); set bits are forbidden.

__device__ __forceinline__ int32_t win_first_free_up(uint32_t word, int32_t p) {
  const int lane = threadIdx.x & 31;
  if (p >= kSmallWindow) return -1;
  const int wl = p >> 5;
  if (lane >= kWords || lane < wl) word = kFull;
  else if (lane == wl) word |= (1u << (p & 31)) - 1u;
  uint32_t fr = ~word;
  unsigned b = __ballot_sync(kFull, fr != 0);
  if (!b) return -1;
  int fl = __ffs(b) - 1;
  uint32_t fw = __shfl_sync(kFull, fr, fl);
  return fl * 32 + __ffs(fw) - 1;
}

__device__ __forceinline__ int32_t win_last_free_down(uint32_t word, int32_t p) {
  const int lane = threadIdx.x & 31;
  if (p < 0) return -1;
  const int wl = p >> 5;
  if (lane >= kWords || lane > wl) word = kFull;
  else if (lane == wl) word |= ~((2u << (p & 31)) - 1u);
  uint32_t fr = ~word;
  unsigned b = __ballot_sync(kFull, fr != 0);
  if (!b) return -1;
  int fl = 31 - __clz(b);
  uint32_t fw = __shfl_sync(kFull, fr, fl);
  return fl * 32 + 31 - __clz(fw);
}

__device__ __forceinline__ int32_t win_kth_free_down(uint32_t word, int32_t top, int32_t k) {
  const int lane = threadIdx.x & 31;
  if (top < 0) return -1;
  const int wl = top >> 5;
  if (lane >= kWords || lane > wl) word = kFull;
  else if (lane == wl) word |= ~((2u << (top & 31)) - 1u);
  uint32_t fr = ~word;
  int32_t cnt = __popc(fr);
  int32_t suf = cnt;  // free colors in lanes >= this lane
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_down_sync(kFull, suf, o);
    if (lane + o < 32) suf += y;
  }
  int32_t above = suf - cnt;
  bool mine = (above <= k) && (k < above + cnt);
  unsigned b = __ballot_sync(kFull, mine);
  if (!b) return -1;
  int32_t res = -1;
  if (mine) {
    int32_t r = k - above;
    uint32_t f = fr;
    while (true) {
      int32_t x = 31 - __clz(f);
      if (r == 0) { res = lane * 32 + x; break; }
      f &= ~(1u << x);
      r--;
    }
  }
  return __shfl_sync(kFull, res, __ffs(b) - 1);
}

// ------------------------------------------- candidate summaries (warp)
// A large vertex's forbidden set F_S (colors of its two-hop neighbours in the
// wave snapshot) is a bitmap g of `words` words; colors beyond 32 * words are
// free.  Its chunk adds at most 63 more colors (the overlay O), so first fit
// needs only the kSumCand smallest free colors of F_S, and the reverse first
// fit needs the free colors of F_S from the k-th below the top on (plus, for
// overlay colors above that window, one bit of g each).  The gather computes
// these summaries from the bitmap in shared memory; the resolve keeps one
// list per vertex (the reverse window when it has one) in shared memory.

// The N smallest colors not in g, ascending, into out[].  g holds `words`
// words (16-byte aligned, words a multiple of 4; colors beyond are free);
// each lane takes four words per step.
template <int N>
__device__ __forceinline__ void take_up(uint32_t fr, int32_t base, int32_t &r, int32_t *out) {
  while (fr && r < N) {
    out[r++] = base + __ffs(fr) - 1;
    fr &= fr - 1u;
  }
}

// Resumable: scans the 16-byte groups from q0 on while fewer than N colors
// are found and q0 < qend (groups at or beyond qend are not read: a caller
// may not have finished them); groups at or beyond W4 are all free.
template <int N>
__device__ __forceinline__ void warp_first_free_from(const uint32_t *g, int32_t W4, int32_t qend,
                                                     int32_t *out, int32_t &got, int32_t &q0) {
  const int lane = threadIdx.x & 31;
  const uint4 *g4 = reinterpret_cast<const uint4 *>(g);
  while (got < N && q0 < qend) {
    const int32_t q = q0 + lane;
    uint4 f = make_uint4(0u, 0u, 0u, 0u);
    if (q < qend) {
      f = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
      if (q < W4) {
        const uint4 b = g4[q];
        f = make_uint4(~b.x, ~b.y, ~b.z, ~b.w);
      }
    }
    const int32_t cnt = __popc(f.x) + __popc(f.y) + __popc(f.z) + __popc(f.w);
    const int32_t inc = warp_incl_scan(cnt);
    int32_t r = got + inc - cnt;
    if (r < N) {
      take_up<N>(f.x, 128 * q, r, out);
      take_up<N>(f.y, 128 * q + 32, r, out);
      take_up<N>(f.z, 128 * q + 64, r, out);
      take_up<N>(f.w, 128 * q + 96, r, out);
    }
    got += __shfl_sync(kFull, inc, 31);
    q0 = (qend - q0 > 32) ? q0 + 32 : qend;
  }
  __syncwarp();
}

template <int N>
__device__ __forceinline__ void warp_first_free(const uint32_t *g, int32_t words, int32_t *out) {
  int32_t got = 0, q0 = 0;
  warp_first_free_from<N>(g, words >> 2, INT32_MAX, out, got, q0);
}

template <int N>
__device__ __forceinline__ void take_down(uint32_t fr, int32_t base, int32_t k, int32_t &r,
                                          int32_t *out) {
  const int32_t c = __popc(fr);
  if (r + c <= k) {  // the whole word lies before the k-th
    r += c;
    return;
  }
  while (fr && r < k + N) {
    const int32_t b = 31 - __clz(fr);
    if (r >= k) out[r - k] = base + b;
    r++;
    fr &= ~(1u << b);
  }
}

template <int N>
__device__ __forceinline__ int32_t warp_kth_free_down(const uint32_t *g, int32_t top, int32_t k,
                                                      int32_t *out) {
  const int lane = threadIdx.x & 31;
  const uint4 *g4 = reinterpret_cast<const uint4 *>(g);
  int32_t seen = 0;
  for (int32_t q0 = top >> 7; q0 >= 0 && seen < k + N; q0 -= 32) {
    const int32_t q = q0 - lane;
    uint4 f = make_uint4(0u, 0u, 0u, 0u);
    if (q >= 0) {
      const uint4 b = g4[q];
      f = make_uint4(~b.x & mask_upto(128 * q, top), ~b.y & mask_upto(128 * q + 32, top),
                     ~b.z & mask_upto(128 * q + 64, top), ~b.w & mask_upto(128 * q + 96, top));
    }
    const int32_t cnt = __popc(f.x) + __popc(f.y) + __popc(f.z) + __popc(f.w);
    const int32_t inc = warp_incl_scan(cnt);
    int32_t r = seen + inc - cnt;  // rank of this lane's highest free color
    if (r + cnt > k && r < k + N) {
      take_down<N>(f.w, 128 * q + 96, k, r, out);
      take_down<N>(f.z, 128 * q + 64, k, r, out);
      take_down<N>(f.y, 128 * q + 32, k, r, out);
      take_down<N>(f.x, 128 * q, k, r, out);
    }
    seen += __shfl_sync(kFull, inc, 31);
  }
  __syncwarp();
  const int32_t have = seen - k;
  return have <= 0 ? 0 : (have < N ? have : N);
}

// One warp: the first-fit summary of a large vertex from its forbidden
// bitmap bm (`words` words, read only) into rec[kSumInts]; the owner of a net
// larger than T (so > T) with a k-th free color and an earlier neighbour in
// its chunk also leaves the bitmap words up to color so - 1 in lb, for the
// resolve's tests of overlay colors.
// The summary's reverse first-fit part, count and mask (its first-fit list
// already in rec[0, kSumCand)).
__device__ __forceinline__ void warp_summarize_rest(const uint32_t *bm, int32_t so, int32_t T,
                                                    int32_t k, unsigned long long adj,
                                                    int32_t *rec, uint32_t *lb) {
  const int lane = threadIdx.x & 31;
  int32_t rc = 0;
  if (so > T) rc = warp_kth_free_down<kSumCand>(bm, so - 1, k, rec + kSumCand);
  if (lane == 0) {
    rec[2 * kSumCand] = rc;
    *reinterpret_cast<unsigned long long *>(rec + 2 * kSumCand + 2) = adj;
  }
  if (rc > 0 && adj != 0ull) {
    // the resolve tests overlay colors in (ak, so - 1] only, ak = the k-th
    // (and only for a vertex with an earlier neighbour in its chunk: the
    // others are colored from the summary alone)
    const int32_t ak = rec[kSumCand];
    const uint4 *b4 = reinterpret_cast<const uint4 *>(bm);
    uint4 *l4 = reinterpret_cast<uint4 *>(lb);
    for (int32_t x = (ak >> 7) + lane; x <= ((so - 1) >> 7); x += 32) l4[x] = b4[x];
  }
  __syncwarp();
}

__device__ __forceinline__ void warp_summarize(const uint32_t *bm, int32_t words, int32_t so,
                                               int32_t T, int32_t k, unsigned long long adj,
                                               int32_t *rec, uint32_t *lb) {
  warp_first_free<kSumCand>(bm, words, rec);
  warp_summarize_rest(bm, so, T, k, adj, rec, lb);
}

__device__ __forceinline__ unsigned long long low_mask64(int32_t n) {
  return n >= 64 ? ~0ull : ((1ull << n) - 1ull);
}

// --------------------------------------------------------- resolve kernel

// Whether vertex (d2, deg) takes the fused small path (must agree with the
// piece count of k_piece_count).
__device__ __forceinline__ bool is_small(int32_t d2, int32_t deg, bool small_ok) {
  return small_ok && d2 <= kSmallD2 && deg <= kSmallMaxDeg;
}

// A 4-byte asynchronous copy global -> shared (both 4-byte aligned), and the
// per-thread group commit / wait around it.
__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A chunk whose earlier vertices spread over more ids than this tests its
// hub chunk-mates pair by pair instead of reading the hubs' member windows.
constexpr int32_t kHubScanSpan = 2048;

// Position of the set bit of v with n set bits below it (v has more than n;
// 0 when it has not).
__device__ __forceinline__ int32_t nth_set_bit32(uint32_t v, int32_t n) {
  int32_t pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const int32_t c = __popc(v & ((1u << w) - 1u));
    if (n >= c) {
      n -= c;
      v >>= w;
      pos += w;
    }
  }
  return pos & 31;
}

// Position of the set bit of v with n set bits below it (v has more than n).
__device__ __forceinline__ int32_t nth_set_bit64(unsigned long long v, int32_t n) {
  int32_t pos = 0;
#pragma unroll
  for (int w = 32; w > 0; w >>= 1) {
    const int32_t c = __popcll(v & ((1ull << w) - 1ull));
    if (n >= c) {
      n -= c;
      v >>= w;
      pos += w;
    }
  }
  return pos;
}

// The entries of the ascending list l[0, cnt) equal to one of the warp's keys
// (two per lane; INT32_MIN: none), as a mask in every lane.  Both searches of
// a lane run side by side.
__device__ __forceinline__ unsigned long long list_marks(const int32_t *l, int32_t cnt,
                                                         int32_t k0, int32_t k1) {
  int32_t p0 = 0, p1 = 0;
#pragma unroll
  for (int w = 32; w > 0; w >>= 1) {
    const bool g0 = p0 + w - 1 < cnt && l[p0 + w - 1] < k0;
    const bool g1 = p1 + w - 1 < cnt && l[p1 + w - 1] < k1;
    if (g0) p0 += w;
    if (g1) p1 += w;
  }
  unsigned long long m = 0ull;
  if (k0 != INT32_MIN && p0 < cnt && l[p0] == k0) m |= 1ull << p0;
  if (k1 != INT32_MIN && p1 < cnt && l[p1] == k1) m |= 1ull << p1;
  const unsigned lo = __reduce_or_sync(kFull, (unsigned)m);
  const unsigned hi = __reduce_or_sync(kFull, (unsigned)(m >> 32));
  return ((unsigned long long)hi << 32) | lo;
}

// The same mask through a scratch bitmap over the list's span (l[cnt - 1] -
// l[0] < kPullBits, else by search): each lane sets the bits of its keys,
// then tests the bits of its two entries.  The scratch is zero before and after.
constexpr int kPullBits = 4096;
__device__ __forceinline__ unsigned long long pull_marks(const int32_t *l, int32_t cnt,
                                                         int32_t k0, int32_t k1,
                                                         uint32_t *scr) {
  const int lane = threadIdx.x & 31;
  const int32_t b = l[0], span = l[cnt - 1] - b;
  if (span >= kPullBits) return list_marks(l, cnt, k0, k1);
  const int32_t e0 = lane < cnt ? l[lane] - b : -1;
  const int32_t e1 = lane + 32 < cnt ? l[lane + 32] - b : -1;
  // keys outside [b, b + span] take no entry (INT32_MIN: out of range)
  const int32_t o0 = (k0 != INT32_MIN && k0 >= b && k0 - b <= span) ? k0 - b : -1;
  const int32_t o1 = (k1 != INT32_MIN && k1 >= b && k1 - b <= span) ? k1 - b : -1;
  if (o0 >= 0) atomicOr(&scr[o0 >> 5], 1u << (o0 & 31));
  if (o1 >= 0) atomicOr(&scr[o1 >> 5], 1u << (o1 & 31));
  __syncwarp();
  const bool t0 = e0 >= 0 && ((scr[e0 >> 5] >> (e0 & 31)) & 1u);
  const bool t1 = e1 >= 0 && ((scr[e1 >> 5] >> (e1 & 31)) & 1u);
  const unsigned long long tk =
      ((unsigned long long)__ballot_sync(kFull, t1) << 32) | __ballot_sync(kFull, t0);
  if (o0 >= 0) scr[o0 >> 5] = 0u;
  if (o1 >= 0) scr[o1 >> 5] = 0u;
  __syncwarp();
  return tk;
}

// First fit, phase B: one warp colors the chunk's vertices that have earlier
// neighbours in the chunk, in order (a vertex's color depends on its earlier
// neighbours' final colors, and on later rounds the chunks are nearly
// complete chains).  Each large vertex has one ascending candidate list in
// shared memory: its 64 smallest free colors, or its reverse first-fit window
// negated.  Lane v % 32 keeps vertex v's color (col, once decided: dec) in a
// register (slot v / 32).  At its step a vertex looks its neighbours' colors
// up in its list (one search per neighbour, all in parallel): x = the first
// entry none takes (first fit), or the (e+1)-th, where e counts the distinct
// neighbour colors in (ak, so - 1] that are free in its forbidden set F_S
// (reverse first fit: each shifts the k-th free color one further down).
// Those F_S bits (fm, in shared memory) are pushed when a neighbour's color
// is decided: the bitmap word is copied then (cp.async, into a landing slot
// of the vertex, one per step parity) and folded in two walked steps later,
// so a copy is waited for only by the vertex right after the one that
// pushed it.  dup holds each vertex's earlier vertices of the same color (an
// overlay is a set).
__device__ __forceinline__ void ff_walk(const WaveArgs &a, int32_t n, int64_t slot0,
                                        unsigned long long large,
                                        const unsigned long long *s_adj, int32_t *s_col,
                                        uint32_t (*s_bm)[kWords], const int32_t *s_sown,
                                        const int32_t *s_k, const int32_t (*s_list)[kSumCand],
                                        const int32_t *s_rcnt, unsigned long long *s_dup,
                                        unsigned long long *s_fm, int32_t *cx, uint32_t *wscr,
                                        uint32_t *pscr, uint32_t *land) {
  const int lane = threadIdx.x & 31;
  unsigned long long adj[2];
  int32_t col[2], lo[2], hi[2];
  bool dec[2];
  // pending fm pushes per step parity: bit (color & 31) | pushing vertex << 5,
  // or -1; the word lands in land[parity][vertex]
  int32_t pb[2][2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int32_t v = lane + 32 * h;
    const bool valid = v < n;
    const bool rff = valid && ((large >> v) & 1ull) && s_rcnt[v] > 0;
    adj[h] = valid ? s_adj[v] : 0ull;
    dec[h] = valid && adj[h] == 0ull;  // colored by step P
    col[h] = dec[h] ? s_col[v] : -1;
    lo[h] = rff ? -s_list[v][0] : INT32_MAX;  // fm tests colors in (lo, hi]
    hi[h] = rff ? s_sown[v] - 1 : INT32_MIN;
    if (valid) s_dup[v] = s_fm[v] = 0ull;
    pb[0][h] = pb[1][h] = -1;
  }
  const unsigned long long decided0 =
      ((unsigned long long)__ballot_sync(kFull, dec[1]) << 32) | __ballot_sync(kFull, dec[0]);
  if (decided0 == low_mask64(n)) return;
  // dup and fm serve only the reverse first fit of undecided vertices
  const bool rff_left = __any_sync(kFull, (!dec[0] && lo[0] < hi[0]) || (!dec[1] && lo[1] < hi[1]));
  const unsigned below = (1u << lane) - 1u;
  // dup among the vertices colored by step P (undecided ones get unique keys)
  if (rff_left) {
    const int32_t k0 = dec[0] ? col[0] : -1 - lane, k1 = dec[1] ? col[1] : -1 - lane;
    const unsigned m0 = __match_any_sync(kFull, k0), m1 = __match_any_sync(kFull, k1);
    unsigned cross = 0u;  // first-half lanes with this lane's second color
    for (int t = 0; t < 32; t++) {
      const int32_t c = __shfl_sync(kFull, k0, t);
      if (dec[1] && c == k1) cross |= 1u << t;
    }
    if (dec[0]) s_dup[lane] = m0 & below;
    if (dec[1]) s_dup[lane + 32] = ((unsigned long long)(m1 & below) << 32) | cross;
  }
  // fm pushes of the colors decided by step P into the undecided reverse
  // first-fit vertices, four loads in flight
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int32_t v = lane + 32 * h;
    unsigned long long todo = (!dec[h] && lo[h] < hi[h]) ? (adj[h] & decided0) : 0ull;
    const uint32_t *lb = a.lbm + (slot0 + v) * a.words;
    unsigned long long fm = 0ull;
    while (todo) {
      int32_t j[4], c[4];
      uint32_t wd[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        j[q] = todo ? __ffsll((long long)todo) - 1 : -1;
        todo &= todo - 1ull;
        c[q] = j[q] >= 0 ? s_col[j[q]] : -1;
        const bool in = j[q] >= 0 && c[q] > lo[h] && c[q] <= hi[h];
        wd[q] = in ? lb[c[q] >> 5] : 0u;
        if (!in) j[q] = -1;
      }
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (j[q] >= 0 && ((wd[q] >> (c[q] & 31)) & 1u) == 0u) fm |= 1ull << j[q];
    }
    if (fm) s_fm[v] = fm;
  }
  __syncwarp();
  int32_t par = 0;  // parity of the walked step
  for (int32_t i = 0; i < n; i++) {
    if ((decided0 >> i) & 1ull) continue;
    // fold the fm pushes of two walked steps ago (their copies are done once
    // at most the last step's group is pending)
    if (rff_left) {
      cp_async_wait<1>();
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int32_t b = par ? pb[1][h] : pb[0][h];
        if (b >= 0 && ((land[par * kMaxChunk + lane + 32 * h] >> (b & 31)) & 1u) == 0u)
          s_fm[lane + 32 * h] |= 1ull << (b >> 5);
        if (par) pb[1][h] = -1; else pb[0][h] = -1;
      }
      __syncwarp();
    }
    const int32_t li = i & 31, hv = i >> 5;
    const unsigned long long am = s_adj[i];
    bool in_o[2];
#pragma unroll
    for (int h = 0; h < 2; h++) in_o[h] = lane + 32 * h < i && ((am >> (lane + 32 * h)) & 1ull);
    int32_t x = -1;
    if (!((large >> i) & 1ull)) {
      // small vertex: its window bitmap with the overlay ORed in (a copy)
      const int32_t so = s_sown[i];
      if (lane < kWords) wscr[lane] = s_bm[i][lane];
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; h++)
        if (in_o[h] && col[h] < kSmallWindow) atomicOr(&wscr[col[h] >> 5], 1u << (col[h] & 31));
      __syncwarp();
      const uint32_t word = (lane < kWords) ? wscr[lane] : kFull;
      if (so > a.T) x = win_kth_free_down(word, so - 1, s_k[i]);
      if (x < 0) x = win_first_free_up(word, 0);
      if (x < 0) {  // cannot happen within the window bounds
        if (lane == 0) atomicOr(a.err, ERR_INTERNAL);
        x = 0;
      }
      __syncwarp();
    } else {
      const int32_t rc = s_rcnt[i];
      const int32_t *l = s_list[i];
      if (rc == 0) {
        // first fit: at most 63 neighbours take at most 63 of the 64 entries
        const unsigned long long tk = pull_marks(l, kSumCand, in_o[0] ? col[0] : INT32_MIN,
                                                 in_o[1] ? col[1] : INT32_MIN, pscr);
        x = l[__ffsll((long long)~tk) - 1];
      } else {
        // reverse first fit: the window entries (colors <= ak, negated) that
        // no neighbour takes, after skipping e of them
        const int32_t ak = -l[0];
        const unsigned long long tk =
            pull_marks(l, rc, (in_o[0] && col[0] <= ak) ? -col[0] : INT32_MIN,
                       (in_o[1] && col[1] <= ak) ? -col[1] : INT32_MIN, pscr);
        unsigned long long fmi = s_fm[i];
        {  // the last walked step's push to i (its copy may be in flight)
          int32_t pj = -1;
          const int32_t b = par ? pb[0][hv] : pb[1][hv];
          if (lane == li && b >= 0) {
            cp_async_wait<0>();
            if (((land[(par ^ 1) * kMaxChunk + i] >> (b & 31)) & 1u) == 0u) pj = b >> 5;
          }
          pj = __shfl_sync(kFull, pj, li);
          if (pj >= 0) fmi |= 1ull << pj;
        }
        bool first[2];
#pragma unroll
        for (int h = 0; h < 2; h++)
          first[h] = in_o[h] && ((fmi >> (lane + 32 * h)) & 1ull) &&
                     (s_dup[lane + 32 * h] & am) == 0ull;
        const int32_t e = __popc(__ballot_sync(kFull, first[0])) +
                          __popc(__ballot_sync(kFull, first[1]));
        const unsigned long long av = ~tk & low_mask64(rc);
        if (__popcll(av) > e) {
          x = -l[nth_set_bit64(av, e)];
        } else if (rc == kSumCand) {
          // e + (taken entries) <= |O| <= 63 < 64 entries
          if (lane == 0) atomicOr(a.err, ERR_INTERNAL);
          x = 0;
        } else {
          // no k-th free color: first fit over the 64 smallest free colors
          const int32_t *rec = a.gsum + (slot0 + i) * kSumInts;
          cx[lane] = rec[lane];
          cx[lane + 32] = rec[32 + lane];
          __syncwarp();
          const unsigned long long tf = pull_marks(cx, kSumCand, in_o[0] ? col[0] : INT32_MIN,
                                                   in_o[1] ? col[1] : INT32_MIN, pscr);
          x = cx[__ffsll((long long)~tf) - 1];
          __syncwarp();
        }
      }
    }
    // ---- i is decided: its duplicates, the later duplicates it leads, and
    // the fm pushes of its color to the later vertices that test it
    if (!rff_left) {
      if (lane == li) {
        col[hv] = x;
        dec[hv] = true;
      }
      if (lane == 0) s_col[i] = x;
      __syncwarp();
      continue;
    }
    const unsigned long long dmask =
        ((unsigned long long)__ballot_sync(kFull, dec[1] && lane + 32 < i && col[1] == x) << 32) |
        __ballot_sync(kFull, dec[0] && lane < i && col[0] == x);
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int32_t v = lane + 32 * h;
      if (v == i) {
        col[h] = x;
        dec[h] = true;
        s_dup[v] = dmask;
      } else if (v > i && v < n) {
        if (dec[h] && col[h] == x) s_dup[v] |= 1ull << i;
        if (!dec[h] && ((adj[h] >> i) & 1ull) && x > lo[h] && x <= hi[h]) {
          cp_async4(&land[par * kMaxChunk + v], a.lbm + (slot0 + v) * a.words + (x >> 5));
          if (par) pb[1][h] = (x & 31) | (i << 5); else pb[0][h] = (x & 31) | (i << 5);
        }
      }
    }
    cp_async_commit();
    par ^= 1;
    if (lane == 0) s_col[i] = x;
    __syncwarp();
  }
  cp_async_wait<0>();  // no copy into the landing slots outlives the chunk
  __syncwarp();
}

template <int POLICY, int NT>
__global__ void __launch_bounds__(NT) k_color_wave(WaveArgs a) {
  constexpr int NW = NT / 32;
  __shared__ int32_t s_w[kMaxChunk], s_ab[kMaxChunk], s_deg[kMaxChunk], s_d2[kMaxChunk];
  __shared__ int32_t s_sown[kMaxChunk], s_k[kMaxChunk], s_col[kMaxChunk];
  __shared__ int32_t s_ppi[kMaxChunk];   // inclusive prefix of small-vertex degrees
  __shared__ int32_t s_next[kMaxChunk];  // next large vertex at or after i
  __shared__ unsigned long long s_adj[kMaxChunk];
  __shared__ uint32_t s_bm[kMaxChunk][kWords];
  __shared__ int32_t s_pstart[kPairCap];
  __shared__ int32_t s_poff[kPairCap + 1];
  __shared__ uint8_t s_pvert[kPairCap];
  __shared__ int32_t s_red[NW + 1];
  __shared__ int32_t s_state[4];  // col_max, col_next, npairs, stop
  constexpr int KC = (POLICY == BGPC_FF) ? kMaxChunk : 1;
  // first fit: each large vertex's candidate list (ascending; a reverse
  // first-fit window is stored negated) and its window length (0: none)
  __shared__ int32_t s_list[KC][kSumCand];
  __shared__ int32_t s_rcnt[KC];
  __shared__ unsigned long long s_dup[KC], s_fm[KC];  // the walk's masks
  __shared__ uint32_t s_land[2 * KC];                 // the walk's landing slots
  __shared__ uint32_t s_pull[(POLICY == BGPC_FF) ? kPullBits / 32 : 1];  // the walk's scratch
  __shared__ int32_t s_cx[(POLICY == BGPC_FF) ? kSumCand : 1];  // a whole summary list
  __shared__ uint32_t s_wscr[(POLICY == BGPC_FF) ? kWords : 1];   // a window with its overlay
  __shared__ unsigned long long s_large;
  extern __shared__ __align__(16) uint32_t s_big[];  // a.words: one large vertex's F

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t gm = a.dev->gmax;
  const int32_t bound = max(max(gm, a.maxnet - 1), 0) + a.C;  // every color of this wave <= bound
  if (bound >= a.words * 32) {
    if (tid == 0 && blockIdx.x == 0) atomicOr(a.err, ERR_COLOR);
    return;
  }
  const bool small_ok = a.small_ok != 0;
  if constexpr (POLICY == BGPC_FF)
    for (int x = tid; x < kPullBits / 32; x += NT) s_pull[x] = 0u;  // kept zero by the walk
  const int32_t col_max0 = max(gm, 0);

  for (int32_t t = (int32_t)blockIdx.x; t < a.nchunks; t += (int32_t)gridDim.x) {
    const int32_t j = a.chunks[t];
    const int32_t p0 = j * a.C;
    const int32_t n = min(a.C, a.m - p0);
    const int64_t slot0 = (int64_t)t * a.C;  // wave-order slot of the chunk's first vertex

    // ---- step 0: per-vertex data
    if (tid < n) {
      int32_t w = a.W[p0 + tid];
      int32_t ab = a.a_ptr[w], ae = a.a_ptr[w + 1];
      int32_t so = a.s_own[w];
      s_w[tid] = w;
      s_ab[tid] = ab;
      s_deg[tid] = ae - ab;
      s_d2[tid] = a.d2tot[w];
      s_sown[tid] = so;
      s_k[tid] = (so > a.T) ? a.kofs[p0 + tid] : 0;
      s_adj[tid] = 0ull;
    }
    for (int x = tid; x < kMaxChunk * kWords; x += NT) (&s_bm[0][0])[x] = 0u;
    if (tid == 0) { s_state[0] = col_max0; s_state[1] = 0; }
    __syncthreads();

    // ---- step 1: small vertices and their (vertex, net) pair offsets
    if (warp == 0) {
      const int i0 = lane, i1 = lane + 32;
      const bool sm0 = i0 < n && is_small(s_d2[i0], s_deg[i0], small_ok);
      const bool sm1 = i1 < n && is_small(s_d2[i1], s_deg[i1], small_ok);
      const int32_t d0 = sm0 ? s_deg[i0] : 0, d1 = sm1 ? s_deg[i1] : 0;
      const int32_t inc0 = warp_incl_scan(d0);
      const int32_t tot0 = __shfl_sync(kFull, inc0, 31);
      const int32_t inc1 = warp_incl_scan(d1) + tot0;
      s_ppi[i0] = inc0;
      s_ppi[i1] = inc1;
      const unsigned lg0 = __ballot_sync(kFull, i0 < n && !sm0);
      const unsigned lg1 = __ballot_sync(kFull, i1 < n && !sm1);
      const unsigned long long large = ((unsigned long long)lg1 << 32) | lg0;
      if (lane == 0) s_large = large;
      const unsigned long long m0 = large >> i0;
      s_next[i0] = m0 ? min(i0 + __ffsll((long long)m0) - 1, n) : n;
      const unsigned long long m1 = large >> i1;
      s_next[i1] = m1 ? min(i1 + __ffsll((long long)m1) - 1, n) : n;
      if (lane == 31) s_state[2] = inc1;
    }
    __syncthreads();

    // ---- step 2: (vertex, net) pairs of the small vertices
    const int32_t P = s_state[2];
    for (int32_t pt = tid; pt < P; pt += NT) {
      int32_t lo = 0, hi = n - 1;  // smallest i with s_ppi[i] > pt
      while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (s_ppi[mid] > pt) hi = mid; else lo = mid + 1;
      }
      const int32_t i = lo;
      const int32_t width = (i == 0) ? s_ppi[0] : s_ppi[i] - s_ppi[i - 1];
      const int32_t tl = pt - (s_ppi[i] - width);
      const int32_t v = a.a_idx[s_ab[i] + tl];
      const int32_t bp = a.b_ptr[v];
      s_pstart[pt] = bp;
      s_poff[pt] = a.b_ptr[v + 1] - bp;
      s_pvert[pt] = (uint8_t)i;
    }
    __syncthreads();

    // ---- step 3: exclusive scan of the pair sizes
    {
      constexpr int PER = (kPairCap + NT - 1) / NT;
      int32_t loc[PER];
      int32_t sum = 0;
#pragma unroll
      for (int q = 0; q < PER; q++) {
        int32_t pt = tid * PER + q;
        loc[q] = (pt < P) ? s_poff[pt] : 0;
        sum += loc[q];
      }
      int32_t total;
      int32_t ex = block_excl_scan<NT>(sum, s_red, &total);
#pragma unroll
      for (int q = 0; q < PER; q++) {
        int32_t pt = tid * PER + q;
        if (pt < P) s_poff[pt] = ex;
        ex += loc[q];
      }
      if (tid == 0) s_poff[P] = total;
    }
    __syncthreads();

    // ---- step 4 (phase A): flattened two-hop gather of the small vertices
    {
      const int32_t E = s_poff[P];
      for (int32_t e0 = tid; e0 < E; e0 += 4 * NT) {
        int32_t val[4], vi[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          int32_t e = e0 + q * NT;
          val[q] = INT32_MIN;
          vi[q] = 0;
          if (e < E) {
            int32_t lo = 0, hi = P - 1;  // largest k with s_poff[k] <= e
            while (lo < hi) {
              int32_t mid = (lo + hi + 1) >> 1;
              if (s_poff[mid] <= e) lo = mid; else hi = mid - 1;
            }
            vi[q] = s_pvert[lo];
            val[q] = a.nc[s_pstart[lo] + (e - s_poff[lo])];
          }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int32_t x = val[q];
          if (x == INT32_MIN) continue;
          const int32_t i = vi[q];
          if (x >= 0) {
            if (x < kSmallWindow) atomicOr(&s_bm[i][x >> 5], 1u << (x & 31));
          } else {
            const int32_t rel = (-2 - x) - p0;
            if (rel >= 0 && rel < i) atomicOr(&s_adj[i], 1ull << rel);
          }
        }
      }
    }
    __syncthreads();

    // ---- step S (first fit): the large vertices' summaries from the gather
    const unsigned long long large = s_large;
    if constexpr (POLICY == BGPC_FF) {
      // two vertices per warp and step, their loads issued together
      for (int32_t iv0 = warp; iv0 < n; iv0 += 2 * NW) {
        int32_t f0[2], f1[2], r0[2], r1[2], rc[2];
        unsigned long long am[2];
        bool lg[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int32_t iv = iv0 + h * NW;
          lg[h] = iv < n && ((large >> iv) & 1ull);
          const int32_t *rec = a.gsum + (slot0 + (lg[h] ? iv : 0)) * kSumInts;
          f0[h] = lg[h] ? rec[lane] : 0;
          f1[h] = lg[h] ? rec[32 + lane] : 0;
          r0[h] = lg[h] ? rec[kSumCand + lane] : 0;
          r1[h] = lg[h] ? rec[kSumCand + 32 + lane] : 0;
          rc[h] = (lg[h] && s_sown[iv] > a.T) ? rec[2 * kSumCand] : 0;
          am[h] = (lg[h] && lane == 0)
                      ? *reinterpret_cast<const unsigned long long *>(rec + 2 * kSumCand + 2)
                      : 0ull;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
          if (!lg[h]) continue;
          const int32_t iv = iv0 + h * NW;
          s_list[iv][lane] = rc[h] > 0 ? -r0[h] : f0[h];
          s_list[iv][lane + 32] = rc[h] > 0 ? -r1[h] : f1[h];
          if (lane == 0) {
            s_rcnt[iv] = rc[h];
            s_adj[iv] = am[h];
          }
        }
      }
      __syncthreads();
    }

    // ---- step P (first fit): a vertex with no earlier neighbour in its
    // chunk sees no overlay, so its color follows from its own forbidden set
    // alone; those vertices are colored all at once, one warp each
    if constexpr (POLICY == BGPC_FF) {
      for (int32_t iv = warp; iv < n; iv += NW) {
        if (s_adj[iv] != 0ull) continue;
        int32_t x;
        const int32_t so = s_sown[iv];
        if ((large >> iv) & 1ull) {
          x = (s_rcnt[iv] > 0) ? -s_list[iv][0] : s_list[iv][0];
        } else {
          const uint32_t word = (lane < kWords) ? s_bm[iv][lane] : kFull;
          x = (so > a.T) ? win_kth_free_down(word, so - 1, s_k[iv]) : -1;
          if (x < 0) x = win_first_free_up(word, 0);
          if (x < 0) {  // cannot happen within the window bounds
            if (lane == 0) atomicOr(a.err, ERR_INTERNAL);
            x = 0;
          }
        }
        if (lane == 0) s_col[iv] = x;
      }
      __syncthreads();
    }

    // ---- phase B (first fit): the vertices with earlier neighbours in the
    // chunk, walked in order by one warp
    if constexpr (POLICY == BGPC_FF) {
      if (warp == 0)
        ff_walk(a, n, slot0, large, s_adj, s_col, s_bm, s_sown, s_k, s_list, s_rcnt, s_dup, s_fm,
                s_cx, s_wscr, s_pull, s_land);
      __syncthreads();
    }

    // ---- phase B (B1, B2): resolve the chunk's vertices in order.  One warp
    // walks the chunk; it stops only at a vertex that needs the whole CTA (a
    // large vertex).
    int32_t i = (POLICY == BGPC_FF) ? n : 0;
    while (i < n) {
      if (warp == 0) {
        int32_t col_max = s_state[0], col_next = s_state[1];
        int32_t ii = i;
        for (; ii < n; ii++) {
          const bool lg = (large >> ii) & 1ull;
          if (lg) break;
          const unsigned long long am = s_adj[ii];
          int32_t x = -1;
          {
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const int32_t jj = lane + 32 * h;
              if (jj < ii && ((am >> jj) & 1ull)) {
                const int32_t c = s_col[jj];
                if (c < kSmallWindow) atomicOr(&s_bm[ii][c >> 5], 1u << (c & 31));
              }
            }
            __syncwarp();
            const uint32_t word = (lane < kWords) ? s_bm[ii][lane] : kFull;
            const int32_t so = s_sown[ii];
            if (so > a.T) x = win_kth_free_down(word, so - 1, s_k[ii]);
            if (x < 0) {
              if (POLICY == BGPC_B1) {
                if ((s_w[ii] & 1) == 0) {
                  x = win_last_free_down(word, col_max);
                  if (x < 0) x = win_first_free_up(word, col_max + 1);
                } else {
                  x = win_first_free_up(word, 0);
                }
              } else if (POLICY == BGPC_B2 || POLICY == BGPC_B2X) {
                x = win_first_free_up(word, col_next);
                if (x < 0 || x > col_max) x = win_first_free_up(word, 0);
              } else {
                x = win_first_free_up(word, 0);
              }
            }
            if (x < 0) {  // cannot happen within the window bounds
              if (lane == 0) atomicOr(a.err, ERR_INTERNAL);
              x = 0;
            }
          }
          col_max = max(col_max, x);
          if (POLICY == BGPC_B2) col_next = min(x + 1, col_max / 3 + 1);
          if (POLICY == BGPC_B2X) col_next = max(x + 1, col_max / 3 + 1);
          if (lane == 0) s_col[ii] = x;
          __syncwarp();
        }
        if (lane == 0) {
          s_state[0] = col_max;
          s_state[1] = col_next;
          s_state[3] = ii;
        }
      }
      __syncthreads();
      const int32_t L = s_state[3];
      if (L < n) {
        // ---- CTA-wide path: the vertex's gathered forbidden set (k_gather)
        // in shared memory, searched with block-wide reductions (B1/B2 only:
        // first fit launches without the dynamic shared bitmap)
        const int64_t slot = slot0 + L;
        uint4 *gsrc = reinterpret_cast<uint4 *>(a.gbm + slot * a.words);
        uint4 *sdst = reinterpret_cast<uint4 *>(s_big);
        for (int32_t x = tid; x < (a.words >> 2); x += NT) {
          sdst[x] = gsrc[x];
          if (POLICY != BGPC_FF) gsrc[x] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (POLICY != BGPC_FF && tid == 0) {
          s_adj[L] = a.gadj[slot];
          a.gadj[slot] = 0ull;
        }
        __syncthreads();
        if (tid < L && ((s_adj[L] >> tid) & 1ull)) {
          const int32_t c = s_col[tid];
          atomicOr(&s_big[c >> 5], 1u << (c & 31));
        }
        __syncthreads();
        const int32_t col_max = s_state[0], col_next = s_state[1];
        int32_t x = -1;
        const int32_t so = s_sown[L];
        if (so > a.T) x = bm_kth_free_down<NT>(s_big, so - 1, s_k[L], s_red);
        if (x < 0) {
          if (POLICY == BGPC_B1) {
            if ((s_w[L] & 1) == 0) {
              x = bm_last_free_down<NT>(s_big, col_max, s_red);
              if (x < 0) x = bm_first_free_up<NT>(s_big, a.words, col_max + 1, s_red);
            } else {
              x = bm_first_free_up<NT>(s_big, a.words, 0, s_red);
            }
          } else if (POLICY == BGPC_B2 || POLICY == BGPC_B2X) {
            x = bm_first_free_up<NT>(s_big, a.words, col_next, s_red);
            if (x > col_max) x = bm_first_free_up<NT>(s_big, a.words, 0, s_red);
          } else {
            x = bm_first_free_up<NT>(s_big, a.words, 0, s_red);
          }
        }
        if (tid == 0) {
          if (x < 0 || x > bound) { atomicOr(a.err, ERR_COLOR); x = 0; }
          s_col[L] = x;
          int32_t cm = max(col_max, x);
          s_state[0] = cm;
          if (POLICY == BGPC_B2) s_state[1] = min(x + 1, cm / 3 + 1);
          if (POLICY == BGPC_B2X) s_state[1] = max(x + 1, cm / 3 + 1);
        }
        __syncthreads();
      }
      i = L + 1;
    }
    if (tid < n) a.stage[p0 + tid] = s_col[tid];
    __syncthreads();
  }
}

// ------------------------------------------------------------ gather kernel
// One work item = up to kPiece nets of one large vertex.  The CTA collects
// the colors of the members of those nets (from the snapshot, via nc) into a
// shared bitmap and the earlier chunk-mates it meets into a 64-bit mask, then
// ORs both into the vertex's global slot.  A heavy vertex is spread over many
// CTAs, so no chunk waits for one SM.  Inside a piece every warp takes an
// equal contiguous slice of the piece's entries (net sizes differ by orders
// of magnitude, so one warp per net would leave most warps waiting) and
// streams it with 16-byte loads.
//
// Hub nets (more than kHubMin members) are not streamed: their published
// colors are kept as one bitmap per net (built at the start of the round,
// extended by every publish), so a member ORs `words` bitmap words instead of
// reading |vtxs(v)| mirror entries, and finds its earlier chunk-mates in the
// net by binary search of their ids in vtxs(v).  On power-law graphs the few
// hub nets carry almost all of the two-hop volume (sum over nets of s^2).

// One mirror word: a published color joins the forbidden bitmap; an earlier
// chunk-mate (queue position in [p0, p0 + rel_hi)) joins the adjacency mask.
__device__ __forceinline__ void take(int32_t x, uint32_t *s_bm, int32_t lim, int32_t p0,
                                     int32_t rel_hi, unsigned long long &adj) {
  // both tests without a branch between them (unsigned compares)
  const uint32_t rel = 0xfffffffeu - (uint32_t)x - (uint32_t)p0;  // -2 - x - p0
  if ((uint32_t)x < (uint32_t)lim) atomicOr(&s_bm[x >> 5], 1u << (x & 31));
  if (x < 0 && rel < (uint32_t)rel_hi) adj |= 1ull << rel;
}

// The lanes of a warp stream src[0, n) (scalar head to a 16-byte boundary,
// int4 body, scalar tail); the head, the tail and the first four int4 groups
// of every lane are loaded together, so a net of up to ~512 members costs one
// round trip.
__device__ __forceinline__ void warp_stream(const int32_t *__restrict__ src, int32_t n,
                                            uint32_t *s_bm, int32_t lim, int32_t p0,
                                            int32_t rel_hi, unsigned long long &adj) {
  const int lane = threadIdx.x & 31;
  const int32_t mis = (int32_t)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
  const int32_t head = mis ? min(n, 4 - mis) : 0;
  const int4 *v = reinterpret_cast<const int4 *>(src + head);
  const int32_t nv = (n - head) >> 2;
  const int32_t t0 = head + (nv << 2);
  const bool hv = lane < head, tv = t0 + lane < n;
  const int32_t hx = hv ? __ldg(src + lane) : 0;
  const int32_t tx = tv ? __ldg(src + t0 + lane) : 0;
  for (int32_t b0 = 0;; b0 += 128) {
    int4 q[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int32_t i = b0 + lane + 32 * k;
      q[k] = (i < nv) ? __ldg(v + i) : make_int4(0, 0, 0, 0);
    }
    if (b0 == 0) {
      if (hv) take(hx, s_bm, lim, p0, rel_hi, adj);
      if (tv) take(tx, s_bm, lim, p0, rel_hi, adj);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (b0 + lane + 32 * k >= nv) continue;
      take(q[k].x, s_bm, lim, p0, rel_hi, adj);
      take(q[k].y, s_bm, lim, p0, rel_hi, adj);
      take(q[k].z, s_bm, lim, p0, rel_hi, adj);
      take(q[k].w, s_bm, lim, p0, rel_hi, adj);
    }
    if (b0 + 128 >= nv) break;
  }
}

// First index of the sorted list l[0, n) whose value is >= u.
__device__ __forceinline__ int32_t lower_bound(const int32_t *__restrict__ l, int32_t n, int32_t u) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (__ldg(l + mid) < u) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Two lower bounds in the sorted list l[0, n) at once, by one warp: lanes
// 0-15 search key0, lanes 16-31 key1, each half probing 16 evenly spaced
// entries per round (the range shrinks 16-fold per dependent load instead of
// 2-fold).  Returns (lower_bound(key0), lower_bound(key1)) in every lane.
__device__ __forceinline__ int2 warp_lower_bounds(const int32_t *__restrict__ l, int32_t n,
                                                  int32_t key0, int32_t key1) {
  const int lane = threadIdx.x & 31;
  const int sl = lane & 15;
  const unsigned half = (lane < 16) ? 0x0000ffffu : 0xffff0000u;
  const int32_t key = (lane < 16) ? key0 : key1;
  int32_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (__any_sync(kFull, lo < hi)) {
    const int32_t step = (hi - lo + 15) >> 4;
    const int32_t e = lo + (sl + 1) * step - 1;  // last entry of sub-range sl
    const bool valid = lo < hi && e < hi;
    const bool below = valid && __ldg(l + e) < key;
    const int32_t cnt = __popc(__ballot_sync(kFull, below) & half);
    const int32_t ec = lo + (cnt + 1) * step - 1;
    if (lo < hi) {
      const int32_t nlo = lo + cnt * step;
      hi = (cnt < 16 && ec < hi) ? ec : hi;
      lo = nlo;
    }
  }
  return make_int2(__shfl_sync(kFull, lo, 0), __shfl_sync(kFull, lo, 16));
}

// Whether vertex u is in the sorted list l[0, n).
__device__ __forceinline__ bool sorted_has(const int32_t *__restrict__ l, int32_t n, int32_t u) {
  const int32_t lo = lower_bound(l, n, u);
  return lo < n && __ldg(l + lo) == u;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_gather(GatherArgs a) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) uint32_t s_bm[];
  __shared__ int32_t s_pstart[kPiece];
  __shared__ int32_t s_poff[kPiece + 1];
  __shared__ int32_t s_hslot[kPiece], s_hbp[kPiece], s_hsz[kPiece];  // hub nets of the piece
  __shared__ int32_t s_info[7];  // p0, rel_hi, whole, nnets, hubs, vertex, pieces
  __shared__ int64_t s_slot;
  __shared__ unsigned long long s_adj;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t sbeg = a.segoff[a.slot_lo], send = a.segoff[a.slot_hi];
  const int32_t lim = a.words * 32;
  for (int32_t x = tid; x < a.words; x += NT) s_bm[x] = 0u;
  if (tid == 0) s_adj = 0ull;
  for (int32_t sg = sbeg + (int32_t)blockIdx.x; sg < send; sg += (int32_t)gridDim.x) {
    // ---- the piece: its vertex and the prefix of its net sizes
    if (warp == 0) {
      // the piece's descriptor: wave-order slot, vertex, first incidence,
      // number of nets | number of pieces of the vertex << 6
      const int4 sm = a.segmap[sg];
      const int32_t u = sm.x, w = sm.y, ibeg = sm.z;
      const int32_t nnets = sm.w & 63, npieces = sm.w >> 6;
      const int32_t j = a.wlist[u / a.C];
      const int32_t p0 = j * a.C;
      const int32_t p = p0 + u % a.C;
      int32_t sz = 0, bp = 0, hub = -1;
      if (lane < nnets) {
        const int32_t v = a.a_idx[ibeg + lane];
        bp = a.b_ptr[v];
        sz = a.b_ptr[v + 1] - bp;
        hub = a.hub_id ? a.hub_id[v] : -1;
      }
      // hub nets are read from their bitmaps; the others are streamed
      const unsigned hubs = __ballot_sync(kFull, hub >= 0);
      if (hub >= 0) {
        const int32_t k = __popc(hubs & ((1u << lane) - 1u));
        s_hslot[k] = hub;
        s_hbp[k] = bp;
        s_hsz[k] = sz;
      }
      const int32_t inc = warp_incl_scan(hub >= 0 ? 0 : sz);
      if (lane < kPiece) {
        s_pstart[lane] = bp;
        s_poff[lane + 1] = inc;
      }
      if (hubs) {
        const int32_t hv = __reduce_add_sync(kFull, hub >= 0 ? sz - 1 : 0);
        if (lane == 0) {
          atomicAdd(&a.dev->trav_hub, (unsigned long long)hv);
          atomicAdd(&a.dev->hub_pairs, (unsigned long long)__popc(hubs));
          atomicAdd(&a.dev->hub_words, (unsigned long long)__popc(hubs) * a.words);
        }
      }
      if (lane == 0) {
        s_poff[0] = 0;
        s_info[0] = p0;
        s_info[1] = p - p0;
        s_info[2] = npieces == 1;
        s_info[3] = nnets;
        s_info[4] = __popc(hubs);
        s_info[5] = w;
        s_info[6] = npieces;
        s_slot = (int64_t)(u - a.slot_lo);
      }
    }
    __syncthreads();
    const int32_t p0 = s_info[0], rel_hi = s_info[1], nnets = s_info[3], nh = s_info[4];
    unsigned long long adj = 0ull;
    if (nh > 0) {
      // hub nets: OR their bitmaps (16 bytes per thread and step) ...
      const int32_t W4 = a.words >> 2;
      const uint4 *nb4 = reinterpret_cast<const uint4 *>(a.nbm);
      for (int32_t t = tid; t < nh * W4; t += NT) {
        const int32_t h = t / W4, x = t - h * W4;
        const uint4 q = __ldg(nb4 + (int64_t)s_hslot[h] * W4 + x);
        if (q.x) atomicOr(&s_bm[4 * x + 0], q.x);
        if (q.y) atomicOr(&s_bm[4 * x + 1], q.y);
        if (q.z) atomicOr(&s_bm[4 * x + 2], q.z);
        if (q.w) atomicOr(&s_bm[4 * x + 3], q.w);
      }
      // ... and find the earlier chunk-mates that are members
      if (a.id_order && rel_hi > 0) {
        // the chunk's ids increase with the position: its earlier members
        // lie between the ids of its first and last earlier vertex, a short
        // stretch of vtxs(v) located by two binary searches (one warp per
        // hub net), whose mirror words carry their queue positions
        const int32_t id_lo = a.W[p0], id_hi = a.W[p0 + rel_hi - 1];
        for (int32_t h = warp; h < nh; h += NW) {
          const int32_t *l = a.b_idx + s_hbp[h];
          const int2 bb = warp_lower_bounds(l, s_hsz[h], id_lo, id_hi + 1);
          const int32_t lb = bb.x, ub = bb.y;
          for (int32_t f = lb + lane; f < ub; f += 32) {
            const int32_t x = a.nc[s_hbp[h] + f];
            const int32_t rel = (-2 - x) - p0;
            if (x < 0 && rel >= 0 && rel < rel_hi) adj |= 1ull << rel;
          }
        }
      } else {
        for (int32_t t = tid; t < nh * rel_hi; t += NT) {
          const int32_t h = t / rel_hi, j = t - h * rel_hi;
          if (sorted_has(a.b_idx + s_hbp[h], s_hsz[h], a.W[p0 + j])) adj |= 1ull << j;
        }
      }
    }
    const int32_t E = s_poff[nnets];
    const int32_t per = (E + NW - 1) / NW;
    const int32_t lo_e = min(E, warp * per), hi_e = min(E, lo_e + per);
    if (lo_e < hi_e) {
      int32_t t = 0;  // first net of the slice: largest t with s_poff[t] <= lo_e
      for (int32_t step = kPiece / 2; step > 0; step >>= 1)
        if (t + step < nnets && s_poff[t + step] <= lo_e) t += step;
      for (; t < nnets && s_poff[t] < hi_e; t++) {
        const int32_t nb = max(lo_e, s_poff[t]), ne = min(hi_e, s_poff[t + 1]);
        warp_stream(a.nc + s_pstart[t] + (nb - s_poff[t]), ne - nb, s_bm, lim, p0, rel_hi, adj);
      }
    }
    const unsigned lo32 = __reduce_or_sync(kFull, (unsigned)(adj & 0xffffffffull));
    const unsigned hi32 = __reduce_or_sync(kFull, (unsigned)(adj >> 32));
    if (lane == 0 && (lo32 | hi32)) atomicOr(&s_adj, ((unsigned long long)hi32 << 32) | lo32);
    __syncthreads();
    const int64_t slot = s_slot;
    uint32_t *g = a.gbm + slot * a.words;
    const bool whole = s_info[2] != 0;
    bool take = false;  // first fit: this CTA writes the vertex's summary
    if (a.summ && !whole) {
      // ---- several pieces: merge into the slot; the last piece to merge
      // takes the slot back (leaving it zero)
      for (int32_t x = tid; x < a.words; x += NT) {
        const uint32_t b = s_bm[x];
        if (b) {
          atomicOr(&g[x], b);
          s_bm[x] = 0u;
        }
      }
      if (tid == 0 && s_adj) atomicOr(&a.gadj[slot], s_adj);
      __threadfence();
      __syncthreads();
      if (tid == 0) s_info[2] = atomicAdd(a.gcnt + slot, 1) == s_info[6] - 1;
      __syncthreads();
      take = s_info[2] != 0;
      if (take) {
        __threadfence();
        for (int32_t x = tid; x < a.words; x += NT) {
          const uint32_t b = __ldcg(g + x);
          if (b) {
            s_bm[x] = b;
            g[x] = 0u;
          }
        }
        if (tid == 0) {
          s_adj = __ldcg(a.gadj + slot);
          a.gadj[slot] = 0ull;
          a.gcnt[slot] = 0;
        }
        __syncthreads();
      }
    } else if (a.summ) {
      take = true;  // one piece: the bitmap is complete
    }
    if (take) {
      if (warp == 0) {
        const int32_t so = a.s_own[s_info[5]];
        warp_summarize(s_bm, a.words, so, a.T, (so > a.T) ? a.kofs[p0 + rel_hi] : 0, s_adj,
                       a.gsum + slot * kSumInts, a.lbm + slot * a.words);
      }
      __syncthreads();
      for (int32_t x = tid; x < a.words; x += NT) s_bm[x] = 0u;
    } else if (!a.summ) {
      // ---- merge into the vertex's slot, leaving the shared bitmap zero
      for (int32_t x = tid; x < a.words; x += NT) {
        const uint32_t b = s_bm[x];
        if (b) {
          if (whole) g[x] = b; else atomicOr(&g[x], b);
          s_bm[x] = 0u;
        }
      }
      if (tid == 0) {
        const unsigned long long m = s_adj;
        if (m) {
          if (whole) a.gadj[slot] = m; else atomicOr(&a.gadj[slot], m);
        }
      }
    }
    __syncthreads();
    if (tid == 0) s_adj = 0ull;
    __syncthreads();
  }
}

// Zero the non-zero 16-byte words of a warp's shared bitmap.
__device__ __forceinline__ void warp_clear(uint4 *bm4, int32_t n4) {
  for (int32_t x = (int32_t)(threadIdx.x & 31); x < n4; x += 32) {
    const uint4 b = bm4[x];
    if (b.x | b.y | b.z | b.w) bm4[x] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncwarp();
}

// The hubs' colors into a warp's bitmap, 16-byte groups [qlo, qhi): each
// lane ORs its own groups of every hub of the piece (two groups of two hubs
// per step, four loads in flight) and updates the bitmap once per group.
// hubs = the lanes whose net is a hub, hub = this lane's hub slot.  The loop
// bounds are the same in every lane: the shuffles need the whole warp.
__device__ __forceinline__ void warp_hub_or(uint4 *s_bm4, const uint4 *nb4, int32_t W4,
                                            unsigned hubs, int32_t hub, int32_t qlo,
                                            int32_t qhi) {
  const int lane = threadIdx.x & 31;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  for (int32_t xb = qlo; xb < qhi; xb += 64) {
    const int32_t x0 = xb + lane;
    const bool v0 = x0 < qhi, v1 = x0 + 32 < qhi;
    uint4 c0 = zero, c1 = zero;
    for (unsigned hm = hubs; hm;) {
      const int32_t s0 = __shfl_sync(kFull, hub, __ffs(hm) - 1);
      hm &= hm - 1u;
      const int32_t s1 = hm ? __shfl_sync(kFull, hub, __ffs(hm) - 1) : -1;
      hm &= hm - 1u;
      const uint4 *h0 = nb4 + (int64_t)s0 * W4 + x0;
      const uint4 q00 = v0 ? __ldg(h0) : zero;
      const uint4 q01 = v1 ? __ldg(h0 + 32) : zero;
      uint4 q10 = zero, q11 = zero;
      if (s1 >= 0) {
        const uint4 *h1 = nb4 + (int64_t)s1 * W4 + x0;
        q10 = v0 ? __ldg(h1) : zero;
        q11 = v1 ? __ldg(h1 + 32) : zero;
      }
      c0 = make_uint4(c0.x | q00.x | q10.x, c0.y | q00.y | q10.y, c0.z | q00.z | q10.z,
                      c0.w | q00.w | q10.w);
      c1 = make_uint4(c1.x | q01.x | q11.x, c1.y | q01.y | q11.y, c1.z | q01.z | q11.z,
                      c1.w | q01.w | q11.w);
    }
    if (v0 && (c0.x | c0.y | c0.z | c0.w)) {
      const uint4 b = s_bm4[x0];
      s_bm4[x0] = make_uint4(b.x | c0.x, b.y | c0.y, b.z | c0.z, b.w | c0.w);
    }
    if (c1.x | c1.y | c1.z | c1.w) {
      const uint4 b = s_bm4[x0 + 32];
      s_bm4[x0 + 32] = make_uint4(b.x | c1.x, b.y | c1.y, b.z | c1.z, b.w | c1.w);
    }
  }
  __syncwarp();
}

// Warp-private form of the gather: every warp takes whole pieces on its own,
// with its own bitmap in shared memory, so no CTA barrier stands between a
// piece's dependent loads (piece -> vertex -> nets -> net extents) and the
// other warps' streaming.  Same results as k_gather: the bitmap and mask of
// a piece are ORed into the vertex's slot the same way.
template <int NT>
__global__ void __launch_bounds__(NT, 4) k_gather_w(GatherArgs a) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) uint32_t s_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *s_bm = s_all + (size_t)warp * a.words;
  uint4 *s_bm4 = reinterpret_cast<uint4 *>(s_bm);
  const int32_t lim = a.words * 32, W4 = a.words >> 2;
  for (int32_t x = lane; x < a.words; x += 32) s_bm[x] = 0u;
  __syncwarp();
  const int32_t sbeg = a.segoff[a.slot_lo], send = a.segoff[a.slot_hi];
  const uint4 *nb4 = reinterpret_cast<const uint4 *>(a.nbm);
  const int64_t nwarps = (int64_t)gridDim.x * NW;
  unsigned long long n_trav_hub = 0, n_hub_pairs = 0, n_hub_groups = 0;  // lane 0's counts
  for (int64_t sg = sbeg + (int64_t)blockIdx.x * NW + warp; sg < send; sg += nwarps) {
    // ---- the piece: its vertex, its chunk and its nets (one net per lane)
    // the piece's descriptor (built by the piece map with full parallelism,
    // so the warp starts with one load instead of a chain of four)
    const int4 sm = a.segmap[sg];
    const int32_t u = sm.x, w = sm.y, ibeg = sm.z;
    const int32_t nnets = sm.w & 63, npieces = sm.w >> 6;
    const int32_t p0 = a.wlist[u / a.C] * a.C;
    const int32_t rel_hi = u % a.C;  // the vertex's index in its chunk
    const bool whole = npieces == 1;
    // hub groups ORed here: all of them, except for a one-piece first-fit
    // vertex, whose summary reads the groups up to its owner's top s - 1
    // (and more only if its first 64 free colors lie beyond them)
    int32_t so = 0, qor = W4;
    if (a.summ && whole) {
      so = a.s_own[w];
      qor = min(W4, max(so > a.T ? ((so - 1) >> 7) + 1 : 0, 2));
    }
    int32_t sz = 0, bp = 0, hub = -1, tp = 0, vnet = 0;
    if (lane < nnets) {
      vnet = a.a_idx[ibeg + lane];
      bp = a.b_ptr[vnet];
      sz = a.b_ptr[vnet + 1] - bp;
      hub = a.hub_id ? a.hub_id[vnet] : -1;
      if (a.id_order && hub >= 0) tp = a.tpos[ibeg + lane];
    }
    const unsigned hubs = __ballot_sync(kFull, hub >= 0);
    unsigned long long adj = 0ull;
    if (hubs) {
      n_trav_hub += (unsigned long long)__reduce_add_sync(kFull, hub >= 0 ? sz - 1 : 0);
      n_hub_pairs += (unsigned long long)__popc(hubs);
      n_hub_groups += (unsigned long long)__popc(hubs) * qor;
      const int32_t id_lo = (a.id_order && rel_hi > 0) ? a.W[p0] : 0;
      warp_hub_or(s_bm4, nb4, W4, hubs, hub, 0, qor);
      // their earlier chunk-mates.  A chunk whose ids spread wide (later
      // rounds, or a caller's rank order): every (hub, earlier chunk-mate)
      // pair is tested directly, one per lane, by bisecting the hub's net id
      // in the chunk-mate's sorted net list (short and contiguous).
      const bool wide = rel_hi > 0 && (!a.id_order || w - id_lo > kHubScanSpan);
      if (wide) {
        const int32_t npairs = __popc(hubs) * rel_hi;
        for (int32_t q0 = 0; q0 < npairs; q0 += 32) {
          const int32_t q = q0 + lane;
          const int32_t k = q < npairs ? q / rel_hi : 0, j = q - k * rel_hi;
          const int32_t hv = __shfl_sync(kFull, vnet, nth_set_bit32(hubs, k));
          if (q < npairs) {
            const int32_t u = a.W[p0 + j];
            int32_t lo = a.a_ptr[u];
            const int32_t end = a.a_ptr[u + 1];
            int32_t hi = end;
            while (lo < hi) {
              const int32_t mid = (lo + hi) >> 1;
              if (__ldg(a.a_idx + mid) < hv) lo = mid + 1; else hi = mid;
            }
            if (lo < end && __ldg(a.a_idx + lo) == hv) adj |= 1ull << j;
          }
        }
      }
      // In id order with a narrow chunk (the first round) the earlier
      // vertices have ids in [id_lo, w), so in the id-sorted vtxs(v) they sit
      // right before w's own entry (its CSC index tp): read backwards from
      // there while the ids stay >= id_lo (one window of 32 per step, usually
      // one step); the mirror words of those entries carry the queue
      // positions.  Four hubs per step: their first windows (ids and mirror
      // words) are loaded together.
      for (unsigned hm = hubs; hm && rel_hi > 0 && !wide;) {
        int32_t f[4], hb[4], id[4], x[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const bool val = hm != 0;
          const int t = val ? __ffs(hm) - 1 : 0;
          f[k] = __shfl_sync(kFull, tp, t) - 1 - lane;
          hb[k] = val ? __shfl_sync(kFull, bp, t) : INT32_MAX;
          hm &= hm - 1u;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const bool ok = f[k] >= hb[k];
          id[k] = ok ? __ldg(a.b_idx + f[k]) : INT32_MIN;
          x[k] = ok ? a.nc[f[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
          bool in = id[k] >= id_lo;
          int32_t xk = x[k];
          // more than 32 entries with ids in [id_lo, w): the next windows
          for (int32_t top = f[k] + lane - 32;;) {
            const int32_t rel = (-2 - xk) - p0;
            if (in && xk < 0 && rel >= 0 && rel < rel_hi) adj |= 1ull << rel;
            if (__ballot_sync(kFull, in) != kFull) break;
            const int32_t g = top - lane;
            in = g >= hb[k] && __ldg(a.b_idx + g) >= id_lo;
            xk = in ? a.nc[g] : 0;
            top -= 32;
          }
        }
      }
      __syncwarp();
    }
    // ---- the other nets: those of up to 64 members four at a time (two
    // words per lane each, eight loads in flight), larger ones streamed
    unsigned few = __ballot_sync(kFull, hub < 0 && sz > 0 && sz <= 64);
    const unsigned lg = __ballot_sync(kFull, hub < 0 && sz > 64);
    while (few) {
      int32_t n[4], b[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int t = few ? __ffs(few) - 1 : 0;
        n[k] = few ? __shfl_sync(kFull, sz, t) : 0;
        b[k] = __shfl_sync(kFull, bp, t);
        few &= few - 1u;
      }
      int32_t x[8];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        x[2 * k] = (lane < n[k]) ? __ldg(a.nc + b[k] + lane) : 0;
        x[2 * k + 1] = (lane + 32 < n[k]) ? __ldg(a.nc + b[k] + lane + 32) : 0;
      }
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (lane < n[k]) take(x[2 * k], s_bm, lim, p0, rel_hi, adj);
        if (lane + 32 < n[k]) take(x[2 * k + 1], s_bm, lim, p0, rel_hi, adj);
      }
    }
    for (unsigned m = lg; m; m &= m - 1u) {
      const int t = __ffs(m) - 1;
      warp_stream(a.nc + __shfl_sync(kFull, bp, t), __shfl_sync(kFull, sz, t), s_bm, lim, p0,
                  rel_hi, adj);
    }
    const unsigned lo32 = __reduce_or_sync(kFull, (unsigned)(adj & 0xffffffffull));
    const unsigned hi32 = __reduce_or_sync(kFull, (unsigned)(adj >> 32));
    const unsigned long long adjm = ((unsigned long long)hi32 << 32) | lo32;
    __syncwarp();
    const int64_t slot = (int64_t)(u - a.slot_lo);
    if (a.summ && whole) {
      // first fit, one piece: the summary straight from the bitmap
      int32_t *rec = a.gsum + slot * kSumInts;
      int32_t got = 0, q0 = 0;
      warp_first_free_from<kSumCand>(s_bm, W4, qor, rec, got, q0);
      // past the groups ORed so far: the hubs' next groups, twice as many
      // each step, until 64 free colors are found (the streamed nets are
      // complete at every group)
      while (got < kSumCand && hubs && qor < W4) {
        const int32_t qn = min(W4, 2 * qor);
        warp_hub_or(s_bm4, nb4, W4, hubs, hub, qor, qn);
        n_hub_groups += (unsigned long long)__popc(hubs) * (qn - qor);
        qor = qn;
        warp_first_free_from<kSumCand>(s_bm, W4, qor, rec, got, q0);
      }
      if (got < kSumCand) warp_first_free_from<kSumCand>(s_bm, W4, INT32_MAX, rec, got, q0);
      warp_summarize_rest(s_bm, so, a.T, (so > a.T) ? a.kofs[p0 + rel_hi] : 0, adjm, rec,
                          a.lbm + slot * a.words);
      warp_clear(s_bm4, W4);
      continue;
    }
    // ---- merge into the vertex's slot, leaving the bitmap zero
    uint4 *g4 = reinterpret_cast<uint4 *>(a.gbm + slot * a.words);
    for (int32_t x = lane; x < W4; x += 32) {
      const uint4 b = s_bm4[x];
      if (b.x | b.y | b.z | b.w) {
        if (whole && !a.summ) {
          g4[x] = b;
        } else {
          unsigned long long *g = reinterpret_cast<unsigned long long *>(g4 + x);
          const unsigned long long lo = ((unsigned long long)b.y << 32) | b.x;
          const unsigned long long hi = ((unsigned long long)b.w << 32) | b.z;
          if (lo) atomicOr(g + 0, lo);
          if (hi) atomicOr(g + 1, hi);
        }
        s_bm4[x] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    if (lane == 0 && adjm) {
      if (whole && !a.summ) a.gadj[slot] = adjm; else atomicOr(&a.gadj[slot], adjm);
    }
    if (a.summ) {
      // first fit, several pieces: the last piece to merge takes the slot
      // back (leaving it zero) and writes the summary
      __threadfence();
      __syncwarp();
      int32_t last = 0;
      if (lane == 0) last = atomicAdd(a.gcnt + slot, 1) == npieces - 1;
      last = __shfl_sync(kFull, last, 0);
      if (last) {
        __threadfence();
        unsigned long long m = 0ull;
        if (lane == 0) {
          m = __ldcg(a.gadj + slot);
          a.gadj[slot] = 0ull;
          a.gcnt[slot] = 0;
        }
        m = __shfl_sync(kFull, m, 0);
        for (int32_t x0 = lane; x0 < W4; x0 += 128) {  // four loads in flight
          uint4 q[4];
#pragma unroll
          for (int k = 0; k < 4; k++)
            q[k] = (x0 + 32 * k < W4) ? __ldcg(g4 + x0 + 32 * k) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (int k = 0; k < 4; k++) {
            if (q[k].x | q[k].y | q[k].z | q[k].w) {
              s_bm4[x0 + 32 * k] = q[k];
              g4[x0 + 32 * k] = make_uint4(0u, 0u, 0u, 0u);
            }
          }
        }
        __syncwarp();
        const int32_t so = a.s_own[w];
        warp_summarize(s_bm, a.words, so, a.T, (so > a.T) ? a.kofs[p0 + rel_hi] : 0, m,
                       a.gsum + slot * kSumInts, a.lbm + slot * a.words);
        warp_clear(s_bm4, W4);
      }
    }
    __syncwarp();
  }
  if (lane == 0 && n_hub_pairs) {
    atomicAdd(&a.dev->trav_hub, n_trav_hub);
    atomicAdd(&a.dev->hub_pairs, n_hub_pairs);
    atomicAdd(&a.dev->hub_words, 4 * n_hub_groups);
  }
}

// --------------------------------------------------- pieces of the round
// Wave-order slot u = (index of its chunk in the wave-ordered chunk list) * C
// + offset in the chunk.  Large vertices get ceil(deg / kPiece) pieces (at
// least one), small ones none.
constexpr int kScanNT = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanNT * kScanPer;

__device__ __forceinline__ int32_t pieces_of(const int32_t *a_ptr, const int32_t *d2tot,
                                             const int32_t *W, const int32_t *wlist, int32_t C,
                                             int32_t m, bool small_ok, int64_t u) {
  const int64_t p = (int64_t)wlist[u / C] * C + u % C;
  if (p >= m) return 0;
  const int32_t w = W[p];
  const int32_t deg = a_ptr[w + 1] - a_ptr[w];
  if (is_small(d2tot[w], deg, small_ok)) return 0;
  return max(1, (deg + kPiece - 1) / kPiece);
}

__global__ void __launch_bounds__(kScanNT) k_piece_count(const int32_t *__restrict__ a_ptr,
                                                         const int32_t *__restrict__ d2tot,
                                                         const int32_t *__restrict__ W,
                                                         const int32_t *__restrict__ wlist,
                                                         int32_t nslots, int32_t C, int32_t m,
                                                         int32_t small_ok,
                                                         int32_t *__restrict__ segoff,
                                                         int32_t *__restrict__ blocksum) {
  __shared__ int32_t red[kScanNT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t c = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    const int64_t u = base + q;
    if (u < nslots) {
      const int32_t k = pieces_of(a_ptr, d2tot, W, wlist, C, m, small_ok != 0, u);
      segoff[u] = k;
      c += k;
    }
  }
  int32_t total;
  block_excl_scan<kScanNT>(c, red, &total);
  if (threadIdx.x == 0) blocksum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanNT) k_piece_blocks(int32_t *__restrict__ blocksum,
                                                          int32_t nblocks, int32_t nslots,
                                                          int32_t *__restrict__ segoff,
                                                          DevScalars *dev) {
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
  if (threadIdx.x == 0) {
    dev->nseg = carry;
    segoff[nslots] = carry;
  }
}

__global__ void __launch_bounds__(kScanNT) k_piece_scatter(int32_t nslots,
                                                           const int32_t *__restrict__ blocksum,
                                                           int32_t *__restrict__ segoff,
                                                           int4 *__restrict__ segmap,
                                                           const int32_t *__restrict__ a_ptr,
                                                           const int32_t *__restrict__ W,
                                                           const int32_t *__restrict__ wlist,
                                                           int32_t C) {
  __shared__ int32_t red[kScanNT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t k[kScanPer];
  int32_t c = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    k[q] = (base + q < nslots) ? segoff[base + q] : 0;
    c += k[q];
  }
  int32_t total;
  int32_t ex = block_excl_scan<kScanNT>(c, red, &total) + blocksum[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    if (base + q < nslots) {
      segoff[base + q] = ex;
      if (k[q] > 0) {
        // piece r of the vertex in slot u: {u, vertex, first incidence,
        // nets | pieces << 6}
        const int32_t u = (int32_t)(base + q);
        const int32_t w = W[wlist[u / C] * C + u % C];
        const int32_t ab = a_ptr[w], ae = a_ptr[w + 1];
        for (int32_t r = 0; r < k[q]; r++) {
          const int32_t ib = ab + r * kPiece;
          segmap[ex + r] = make_int4(u, w, ib, min(ae - ib, kPiece) | (k[q] << 6));
        }
      }
      ex += k[q];
    }
  }
}

// Publish: colors of the wave's positions go to c[] and to every CSC entry
// of their edges (nc), and the running max color is updated.  ihub[i] is the
// hub slot of CSR entry i's net (-1: not a hub), read in CSR order instead of
// looking the net up at random.  Large vertices are published piece by piece
// from the wave's piece map (one warp per piece of up to 32 nets, one lane
// per incidence; every piece also writes the vertex's color), so a vertex of
// thousands of nets is spread over many warps; small vertices (at most 16
// nets, no pieces) take half a warp each.
__global__ void k_publish(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ d2tot,
                          const int32_t *__restrict__ ihub, const int32_t *__restrict__ tpos,
                          const int32_t *__restrict__ W, const int32_t *__restrict__ stage,
                          const int32_t *__restrict__ wlist, int32_t C, int32_t m,
                          int32_t small_ok, int32_t slot_lo, int32_t slot_hi,
                          const int32_t *__restrict__ segoff, const int4 *__restrict__ segmap,
                          int32_t *__restrict__ nc, int32_t *__restrict__ colors,
                          uint32_t *__restrict__ nbm, int32_t words, DevScalars *dev) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t mx = -1;
  // large vertices: their pieces
  const int32_t sbeg = segoff[slot_lo], send = segoff[slot_hi];
  for (int64_t sg = sbeg + warp; sg < send; sg += nwarps) {
    const int4 sm = segmap[sg];
    const int32_t u = sm.x, w = sm.y, ib = sm.z, nn = sm.w & 63;
    const int32_t col = stage[wlist[u / C] * C + u % C];
    if (lane < nn) {
      const int32_t i = ib + lane;
      nc[tpos[i]] = col;
      if (ihub) {  // the color joins the bitmap of every hub net of w
        const int32_t h = ihub[i];
        if (h >= 0) atomicOr(&nbm[(int64_t)h * words + (col >> 5)], 1u << (col & 31));
      }
    }
    if (lane == 0) colors[w] = col;
    mx = max(mx, col);
  }
  // small vertices: half a warp each
  if (small_ok) {
    const int32_t hl = lane & 15;
    for (int64_t u = (int64_t)slot_lo + 2 * warp + (lane >> 4); u < slot_hi; u += 2 * nwarps) {
      const int64_t p = (int64_t)wlist[u / C] * C + u % C;
      if (p >= m) continue;
      const int32_t w = W[p];
      const int32_t beg = a_ptr[w], deg = a_ptr[w + 1] - beg;
      if (!is_small(d2tot[w], deg, true)) continue;
      const int32_t col = stage[p];
      if (hl < deg) {
        const int32_t i = beg + hl;
        nc[tpos[i]] = col;
        if (ihub) {
          const int32_t h = ihub[i];
          if (h >= 0) atomicOr(&nbm[(int64_t)h * words + (col >> 5)], 1u << (col & 31));
        }
      }
      if (hl == 0) colors[w] = col;
      mx = max(mx, col);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (lane == 0 && mx >= 0) atomicMax(&dev->gmax, mx);
}

constexpr int kWaveNT = 256;
constexpr int kGatherNT = 256;

// Lets the kernel take all the dynamic shared memory the device allows next to
// its static arrays.  Always the same value, so concurrent callers (the
// batched entry point colors graphs from several host threads) never see a
// smaller limit than the one they launch with.
template <typename K>
cudaError_t allow_dynamic_smem(K kern) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

template <int POLICY>
cudaError_t launch_policy(const WaveArgs &a, int sms, cudaStream_t s) {
  auto kern = k_color_wave<POLICY, kWaveNT>;
  // first fit resolves from the gather's summaries: no bitmap in shared memory
  const size_t smem = (POLICY == BGPC_FF) ? 0 : (size_t)a.words * 4;
  cudaError_t e = allow_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWaveNT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * sms;
  if (grid > a.nchunks) grid = a.nchunks;
  kern<<<grid, kWaveNT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int32_t wave_max_words(int smem_optin) {
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, k_color_wave<BGPC_FF, kWaveNT>) == cudaSuccess)
    stat = fa.sharedSizeBytes;
  else
    cudaGetLastError();
  long long room = ((long long)smem_optin - (long long)stat - 1024) / 4;
  return room > 0 ? (int32_t)(room & ~3LL) : 0;
}

cudaError_t launch_color_wave(int policy, const WaveArgs &a, int sms, cudaStream_t s) {
  if (a.nchunks <= 0) return cudaSuccess;
  switch (policy) {
    case BGPC_B1: return launch_policy<BGPC_B1>(a, sms, s);
    case BGPC_B2: return launch_policy<BGPC_B2>(a, sms, s);
    case BGPC_B2X: return launch_policy<BGPC_B2X>(a, sms, s);
    default: return launch_policy<BGPC_FF>(a, sms, s);
  }
}

cudaError_t launch_gather(const GatherArgs &a, bool cta_only, int sms, cudaStream_t s) {
  if (a.slot_hi <= a.slot_lo) return cudaSuccess;
  if (!cta_only) {  // warp-private pieces when eight bitmaps fit beside each other
    auto kw = k_gather_w<kGatherNT>;
    const size_t smem_w = (size_t)(kGatherNT / 32) * a.words * 4;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem_w + 1024 <= (size_t)optin / 2) {  // at least two CTAs per SM
      cudaError_t e = allow_dynamic_smem(kw);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kw, kGatherNT, smem_w);
      if (e != cudaSuccess) return e;
      if (per_sm >= 1) {
        kw<<<per_sm * sms, kGatherNT, smem_w, s>>>(a);
        return cudaGetLastError();
      }
    }
  }
  auto kern = k_gather<kGatherNT>;
  const size_t smem = (size_t)a.words * 4;
  cudaError_t e = allow_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGatherNT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  kern<<<per_sm * sms, kGatherNT, smem, s>>>(a);
  return cudaGetLastError();
}

int launch_pieces(const int32_t *a_ptr, const int32_t *d2tot, const int32_t *W,
                  const int32_t *wlist, int32_t nch, int32_t C, int32_t m, int32_t small_ok,
                  int32_t *segoff, int32_t *blocksum, int4 *segmap, DevScalars *dev,
                  cudaStream_t s) {
  const int32_t nslots = nch * C;
  if (nslots <= 0) return 0;
  const int nblocks = div_up(nslots, kScanTile);
  k_piece_count<<<nblocks, kScanNT, 0, s>>>(a_ptr, d2tot, W, wlist, nslots, C, m, small_ok,
                                            segoff, blocksum);
  k_piece_blocks<<<1, kScanNT, 0, s>>>(blocksum, nblocks, nslots, segoff, dev);
  k_piece_scatter<<<nblocks, kScanNT, 0, s>>>(nslots, blocksum, segoff, segmap, a_ptr, W,
                                              wlist, C);
  return 3;
}

int launch_publish(const int32_t *a_ptr, const int32_t *d2tot, const int32_t *ihub,
                   const int32_t *tpos, const int32_t *W, const int32_t *stage,
                   const int32_t *wlist, int32_t C, int32_t m, int32_t small_ok,
                   int32_t slot_lo, int32_t slot_hi, const int32_t *segoff, const int4 *segmap,
                   int32_t *nc, int32_t *colors, uint32_t *nbm, int32_t words, DevScalars *dev,
                   int sms, cudaStream_t s) {
  if (slot_hi <= slot_lo) return 0;
  // one resident set (8 CTAs of 256 per SM), grid-stride over pieces and slots
  long long grid = div_up((long long)(slot_hi - slot_lo) * 32, 256);
  if (grid > (long long)sms * 8) grid = (long long)sms * 8;
  if (grid < 1) grid = 1;
  k_publish<<<(int)grid, 256, 0, s>>>(a_ptr, d2tot, ihub, tpos, W, stage, wlist, C, m, small_ok,
                                      slot_lo, slot_hi, segoff, segmap, nc, colors, nbm, words,
                                      dev);
  return 1;
}

// ---------------------------------------------------------- hub nets
// Nets with more than H members get a slot (order of the slots is irrelevant).
// The hub threshold: the smallest ladder size whose nets' first-round bitmaps
// (the round-0 width: every color <= max(maxnet - 1, 0) + C * Q) take at most
// budget_words words; then hub_id[v] = the slot of net v if it is larger, or -1.
__global__ void k_hub_select(const int32_t *__restrict__ b_ptr, int32_t n_b, int32_t C,
                             int32_t Q, int64_t budget_words, int32_t *__restrict__ hub_id,
                             int32_t *__restrict__ hub_net, DevScalars *dev) {
  __shared__ int32_t s_H;
  if (threadIdx.x == 0) {
    const int64_t ncol = (int64_t)max(dev->maxnet - 1, 0) + (int64_t)C * Q + C + 2;
    const int64_t words0 = ((ncol + 31) / 32 + 3) & ~(int64_t)3;
    int32_t H = INT32_MAX;
    int64_t above = 0;  // nets larger than hub_ladder(k)
    for (int k = kHubLadder - 1; k >= 0; k--) {
      above += dev->hub_hist[k];
      if (above * words0 > budget_words) break;
      H = hub_ladder(k);
    }
    s_H = H;
    if (blockIdx.x == 0) dev->hub_H = H;
  }
  __syncthreads();
  const int32_t H = s_H;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_b;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t h = -1;
    if (b_ptr[v + 1] - b_ptr[v] > H) {
      h = atomicAdd(&dev->nhub, 1);
      hub_net[h] = (int32_t)v;
    }
    hub_id[v] = h;
  }
}

// Bitmap of the published colors of each hub net (one CTA per net, the
// bitmap assembled in shared memory, written out whole).
__global__ void __launch_bounds__(256) k_hub_build(const int32_t *__restrict__ b_ptr,
                                                   const int32_t *__restrict__ nc,
                                                   const int32_t *__restrict__ hub_net,
                                                   int32_t nhub, int32_t words,
                                                   uint32_t *__restrict__ nbm) {
  extern __shared__ __align__(16) uint32_t s_bm[];
  const int32_t lim = words * 32;
  for (int32_t h = blockIdx.x; h < nhub; h += gridDim.x) {
    for (int32_t x = threadIdx.x; x < words; x += blockDim.x) s_bm[x] = 0u;
    __syncthreads();
    const int32_t v = hub_net[h];
    const int32_t beg = b_ptr[v], end = b_ptr[v + 1];
    // four members per thread and step, their loads issued together
    for (int32_t f0 = beg + threadIdx.x; f0 < end; f0 += 4 * blockDim.x) {
      int32_t c[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int32_t f = f0 + q * (int32_t)blockDim.x;
        c[q] = f < end ? nc[f] : -1;
      }
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (c[q] >= 0 && c[q] < lim) atomicOr(&s_bm[c[q] >> 5], 1u << (c[q] & 31));
    }
    __syncthreads();
    for (int32_t x = threadIdx.x; x < words; x += blockDim.x)
      nbm[(int64_t)h * words + x] = s_bm[x];
    __syncthreads();
  }
}

int launch_hub_select(const int32_t *b_ptr, int32_t n_b, int32_t C, int32_t Q,
                      int64_t budget_words, int32_t *hub_id, int32_t *hub_net, DevScalars *dev,
                      int sms, cudaStream_t s) {
  if (n_b <= 0) return 0;
  long long grid = div_up(n_b, 256);
  if (grid > (long long)sms * 8) grid = (long long)sms * 8;
  k_hub_select<<<(int)grid, 256, 0, s>>>(b_ptr, n_b, C, Q, budget_words, hub_id, hub_net, dev);
  return 1;
}

int launch_hub_build(const int32_t *b_ptr, const int32_t *nc, const int32_t *hub_net,
                     int32_t nhub, int32_t words, uint32_t *nbm, int sms, cudaStream_t s) {
  if (nhub <= 0) return 0;
  if (allow_dynamic_smem(k_hub_build) != cudaSuccess) return 0;  // reported by the caller
  const int grid = nhub < sms * 8 ? nhub : sms * 8;  // one resident set at 256 threads
  k_hub_build<<<grid, 256, (size_t)words * 4, s>>>(b_ptr, nc, hub_net, nhub, words, nbm);
  return 1;
}

}  // namespace bgpc
