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

// ------------------------------------------------ byte-map searches (CTA)
// bytes[x] != 0 means color x is forbidden.  `lim` is a multiple of 16.

// Smallest free x with p <= x < lim, or lim.
template <int NT>
__device__ int32_t bytes_first_free_up(const uint8_t *bytes, int32_t p, int32_t lim,
                                       int32_t *red) {
  for (int32_t base = p & ~15; base < lim; base += NT * 16) {
    int32_t x0 = base + (int32_t)threadIdx.x * 16;
    int32_t found = INT32_MAX;
    if (x0 < lim) {
      uint4 v = *reinterpret_cast<const uint4 *>(bytes + x0);
      uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        int32_t lo = x0 + 4 * q;
        uint32_t z = __vcmpeq4(wv[q], 0u);
        if (lo + 4 <= p) z = 0;
        else if (lo < p) z &= ~((1u << (8 * (p - lo))) - 1u);
        if (z && found == INT32_MAX) found = lo + ((__ffs(z) - 1) >> 3);
      }
    }
    found = block_min<NT>(found, red);
    if (found != INT32_MAX) return found;
  }
  return lim;
}

// Largest free x with 0 <= x <= p, or -1.
template <int NT>
__device__ int32_t bytes_last_free_down(const uint8_t *bytes, int32_t p, int32_t *red) {
  for (int32_t top = p; top >= 0; top -= NT * 16) {
    int32_t hi = top - 16 * (int32_t)threadIdx.x, lo = max(hi - 15, 0);
    int32_t found = -1;
    for (int32_t x = hi; x >= lo; x--)
      if (bytes[x] == 0) { found = x; break; }
    found = block_max<NT>(found, red);
    if (found >= 0) return found;
  }
  return -1;
}

// The k-th (0-based) free color counting down from top, or -1.
template <int NT>
__device__ int32_t bytes_kth_free_down(const uint8_t *bytes, int32_t top, int32_t k,
                                       int32_t *red) {
  int32_t remaining = k;
  for (int32_t t0 = top; t0 >= 0; t0 -= NT * 16) {
    int32_t hi = t0 - 16 * (int32_t)threadIdx.x, lo = max(hi - 15, 0);
    int32_t cnt = 0;
    for (int32_t x = hi; x >= lo; x--) cnt += (bytes[x] == 0);
    int32_t total;
    int32_t excl = block_excl_scan<NT>(cnt, red, &total);
    if (remaining < total) {
      int32_t res = -1;
      if (cnt > 0 && excl <= remaining && remaining < excl + cnt) {
        int32_t r = remaining - excl;
        for (int32_t x = hi; x >= lo; x--) {
          if (bytes[x] == 0) {
            if (r == 0) { res = x; break; }
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

// ------------------------------------------------------------------ kernel

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
  __shared__ int32_t s_state[4];  // col_max, col_next, npairs
  extern __shared__ __align__(16) uint8_t s_bytes[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t gm = a.dev->gmax;
  const int32_t bound = max(max(gm, a.maxnet - 1), 0) + a.C;  // every color of this wave <= bound
  const int32_t need = ((bound + 1) + 15) & ~15;
  if (need > a.cbw) {
    if (tid == 0 && blockIdx.x == 0) atomicOr(a.err, ERR_COLOR);
    return;
  }
  const bool small_ok = (POLICY == BGPC_FF) || (bound < kSmallWindow);
  const int32_t col_max0 = max(gm, 0);

  for (int32_t t = (int32_t)blockIdx.x; t < a.nchunks; t += (int32_t)gridDim.x) {
    const int32_t j = a.chunks[t];
    const int32_t p0 = j * a.C;
    const int32_t n = min(a.C, a.m - p0);

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

    // ---- step 1: which vertices take the small path; their pair offsets
    if (warp == 0) {
      const int i0 = lane, i1 = lane + 32;
      bool c0 = small_ok && i0 < n && s_d2[i0] <= kSmallD2;
      bool c1 = small_ok && i1 < n && s_d2[i1] <= kSmallD2;
      int32_t d0 = c0 ? s_deg[i0] : 0, d1 = c1 ? s_deg[i1] : 0;
      int32_t inc0 = warp_incl_scan(d0);
      int32_t tot0 = __shfl_sync(kFull, inc0, 31);
      int32_t inc1 = warp_incl_scan(d1) + tot0;
      bool sm0 = c0 && inc0 <= kPairCap;
      bool sm1 = c1 && inc1 <= kPairCap;
      // non-small vertices get zero width in the pair prefix
      if (!sm0) d0 = 0;
      if (!sm1) d1 = 0;
      inc0 = warp_incl_scan(d0);
      tot0 = __shfl_sync(kFull, inc0, 31);
      inc1 = warp_incl_scan(d1) + tot0;
      s_ppi[i0] = inc0;
      if (i1 < kMaxChunk) s_ppi[i1] = inc1;
      unsigned lg0 = __ballot_sync(kFull, i0 < n && !sm0);
      unsigned lg1 = __ballot_sync(kFull, i1 < n && !sm1);
      unsigned long long large = ((unsigned long long)lg1 << 32) | lg0;
      unsigned long long m0 = large >> i0;
      s_next[i0] = m0 ? min(i0 + __ffsll((long long)m0) - 1, n) : n;
      unsigned long long m1 = (i1 < 64) ? (large >> i1) : 0ull;
      s_next[i1] = m1 ? min(i1 + __ffsll((long long)m1) - 1, n) : n;
      if (lane == 31) s_state[2] = inc1;
    }
    __syncthreads();

    // ---- step 2: (vertex, net) pairs of the small vertices
    const int32_t P = s_state[2];
    for (int32_t t = tid; t < P; t += NT) {
      int32_t lo = 0, hi = n - 1;  // smallest i with s_ppi[i] > t
      while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (s_ppi[mid] > t) hi = mid; else lo = mid + 1;
      }
      const int32_t i = lo;
      const int32_t width = (i == 0) ? s_ppi[0] : s_ppi[i] - s_ppi[i - 1];
      const int32_t tl = t - (s_ppi[i] - width);
      const int32_t v = a.a_idx[s_ab[i] + tl];
      const int32_t bp = a.b_ptr[v];
      s_pstart[t] = bp;
      s_poff[t] = a.b_ptr[v + 1] - bp;
      s_pvert[t] = (uint8_t)i;
    }
    __syncthreads();

    // ---- step 3: exclusive scan of the pair sizes
    {
      constexpr int PER = (kPairCap + NT - 1) / NT;
      int32_t loc[PER];
      int32_t sum = 0;
#pragma unroll
      for (int q = 0; q < PER; q++) {
        int32_t t = tid * PER + q;
        loc[q] = (t < P) ? s_poff[t] : 0;
        sum += loc[q];
      }
      int32_t total;
      int32_t ex = block_excl_scan<NT>(sum, s_red, &total);
#pragma unroll
      for (int q = 0; q < PER; q++) {
        int32_t t = tid * PER + q;
        if (t < P) s_poff[t] = ex;
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

    // ---- phase B: resolve the chunk's vertices in order
    int32_t i = 0;
    while (i < n) {
      const int32_t L = s_next[i];
      if (warp == 0 && i < L) {
        int32_t col_max = s_state[0], col_next = s_state[1];
        for (int32_t ii = i; ii < L; ii++) {
          const unsigned long long am = s_adj[ii];
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
          int32_t x = -1;
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
          col_max = max(col_max, x);
          if (POLICY == BGPC_B2) col_next = min(x + 1, col_max / 3 + 1);
          if (POLICY == BGPC_B2X) col_next = max(x + 1, col_max / 3 + 1);
          if (lane == 0) s_col[ii] = x;
          __syncwarp();
        }
        if (lane == 0) { s_state[0] = col_max; s_state[1] = col_next; }
      }
      __syncthreads();
      if (L < n) {
        // ---- large vertex: CTA-wide gather into the byte map
        for (int32_t x = tid * 16; x < need; x += NT * 16)
          *reinterpret_cast<uint4 *>(s_bytes + x) = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        const int32_t ab = s_ab[L], deg = s_deg[L];
        int bad = 0;
        for (int32_t t = warp; t < deg; t += NW) {
          const int32_t v = a.a_idx[ab + t];
          const int32_t beg = a.b_ptr[v], end = a.b_ptr[v + 1];
          for (int32_t e0 = beg + lane; e0 < end; e0 += 128) {
            int32_t val[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
              int32_t e = e0 + 32 * q;
              val[q] = (e < end) ? a.nc[e] : INT32_MIN;
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
              const int32_t x = val[q];
              if (x == INT32_MIN) continue;
              if (x >= 0) {
                if (x < need) s_bytes[x] = 1; else bad = 1;
              } else {
                const int32_t rel = (-2 - x) - p0;
                if (rel >= 0 && rel < L) atomicOr(&s_adj[L], 1ull << rel);
              }
            }
          }
        }
        if (bad) atomicOr(a.err, ERR_COLOR);
        __syncthreads();
        if (tid < L && ((s_adj[L] >> tid) & 1ull)) s_bytes[s_col[tid]] = 1;
        __syncthreads();
        const int32_t col_max = s_state[0], col_next = s_state[1];
        int32_t x = -1;
        const int32_t so = s_sown[L];
        if (so > a.T) x = bytes_kth_free_down<NT>(s_bytes, so - 1, s_k[L], s_red);
        if (x < 0) {
          if (POLICY == BGPC_B1) {
            if ((s_w[L] & 1) == 0) {
              x = bytes_last_free_down<NT>(s_bytes, col_max, s_red);
              if (x < 0) x = bytes_first_free_up<NT>(s_bytes, col_max + 1, need, s_red);
            } else {
              x = bytes_first_free_up<NT>(s_bytes, 0, need, s_red);
            }
          } else if (POLICY == BGPC_B2 || POLICY == BGPC_B2X) {
            x = bytes_first_free_up<NT>(s_bytes, col_next, need, s_red);
            if (x > col_max) x = bytes_first_free_up<NT>(s_bytes, 0, need, s_red);
          } else {
            x = bytes_first_free_up<NT>(s_bytes, 0, need, s_red);
          }
        }
        if (tid == 0) {
          if (x < 0 || x >= need) { atomicOr(a.err, ERR_COLOR); x = 0; }
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

// Publish: colors of the wave's positions go to c[] and to every CSC entry
// of their edges (nc), and the running max color is updated.
__global__ void k_publish(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ tpos,
                          const int32_t *__restrict__ W, const int32_t *__restrict__ stage,
                          const int32_t *__restrict__ chunks, int32_t nchunks, int32_t C,
                          int32_t m, int32_t *__restrict__ nc, int32_t *__restrict__ colors,
                          DevScalars *dev) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t mx = -1;
  const int64_t total = (int64_t)nchunks * C;
  for (int64_t t = warp; t < total; t += nwarps) {
    const int64_t p = (int64_t)chunks[t / C] * C + t % C;
    if (p >= m) continue;
    const int32_t w = W[p], col = stage[p];
    const int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    for (int32_t i = beg + lane; i < end; i += 32) nc[tpos[i]] = col;
    if (lane == 0) colors[w] = col;
    mx = max(mx, col);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (lane == 0 && mx >= 0) atomicMax(&dev->gmax, mx);
}

template <int POLICY, int NT>
cudaError_t launch_policy(const WaveArgs &a, int sms, int smem_optin, cudaStream_t s) {
  auto kern = k_color_wave<POLICY, NT>;
  size_t smem = (size_t)a.cbw;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * sms;
  if (grid > a.nchunks) grid = a.nchunks;
  (void)smem_optin;
  kern<<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t wave_smem_bytes(int32_t cbw) { return (size_t)cbw; }

int32_t wave_max_cbw(int smem_optin) {
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, k_color_wave<BGPC_FF, 256>) == cudaSuccess) stat = fa.sharedSizeBytes;
  else cudaGetLastError();
  long long room = (long long)smem_optin - (long long)stat - 1024;
  return room > 0 ? (int32_t)(room & ~15LL) : 0;
}

cudaError_t launch_color_wave(int policy, const WaveArgs &a, int sms, int smem_optin,
                              cudaStream_t s) {
  if (a.nchunks <= 0) return cudaSuccess;
  switch (policy) {
    case BGPC_B1: return launch_policy<BGPC_B1, 256>(a, sms, smem_optin, s);
    case BGPC_B2: return launch_policy<BGPC_B2, 256>(a, sms, smem_optin, s);
    case BGPC_B2X: return launch_policy<BGPC_B2X, 256>(a, sms, smem_optin, s);
    default: return launch_policy<BGPC_FF, 256>(a, sms, smem_optin, s);
  }
}

int launch_publish(const int32_t *a_ptr, const int32_t *tpos, const int32_t *W,
                   const int32_t *stage, const int32_t *chunks, int32_t nchunks, int32_t C,
                   int32_t m, int32_t *nc, int32_t *colors, DevScalars *dev, int sms,
                   cudaStream_t s) {
  if (nchunks <= 0) return 0;
  long long warps = (long long)nchunks * C;
  long long grid = div_up(warps * 32, 256);
  if (grid > (long long)sms * 16) grid = (long long)sms * 16;
  k_publish<<<(int)grid, 256, 0, s>>>(a_ptr, tpos, W, stage, chunks, nchunks, C, m, nc, colors,
                                      dev);
  return 1;
}

}  // namespace bgpc
