// Learned vertex order: per-vertex features of the bipartite graph, a small
// MLP (forward pass, gradient of the mean squared error, Adam step) and the
// rank of a score vector.  The paper colors in a given vertex order and
// compares static orders (Sec. VI, Table II); a learned score replaces the
// static heuristic, and the rank it induces is passed as bgpc_opts_t.rank.
//
// All arithmetic is float32 on CUDA cores: the MLP is 8 -> 64 -> 64 -> 1, a
// few kFLOP per vertex, negligible next to one coloring sweep, so it does not
// pay to reshape it for the tensor cores.  The gradient is reduced in a fixed
// order (fixed grid, tile t always on block t mod kGradBlocks, block partials
// summed in block order), so it does not depend on timing or on the GPU.
#include <cuda_bf16.h>
#include <math.h>

#include "bgpc_internal.cuh"

using namespace bgpc;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNT = 256;
constexpr int kIn = BGPC_MLP_IN, kHid = BGPC_MLP_HIDDEN, kP = BGPC_MLP_PARAMS;
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 576, kOffB2 = 4672, kOffW3 = 4736,
              kOffB3 = 4800;
static_assert(kOffB1 == kOffW1 + kHid * kIn && kOffW2 == kOffB1 + kHid &&
                  kOffB2 == kOffW2 + kHid * kHid && kOffW3 == kOffB2 + kHid &&
                  kOffB3 == kOffW3 + kHid && kOffB3 + 1 == kP,
              "parameter packing");
constexpr int kPpad = (kP + 3) & ~3;
constexpr int kGradBlocks = 256;  // fixed grid of the gradient kernel
constexpr int kTile = kNT;        // vertices per gradient tile, one per thread
constexpr int kRow = kHid + 1;    // padded activation row in shared memory
constexpr int kOwn = (kP + kNT - 1) / kNT;  // parameters accumulated by each thread
constexpr int kPartStride = kP + 1;         // block partial: 4801 gradients + loss
constexpr size_t kGradSmem =
    sizeof(float) * ((size_t)kPpad + (size_t)kTile * kIn + 2 * (size_t)kTile * kRow + kTile);
constexpr int kScanNT = 1024, kScanPer = 4, kScanTile = kScanNT * kScanPer;

struct Guard {
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

#define CU(call)                                                             \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      cudaGetLastError();                                                    \
      return e_ == cudaErrorMemoryAllocation ? BGPC_ENOMEM : BGPC_ECUDA;     \
    }                                                                        \
  } while (0)

// ------------------------------------------------------------- features
// One warp per vertex; the lanes stride over its nets.
__global__ void k_features(const int32_t *__restrict__ a_ptr, const int32_t *__restrict__ a_idx,
                           const int32_t *__restrict__ b_ptr, int32_t n_a, int32_t T,
                           float *__restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_a; w += nwarps) {
    const int32_t beg = a_ptr[w], end = a_ptr[w + 1];
    long long cnt = 0, sum = 0, sum1 = 0, sq = 0, nbig = 0;
    int32_t mx = 0, mn = INT32_MAX;
    for (int32_t i = beg + lane; i < end; i += 32) {
      const int32_t v = a_idx[i];
      const int32_t s = b_ptr[v + 1] - b_ptr[v];
      cnt++;
      sum += s;
      sum1 += s - 1;
      sq += (long long)s * s;
      nbig += (s > T);
      mx = max(mx, s);
      mn = min(mn, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(kFull, cnt, o);
      sum += __shfl_xor_sync(kFull, sum, o);
      sum1 += __shfl_xor_sync(kFull, sum1, o);
      sq += __shfl_xor_sync(kFull, sq, o);
      nbig += __shfl_xor_sync(kFull, nbig, o);
      mx = max(mx, __shfl_xor_sync(kFull, mx, o));
      mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    }
    if (lane < kIn) {
      float out = 0.f;
      if (cnt > 0) {
        double raw;
        switch (lane) {
          case 0: raw = (double)cnt; break;
          case 1: raw = (double)sum / (double)cnt; break;
          case 2: raw = (double)mx; break;
          case 3: raw = (double)sum; break;
          case 4: raw = (double)sum1; break;
          case 5: raw = (double)mn; break;
          case 6: raw = (double)nbig; break;
          default: raw = (double)sq / (double)sum; break;
        }
        out = (float)log1p(raw);
      }
      X[w * kIn + lane] = out;
    }
  }
}

// ------------------------------------------------------------- bfloat16
__device__ __forceinline__ uint16_t to_bf16(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float from_bf16(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__global__ void k_mlp_sync(const float *__restrict__ w, uint16_t *__restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kP) wb[p] = to_bf16(w[p]);
}

__device__ __forceinline__ void load_weights(const uint16_t *__restrict__ wb, float *Ws) {
  for (int p = threadIdx.x; p < kP; p += blockDim.x) Ws[p] = from_bf16(wb[p]);
}

// h1 = relu(W1 x + b1) for one vertex, into registers.
__device__ __forceinline__ void layer1(const float *Ws, const float (&x)[kIn], float (&h1)[kHid]) {
#pragma unroll
  for (int o = 0; o < kHid; o++) {
    float z = Ws[kOffB1 + o];
#pragma unroll
    for (int k = 0; k < kIn; k++) z = fmaf(Ws[kOffW1 + o * kIn + k], x[k], z);
    h1[o] = fmaxf(z, 0.f);
  }
}

// ------------------------------------------------------------- forward
// One thread per vertex; the bfloat16 weights are widened into shared memory.
__global__ void __launch_bounds__(kNT) k_mlp_forward(const uint16_t *__restrict__ wb,
                                                     const float *__restrict__ X, int32_t n,
                                                     float *__restrict__ score) {
  __shared__ float Ws[kPpad];
  load_weights(wb, Ws);
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    // keep the shared weights out of registers across vertices (the compiler
    // would otherwise hoist all 512 W1 loads out of this loop and spill)
    asm volatile("" ::: "memory");
    float x[kIn], h1[kHid];
#pragma unroll
    for (int k = 0; k < kIn; k++) x[k] = X[v * kIn + k];
    layer1(Ws, x, h1);
    float s = Ws[kOffB3];
#pragma unroll 1
    for (int o = 0; o < kHid; o++) {
      float z = Ws[kOffB2 + o];
#pragma unroll
      for (int i = 0; i < kHid; i++) z = fmaf(Ws[kOffW2 + o * kHid + i], h1[i], z);
      s = fmaf(Ws[kOffW3 + o], fmaxf(z, 0.f), s);
    }
    score[v] = s;
  }
}

// ------------------------------------------------------------- gradient
// Block b handles the tiles b, b + kGradBlocks, ... of kTile vertices.  Per
// tile: (a) every thread runs the forward pass of its vertex and keeps x, h1,
// h2 and dL/ds in shared memory; (c) every thread accumulates the gradients
// of the W2, b2, W3, b3 entries it owns (parameter p belongs to thread
// p mod kNT) over the tile; (d) every thread backpropagates its vertex to
// dL/dz1 (over h2's storage); (e) W1 and b1 entries as in (c).  The block's
// sums go to part[b]; the loss sum of (s - y)^2 to part[b][kP].
__global__ void __launch_bounds__(kNT) k_mlp_grad(const uint16_t *__restrict__ wb,
                                                  const float *__restrict__ X,
                                                  const float *__restrict__ y, int32_t n,
                                                  float ds_scale, float *__restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  float *Ws = sm;
  float *Xs = Ws + kPpad;
  float *H1 = Xs + kTile * kIn;
  float *H2 = H1 + kTile * kRow;  // h2, then dL/dz1
  float *DS = H2 + kTile * kRow;
  __shared__ float red[kNT / 32];
  const int tid = threadIdx.x;
  load_weights(wb, Ws);
  __syncthreads();
  float acc[kOwn];
#pragma unroll
  for (int j = 0; j < kOwn; j++) acc[j] = 0.f;
  float lacc = 0.f;
  const int64_t ntiles = ((int64_t)n + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // (a) forward of vertex v
    const int64_t v = tile * kTile + tid;
    const bool live = v < n;
    float x[kIn], h1[kHid];
#pragma unroll
    for (int k = 0; k < kIn; k++) {
      x[k] = live ? X[v * kIn + k] : 0.f;
      Xs[tid * kIn + k] = x[k];
    }
    layer1(Ws, x, h1);
#pragma unroll
    for (int o = 0; o < kHid; o++) H1[tid * kRow + o] = h1[o];
    float s = Ws[kOffB3];
#pragma unroll 1
    for (int o = 0; o < kHid; o++) {
      float z = Ws[kOffB2 + o];
#pragma unroll
      for (int i = 0; i < kHid; i++) z = fmaf(Ws[kOffW2 + o * kHid + i], h1[i], z);
      const float h2 = fmaxf(z, 0.f);
      H2[tid * kRow + o] = h2;
      s = fmaf(Ws[kOffW3 + o], h2, s);
    }
    const float d = live ? s - y[v] : 0.f;
    lacc = fmaf(d, d, lacc);
    DS[tid] = d * ds_scale;
    __syncthreads();
    // (c) W2, b2, W3, b3
#pragma unroll
    for (int j = 0; j < kOwn; j++) {
      const int p = tid + j * kNT;
      if (p >= kOffW2 && p < kOffB2) {
        const int o = (p - kOffW2) / kHid, i = (p - kOffW2) % kHid;
        float t = 0.f;
        for (int u = 0; u < kTile; u++)
          if (H2[u * kRow + o] > 0.f) t = fmaf(DS[u], H1[u * kRow + i], t);
        acc[j] = fmaf(Ws[kOffW3 + o], t, acc[j]);
      } else if (p >= kOffB2 && p < kOffW3) {
        const int o = p - kOffB2;
        float t = 0.f;
        for (int u = 0; u < kTile; u++)
          if (H2[u * kRow + o] > 0.f) t += DS[u];
        acc[j] = fmaf(Ws[kOffW3 + o], t, acc[j]);
      } else if (p >= kOffW3 && p < kOffB3) {
        const int i = p - kOffW3;
        float t = 0.f;
        for (int u = 0; u < kTile; u++) t = fmaf(DS[u], H2[u * kRow + i], t);
        acc[j] += t;
      } else if (p == kOffB3) {
        float t = 0.f;
        for (int u = 0; u < kTile; u++) t += DS[u];
        acc[j] += t;
      }
    }
    // (d) dL/dz1 of vertex tid (its dL/dz2 first, from its own h2 row)
    float dz2[kHid];
#pragma unroll
    for (int o = 0; o < kHid; o++)
      dz2[o] = (H2[tid * kRow + o] > 0.f) ? DS[tid] * Ws[kOffW3 + o] : 0.f;
    __syncthreads();  // every thread is done reading h2
#pragma unroll 1
    for (int i = 0; i < kHid; i++) {
      float t = 0.f;
#pragma unroll
      for (int o = 0; o < kHid; o++) t = fmaf(Ws[kOffW2 + o * kHid + i], dz2[o], t);
      H2[tid * kRow + i] = (H1[tid * kRow + i] > 0.f) ? t : 0.f;
    }
    __syncthreads();
    // (e) W1, b1
#pragma unroll
    for (int j = 0; j < kOwn; j++) {
      const int p = tid + j * kNT;
      if (p < kOffB1) {
        const int o = p / kIn, k = p % kIn;
        float t = 0.f;
        for (int u = 0; u < kTile; u++) t = fmaf(H2[u * kRow + o], Xs[u * kIn + k], t);
        acc[j] += t;
      } else if (p < kOffW2) {
        const int o = p - kOffB1;
        float t = 0.f;
        for (int u = 0; u < kTile; u++) t += H2[u * kRow + o];
        acc[j] += t;
      }
    }
    __syncthreads();  // the next tile overwrites Xs, H1, H2, DS
  }
  float *out = part + (size_t)blockIdx.x * kPartStride;
#pragma unroll
  for (int j = 0; j < kOwn; j++) {
    const int p = tid + j * kNT;
    if (p < kP) out[p] = acc[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(kFull, lacc, o);
  if ((tid & 31) == 0) red[tid >> 5] = lacc;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int i = 0; i < kNT / 32; i++) t += red[i];
    out[kP] = t;
  }
}

// grad[p] = sum over blocks of part[b][p] (block order); loss = sum / n.
__global__ void k_mlp_reduce(const float *__restrict__ part, float inv_n,
                             float *__restrict__ grad, float *__restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kP) return;
  float t = 0.f;
  for (int b = 0; b < kGradBlocks; b++) t += part[(size_t)b * kPartStride + p];
  if (p < kP) grad[p] = t;
  else *loss = t * inv_n;
}

__global__ void k_mlp_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                           uint16_t *__restrict__ wb, const float *__restrict__ g, float lr,
                           float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kP) return;
  const float gp = g[p];
  const float mp = 0.9f * m[p] + 0.1f * gp;
  const float vp = 0.999f * v[p] + 0.001f * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float wn = w[p] - lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
  w[p] = wn;
  wb[p] = to_bf16(wn);
}

// ------------------------------------------------------------- rank
// Ascending key = decreasing score; -0.0 and +0.0 map to the same key.
__device__ __forceinline__ uint32_t desc_key(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u << 1) == 0u) u = 0u;
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ~u;
}

__global__ void k_rank_init(const float *__restrict__ score, int32_t n, uint32_t *__restrict__ key,
                            int32_t *__restrict__ val, int32_t *err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float f = score[i];
    if (f != f) atomicOr(err, ERR_RANGE);
    key[i] = desc_key(f);
    val[i] = (int32_t)i;
  }
}

// Digit counts of one tile of kNT keys: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kNT) k_radix_hist(const uint32_t *__restrict__ key, int32_t n,
                                                    int shift, int32_t ntiles,
                                                    int32_t *__restrict__ hist) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x;
  if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: an element goes to the start of its digit in this tile
// (scanned counts) plus the number of equal digits before it in the tile
// (earlier warps, then earlier lanes of its warp).
__global__ void __launch_bounds__(kNT) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                       const int32_t *__restrict__ vin, int32_t n,
                                                       int shift, int32_t ntiles,
                                                       const int32_t *__restrict__ off,
                                                       uint32_t *__restrict__ kout,
                                                       int32_t *__restrict__ vout) {
  constexpr int NW = kNT / 32;
  __shared__ int32_t wc[NW][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < NW * 256; i += kNT) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x;
  const bool live = i < n;
  uint32_t k = 0u;
  int32_t val = 0;
  int d = -1 - lane;  // distinct dummies for lanes past the end
  if (live) {
    k = kin[i];
    val = vin[i];
    d = (int)((k >> shift) & 255u);
  }
  const unsigned peers = __match_any_sync(kFull, d);
  const int before = __popc(peers & ((1u << lane) - 1u));
  if (live && before == 0) wc[warp][d] = __popc(peers);
  __syncthreads();
  {  // exclusive prefix over the warps, one thread per digit
    int32_t run = 0;
    for (int w = 0; w < NW; w++) {
      const int32_t t = wc[w][threadIdx.x];
      wc[w][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
  if (live) {
    const int64_t pos = (int64_t)off[(int64_t)d * ntiles + blockIdx.x] + wc[warp][d] + before;
    kout[pos] = k;
    vout[pos] = val;
  }
}

__global__ void k_rank_write(const int32_t *__restrict__ val, int32_t n, int32_t *__restrict__ rank) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    rank[val[p]] = (int32_t)p;
}

// ---- exclusive scan of int32 (tile scan, scan of tile sums, add)
template <int NT>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *red, int32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) red[warp] = inc;
  __syncthreads();
  int32_t before = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < NT / 32; i++) {
    const int32_t r = red[i];
    before += (i < warp) ? r : 0;
    tot += r;
  }
  __syncthreads();
  *total = tot;
  return before + inc - v;
}

__global__ void __launch_bounds__(kScanNT) k_scan_tiles(int32_t *__restrict__ a, int64_t len,
                                                        int32_t *__restrict__ sums) {
  __shared__ int32_t red[kScanNT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t x[kScanPer];
  int32_t c = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    x[q] = (base + q < len) ? a[base + q] : 0;
    c += x[q];
  }
  int32_t total;
  int32_t ex = block_excl_scan<kScanNT>(c, red, &total);
#pragma unroll
  for (int q = 0; q < kScanPer; q++) {
    if (base + q < len) a[base + q] = ex;
    ex += x[q];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanNT) k_scan_sums(int32_t *__restrict__ sums, int32_t nb) {
  __shared__ int32_t red[kScanNT / 32];
  int32_t carry = 0;
  for (int32_t b0 = 0; b0 < nb; b0 += kScanNT) {
    const int32_t b = b0 + (int32_t)threadIdx.x;
    const int32_t x = (b < nb) ? sums[b] : 0;
    int32_t total;
    const int32_t ex = block_excl_scan<kScanNT>(x, red, &total);
    if (b < nb) sums[b] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanNT) k_scan_add(int32_t *__restrict__ a, int64_t len,
                                                      const int32_t *__restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  const int32_t add = sums[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kScanPer; q++)
    if (base + q < len) a[base + q] += add;
}

int grid_for(int64_t items, int per_block, int cap) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

bool bad_graph(const bgpc_graph_t *g) {
  if (!g || g->n_a < 0 || g->n_b < 0 || g->nnz < 0) return true;
  if (g->n_a > 0 && (!g->a_ptr || !g->b_ptr)) return true;
  if (g->nnz > 0 && (!g->a_idx || !g->b_idx)) return true;
  return false;
}

bool bad_mlp(const bgpc_mlp_t *m) { return !m || !m->w || !m->w_bf16; }

int grad_impl(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, const float *X, const float *y, int32_t n,
              float *grad, float *loss, cudaStream_t s) {
  if ((int64_t)kGradSmem > (int64_t)ctx->smem_optin) return BGPC_EINVAL;
  CU(grow(ctx->mpart, (size_t)kGradBlocks * kPartStride + 4));
  float *part = ctx->mpart.p;
  float *dloss = part + (size_t)kGradBlocks * kPartStride;
  CU(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)kGradSmem));
  k_mlp_grad<<<kGradBlocks, kNT, kGradSmem, s>>>(mlp->w_bf16, X, y, n, 2.0f / (float)n, part);
  k_mlp_reduce<<<(kP + 1 + kNT - 1) / kNT, kNT, 0, s>>>(part, 1.0f / (float)n, grad, dloss);
  CU(cudaGetLastError());
  if (loss) {
    CU(cudaMemcpyAsync(loss, dloss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
  }
  return BGPC_OK;
}

int adam_impl(bgpc_mlp_t *mlp, const float *grad, float lr, cudaStream_t s) {
  const int64_t t = mlp->step + 1;
  const double c1 = 1.0 / (1.0 - pow(0.9, (double)t));
  const double c2 = 1.0 / (1.0 - pow(0.999, (double)t));
  k_mlp_adam<<<(kP + kNT - 1) / kNT, kNT, 0, s>>>(mlp->w, mlp->adam_m, mlp->adam_v, mlp->w_bf16,
                                                  grad, lr, (float)c1, (float)c2);
  CU(cudaGetLastError());
  mlp->step = t;
  return BGPC_OK;
}

}  // namespace

// Exclusive scan of a[0, len) in place (sums: ceil(len / 4096) scratch ints).
int bgpc::launch_excl_scan(int32_t *a, int64_t len, int32_t *sums, cudaStream_t s) {
  if (len <= 0) return 0;
  const int32_t nsb = (int32_t)((len + kScanTile - 1) / kScanTile);
  k_scan_tiles<<<nsb, kScanNT, 0, s>>>(a, len, sums);
  k_scan_sums<<<1, kScanNT, 0, s>>>(sums, nsb);
  k_scan_add<<<nsb, kScanNT, 0, s>>>(a, len, sums);
  return 3;
}

extern "C" {

int bgpc_features(bgpc_ctx_t *ctx, const bgpc_graph_t *g, int32_t big_net, float *X,
                  void *stream) {
  if (!ctx || bad_graph(g) || big_net < 0) return BGPC_EINVAL;
  if (g->n_a == 0) return BGPC_OK;
  if (!X) return BGPC_EINVAL;
  Guard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  k_features<<<grid_for((int64_t)g->n_a * 32, kNT, ctx->num_sms * 16), kNT, 0, s>>>(
      g->a_ptr, g->a_idx, g->b_ptr, g->n_a, big_net, X);
  CU(cudaGetLastError());
  return BGPC_OK;
}

int bgpc_mlp_sync(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, void *stream) {
  if (!ctx || bad_mlp(mlp)) return BGPC_EINVAL;
  Guard guard(ctx->device);
  k_mlp_sync<<<(kP + kNT - 1) / kNT, kNT, 0, (cudaStream_t)stream>>>(mlp->w, mlp->w_bf16);
  CU(cudaGetLastError());
  return BGPC_OK;
}

int bgpc_mlp_forward(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, const float *X, int32_t n,
                     float *score, void *stream) {
  if (!ctx || !mlp || !mlp->w_bf16 || n < 0) return BGPC_EINVAL;
  if (n == 0) return BGPC_OK;
  if (!X || !score) return BGPC_EINVAL;
  Guard guard(ctx->device);
  k_mlp_forward<<<grid_for(n, kNT, ctx->num_sms * 8), kNT, 0, (cudaStream_t)stream>>>(
      mlp->w_bf16, X, n, score);
  CU(cudaGetLastError());
  return BGPC_OK;
}

int bgpc_mlp_grad(bgpc_ctx_t *ctx, const bgpc_mlp_t *mlp, const float *X, const float *y,
                  int32_t n, float *grad, float *loss, void *stream) {
  if (!ctx || !mlp || !mlp->w_bf16 || n < 1 || !X || !y || !grad) return BGPC_EINVAL;
  Guard guard(ctx->device);
  return grad_impl(ctx, mlp, X, y, n, grad, loss, (cudaStream_t)stream);
}

int bgpc_mlp_adam(bgpc_ctx_t *ctx, bgpc_mlp_t *mlp, const float *grad, float lr, void *stream) {
  if (!ctx || bad_mlp(mlp) || !mlp->adam_m || !mlp->adam_v || !grad || mlp->step < 0)
    return BGPC_EINVAL;
  Guard guard(ctx->device);
  return adam_impl(mlp, grad, lr, (cudaStream_t)stream);
}

int bgpc_mlp_train_step(bgpc_ctx_t *ctx, bgpc_mlp_t *mlp, const float *X, const float *y,
                        int32_t n, float lr, float *loss, void *stream) {
  if (!ctx || bad_mlp(mlp) || !mlp->adam_m || !mlp->adam_v || n < 1 || !X || !y ||
      mlp->step < 0)
    return BGPC_EINVAL;
  Guard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  CU(grow(ctx->mgrad, (size_t)kP));
  int rc = grad_impl(ctx, mlp, X, y, n, ctx->mgrad.p, loss, s);
  if (rc) return rc;
  return adam_impl(mlp, ctx->mgrad.p, lr, s);
}

int bgpc_rank_from_scores(bgpc_ctx_t *ctx, const float *score, int32_t n, int32_t *rank,
                          void *stream) {
  if (!ctx || n < 0) return BGPC_EINVAL;
  if (n == 0) return BGPC_OK;
  if (!score || !rank) return BGPC_EINVAL;
  Guard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t ntiles = (int32_t)(((int64_t)n + kNT - 1) / kNT);
  const int64_t hlen = (int64_t)ntiles * 256;
  const int32_t nsb = (int32_t)((hlen + kScanTile - 1) / kScanTile);
  CU(grow(ctx->rkey0, (size_t)n));
  CU(grow(ctx->rkey1, (size_t)n));
  CU(grow(ctx->rval0, (size_t)n));
  CU(grow(ctx->rval1, (size_t)n));
  CU(grow(ctx->rhist, (size_t)hlen));
  CU(grow(ctx->rsum, (size_t)nsb));
  CU(cudaMemsetAsync(&ctx->dev->err, 0, sizeof(int32_t), s));
  k_rank_init<<<grid_for(n, kNT, ctx->num_sms * 16), kNT, 0, s>>>(score, n, ctx->rkey0.p,
                                                                    ctx->rval0.p, &ctx->dev->err);
  uint32_t *kin = ctx->rkey0.p, *kout = ctx->rkey1.p;
  int32_t *vin = ctx->rval0.p, *vout = ctx->rval1.p;
  for (int shift = 0; shift < 32; shift += 8) {
    k_radix_hist<<<ntiles, kNT, 0, s>>>(kin, n, shift, ntiles, ctx->rhist.p);
    k_scan_tiles<<<nsb, kScanNT, 0, s>>>(ctx->rhist.p, hlen, ctx->rsum.p);
    k_scan_sums<<<1, kScanNT, 0, s>>>(ctx->rsum.p, nsb);
    k_scan_add<<<nsb, kScanNT, 0, s>>>(ctx->rhist.p, hlen, ctx->rsum.p);
    k_radix_scatter<<<ntiles, kNT, 0, s>>>(kin, vin, n, shift, ntiles, ctx->rhist.p, kout, vout);
    uint32_t *tk = kin;
    kin = kout;
    kout = tk;
    int32_t *tv = vin;
    vin = vout;
    vout = tv;
  }
  k_rank_write<<<grid_for(n, kNT, ctx->num_sms * 16), kNT, 0, s>>>(vin, n, rank);
  CU(cudaGetLastError());
  int32_t err = 0;
  CU(cudaMemcpyAsync(&err, &ctx->dev->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return err ? BGPC_EINVAL : BGPC_OK;
}

}  // extern "C"
