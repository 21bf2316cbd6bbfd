// Color-set statistics (Sec. VI-C, Table VI: number of color sets, average
// cardinality, standard deviation) and the validity check of a coloring
// (Sec. II: two V_A vertices sharing a net must differ).
#include "bgpc_internal.cuh"

namespace bgpc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNT = 256;

__global__ void k_card(const int32_t *__restrict__ colors, int32_t n,
                       unsigned long long *__restrict__ card, int32_t ncard, int32_t *err) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = colors[u];
    if (c < 0 || c >= ncard) atomicOr(err, ERR_COLOR);
    else atomicAdd(&card[c], 1ull);
  }
}

// acc[0] = non-empty sets, acc[1] = max, acc[2] = sum, acc[3] = sum of squares
__global__ void k_card_stats(const unsigned long long *__restrict__ card, int32_t ncard,
                             DevScalars *dev) {
  unsigned long long sets = 0, mx = 0, sum = 0, sq = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ncard;
       k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = card[k];
    sets += (x > 0);
    mx = x > mx ? x : mx;
    sum += x;
    sq += x * x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sets += __shfl_xor_sync(kFull, sets, o);
    unsigned long long y = __shfl_xor_sync(kFull, mx, o);
    mx = y > mx ? y : mx;
    sum += __shfl_xor_sync(kFull, sum, o);
    sq += __shfl_xor_sync(kFull, sq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&dev->acc[0], sets);
    atomicMax(&dev->acc[1], mx);
    atomicAdd(&dev->acc[2], sum);
    atomicAdd(&dev->acc[3], sq);
  }
}

__global__ void k_bad_uncolored(const int32_t *__restrict__ colors, int32_t n, int32_t ncolors,
                                uint8_t *__restrict__ bad) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = colors[u];
    bad[u] = (c < 0 || c >= ncolors) ? 1 : 0;
  }
}

__global__ void k_validate_warp(const int32_t *__restrict__ b_ptr, const int32_t *__restrict__ b_idx,
                                int32_t n_b, const int32_t *__restrict__ colors,
                                uint8_t *__restrict__ bad) {
  const int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n_b; v += nwarps) {
    const int32_t beg = b_ptr[v], size = b_ptr[v + 1] - beg;
    if (size < 2 || size > kDetectWarpMax) continue;
    int32_t u = -1, c = -1 - lane;
    if (lane < size) {
      u = b_idx[beg + lane];
      const int32_t cu = colors[u];
      if (cu >= 0) c = cu;
    }
    const unsigned grp = __match_any_sync(kFull, c);
    if (u >= 0 && c >= 0 && __popc(grp) > 1) bad[u] = 1;
  }
}

__global__ void __launch_bounds__(kNT) k_validate_table(const int32_t *__restrict__ b_ptr,
                                                        const int32_t *__restrict__ b_idx,
                                                        const int32_t *__restrict__ colors,
                                                        const int32_t *__restrict__ bigd,
                                                        int32_t nbig, int32_t *__restrict__ vtab,
                                                        int32_t tabcap, uint8_t *__restrict__ bad) {
  int32_t *tab = vtab + (size_t)blockIdx.x * (size_t)tabcap;
  for (int32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const int32_t v = bigd[b];
    const int32_t beg = b_ptr[v], end = b_ptr[v + 1];
    for (int32_t f = beg + threadIdx.x; f < end; f += kNT) {
      const int32_t c = colors[b_idx[f]];
      if (c >= 0 && c < tabcap) atomicAdd(&tab[c], 1);
    }
    __syncthreads();
    for (int32_t f = beg + threadIdx.x; f < end; f += kNT) {
      const int32_t u = b_idx[f];
      const int32_t c = colors[u];
      if (c >= 0 && c < tabcap && tab[c] > 1) bad[u] = 1;
    }
    __syncthreads();
    for (int32_t f = beg + threadIdx.x; f < end; f += kNT) {
      const int32_t c = colors[b_idx[f]];
      if (c >= 0 && c < tabcap) tab[c] = 0;
    }
    __syncthreads();
  }
}

__global__ void k_count_bad(const uint8_t *__restrict__ bad, int32_t n, DevScalars *dev) {
  unsigned long long acc = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x)
    acc += bad[u];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&dev->acc[0], acc);
}

inline int grid_for(long long n, int cap) {
  long long g = div_up(n, kNT);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int launch_card(const int32_t *colors, int32_t n, unsigned long long *card, int32_t ncard,
                 int32_t *err, cudaStream_t s) {
  cudaMemsetAsync(card, 0, sizeof(unsigned long long) * (size_t)ncard, s);
  if (n <= 0) return 0;
  k_card<<<grid_for(n, 4096), kNT, 0, s>>>(colors, n, card, ncard, err);
  return 1;
}

int launch_card_stats(const unsigned long long *card, int32_t ncard, DevScalars *dev,
                       cudaStream_t s) {
  cudaMemsetAsync(dev->acc, 0, sizeof(dev->acc), s);
  if (ncard <= 0) return 0;
  k_card_stats<<<grid_for(ncard, 1184), kNT, 0, s>>>(card, ncard, dev);
  return 1;
}

int launch_validate(const bgpc_graph_t &g, const int32_t *colors, const int32_t *bigd,
                     int32_t nbigd, int32_t *vtab, int32_t tabcap, int32_t nslots,
                     uint8_t *bad, DevScalars *dev, int sms, cudaStream_t s) {
  cudaMemsetAsync(dev->acc, 0, sizeof(dev->acc), s);
  if (g.n_a <= 0) return 0;
  k_bad_uncolored<<<grid_for(g.n_a, 4096), kNT, 0, s>>>(colors, g.n_a, tabcap, bad);
  if (g.n_b > 0) {
    long long wg = div_up((long long)g.n_b * 32, kNT);
    if (wg > (long long)sms * 16) wg = (long long)sms * 16;
    k_validate_warp<<<(int)wg, kNT, 0, s>>>(g.b_ptr, g.b_idx, g.n_b, colors, bad);
  }
  if (nbigd > 0) {
    int grid = nbigd < nslots ? nbigd : nslots;
    k_validate_table<<<grid, kNT, 0, s>>>(g.b_ptr, g.b_idx, colors, bigd, nbigd, vtab, tabcap,
                                          bad);
  }
  k_count_bad<<<grid_for(g.n_a, 1184), kNT, 0, s>>>(bad, g.n_a, dev);
  return 2 + (g.n_b > 0) + (nbigd > 0);
}

}  // namespace bgpc
