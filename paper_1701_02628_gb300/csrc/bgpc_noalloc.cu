// Color-set statistics for callers that cannot allocate device memory.
//
// bgpc_color_sets needs a caller-provided cardinality array, and the coloring
// path keeps its histogram in context scratch that is grown with cudaMalloc.
// Some callers can do neither: code running under an allocator that owns all
// device memory (a framework's caching allocator or a fixed memory budget
// leaves nothing for a second allocator), and latency-critical loops that
// must never enter the driver's allocator (cudaMalloc and cudaFree can
// synchronise the whole device).  bgpc_color_sets_noalloc serves them: its
// histogram and accumulators live in one file-scope device array of fixed
// size, so the call allocates nothing.
//
// Costs and rules of that choice:
//  * every GPU that loads this library holds the array (8 MiB + 128 B) until
//    the process exits;
//  * host code cannot use the array's name as a device address; its address
//    is looked up once per device with cudaGetSymbolAddress, on the first call
//    made on that device (make that first call before any stream capture, and
//    do not call it again after cudaDeviceReset: the cached address would be
//    stale);
//  * every call shares the array: calls that overlap on the GPU (other
//    streams, other host threads) race and give wrong statistics;
//  * colors must lie in [0, max_colors) with max_colors <= 2^20, and the
//    colors array must be reachable from the current device;
//  * the call copies the accumulators to the host and synchronises `stream`.
#include <math.h>

#include <mutex>

#include "bgpc_internal.cuh"

namespace {

constexpr int kNT = 256;
constexpr int kAcc = 16;  // leading words: accumulators and the error flag
constexpr int32_t kMaxColors = BGPC_NOALLOC_MAX_COLORS;

// [0, kAcc): acc[0] sets, acc[1] max, acc[2] sum, acc[3] sum of squares,
// acc[4] out-of-range flag; [kAcc, kAcc + kMaxColors): cardinality per color.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kAcc + kMaxColors];

std::mutex g_mu;
unsigned long long *g_addr[64] = {nullptr};

__global__ void k_na_clear(unsigned long long *scr, int32_t ncolors) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)kAcc + ncolors;
       i += (int64_t)gridDim.x * blockDim.x)
    scr[i] = 0ull;
}

__global__ void k_na_hist(const int32_t *__restrict__ colors, int32_t n, int32_t ncolors,
                          unsigned long long *scr) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = colors[u];
    if (c < 0 || c >= ncolors) scr[4] = 1ull;
    else atomicAdd(&scr[kAcc + c], 1ull);
  }
}

__global__ void k_na_reduce(int32_t ncolors, unsigned long long *scr) {
  unsigned long long sets = 0, mx = 0, sum = 0, sq = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ncolors;
       k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = scr[kAcc + k];
    sets += (x > 0);
    mx = x > mx ? x : mx;
    sum += x;
    sq += x * x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sets += __shfl_xor_sync(0xffffffffu, sets, o);
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (sets) atomicAdd(&scr[0], sets);
    if (mx) atomicMax(&scr[1], mx);
    if (sum) atomicAdd(&scr[2], sum);
    if (sq) atomicAdd(&scr[3], sq);
  }
}

int grid_for(long long n) {
  long long g = (n + kNT - 1) / kNT;
  if (g > 2048) g = 2048;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

extern "C" int bgpc_color_sets_noalloc(const int32_t *colors, int32_t n, int32_t max_colors,
                                       int32_t *n_sets, int32_t *max_card, double *mean_card,
                                       double *std_card, void *stream) {
  if (n < 0 || (n > 0 && !colors)) return BGPC_EINVAL;
  if (max_colors < 1 || max_colors > kMaxColors) return BGPC_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return BGPC_ECUDA;
  }
  if (n > 0) {
    // the kernels run on the current device: a colors array on another one
    // would be dereferenced through the wrong address space
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, colors) != cudaSuccess) {
      cudaGetLastError();
      return BGPC_EINVAL;
    }
    if (at.type == cudaMemoryTypeUnregistered ||
        (at.type == cudaMemoryTypeDevice && at.device != dev))
      return BGPC_EINVAL;
  }
  unsigned long long *scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return BGPC_ECUDA;
      }
      g_addr[dev] = static_cast<unsigned long long *>(p);
    }
    scr = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_na_clear<<<grid_for((long long)kAcc + max_colors), kNT, 0, s>>>(scr, max_colors);
  if (n > 0) k_na_hist<<<grid_for(n), kNT, 0, s>>>(colors, n, max_colors, scr);
  k_na_reduce<<<grid_for(max_colors), kNT, 0, s>>>(max_colors, scr);
  unsigned long long acc[kAcc];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(acc, scr, sizeof(acc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return BGPC_ECUDA;
  }
  if (acc[4]) return BGPC_EINVAL;
  const double sets = (double)acc[0];
  const double mean = sets > 0 ? (double)acc[2] / sets : 0.0;
  const double var = sets > 0 ? (double)acc[3] / sets - mean * mean : 0.0;
  if (n_sets) *n_sets = (int32_t)acc[0];
  if (max_card) *max_card = (int32_t)acc[1];
  if (mean_card) *mean_card = mean;
  if (std_card) *std_card = var > 0 ? sqrt(var) : 0.0;
  return BGPC_OK;
}
