// Smallest-last vertex order (the static order the paper compares with the
// natural one: Sec. VI, Tables II and IV) as a rank for bgpc_color.
//
// On the conflict graph of BGPC (u ~ w iff they share a net) the vertices are
// removed one at a time, always a remaining vertex of smallest remaining
// degree (ties: the smallest id); the coloring order is the reverse of the
// removal order.  Each removal depends on all the earlier ones, so the order
// is built by one host thread: the graph is copied from the device, the
// distinct two-hop neighbour lists are built, and a binary heap keyed by
// (degree, id) with lazy deletion yields the removals in O(E2 log n).  Only
// the order is built here; the coloring in that order runs on the GPU.
#include <stdint.h>
#include <string.h>

#include <functional>
#include <queue>
#include <vector>

#include "bgpc_internal.cuh"

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int bgpc_rank_smallest_last(bgpc_ctx_t *ctx, const bgpc_graph_t *g, int64_t max_pairs,
                                       int32_t *rank, int32_t *degeneracy, void *stream) {
  if (!ctx || !g || g->n_a < 0 || g->n_b < 0 || g->nnz < 0 || max_pairs < 0) return BGPC_EINVAL;
  if (g->n_a > 0 && (!rank || !g->a_ptr || !g->b_ptr)) return BGPC_EINVAL;
  if (g->nnz > 0 && (!g->a_idx || !g->b_idx)) return BGPC_EINVAL;
  if (degeneracy) *degeneracy = 0;
  const int32_t n = g->n_a;
  if (n == 0) return BGPC_OK;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> ap((size_t)n + 1), ai((size_t)g->nnz), bp((size_t)g->n_b + 1),
      bi((size_t)g->nnz);
  if (cudaMemcpyAsync(ap.data(), g->a_ptr, sizeof(int32_t) * ap.size(), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(bp.data(), g->b_ptr, sizeof(int32_t) * bp.size(), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      (g->nnz > 0 &&
       (cudaMemcpyAsync(ai.data(), g->a_idx, sizeof(int32_t) * ai.size(),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(bi.data(), g->b_idx, sizeof(int32_t) * bi.size(),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)) ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return BGPC_ECUDA;
  }
  if (ap[0] != 0 || ap[(size_t)n] != g->nnz || bp[(size_t)g->n_b] != g->nnz) return BGPC_EINVAL;
  // distinct two-hop neighbour lists (the conflict graph), counted then filled
  std::vector<int32_t> mark((size_t)n, -1);
  std::vector<int64_t> np((size_t)n + 1, 0);
  for (int32_t w = 0; w < n; w++) {
    int64_t cnt = 0;
    for (int32_t e = ap[(size_t)w]; e < ap[(size_t)w + 1]; e++) {
      const int32_t v = ai[(size_t)e];
      if (v < 0 || v >= g->n_b) return BGPC_EINVAL;
      for (int32_t f = bp[(size_t)v]; f < bp[(size_t)v + 1]; f++) {
        const int32_t u = bi[(size_t)f];
        if (u < 0 || u >= n) return BGPC_EINVAL;
        if (u != w && mark[(size_t)u] != w) {
          mark[(size_t)u] = w;
          cnt++;
        }
      }
    }
    np[(size_t)w + 1] = np[(size_t)w] + cnt;
    if (np[(size_t)w + 1] > max_pairs) return BGPC_ENOMEM;
  }
  std::vector<int32_t> nb((size_t)np[(size_t)n]);
  std::fill(mark.begin(), mark.end(), -1);
  for (int32_t w = 0; w < n; w++) {
    int64_t o = np[(size_t)w];
    for (int32_t e = ap[(size_t)w]; e < ap[(size_t)w + 1]; e++) {
      const int32_t v = ai[(size_t)e];
      for (int32_t f = bp[(size_t)v]; f < bp[(size_t)v + 1]; f++) {
        const int32_t u = bi[(size_t)f];
        if (u != w && mark[(size_t)u] != w) {
          mark[(size_t)u] = w;
          nb[(size_t)o++] = u;
        }
      }
    }
  }
  // removals in (degree, id) order; a heap entry is stale once the vertex's
  // degree has dropped or it has been removed
  std::vector<int32_t> deg((size_t)n);
  std::vector<uint8_t> gone((size_t)n, 0);
  using Key = unsigned long long;
  std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
  for (int32_t w = 0; w < n; w++) {
    deg[(size_t)w] = (int32_t)(np[(size_t)w + 1] - np[(size_t)w]);
    heap.push(((Key)(uint32_t)deg[(size_t)w] << 32) | (uint32_t)w);
  }
  std::vector<int32_t> h_rank((size_t)n);
  int32_t dg = 0;
  for (int32_t step = 0; step < n; step++) {
    int32_t w = -1;
    while (!heap.empty()) {
      const Key k = heap.top();
      heap.pop();
      const int32_t x = (int32_t)(k & 0xffffffffull), d = (int32_t)(k >> 32);
      if (!gone[(size_t)x] && d == deg[(size_t)x]) {
        w = x;
        break;
      }
    }
    if (w < 0) return BGPC_EINTERNAL;
    gone[(size_t)w] = 1;
    if (deg[(size_t)w] > dg) dg = deg[(size_t)w];
    h_rank[(size_t)w] = n - 1 - step;
    for (int64_t o = np[(size_t)w]; o < np[(size_t)w + 1]; o++) {
      const int32_t u = nb[(size_t)o];
      if (gone[(size_t)u]) continue;
      deg[(size_t)u]--;
      heap.push(((Key)(uint32_t)deg[(size_t)u] << 32) | (uint32_t)u);
    }
  }
  if (cudaMemcpyAsync(rank, h_rank.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return BGPC_ECUDA;
  }
  if (degeneracy) *degeneracy = dg;
  return BGPC_OK;
}
