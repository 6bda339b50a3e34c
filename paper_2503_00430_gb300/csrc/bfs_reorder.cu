// Upload-time layout option BFS_DEGREE_ORDER: every adjacency list of the
// library's device copy is stored with the highest-degree neighbours first
// (ties by id).  Distances do not depend on the order of a list; a bottom-up
// scan (Listing 2/3), which stops at the first neighbour in the frontier,
// meets one sooner because high-degree vertices enter the frontier early.
// The sort is a one-time preprocessing step done with CUB's segmented sort
// (CUDA toolkit source library); no BFS kernel uses CUB.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include "bfs_internal.cuh"

namespace gbfs {

namespace {

// key = (0xffffffff - min(deg(u), 0xffffffff)) << 32 | u: ascending keys give
// degree-descending, id-ascending order.
template <typename RP>
__global__ void k_degree_keys(const RP* rp, const int* col, long long m, unsigned long long* keys) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long j = tid; j < m; j += nth) {
    const int u = col[j];
    long long d = (long long)rp[(long long)u + 1] - (long long)rp[u];
    if (d > 0xffffffffll) d = 0xffffffffll;
    keys[j] = ((0xffffffffull - (unsigned long long)d) << 32) | (unsigned long long)(unsigned)u;
  }
}

__global__ void k_keys_to_col(const unsigned long long* keys, long long m, int* col) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long j = tid; j < m; j += nth) col[j] = (int)(unsigned)(keys[j] & 0xffffffffull);
}

template <typename RP>
int reorder_impl(bfs_graph* g) {
  const long long m = g->m;
  if (m == 0) return BFS_OK;
  if (m >= (1ll << 31)) return BFS_EINVAL;  // the segmented sort takes 32-bit item counts
  const RP* rp = reinterpret_cast<const RP*>(g->rp);
  unsigned long long *k_in = nullptr, *k_out = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  int rc = BFS_OK;
  do {
    cudaError_t e = cudaMalloc(&k_in, sizeof(unsigned long long) * (size_t)m);
    if (e == cudaSuccess) e = cudaMalloc(&k_out, sizeof(unsigned long long) * (size_t)m);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc (reorder keys)", __FILE__, __LINE__); break; }
    const int grid = g->num_sms * 8, block = 256;
    k_degree_keys<RP><<<grid, block>>>(rp, g->col, m, k_in);
    e = cub::DeviceSegmentedSort::SortKeys(nullptr, tmp_bytes, k_in, k_out, (int)m, (int)g->n, rp, rp + 1);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes);
    if (e == cudaSuccess)
      e = cub::DeviceSegmentedSort::SortKeys(tmp, tmp_bytes, k_in, k_out, (int)m, (int)g->n, rp, rp + 1);
    if (e != cudaSuccess) { rc = cuda_fail(e, "segmented sort", __FILE__, __LINE__); break; }
    k_keys_to_col<<<grid, block>>>(k_out, m, g->col);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { rc = cuda_fail(e, "reorder", __FILE__, __LINE__); break; }
  } while (0);
  cudaFree(k_in);
  cudaFree(k_out);
  cudaFree(tmp);
  return rc;
}

}  // namespace

namespace {

template <typename RP>
__global__ void k_degrees(const RP* rp, long long n, unsigned* deg, int* ids) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += nth) {
    const long long d = (long long)rp[v + 1] - (long long)rp[v];
    deg[v] = d > 0xffffffffll ? 0xffffffffu : (unsigned)d;
    ids[v] = (int)v;
  }
}

template <typename RP>
int degree_order_impl(bfs_graph* g, int* order) {
  const long long n = g->n;
  unsigned *k_in = nullptr, *k_out = nullptr;
  int* ids = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  int rc = BFS_OK;
  do {
    cudaError_t e = cudaMalloc(&k_in, sizeof(unsigned) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&k_out, sizeof(unsigned) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&ids, sizeof(int) * (size_t)n);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc (degree order)", __FILE__, __LINE__); break; }
    k_degrees<RP><<<g->num_sms * 8, 256>>>(reinterpret_cast<const RP*>(g->rp), n, k_in, ids);
    e = cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp_bytes, k_in, k_out, ids, order, (int)n);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes);
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, k_in, k_out, ids, order, (int)n);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { rc = cuda_fail(e, "degree order sort", __FILE__, __LINE__); break; }
  } while (0);
  cudaFree(k_in);
  cudaFree(k_out);
  cudaFree(ids);
  cudaFree(tmp);
  return rc;
}

}  // namespace

// Vertex ids ordered by degree, highest first (stable in id): the processing
// order of multi-source pull levels, so that a warp's lanes scan lists of
// similar length.
int vertices_by_degree(bfs_graph* g, int* order) {
  return g->rp_bits == 32 ? degree_order_impl<int>(g, order) : degree_order_impl<long long>(g, order);
}

namespace {

// new_of[old_of[i]] = i and the degree of new vertex i (deg[n] = 0, so an
// exclusive scan over n + 1 entries gives the renumbered row pointers).
template <typename RP>
__global__ void k_inverse_degrees(const RP* rp, const int* old_of, long long n, int* new_of, RP* deg) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i <= n; i += nth) {
    if (i == n) {
      deg[n] = 0;
      continue;
    }
    const int o = old_of[i];
    new_of[o] = (int)i;
    deg[i] = rp[(long long)o + 1] - rp[o];
  }
}

// Warp per new vertex: its list, neighbour ids renumbered.
template <typename RP>
__global__ void k_relabel_lists(const RP* rp, const int* col, const RP* rp2, const int* old_of, const int* new_of,
                                long long n, int* col2) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  for (long long i = gw; i < n; i += nwarps) {
    const int o = old_of[i];
    const long long s = (long long)rp[o], d = (long long)rp[(long long)o + 1] - s, s2 = (long long)rp2[i];
    for (long long j = lane; j < d; j += 32) col2[s2 + j] = new_of[col[s + j]];
  }
}

template <typename RP>
int relabel_impl(bfs_graph* g, Relabel* r) {
  const long long n = g->n, m = g->m;
  const size_t mpad = (size_t)((m + 3) / 4 * 4 + 4);
  RP* rp2 = nullptr;
  RP* deg = nullptr;
  int* tmp_col = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  int rc = BFS_OK;
  do {
    cudaError_t e = cudaMalloc(&r->old_of, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&r->new_of, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&rp2, sizeof(RP) * (size_t)(n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&deg, sizeof(RP) * (size_t)(n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&r->col, sizeof(int) * mpad);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc (relabel)", __FILE__, __LINE__); break; }
    r->rp = rp2;
    rc = degree_order_impl<RP>(g, r->old_of);
    if (rc != BFS_OK) break;
    const int grid = g->num_sms * 8, block = 256;
    k_inverse_degrees<RP><<<grid, block>>>(reinterpret_cast<const RP*>(g->rp), r->old_of, n, r->new_of, deg);
    e = cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, deg, rp2, n + 1);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes);
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, deg, rp2, n + 1);
    if (e != cudaSuccess) { rc = cuda_fail(e, "relabel scan", __FILE__, __LINE__); break; }
    cudaFree(tmp);
    tmp = nullptr;
    e = cudaMemset(r->col + m, 0, sizeof(int) * (mpad - (size_t)m));
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemset (relabel)", __FILE__, __LINE__); break; }
    // Degree-ordered lists map to ascending new ids; other lists are sorted
    // after renumbering (the segmented sort takes 32-bit counts).
    const bool sort = !g->deg_ordered && m > 0 && m < (1ll << 31);
    if (sort) {
      e = cudaMalloc(&tmp_col, sizeof(int) * (size_t)m);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc (relabel sort)", __FILE__, __LINE__); break; }
    }
    k_relabel_lists<RP><<<grid, block>>>(reinterpret_cast<const RP*>(g->rp), g->col, rp2, r->old_of, r->new_of, n,
                                         sort ? tmp_col : r->col);
    if (sort) {
      e = cub::DeviceSegmentedSort::SortKeys(nullptr, tmp_bytes, tmp_col, r->col, (int)m, (int)n, rp2, rp2 + 1);
      if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes);
      if (e == cudaSuccess)
        e = cub::DeviceSegmentedSort::SortKeys(tmp, tmp_bytes, tmp_col, r->col, (int)m, (int)n, rp2, rp2 + 1);
      if (e != cudaSuccess) { rc = cuda_fail(e, "relabel sort", __FILE__, __LINE__); break; }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { rc = cuda_fail(e, "relabel", __FILE__, __LINE__); break; }
    r->n_live = n - g->isolated;
  } while (0);
  cudaFree(deg);
  cudaFree(tmp_col);
  cudaFree(tmp);
  return rc;
}

}  // namespace

int ensure_relabel(bfs_graph* g) {
  if (g->rl) return BFS_OK;
  Relabel* r = new Relabel();
  const int rc = g->rp_bits == 32 ? relabel_impl<int>(g, r) : relabel_impl<long long>(g, r);
  if (rc != BFS_OK) {
    cudaFree(r->rp);
    cudaFree(r->col);
    cudaFree(r->new_of);
    cudaFree(r->old_of);
    delete r;
    return rc;
  }
  g->rl = r;
  return BFS_OK;
}

void free_relabel(bfs_graph* g) {
  if (!g->rl) return;
  cudaFree(g->rl->head);
  cudaFree(g->rl->init_vis);
  free(g->rl->h_new_of);
  cudaFree(g->rl->rp);
  cudaFree(g->rl->col);
  cudaFree(g->rl->new_of);
  cudaFree(g->rl->old_of);
  delete g->rl;
  g->rl = nullptr;
}

int reorder_by_degree(bfs_graph* g) {
  return g->rp_bits == 32 ? reorder_impl<int>(g) : reorder_impl<long long>(g);
}

}  // namespace gbfs
