// Upload-time layout option BFS_DEGREE_ORDER: every adjacency list of the
// library's device copy is stored with the highest-degree neighbours first
// (ties by id).  Distances do not depend on the order of a list; a bottom-up
// scan (Listing 2/3), which stops at the first neighbour in the frontier,
// meets one sooner because high-degree vertices enter the frontier early.
// The sort is a one-time preprocessing step done with CUB's segmented sort
// (CUDA toolkit source library); no BFS kernel uses CUB.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cub/device/device_radix_sort.cuh>
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

int reorder_by_degree(bfs_graph* g) {
  return g->rp_bits == 32 ? reorder_impl<int>(g) : reorder_impl<long long>(g);
}

}  // namespace gbfs
