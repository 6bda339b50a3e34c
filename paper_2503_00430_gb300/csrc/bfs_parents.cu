// bfs_parents: a BFS tree (Graph500-style parent array) from a distance array.
//
// The paper computes distances only; a parent array is the usual companion
// output.  Parents are not unique, so the rule is fixed: the parent of a
// reached vertex v other than the source is the first vertex u of v's list
// (in the library's list order) with dist[u] = dist[v] - 1 - the bottom-up
// test of Listing 2 run once more on the finished distances.  The source (the
// vertex at distance 0) is its own parent; unreached vertices get -1.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bfs_internal.cuh"

namespace gbfs {
namespace {

constexpr int kParLane = 32;  // entries a lane scans on its own before the warp takes over

template <typename RP>
__device__ __forceinline__ long long par_rp(const void* rp, long long i) {
  return (long long)__ldg(reinterpret_cast<const RP*>(rp) + i);
}

// A warp takes 32 consecutive vertices: each lane scans the first kParLane
// entries of its vertex; vertices still unresolved with longer lists are then
// scanned by the whole warp, 32 entries per step, one vertex at a time.
template <typename RP>
__global__ void __launch_bounds__(256) k_parents(const void* rp, const int* col, const int* dist, long long n,
                                                 int* parent) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  for (long long base = tid - lane; base < n; base += nth) {
    const long long v = base + lane;
    int d = -1;
    long long s = 0, e = 0, j = 0;
    int p = -1;
    bool open = false;
    if (v < n) {
      d = __ldg(dist + v);
      if (d == 0) {
        p = (int)v;
      } else if (d > 0) {
        s = par_rp<RP>(rp, v);
        e = par_rp<RP>(rp, v + 1);
        const long long stop = e - s > kParLane ? s + kParLane : e;
        for (j = s; j < stop; ++j) {
          const int u = __ldg(col + j);
          if (__ldg(dist + u) == d - 1) {
            p = u;
            break;
          }
        }
        open = p < 0 && j < e;  // parent lies further down a long list
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, open);
    while (todo) {
      const int l = __ffs(todo) - 1;
      todo &= todo - 1;
      const long long js = __shfl_sync(0xffffffffu, j, l), je = __shfl_sync(0xffffffffu, e, l);
      const int dl = __shfl_sync(0xffffffffu, d, l);
      int found = -1;
      for (long long k0 = js; k0 < je && found < 0; k0 += 32) {
        const long long k = k0 + lane;
        int u = -1;
        bool hit = false;
        if (k < je) {
          u = __ldg(col + k);
          hit = __ldg(dist + u) == dl - 1;
        }
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        if (b) found = __shfl_sync(0xffffffffu, u, __ffs(b) - 1);
      }
      if ((int)lane == l) p = found;
    }
    if (v < n) parent[v] = p;
  }
}

}  // namespace

int run_parents(bfs_graph* g, const int* dist, int* parent, cudaStream_t s) {
  const int grid = g->num_sms * 8, block = 256;
  if (g->rp_bits == 32)
    k_parents<int><<<grid, block, 0, s>>>(g->rp, g->col, dist, g->n, parent);
  else
    k_parents<long long><<<grid, block, 0, s>>>(g->rp, g->col, dist, g->n, parent);
  GBFS_CUDA(cudaGetLastError());
  return BFS_OK;
}

}  // namespace gbfs
