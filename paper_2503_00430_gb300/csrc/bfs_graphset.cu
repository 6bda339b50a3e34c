// Graph sets: one persistent launch over many independent small graphs, one
// BFS source each.
//
// Every block takes graphs, largest first, from a shared counter and runs the
// paper's hybrid BFS (Section 2, Listing 2 with Listing 3's visited bitmap) on
// one graph at a time, entirely inside the block: the visited, frontier and
// next-frontier bitmaps live in shared memory and __syncthreads() is the level
// barrier.  Top-down levels expand the frontier bitmap a word per warp: the
// lists of the word's frontier vertices are concatenated and dealt to the
// lanes 32 entries per step (claims by shared-memory atomicOr); bottom-up
// levels give each warp 32 consecutive vertices that scan their lists in
// aligned 128-bit groups of four entries for a frontier neighbour and stop at
// the first one.  The direction follows the edge-count
// rule with the graph's own counters.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "bfs_internal.cuh"
#include "bfs_device.cuh"

struct bfs_graphset {
  int count = 0;
  long long total_v = 0, total_e = 0;
  long long max_n = 0;
  int device = 0, num_sms = 0;
  long long* voff = nullptr;   // [count+1]
  long long* eoff = nullptr;   // [count+1]
  long long* rp = nullptr;     // [total_v + count] local row pointers
  int* col = nullptr;          // [total_e + 4] local neighbour ids
  int* order = nullptr;        // graph ids, largest first
  int* d_src = nullptr;        // [count]
  unsigned long long* ctrl = nullptr;  // [8]: next graph, levels, td levels, bu levels, max levels
  unsigned long long* h_ctrl = nullptr;
  int* staging = nullptr;      // host-output staging
  std::mutex mu;
};

namespace gbfs {

namespace {

struct GsArgs {
  const long long* voff;
  const long long* eoff;
  const long long* rp;
  const int* col;
  const int* order;
  const int* src;
  int* dist;
  unsigned long long* ctrl;
  int count;
  int nwmax;
  int alpha, beta;
};

__global__ void __launch_bounds__(512) k_graphset(GsArgs A) {
  extern __shared__ unsigned gs_smem[];
  unsigned* vis = gs_smem;
  unsigned* bmA = gs_smem + A.nwmax;
  unsigned* bmB = gs_smem + 2 * A.nwmax;
  __shared__ int s_t;
  __shared__ unsigned long long s_nf, s_mf;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  unsigned long long lv_total = 0, td_total = 0, bu_total = 0, lv_max = 0;
  for (;;) {
    if (threadIdx.x == 0) s_t = (int)atomicAdd(&A.ctrl[0], 1ull);
    __syncthreads();
    const int t = s_t;
    if (t >= A.count) break;
    const int gi = A.order[t];
    const long long vb = A.voff[gi];
    const int n = (int)(A.voff[gi + 1] - vb);
    const long long* rp = A.rp + vb + gi;
    const long long cbase = A.eoff[gi];
    const int* col = A.col + cbase;
    int* dist = A.dist + vb;
    const int src = A.src[gi];
    const long long m = A.eoff[gi + 1] - A.eoff[gi];
    const int nw = (n + 31) / 32;
    // init: dist = -1, bitmaps clear (padding bits past n marked visited)
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
      const int hi = n - 32 * w;
      vis[w] = hi >= 32 ? 0u : ~((1u << hi) - 1u);
      bmA[w] = 0u;
    }
    for (int v = threadIdx.x; v < n; v += blockDim.x) dist[v] = -1;
    __syncthreads();
    if (threadIdx.x == 0) {
      dist[src] = 0;
      vis[src >> 5] |= 1u << (src & 31);
      bmA[src >> 5] |= 1u << (src & 31);
    }
    unsigned* front = bmA;
    unsigned* next = bmB;
    bool td = true;
    long long nf_cur = 1, edges_visited = rp[src + 1] - rp[src];
    int L = 0;
    __syncthreads();
    for (;;) {
      for (int w = threadIdx.x; w < nw; w += blockDim.x) next[w] = 0u;
      if (threadIdx.x == 0) {
        s_nf = 0;
        s_mf = 0;
      }
      __syncthreads();
      unsigned long long my_nf = 0, my_mf = 0;
      if (td) {
        // One warp per frontier word: the lists of the word's frontier vertices
        // are concatenated (exclusive scan of their lengths) and dealt to the
        // lanes 32 entries per step, so a step issues its neighbour loads
        // together instead of one list walk per lane.
        for (int w = (int)warp; w < nw; w += (int)nwarp) {
          const unsigned word = front[w];
          if (!word) continue;
          long long s = 0;
          int len = 0;
          if ((word >> lane) & 1u) {
            const int u = 32 * w + (int)lane;
            s = rp[u];
            len = (int)(rp[u + 1] - s);
          }
          const int incl = dev::warp_incl_scan(len);
          const int excl = incl - len;
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          for (int base = 0; base < total; base += 32) {
            const int e = base + (int)lane;
            const int o = dev::owner_of(excl, e);
            const long long so = __shfl_sync(0xffffffffu, s, o);
            const int eo = __shfl_sync(0xffffffffu, excl, o);
            if (e >= total) continue;
            const int v = __ldg(col + so + (e - eo));
            const unsigned bit = 1u << (v & 31);
            if (vis[v >> 5] & bit) continue;
            if (atomicOr(&vis[v >> 5], bit) & bit) continue;
            dist[v] = L + 1;
            atomicOr(&next[v >> 5], bit);
            my_nf += 1;
            my_mf += (unsigned long long)(rp[v + 1] - rp[v]);
          }
        }
      } else {
        // One warp per 32 consecutive vertices: stop at the first frontier neighbour.
        for (int w = (int)warp; w < nw; w += (int)nwarp) {
          const unsigned vw = vis[w];
          if (vw == 0xffffffffu) continue;
          const int v = 32 * w + (int)lane;
          bool found = false;
          long long d = 0;
          if (!((vw >> lane) & 1u)) {
            const long long s = rp[v], e = rp[v + 1];
            d = e - s;
            // Aligned groups of four entries of the whole column array (16-byte
            // aligned, 4 spare entries past the last list), masked to [s, e).
            const long long gs = cbase + s, ge = cbase + e;
            for (long long a = gs & ~3ll; a < ge && !found; a += 4) {
              const int4 q = __ldg(reinterpret_cast<const int4*>(A.col + a));
              const int c4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (a + t >= gs && a + t < ge && ((front[c4[t] >> 5] >> (c4[t] & 31)) & 1u)) found = true;
            }
          }
          const unsigned fm = __ballot_sync(0xffffffffu, found);
          if (lane == 0 && fm) {
            next[w] = fm;
            vis[w] = vw | fm;  // this warp owns the word during the level
          }
          if (found) {
            dist[v] = L + 1;
            my_nf += 1;
            my_mf += (unsigned long long)d;
          }
        }
      }
      if (my_nf) {
        atomicAdd(&s_nf, my_nf);
        atomicAdd(&s_mf, my_mf);
      }
      __syncthreads();
      const long long nf = (long long)s_nf, mf = (long long)s_mf;
      if (td) ++td_total; else ++bu_total;
      ++L;
      if (nf == 0) break;
      edges_visited += mf;
      const bool ntd = next_is_top_down(BFS_POLICY_EDGES, A.alpha, A.beta, 20, 0ull, L, td, nf, nf_cur, mf,
                                        m - edges_visited, n);
      td = ntd;
      nf_cur = nf;
      unsigned* tmp = front;
      front = next;
      next = tmp;
      __syncthreads();
    }
    lv_total += (unsigned long long)L;
    if ((unsigned long long)L > lv_max) lv_max = (unsigned long long)L;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&A.ctrl[1], lv_total);
    atomicAdd(&A.ctrl[2], td_total);
    atomicAdd(&A.ctrl[3], bu_total);
    atomicMax(&A.ctrl[4], lv_max);
  }
}

void release(bfs_graphset* s) {
  if (!s) return;
  cudaFree(s->voff);
  cudaFree(s->eoff);
  cudaFree(s->rp);
  cudaFree(s->col);
  cudaFree(s->order);
  cudaFree(s->d_src);
  cudaFree(s->ctrl);
  cudaFree(s->staging);
  if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
  delete s;
}

size_t smem_bytes(const bfs_graphset* s) { return 3 * sizeof(unsigned) * (size_t)((s->max_n + 31) / 32); }

}  // namespace
}  // namespace gbfs

using namespace gbfs;

extern "C" {

int bfs_graphset_upload(const int64_t* voff, const int64_t* eoff, const int64_t* row_ptr, const int32_t* col,
                        int32_t count, int flags, bfs_graphset** out) {
  GBFS_NVTX("bfs_graphset_upload");
  if (!out) return BFS_EINVAL;
  *out = nullptr;
  if (!voff || !eoff || !row_ptr || count < 1) return BFS_EINVAL;
  if (voff[0] != 0 || eoff[0] != 0) return BFS_EINVAL;
  long long max_n = 0;
  for (int i = 0; i < count; ++i) {
    const long long n = voff[i + 1] - voff[i], m = eoff[i + 1] - eoff[i];
    if (n < 1 || m < 0) return BFS_EINVAL;
    max_n = std::max(max_n, n);
  }
  // Bitmaps of the largest graph live in shared memory (3 x n/8 bytes).
  if (max_n > (1ll << 19)) return BFS_EINVAL;
  const long long tv = voff[count], te = eoff[count];
  if (te > 0 && !col) return BFS_EINVAL;
  if (flags & BFS_VALIDATE) {
    for (int i = 0; i < count; ++i) {
      const int64_t* rp = row_ptr + voff[i] + i;
      const long long n = voff[i + 1] - voff[i];
      if (rp[0] != 0 || rp[n] != eoff[i + 1] - eoff[i]) return BFS_EINVAL;
      for (long long v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return BFS_EINVAL;
      for (long long j = eoff[i]; j < eoff[i + 1]; ++j)
        if (col[j] < 0 || col[j] >= n) return BFS_EINVAL;
    }
  }
  bfs_graphset* s = new bfs_graphset();
  s->count = count;
  s->total_v = tv;
  s->total_e = te;
  s->max_n = max_n;
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (voff[a + 1] - voff[a]) + (eoff[a + 1] - eoff[a]) > (voff[b + 1] - voff[b]) + (eoff[b + 1] - eoff[b]);
  });
  int rc = BFS_OK;
  do {
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->voff, sizeof(long long) * (size_t)(count + 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->eoff, sizeof(long long) * (size_t)(count + 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->rp, sizeof(long long) * (size_t)(tv + count));
    if (e == cudaSuccess) e = cudaMalloc(&s->col, sizeof(int) * (size_t)(te + 4));
    if (e == cudaSuccess) e = cudaMalloc(&s->order, sizeof(int) * (size_t)count);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_src, sizeof(int) * (size_t)count);
    if (e == cudaSuccess) e = cudaMalloc(&s->ctrl, sizeof(unsigned long long) * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ctrl, sizeof(unsigned long long) * 8);
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph-set allocation", __FILE__, __LINE__); break; }
    e = cudaMemcpy(s->voff, voff, sizeof(long long) * (size_t)(count + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->eoff, eoff, sizeof(long long) * (size_t)(count + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->rp, row_ptr, sizeof(long long) * (size_t)(tv + count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && te > 0) e = cudaMemcpy(s->col, col, sizeof(int) * (size_t)te, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->col + te, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemcpy(s->order, order.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_graphset),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(s));
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph-set upload", __FILE__, __LINE__); break; }
  } while (0);
  if (rc != BFS_OK) {
    release(s);
    return rc;
  }
  *out = s;
  return BFS_OK;
}

}  // extern "C"

namespace gbfs {
long long graphset_total_vertices(const bfs_graphset* s) { return s->total_v; }
int graphset_count(const bfs_graphset* s) { return s->count; }
}  // namespace gbfs

extern "C" {

void bfs_graphset_free(bfs_graphset* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  release(s);
}

int bfs_graphset_run(bfs_graphset* s, const int32_t* srcs, int32_t* dist, const bfs_params* params,
                     bfs_graphset_stats* stats, void* stream) {
  GBFS_NVTX("bfs_graphset_run");
  if (!s || !srcs || !dist) return BFS_EINVAL;
  bfs_params p;
  if (params) p = *params; else bfs_params_default(&p);
  if (p.alpha < 1 || p.beta < 1 || p.threads_per_block < 64 || p.threads_per_block > 512 ||
      (p.threads_per_block & 31))
    return BFS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GBFS_CUDA(cudaMemcpyAsync(s->d_src, srcs, sizeof(int) * (size_t)s->count, cudaMemcpyHostToDevice, st));
  GBFS_CUDA(cudaStreamSynchronize(st));
  std::vector<int> hsrc(srcs, srcs + s->count);
  std::vector<long long> hv(s->count + 1);
  GBFS_CUDA(cudaMemcpy(hv.data(), s->voff, sizeof(long long) * (size_t)(s->count + 1), cudaMemcpyDeviceToHost));
  for (int i = 0; i < s->count; ++i)
    if (hsrc[i] < 0 || hsrc[i] >= hv[i + 1] - hv[i]) return BFS_EINVAL;
  int* out = dist;
  const bool host_out = !is_device_pointer(dist);
  if (host_out) {
    if (!s->staging) GBFS_CUDA(cudaMalloc(&s->staging, sizeof(int) * (size_t)s->total_v));
    out = s->staging;
  }
  GBFS_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(unsigned long long) * 8, st));
  GsArgs A{};
  A.voff = s->voff;
  A.eoff = s->eoff;
  A.rp = s->rp;
  A.col = s->col;
  A.order = s->order;
  A.src = s->d_src;
  A.dist = out;
  A.ctrl = s->ctrl;
  A.count = s->count;
  A.nwmax = (int)((s->max_n + 31) / 32);
  A.alpha = p.alpha;
  A.beta = p.beta;
  const size_t smem = smem_bytes(s);
  int per_sm = 0;
  GBFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(&k_graphset),
                                                          p.threads_per_block, smem));
  if (per_sm < 1) return BFS_ENOMEM;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  k_graphset<<<per_sm * s->num_sms, p.threads_per_block, smem, st>>>(A);
  GBFS_CUDA(cudaGetLastError());
  GBFS_CUDA(cudaMemcpyAsync(s->h_ctrl, s->ctrl, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, st));
  if (host_out)
    GBFS_CUDA(cudaMemcpyAsync(dist, out, sizeof(int) * (size_t)s->total_v, cudaMemcpyDeviceToHost, st));
  GBFS_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->graphs = s->count;
    stats->levels = (int64_t)s->h_ctrl[1];
    stats->td_levels = (int64_t)s->h_ctrl[2];
    stats->bu_levels = (int64_t)s->h_ctrl[3];
    stats->max_levels = (int32_t)s->h_ctrl[4];
    stats->blocks = per_sm * s->num_sms;
  }
  return BFS_OK;
}

}  // extern "C"
