// Autotuner: picks bfs_params for a graph by coordinate descent.
//
// The paper tunes by hand (static vs dynamic scheduling, Section 2; alpha and
// beta of the edge-count rule it cites); here every candidate setting of one
// parameter at a time is timed on sample sources (median of the per-source
// CUDA-event times), the fastest is kept, and every candidate's distances must
// hash identically to the starting setting's (the distances are unique, so a
// parameter can only change speed - a mismatch is reported as an error).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bfs_internal.cuh"

namespace gbfs {
namespace {

__device__ __forceinline__ unsigned long long tmix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Order-independent hash of a distance array.
__global__ void k_dist_hash(const int* d, long long n, unsigned long long* out) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long h = 0;
  for (long long v = tid; v < n; v += nth) h += tmix(((unsigned long long)v << 32) ^ (unsigned)d[v]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31u) == 0) atomicAdd(out, h);
}

struct Trial {
  double median_ms = 0;
  unsigned long long hash = 0;
  int rc = BFS_OK;
};

Trial run_trial(bfs_graph* g, const int* srcs, int k, const bfs_params& p, int* dist, unsigned long long* d_hash,
                cudaStream_t s) {
  Trial t;
  std::vector<float> ms;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  unsigned long long hsum = 0;
  for (int i = 0; i < k && t.rc == BFS_OK; ++i) {
    for (int rep = 0; rep < 2 && t.rc == BFS_OK; ++rep) {  // first run warms the workspace and caches
      cudaEventRecord(a, s);
      t.rc = run_single(g, srcs[i], dist, p, nullptr, nullptr, 0, s);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      if (rep == 1) {
        float x = 0;
        cudaEventElapsedTime(&x, a, b);
        ms.push_back(x);
      }
    }
    if (t.rc != BFS_OK) break;
    cudaMemsetAsync(d_hash, 0, sizeof(unsigned long long), s);
    k_dist_hash<<<g->num_sms * 4, 256, 0, s>>>(dist, g->n, d_hash);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, d_hash, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    hsum = hsum * 0x9E3779B97F4A7C15ull + h;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!ms.empty()) {
    std::sort(ms.begin(), ms.end());
    t.median_ms = ms[ms.size() / 2];
  }
  t.hash = hsum;
  return t;
}

}  // namespace
}  // namespace gbfs

using namespace gbfs;

extern "C" int bfs_tune(bfs_graph* g, const int32_t* srcs, int32_t k, const bfs_params* base, bfs_params* out,
                        bfs_tune_report* report) {
  if (!g || !srcs || k <= 0 || !out) return BFS_EINVAL;
  for (int i = 0; i < k; ++i)
    if (srcs[i] < 0 || (int64_t)srcs[i] >= g->n) return BFS_EINVAL;
  bfs_params cur;
  if (base) cur = *base; else bfs_params_default(&cur);
  cur.launch = BFS_LAUNCH_PERSISTENT;
  std::lock_guard<std::mutex> lock(g->mu);
  int rc = ensure_single_ws(g);
  if (rc != BFS_OK) return rc;
  int* dist = nullptr;
  unsigned long long* d_hash = nullptr;
  GBFS_CUDA(cudaMalloc(&dist, sizeof(int) * (size_t)g->n));
  GBFS_CUDA(cudaMalloc(&d_hash, sizeof(unsigned long long)));
  cudaStream_t s;
  GBFS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  Trial best = run_trial(g, srcs, k, cur, dist, d_hash, s);
  const unsigned long long ref_hash = best.hash;
  const double start_ms = best.median_ms;
  int trials = 1;
  rc = best.rc;
  // Coordinate descent over the tunable fields, two sweeps.
  struct Field {
    int32_t bfs_params::*f;
    std::vector<int32_t> vals;
  };
  const bool small_world = (double)g->m >= 7.0 * (double)g->n;
  std::vector<Field> fields = {
      {&bfs_params::policy, {BFS_POLICY_EDGES, BFS_POLICY_FRONTIER, BFS_POLICY_TD_ONLY}},
      {&bfs_params::alpha, {2, 4, 8, 14, 24, 48, 96}},
      {&bfs_params::beta, {6, 12, 24, 48, 96}},
      {&bfs_params::tau_inv, {5, 10, 20, 40, 80}},
      {&bfs_params::chunk, {256, 512, 1024, 4096}},
      {&bfs_params::small_max, {8, 16, 32}},
      {&bfs_params::bu_thread_max, {0, 8, 32, 128}},
      {&bfs_params::bu_warp_min, {8, 32, 128, 1024}},
      {&bfs_params::bu_chunk, {0, 1, 4}},
      {&bfs_params::threads_per_block, {256, 512, 1024}},
  };
  if (!small_world) fields.erase(fields.begin() + 1, fields.begin() + 4);  // top-down-only class: no switch rule
  for (int sweep = 0; sweep < 2 && rc == BFS_OK; ++sweep) {
    for (const Field& fd : fields) {
      for (int32_t v : fd.vals) {
        if (cur.*(fd.f) == v) continue;
        bfs_params cand = cur;
        cand.*(fd.f) = v;
        // Only settings that can change the work of the current policy.
        if (fd.f == &bfs_params::tau_inv && cand.policy != BFS_POLICY_FRONTIER) continue;
        if ((fd.f == &bfs_params::alpha || fd.f == &bfs_params::beta) && cand.policy != BFS_POLICY_EDGES) continue;
        Trial t = run_trial(g, srcs, k, cand, dist, d_hash, s);
        ++trials;
        if (t.rc != BFS_OK) {
          if (t.rc == BFS_EINVAL) continue;  // e.g. an occupancy the block shape does not allow
          rc = t.rc;
          break;
        }
        if (t.hash != ref_hash) {
          rc = BFS_ECUDA;  // a parameter changed the distances: never expected
          break;
        }
        if (t.median_ms < best.median_ms * 0.98) {
          best = t;
          cur = cand;
        }
      }
      if (rc != BFS_OK) break;
    }
  }
  cudaStreamDestroy(s);
  cudaFree(dist);
  cudaFree(d_hash);
  if (rc != BFS_OK) return rc;
  *out = cur;
  if (report) {
    memset(report, 0, sizeof(*report));
    report->trials = trials;
    report->start_ms = start_ms;
    report->best_ms = best.median_ms;
    report->sources = k;
  }
  return BFS_OK;
}
