// C ABI: graph upload / validation / release, single-source entry points,
// error strings and parameter defaults.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "bfs_internal.cuh"

namespace gbfs {

// Parent arrays (bfs_parents.cu).
int run_parents(bfs_graph* g, const int* dist, int* parent, cudaStream_t s);
void free_parent_ws_of(const bfs_graph* g);

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  fprintf(stderr, "libbfs: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return BFS_ENOMEM;
  }
  return BFS_ECUDA;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory registered with CUDA (pinned),
// through which kernels can store into it directly; null for pageable memory.
void* pinned_device_alias(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

namespace {

// Validation result bits.
enum : unsigned { kBadFirst = 1, kBadLast = 2, kBadOrder = 4, kBadCol = 8 };

template <typename RP>
__global__ void k_validate_rows(const RP* rp, long long n, long long m, unsigned* bad) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  if (tid == 0) {
    if (rp[0] != 0) atomicOr(bad, kBadFirst);
    if ((long long)rp[n] != m) atomicOr(bad, kBadLast);
  }
  for (long long v = tid; v < n; v += nth)
    if (rp[v + 1] < rp[v]) atomicOr(bad, kBadOrder);
}

__global__ void k_validate_cols(const int* col, long long m, long long n, unsigned* bad) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long j = tid; j < m; j += nth) {
    const int c = col[j];
    if (c < 0 || (long long)c >= n) atomicOr(bad, kBadCol);
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Symmetry: the multiset of arcs (u,v) equals that of (v,u) iff (with
// overwhelming probability) the sums of a 64-bit hash of (u,v) and of (v,u)
// over all arcs agree, for two independent hashes.
template <typename RP>
__global__ void k_symmetry_hash(const RP* rp, const int* col, long long n, unsigned long long* sums) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long a0 = 0, a1 = 0, b0 = 0, b1 = 0;
  for (long long u = gw; u < n; u += nwarps) {
    for (long long j = (long long)rp[u] + lane; j < (long long)rp[u + 1]; j += 32) {
      const unsigned long long v = (unsigned long long)col[j];
      const unsigned long long fw = ((unsigned long long)u << 32) | v, bw = (v << 32) | (unsigned long long)u;
      a0 += mix64(fw ^ 0x1234567ull);
      a1 += mix64(fw * 0x9E3779B97F4A7C15ull + 7ull);
      b0 += mix64(bw ^ 0x1234567ull);
      b1 += mix64(bw * 0x9E3779B97F4A7C15ull + 7ull);
    }
  }
  atomicAdd(&sums[0], a0);
  atomicAdd(&sums[1], a1);
  atomicAdd(&sums[2], b0);
  atomicAdd(&sums[3], b1);
}

// Degree facts and the visited-mask of vertices that BFS never needs to scan:
// degree-0 vertices (reachable only as the source) and padding bits >= n.
template <typename RP>
__global__ void k_degree_mask(const RP* rp, long long n, int nw, unsigned* mask, unsigned long long* facts) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long mx = 0, iso = 0;
  for (long long w = gw; w < nw; w += nwarps) {
    const long long v = w * 32 + lane;
    bool set = true;
    if (v < n) {
      const long long d = (long long)rp[v + 1] - (long long)rp[v];
      set = d == 0;
      if (d > (long long)mx) mx = (unsigned long long)d;
      iso += set ? 1 : 0;
    }
    const unsigned word = __ballot_sync(kFull, set);
    if (lane == 0) mask[w] = word;
  }
  atomicMax(&facts[0], mx);
  atomicAdd(&facts[1], iso);
}

template <typename RP>
int validate_and_facts(bfs_graph* g, int flags) {
  unsigned long long* d_buf = nullptr;
  GBFS_CUDA(cudaMalloc(&d_buf, 8 * sizeof(unsigned long long)));
  GBFS_CUDA(cudaMemset(d_buf, 0, 8 * sizeof(unsigned long long)));
  const RP* rp = reinterpret_cast<const RP*>(g->rp);
  const int grid = g->num_sms * 4, block = 256;
  unsigned long long h[8] = {0};
  int rc = BFS_OK;
  if (flags & (BFS_VALIDATE | BFS_VALIDATE_SYMMETRY)) {
    unsigned* bad = reinterpret_cast<unsigned*>(d_buf + 7);
    k_validate_rows<RP><<<grid, block>>>(rp, g->n, g->m, bad);
    k_validate_cols<<<grid, block>>>(g->col, g->m, g->n, bad);
    cudaError_t e = cudaMemcpy(h, d_buf, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaFree(d_buf);
      return cuda_fail(e, "validate", __FILE__, __LINE__);
    }
    if ((unsigned)h[7] != 0) rc = BFS_EINVAL;
    if (rc == BFS_OK && (flags & BFS_VALIDATE_SYMMETRY)) {
      k_symmetry_hash<RP><<<grid, block>>>(rp, g->col, g->n, d_buf);
      e = cudaMemcpy(h, d_buf, sizeof(h), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        cudaFree(d_buf);
        return cuda_fail(e, "symmetry", __FILE__, __LINE__);
      }
      if (h[0] != h[2] || h[1] != h[3]) rc = BFS_EINVAL;
    }
  }
  if (rc == BFS_OK) {
    cudaMemset(d_buf, 0, 8 * sizeof(unsigned long long));
    k_degree_mask<RP><<<grid, block>>>(rp, g->n, g->nw, g->init_vis, d_buf);
    cudaError_t e = cudaMemcpy(h, d_buf, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaFree(d_buf);
      return cuda_fail(e, "degree facts", __FILE__, __LINE__);
    }
    g->max_deg = (long long)h[0];
    g->isolated = (long long)h[1];
    // Degrees are handled as int32 inside the kernels (with room for one chunk).
    if (g->max_deg >= (1ll << 31) - (1ll << 16)) rc = BFS_EINVAL;
  }
  cudaFree(d_buf);
  return rc;
}

void release_graph(bfs_graph* g) {
  if (!g) return;
  free_single_ws(g);
  free_multi_ws(g);
  free_relabel(g);
  free_nonatomic_ws(g->na);
  g->na = nullptr;
  free_parent_ws_of(g);
  if (g->rp) cudaFree(g->rp);
  if (g->col) cudaFree(g->col);
  if (g->init_vis) cudaFree(g->init_vis);
  if (g->head) cudaFree(g->head);
  delete g;
}

// head[v] = {col[s] or -1, col[s+1] or -1, s, degree} with s = rp[v].
template <typename RP>
__global__ void k_build_head(const RP* rp, const int* col, long long n, int4* head) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += nth) {
    const long long s = (long long)rp[v];
    const long long d = (long long)rp[v + 1] - s;
    head[v] = make_int4(d > 0 ? col[s] : -1, d > 1 ? col[s + 1] : -1, (int)s, (int)d);
  }
}

}  // namespace

// The per-vertex head table (built after any reordering of the lists).  List
// starts are stored as int32, so graphs with m >= 2^31 get none.
int build_head(bfs_graph* g) {
  if (g->m >= ((long long)1 << 31) - 8) return BFS_OK;
  GBFS_CUDA(cudaMalloc(&g->head, sizeof(int4) * (size_t)g->n));
  const int grid = g->num_sms * 4, block = 256;
  if (g->rp_bits == 32)
    k_build_head<int><<<grid, block>>>(static_cast<const int*>(g->rp), g->col, g->n, g->head);
  else
    k_build_head<long long><<<grid, block>>>(static_cast<const long long*>(g->rp), g->col, g->n, g->head);
  GBFS_CUDA(cudaGetLastError());
  GBFS_CUDA(cudaDeviceSynchronize());
  return BFS_OK;
}

// Head table and visited mask of the degree-renumbered copy, and its new_of
// on the host, for single-source queries that run on it.
int ensure_relabel_single(bfs_graph* g) {
  int rc = ensure_relabel(g);
  if (rc != BFS_OK) return rc;
  Relabel* r = g->rl;
  if (r->h_new_of) return BFS_OK;
  const int grid = g->num_sms * 4, block = 256;
  GBFS_CUDA(cudaMalloc(&r->init_vis, sizeof(unsigned) * (size_t)g->nw));
  unsigned long long* d_facts = nullptr;
  GBFS_CUDA(cudaMalloc(&d_facts, 8 * sizeof(unsigned long long)));
  GBFS_CUDA(cudaMemset(d_facts, 0, 8 * sizeof(unsigned long long)));
  if (g->rp_bits == 32)
    k_degree_mask<int><<<grid, block>>>(static_cast<const int*>(r->rp), g->n, g->nw, r->init_vis, d_facts);
  else
    k_degree_mask<long long><<<grid, block>>>(static_cast<const long long*>(r->rp), g->n, g->nw, r->init_vis, d_facts);
  if (g->head) {
    GBFS_CUDA(cudaMalloc(&r->head, sizeof(int4) * (size_t)g->n));
    if (g->rp_bits == 32)
      k_build_head<int><<<grid, block>>>(static_cast<const int*>(r->rp), r->col, g->n, r->head);
    else
      k_build_head<long long><<<grid, block>>>(static_cast<const long long*>(r->rp), r->col, g->n, r->head);
  }
  GBFS_CUDA(cudaGetLastError());
  GBFS_CUDA(cudaDeviceSynchronize());
  cudaFree(d_facts);
  int* h = static_cast<int*>(malloc(sizeof(int) * (size_t)g->n));
  if (!h) return BFS_ENOMEM;
  const cudaError_t e = cudaMemcpy(h, r->new_of, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(h);
    return cuda_fail(e, "cudaMemcpy (new_of)", __FILE__, __LINE__);
  }
  r->h_new_of = h;
  return BFS_OK;
}

int ensure_single_ws(bfs_graph* g) {
  SingleWs& ws = g->ws;
  if (ws.ready) return BFS_OK;
  const size_t nwb = sizeof(unsigned) * (size_t)g->nw;
  ws.cap = g->n + g->m / 256 + 2;
  GBFS_CUDA(cudaMalloc(&ws.vis, nwb));
  GBFS_CUDA(cudaMalloc(&ws.lv8, (size_t)(g->n + 15) / 16 * 16));
  for (int i = 0; i < 2; ++i) {
    GBFS_CUDA(cudaMalloc(&ws.bm[i], nwb));
    GBFS_CUDA(cudaMemset(ws.bm[i], 0, nwb));
    GBFS_CUDA(cudaMalloc(&ws.qv[i], sizeof(int) * (size_t)g->n));
    GBFS_CUDA(cudaMalloc(&ws.it[i], sizeof(unsigned long long) * (size_t)ws.cap));
    GBFS_CUDA(cudaMalloc(&ws.mg[i], sizeof(MegaRec) * (size_t)(g->m / 8192 + 2)));
  }
  GBFS_CUDA(cudaMalloc(&ws.ctrl, sizeof(Ctrl)));
  GBFS_CUDA(cudaMemset(ws.ctrl, 0, sizeof(Ctrl)));
  GBFS_CUDA(cudaMalloc(&ws.sticky, sizeof(int)));
  GBFS_CUDA(cudaMemset(ws.sticky, 0, sizeof(int)));
  GBFS_CUDA(cudaMallocHost(&ws.h_ctrl, sizeof(Ctrl)));
  GBFS_CUDA(cudaMallocHost(&ws.h_slot, sizeof(Slot)));
  GBFS_CUDA(cudaEventCreateWithFlags(&ws.done, cudaEventDisableTiming));
  ws.ready = true;
  return BFS_OK;
}

void free_single_ws(bfs_graph* g) {
  SingleWs& ws = g->ws;
  if (ws.done) cudaEventSynchronize(ws.done);
  if (ws.gexec) cudaGraphExecDestroy(ws.gexec);
  if (ws.graph) cudaGraphDestroy(ws.graph);
  cudaFree(ws.vis);
  for (int i = 0; i < 2; ++i) {
    cudaFree(ws.bm[i]);
    cudaFree(ws.qv[i]);
    cudaFree(ws.it[i]);
    cudaFree(ws.mg[i]);
  }
  cudaFree(ws.ctrl);
  cudaFree(ws.sticky);
  cudaFree(ws.dist_tmp);
  cudaFree(ws.lv8);
  cudaFree(ws.lst);
  if (ws.h_ctrl) cudaFreeHost(ws.h_ctrl);
  if (ws.h_slot) cudaFreeHost(ws.h_slot);
  if (ws.done) cudaEventDestroy(ws.done);
  ws = SingleWs();
}

static int check_params(const bfs_params& p) {
  if (p.policy < 0 || p.policy > BFS_POLICY_LOCAL) return BFS_EINVAL;
  if (p.local_levels < 1 || p.local_levels > 4096) return BFS_EINVAL;
  if (p.local_threads < 64 || p.local_threads > 512 || (p.local_threads & 31)) return BFS_EINVAL;
  if (p.launch < 0 || p.launch > BFS_LAUNCH_GRAPH) return BFS_EINVAL;
  if (p.alpha < 1 || p.beta < 1 || p.tau_inv < 1) return BFS_EINVAL;
  if (p.small_max < 1 || p.small_max > 32) return BFS_EINVAL;
  if (p.chunk < 256 || p.chunk > 65535) return BFS_EINVAL;
  if (p.bu_warp_min < 0 || p.bu_warp_min > (1 << 24)) return BFS_EINVAL;
  if (p.threads_per_block < 64 || p.threads_per_block > 1024 || (p.threads_per_block & 31)) return BFS_EINVAL;
  if (p.blocks_per_sm < 0 || p.timeout_ms < 1 || p.test_barrier_extra < 0) return BFS_EINVAL;
  if (p.bu_chunk < 0 || p.bu_chunk > 65536) return BFS_EINVAL;
  if (p.bu_thread_max < 0 || p.bu_thread_max > (1 << 20)) return BFS_EINVAL;
  if (p.ms_lanes < 1 || p.ms_lanes > 256 || p.ms_ring < 2 || p.ms_ring > 16 || p.ms_heavy_min < 0) return BFS_EINVAL;
  if (p.ms_degree_order < 0 || p.ms_degree_order > 1) return BFS_EINVAL;
  if (p.ms_alpha < 1) return BFS_EINVAL;
  if (p.ms_relabel < 0 || p.ms_relabel > 1) return BFS_EINVAL;
  if (p.relabel < 0 || p.relabel > 1) return BFS_EINVAL;
  return BFS_OK;
}

}  // namespace gbfs

using namespace gbfs;

extern "C" {

const char* bfs_strerror(int code) {
  switch (code) {
    case BFS_OK: return "success";
    case BFS_EINVAL: return "invalid argument";
    case BFS_ENOMEM: return "out of memory or over the memory budget";
    case BFS_ECUDA: return "CUDA runtime error";
    case BFS_ETIMEOUT: return "device-side wait timed out";
    case BFS_EAGAIN: return "queue full, try again";
    case BFS_ERANGE: return "distance does not fit the output type";
    case BFS_ENOTFOUND: return "unknown ticket or graph id";
    default: return "unknown error code";
  }
}

int bfs_version(void) { return 10000; }

int bfs_debug_bounds(uint64_t* first_violation, int* checked, int reset) {
  if (!first_violation) return BFS_EINVAL;
  unsigned long long a = 0, b = 0;
  const bool ca = bounds_read_single(&a, reset != 0);
  const bool cb = bounds_read_local(&b, reset != 0);
  if (checked) *checked = (ca || cb) ? 1 : 0;
  *first_violation = a ? a : b;
  return cudaGetLastError() == cudaSuccess ? BFS_OK : BFS_ECUDA;
}

void bfs_params_default(bfs_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->policy = BFS_POLICY_AUTO;
  p->launch = BFS_LAUNCH_PERSISTENT;
  p->alpha = 14;
  p->beta = 24;
  p->tau_inv = 20;
  p->large_diameter_degree = 7;
  p->small_max = 32;
  p->chunk = 256;
  p->bu_warp_min = 32;
  p->threads_per_block = 512;
  p->blocks_per_sm = 0;
  p->timeout_ms = 10000;
  p->script = 0;
  p->test_barrier_extra = 0;
  p->bu_chunk = 0;
  p->bu_thread_max = 32;
  p->ms_lanes = 256;
  p->ms_ring = 16;
  p->ms_heavy_min = 256;
  p->ms_degree_order = 1;
  p->ms_alpha = 2;
  p->ms_relabel = 1;
  p->local_levels = 16;
  p->local_threads = 64;
}

int bfs_graph_upload(const void* row_ptr, int row_ptr_bits, const int32_t* col_idx, int64_t n, int64_t m,
                     int flags, bfs_graph** out) {
  GBFS_NVTX("bfs_graph_upload");
  if (!out) return BFS_EINVAL;
  *out = nullptr;
  if (!row_ptr || (m > 0 && !col_idx)) return BFS_EINVAL;
  if (n < 1 || n >= ((int64_t)1 << 31) || m < 0 || m >= ((int64_t)1 << 39)) return BFS_EINVAL;
  if (row_ptr_bits != 32 && row_ptr_bits != 64) return BFS_EINVAL;
  if (row_ptr_bits == 32 && m >= ((int64_t)1 << 31)) return BFS_EINVAL;
  const bool dev = (flags & BFS_DEVICE_PTRS) != 0;
  bfs_graph* g = new (std::nothrow) bfs_graph();
  if (!g) return BFS_ENOMEM;
  g->n = n;
  g->m = m;
  g->rp_bits = row_ptr_bits;
  g->nw = (int)((n + 31) / 32);
  int rc = BFS_OK;
  do {
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__); break; }
    e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaDeviceGetAttribute", __FILE__, __LINE__); break; }
    const size_t rpb = (size_t)(row_ptr_bits / 8) * (size_t)(n + 1);
    const size_t mpad = (size_t)((m + 3) / 4 * 4 + 4);
    e = cudaMalloc(&g->rp, rpb);
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(int) * mpad);
    if (e == cudaSuccess) e = cudaMalloc(&g->init_vis, sizeof(unsigned) * (size_t)g->nw);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc (graph)", __FILE__, __LINE__); break; }
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = cudaMemcpy(g->rp, row_ptr, rpb, kind);
    if (e == cudaSuccess) e = cudaMemset(g->col + m, 0, sizeof(int) * (mpad - (size_t)m));
    if (e == cudaSuccess && m > 0) e = cudaMemcpy(g->col, col_idx, sizeof(int) * (size_t)m, kind);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpy (graph)", __FILE__, __LINE__); break; }
    rc = row_ptr_bits == 32 ? validate_and_facts<int>(g, flags) : validate_and_facts<long long>(g, flags);
    if (rc == BFS_OK && (flags & BFS_DEGREE_ORDER)) {
      rc = reorder_by_degree(g);
      g->deg_ordered = rc == BFS_OK;
    }
    if (rc == BFS_OK && !(flags & BFS_NO_HEAD)) rc = build_head(g);
  } while (0);
  if (rc != BFS_OK) {
    release_graph(g);
    return rc;
  }
  *out = g;
  return BFS_OK;
}

void bfs_graph_free(bfs_graph* g) {
  GBFS_NVTX("bfs_graph_free");
  if (!g) return;
  cudaDeviceSynchronize();
  release_graph(g);
}

int bfs_graph_info(const bfs_graph* g, int64_t* n, int64_t* m, int64_t* max_degree, int64_t* isolated) {
  if (!g) return BFS_EINVAL;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (max_degree) *max_degree = g->max_deg;
  if (isolated) *isolated = g->isolated;
  return BFS_OK;
}

int bfs_single_ex(bfs_graph* g, int32_t src, int32_t* dist, const bfs_params* params, bfs_stats* stats,
                  bfs_level_stat* levels, int32_t level_cap, void* stream) {
  GBFS_NVTX("bfs_single_ex");
  if (!g || !dist) return BFS_EINVAL;
  if (src < 0 || (int64_t)src >= g->n) return BFS_EINVAL;
  if (level_cap < 0 || (level_cap > 0 && !levels)) return BFS_EINVAL;
  bfs_params p;
  if (params) {
    p = *params;
  } else {
    bfs_params_default(&p);
  }
  int rc = check_params(p);
  if (rc != BFS_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  rc = ensure_single_ws(g);
  if (rc != BFS_OK) return rc;
  if (p.relabel) {
    rc = ensure_relabel_single(g);
    if (rc != BFS_OK) return rc;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (is_device_pointer(dist)) return run_single(g, src, dist, p, stats, levels, level_cap, s);
  // Pinned host output: the kernel stores the distances straight into it (the
  // transfer to the host overlaps the final expansion instead of following it).
  // The multi-level local kernel relaxes distances with atomics: staged instead.
  if (!uses_local_kernel(g, p))
    if (int* alias = static_cast<int*>(pinned_device_alias(dist)))
      return run_single(g, src, alias, p, stats, levels, level_cap, s);
  SingleWs& ws = g->ws;
  if (!ws.dist_tmp) GBFS_CUDA(cudaMalloc(&ws.dist_tmp, sizeof(int) * (size_t)g->n));
  rc = run_single(g, src, ws.dist_tmp, p, stats, levels, level_cap, s);
  if (rc != BFS_OK) return rc;
  GBFS_CUDA(cudaMemcpyAsync(dist, ws.dist_tmp, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  GBFS_CUDA(cudaEventRecord(ws.done, s));
  GBFS_CUDA(cudaStreamSynchronize(s));
  return BFS_OK;
}

int bfs_single(bfs_graph* g, int32_t src, int32_t* dist, void* stream) {
  return bfs_single_ex(g, src, dist, nullptr, nullptr, nullptr, 0, stream);
}

int bfs_single_async(bfs_graph* g, int32_t src, int32_t* dist, const bfs_params* params, void* stream) {
  GBFS_NVTX("bfs_single_async");
  if (!g || !dist) return BFS_EINVAL;
  if (src < 0 || (int64_t)src >= g->n) return BFS_EINVAL;
  bfs_params p;
  if (params) {
    p = *params;
  } else {
    bfs_params_default(&p);
  }
  int rc = check_params(p);
  if (rc != BFS_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  rc = ensure_single_ws(g);
  if (rc != BFS_OK) return rc;
  if (p.relabel) {
    rc = ensure_relabel_single(g);
    if (rc != BFS_OK) return rc;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* out = is_device_pointer(dist) ? dist : nullptr;
  if (!out && !uses_local_kernel(g, p)) out = static_cast<int*>(pinned_device_alias(dist));
  if (!out) return BFS_EINVAL;  // pageable host memory would need a staged copy and a wait
  return run_single(g, src, out, p, nullptr, nullptr, 0, s, false);
}

int bfs_single_wait(bfs_graph* g) {
  GBFS_NVTX("bfs_single_wait");
  if (!g) return BFS_EINVAL;
  std::lock_guard<std::mutex> lock(g->mu);
  SingleWs& ws = g->ws;
  if (!ws.ready) return BFS_OK;
  GBFS_CUDA(cudaEventSynchronize(ws.done));
  // Queries before the last one left their status in the sticky word (folded
  // when the next query was enqueued); the last one's is still in the block.
  int sticky = 0, last = 0;
  GBFS_CUDA(cudaMemcpy(&sticky, ws.sticky, sizeof(int), cudaMemcpyDeviceToHost));
  GBFS_CUDA(cudaMemcpy(&last, &ws.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (sticky != 0) GBFS_CUDA(cudaMemset(ws.sticky, 0, sizeof(int)));
  if (last != 0) GBFS_CUDA(cudaMemset(&ws.ctrl->status, 0, sizeof(int)));
  return sticky != 0 ? sticky : last;
}

int bfs_multi_ex(bfs_graph* g, const int32_t* srcs, int32_t k, void* dist, int dist_bits, const bfs_params* params,
                 bfs_multi_stats* stats, void* stream) {
  GBFS_NVTX("bfs_multi_ex");
  if (!g || !srcs || !dist || k <= 0) return BFS_EINVAL;
  if (dist_bits != 8 && dist_bits != 32) return BFS_EINVAL;
  for (int32_t i = 0; i < k; ++i)
    if (srcs[i] < 0 || (int64_t)srcs[i] >= g->n) return BFS_EINVAL;
  bfs_params p;
  if (params) {
    p = *params;
  } else {
    bfs_params_default(&p);
  }
  int rc = check_params(p);
  if (rc != BFS_OK) return rc;
  if (stats) memset(stats, 0, sizeof(*stats));
  std::lock_guard<std::mutex> lock(g->mu);
  return run_multi(g, srcs, k, dist, dist_bits, p, stats, reinterpret_cast<cudaStream_t>(stream));
}

int bfs_parents(bfs_graph* g, const int32_t* dist, int32_t* parent, void* stream) {
  GBFS_NVTX("bfs_parents");
  if (!g || !dist || !parent) return BFS_EINVAL;
  if (!is_device_pointer(dist) || !is_device_pointer(parent)) return BFS_EINVAL;
  std::lock_guard<std::mutex> lock(g->mu);
  return run_parents(g, dist, parent, reinterpret_cast<cudaStream_t>(stream));
}

int bfs_single_nonatomic_ex(bfs_graph* g, int32_t src, int32_t* dist, int mode, bfs_dup_stats* stats,
                            bfs_dup_level* levels, int32_t level_cap, void* stream) {
  GBFS_NVTX("bfs_single_nonatomic");
  if (!g || !dist) return BFS_EINVAL;
  if (src < 0 || (int64_t)src >= g->n) return BFS_EINVAL;
  if (mode != BFS_DUP_DEDUP && mode != BFS_DUP_EXPAND) return BFS_EINVAL;
  if (level_cap < 0 || (level_cap > 0 && !levels)) return BFS_EINVAL;
  if (!is_device_pointer(dist)) return BFS_EINVAL;
  std::lock_guard<std::mutex> lock(g->mu);
  return run_nonatomic(g, src, dist, mode, stats, levels, level_cap, reinterpret_cast<cudaStream_t>(stream));
}

int bfs_single_nonatomic(bfs_graph* g, int32_t src, int32_t* dist, bfs_dup_stats* stats, bfs_dup_level* levels,
                         int32_t level_cap, void* stream) {
  return bfs_single_nonatomic_ex(g, src, dist, BFS_DUP_DEDUP, stats, levels, level_cap, stream);
}

int bfs_multi(bfs_graph* g, const int32_t* srcs, int32_t k, void* dist, int dist_bits, void* stream) {
  return bfs_multi_ex(g, srcs, k, dist, dist_bits, nullptr, nullptr, stream);
}

}  // extern "C"
