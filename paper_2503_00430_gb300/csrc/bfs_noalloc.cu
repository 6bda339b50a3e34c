// bfs_single_noalloc: single-source BFS that allocates no memory at all.
//
// Who needs it: code that must not call cudaMalloc (or any allocator) at the
// moment it runs a BFS - for example a caller that runs inside a memory pool
// or arena it does not own and may not grow, a real-time or signal-like
// context where an allocation could block on the driver's allocator lock or
// trigger an implicit device synchronisation, or a host that has reserved all
// device memory up front.  Such a caller hands over its graph and its output
// buffer as plain device pointers; everything else the kernel needs lives in
// one statically sized device array declared in this file.
//
// The array (kNoallocScratchBytes = 64 MiB) is created by the CUDA runtime
// together with this file's device code and stays reserved on every GPU that
// loads it until the process exits.  Graphs whose scratch does not fit are
// rejected with BFS_ENOMEM.  All calls share the array and it keeps the last
// call's contents, so calls that can overlap on the GPU (different streams,
// or different host threads without ordering) race and corrupt each other;
// callers must order them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "bfs_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;
constexpr int kMaxDevices = 64;

// The scratch array itself.  Host code must not use this name as an address:
// on the host it is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte layout of the scratch for a graph with n vertices and m entries.
struct Layout {
  size_t ctrl, init_vis, vis, bm0, bm1, qv0, qv1, it0, it1, mg0, mg1, total;
  long long cap;
};

Layout layout_for(long long n, long long m) {
  Layout L{};
  const size_t nwb = sizeof(unsigned) * (size_t)((n + 31) / 32);
  L.cap = n + m / 256 + 2;
  size_t off = 0;
  L.ctrl = off; off += round256(sizeof(gbfs::Ctrl));
  L.init_vis = off; off += round256(nwb);
  L.vis = off; off += round256(nwb);
  L.bm0 = off; off += round256(nwb);
  L.bm1 = off; off += round256(nwb);
  L.qv0 = off; off += round256(sizeof(int) * (size_t)n);
  L.qv1 = off; off += round256(sizeof(int) * (size_t)n);
  L.it0 = off; off += round256(sizeof(unsigned long long) * (size_t)L.cap);
  L.it1 = off; off += round256(sizeof(unsigned long long) * (size_t)L.cap);
  L.mg0 = off; off += round256(sizeof(gbfs::MegaRec) * (size_t)(m / 8192 + 2));
  L.mg1 = off; off += round256(sizeof(gbfs::MegaRec) * (size_t)(m / 8192 + 2));
  L.total = off;
  return L;
}

// Visited mask of vertices BFS never scans: degree 0, and padding bits >= n.
template <typename RP>
__global__ void k_noalloc_mask(const RP* rp, long long n, int nw, unsigned* mask) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  for (long long w = gw; w < nw; w += nwarps) {
    const long long v = w * 32 + lane;
    bool set = true;
    if (v < n) set = rp[v + 1] == rp[v];
    const unsigned word = __ballot_sync(0xffffffffu, set);
    if (lane == 0) mask[w] = word;
  }
}

// Per-device set-up: the device address of the scratch array (with this
// device current) and its SM count.  Runs once per device, on the first call.
int setup_device(int dev, void** scratch, int* num_sms) {
  if (dev < 0 || dev >= kMaxDevices) return BFS_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return gbfs::cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return gbfs::cuda_fail(e, "cudaDeviceGetAttribute", __FILE__, __LINE__);
    g_num_sms[dev] = sms;
    g_scratch_dev[dev] = p;
  }
  *scratch = g_scratch_dev[dev];
  *num_sms = g_num_sms[dev];
  return BFS_OK;
}

}  // namespace

extern "C" int bfs_single_noalloc(const void* row_ptr, int row_ptr_bits, const int32_t* col_idx, int64_t n,
                                  int64_t m, int32_t src, int32_t* dist, void* stream) {
  GBFS_NVTX("bfs_single_noalloc");
  using namespace gbfs;
  if (!row_ptr || !dist || (m > 0 && !col_idx)) return BFS_EINVAL;
  if (row_ptr_bits != 32 && row_ptr_bits != 64) return BFS_EINVAL;
  if (n < 1 || n >= ((int64_t)1 << 31) || m < 0 || (row_ptr_bits == 32 && m >= ((int64_t)1 << 31)))
    return BFS_EINVAL;
  if (src < 0 || (int64_t)src >= n) return BFS_EINVAL;
  // The kernel reads neighbour ids with aligned 16-byte loads, row pointers and
  // distances with naturally aligned loads and stores: a misaligned view (an
  // offset slice, a pool sub-allocation) would fault on the device, so it is
  // rejected here, before anything is launched.
  if ((m > 0 && (reinterpret_cast<uintptr_t>(col_idx) & 15u) != 0) ||
      (reinterpret_cast<uintptr_t>(row_ptr) & (uintptr_t)(row_ptr_bits / 8 - 1)) != 0 ||
      (reinterpret_cast<uintptr_t>(dist) & 3u) != 0)
    return BFS_EINVAL;
  const Layout lay = layout_for(n, m);
  if (lay.total > kNoallocScratchBytes) return BFS_ENOMEM;  // graph too large for the static scratch
  int dev = 0;
  GBFS_CUDA(cudaGetDevice(&dev));
  void* base = nullptr;
  int num_sms = 0;
  int rc = setup_device(dev, &base, &num_sms);
  if (rc != BFS_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bfs_params p;
  bfs_params_default(&p);
  KParams K;
  K.rp = row_ptr;
  K.col = col_idx;
  K.n = n;
  K.m = m;
  K.nw = (int)((n + 31) / 32);
  K.src = src;
  K.init_vis = reinterpret_cast<unsigned*>(b + lay.init_vis);
  K.head = nullptr;
  K.lv8 = nullptr;
  K.n_live = n;
  K.dist = dist;
  K.vis = reinterpret_cast<unsigned*>(b + lay.vis);
  K.bm0 = reinterpret_cast<unsigned*>(b + lay.bm0);
  K.bm1 = reinterpret_cast<unsigned*>(b + lay.bm1);
  K.qv0 = reinterpret_cast<int*>(b + lay.qv0);
  K.qv1 = reinterpret_cast<int*>(b + lay.qv1);
  K.it0 = reinterpret_cast<unsigned long long*>(b + lay.it0);
  K.it1 = reinterpret_cast<unsigned long long*>(b + lay.it1);
  K.cap = lay.cap;
  K.mg0 = reinterpret_cast<MegaRec*>(b + lay.mg0);
  K.mg1 = reinterpret_cast<MegaRec*>(b + lay.mg1);
  K.ctrl = reinterpret_cast<Ctrl*>(b + lay.ctrl);
  K.lst = nullptr;
  K.lst_cap = 0;
  // Section 3's graph classes: average degree below 7 -> top-down only, else the edge-count rule.
  K.policy = ((double)m < (double)p.large_diameter_degree * (double)n) ? BFS_POLICY_TD_ONLY : BFS_POLICY_EDGES;
  K.alpha = p.alpha;
  K.beta = p.beta;
  K.tau_inv = p.tau_inv;
  K.script = 0;
  K.small_max = p.small_max;
  K.chunk = p.chunk;
  K.bu_warp_min = p.bu_warp_min;
  K.bu_chunk = p.bu_chunk;
  K.bu_thread_max = p.bu_thread_max;
  K.need_qv = K.policy != BFS_POLICY_TD_ONLY;
  K.timeout_ns = (long long)p.timeout_ms * 1000000ll;
  K.barrier_extra = 0;
  K.col_cap = (m + 3) / 4 * 4;  // 16-byte loads stay inside the block holding the last entry
  K.mg_cap = m / 8192 + 2;
  // The previous call left its control block behind: it must start at zero.
  GBFS_CUDA(cudaMemsetAsync(K.ctrl, 0, sizeof(Ctrl), s));
  const int mask_grid = num_sms * 4;
  if (row_ptr_bits == 32)
    k_noalloc_mask<int><<<mask_grid, 256, 0, s>>>(static_cast<const int*>(row_ptr), n, K.nw,
                                                  const_cast<unsigned*>(K.init_vis));
  else
    k_noalloc_mask<long long><<<mask_grid, 256, 0, s>>>(static_cast<const long long*>(row_ptr), n, K.nw,
                                                        const_cast<unsigned*>(K.init_vis));
  GBFS_CUDA(cudaGetLastError());
  rc = launch_persistent_prepared(K, row_ptr_bits, num_sms, p.threads_per_block, s);
  if (rc != BFS_OK) return rc;
  int status = 0;
  GBFS_CUDA(cudaMemcpyAsync(&status, &K.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  GBFS_CUDA(cudaStreamSynchronize(s));
  return status;
}
