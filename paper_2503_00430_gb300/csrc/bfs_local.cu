// Multi-level local expansion for large-diameter graphs (BFS_POLICY_LOCAL).
//
// Paper mapping: Section 2, "Other Optimizations" (c) lets threads run several
// top-down levels on their own part of the frontier without merging in
// between; Section 3 gives large-diameter graphs (average degree below 7) a
// top-down-only path because their thousands of levels are dominated by
// synchronisation.  On this GPU a level of a 4096 x 4096 grid costs ~9 us in
// the level-synchronous persistent kernel: a chain of dependent global
// accesses (work item, neighbour ids, visited word, claim, head record) plus
// the same-address append atomics of every warp, then the grid barrier.
//
// Here one persistent cooperative launch runs "super-steps".  In a super-step
// every block takes a contiguous share of the global frontier queue and
// expands it for up to K levels on its own, with the next local frontier kept
// in shared memory and only __syncthreads between local levels; vertices found
// at the K-th local level (or when the shared queue is full) go to the next
// global queue.  Then one grid barrier.  A block only sees its own share of
// the frontier, so it can reach a vertex along a path that is not a shortest
// one before the block that owns the shortest path gets there: distances are
// therefore relaxed with atomicMin (label correcting) instead of the plain
// stores of the level-synchronous path, and every vertex whose label drops is
// expanded again by the thread that lowered it.  When a super-step ends with
// an empty global queue, no label can drop any more: every arc (u, v) has
// dist[v] <= dist[u] + 1 and every label is the length of a real path, so the
// labels are the BFS distances (a fixpoint of the relaxation the paper's
// Listing 1 applies, dist[src] + 1 < dist[dst]).
//
// Layout: dist is the caller's int32 output, used as unsigned so that the
// "unreached" value 0xffffffff is both the atomicMin identity and -1; no
// visited bitmap and no level bytes.  Two global queues (int32, n entries
// each) with one "queued" bitmap each, so a vertex enters a global queue at
// most once per super-step (capacity n suffices).
#include <cuda_runtime.h>
#include <stdint.h>

#include "bfs_device.cuh"
#include "bfs_internal.cuh"

namespace gbfs {

namespace {

using namespace dev;

// Bounds-checked build: as in bfs_single.cu, each data-dependent global index
// is checked and the first violation recorded (the access goes to element 0).
#ifdef GBFS_DEBUG_BOUNDS
__device__ unsigned long long g_local_bounds_err;
__device__ __forceinline__ long long lchk(long long i, long long lim, int site) {
  if (i >= 0 && i < lim) return i;
  atomicCAS(&g_local_bounds_err, 0ull,
            (1ull << 63) | ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
  return 0;
}
#define LCHK(i, lim, site) lchk((long long)(i), (long long)(lim), (site))
#else
#define LCHK(i, lim, site) (i)
#endif

constexpr unsigned kInf = 0xffffffffu;
constexpr int kLocalWindow = 1 << 20;  // row entries per lane per pass of a warp group
constexpr int kLocalThreads = 512;     // largest block of the local kernel

// A vertex of a block-local frontier: its label and its row (first two
// neighbours from the head table when there is one).
struct LocalEntry {
  long long start;  // first list entry
  int deg;
  int label;        // distance it was given when queued
  int u;
  int n0, n1;       // first two neighbours (head table), -1 if missing or no head table
  int pad;
};

struct LParams {
  const void* rp;
  const int* col;
  const int4* head;   // or null: read rp
  long long n, m;
  int nw;
  int src;
  unsigned* dist;     // caller's int32[n] viewed as unsigned
  int* q0;
  int* q1;
  unsigned* qb0;      // vertex is in q0 (bitmap, nw words)
  unsigned* qb1;
  Ctrl* ctrl;         // barrier, status, slot[s & 3].nv = |global queue s|, statistics
  bfs_level_stat* lst;
  int lst_cap;
  int K;              // levels per super-step
  int cap_local;      // LocalEntry slots per shared-memory queue
  long long timeout_ns;
  int barrier_extra;
};

template <typename RP>
__device__ __forceinline__ void row_of(const LParams& P, int v, long long& start, int& deg, int& n0, int& n1) {
  if (P.head) {
    const int4 h = __ldg(P.head + LCHK(v, P.n, 101));
    n0 = h.x;
    n1 = h.y;
    start = h.z;
    deg = h.w;
  } else {
    start = rp_at<RP>(P.rp, LCHK(v, P.n + 1, 102));
    deg = (int)(rp_at<RP>(P.rp, LCHK((long long)v + 1, P.n + 1, 103)) - start);
    n0 = n1 = -1;
  }
}

// Per-thread counters of one super-step (statistics variant only).
struct LAcc {
  unsigned long long expanded = 0, examined = 0, improved = 0;
};

// Warp-collective: append the improved candidates of this lane (mask `imp`,
// up to four) to the next global queue, each vertex at most once per queue.
__device__ __forceinline__ void append_global(const LParams& P, int s, const int (&v)[4], unsigned imp) {
  unsigned* qbn = ((s + 1) & 1) ? P.qb1 : P.qb0;
  int* qn = ((s + 1) & 1) ? P.q1 : P.q0;
  unsigned take = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((imp >> k) & 1u) {
      const unsigned bit = 1u << (v[k] & 31);
      if (!(atomicOr(qbn + LCHK(v[k] >> 5, P.nw, 104), bit) & bit)) take |= 1u << k;
    }
  const int cnt = __popc(take);
  if (__ballot_sync(kFull, cnt != 0) == 0) return;
  const int incl = warp_incl_scan(cnt);
  const int tot = __shfl_sync(kFull, incl, 31);
  unsigned long long b = 0;
  if (lane_id() == 31) b = atomicAdd(&P.ctrl->slot[(s + 1) & 3].nv, (unsigned long long)tot);
  b = __shfl_sync(kFull, b, 31) + (unsigned long long)(incl - cnt);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((take >> k) & 1u) qn[LCHK(b++, P.n, 105)] = v[k];
}

// Warp-collective: expand `count` entries of one local frontier (level 0 of a
// super-step: entries lo.. of the global queue; later levels: shared queue A)
// and relax every neighbour to label + 1.  Improved neighbours go to shared
// queue B while `to_local`, else (or when B is full) to the next global queue.
template <typename RP, bool STATS>
__device__ __forceinline__ void expand_local(const LParams& P, int s, bool from_global, const int* gq, long long lo, long long count,
                             const LocalEntry* A, LocalEntry* B, int* nB, bool to_local, LAcc& acc) {
  const unsigned lane = lane_id();
  const int warp = (int)(threadIdx.x >> 5), nwarps = (int)(blockDim.x >> 5);
  unsigned* qb = (s & 1) ? P.qb1 : P.qb0;
  for (long long base = (long long)warp * 32; base < count; base += (long long)nwarps * 32) {
    const long long i = base + lane;
    bool have = i < count;
    int u = -1, label = 0, deg = 0, n0 = -1, n1 = -1;
    long long start = 0;
    if (have) {
      if (from_global) {
        u = gq[LCHK(lo + i, P.n, 106)];
        const unsigned bit = 1u << (u & 31);
        atomicAnd(qb + LCHK(u >> 5, P.nw, 107), ~bit);  // leaves the queue: it may be queued again from now on
        row_of<RP>(P, u, start, deg, n0, n1);
        label = (int)ld_relaxed_u32(P.dist + LCHK(u, P.n, 108));
      } else {
        const LocalEntry& e = A[LCHK(i, P.cap_local, 109)];
        u = e.u;
        label = e.label;
        start = e.start;
        deg = e.deg;
        n0 = e.n0;
        n1 = e.n1;
        // A lower label means another thread lowered it and expands u itself.
        if ((int)ld_relaxed_u32(P.dist + LCHK(u, P.n, 110)) < label) have = false;
      }
    }
    if (!have) deg = 0;
    if (STATS && have) acc.expanded += 1;
    const int skip = P.head ? 2 : 0;  // entries 0 and 1 come from the head record
    // Rows are taken in windows of at most kLocalWindow entries per lane, so the
    // warp's scan of 32 lengths stays within int even for hub vertices.
    long long done = 0;
    for (;;) {
      const long long left = (long long)deg - done;
      const int take = left < (long long)kLocalWindow ? (int)left : kLocalWindow;
      if (__ballot_sync(kFull, take > 0) == 0) break;
      const int incl = warp_incl_scan(take);
      const int excl = incl - take;
      const int total = __shfl_sync(kFull, incl, 31);
      for (int b0 = 0; b0 < total; b0 += 128) {
        int v[4], lab[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = b0 + 32 * k + (int)lane;
          const int o = owner_of(excl, e);
          const long long off = (long long)(e - __shfl_sync(kFull, excl, o)) + __shfl_sync(kFull, done, o);
          const long long so = __shfl_sync(kFull, start, o);
          const int h0 = __shfl_sync(kFull, n0, o), h1 = __shfl_sync(kFull, n1, o);
          lab[k] = __shfl_sync(kFull, label, o) + 1;
          v[k] = -1;
          if (e < total) v[k] = off < skip ? (off == 0 ? h0 : h1) : __ldg(P.col + LCHK(so + off, P.m, 111));
        }
        unsigned imp = 0;
        long long rs[4];
        int rd[4], r0[4], r1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          rs[k] = 0;
          rd[k] = 0;
          r0[k] = r1[k] = -1;
          if (v[k] >= 0) {
            const unsigned old = atomicMin(P.dist + LCHK(v[k], P.n, 112), (unsigned)lab[k]);
            if (old > (unsigned)lab[k]) imp |= 1u << k;
            if (to_local) row_of<RP>(P, v[k], rs[k], rd[k], r0[k], r1[k]);  // issued with the claim
            if (STATS) acc.examined += 1;
          }
        }
        if (STATS) acc.improved += (unsigned long long)__popc(imp);
        unsigned glob = imp;
        if (to_local) {
          const int cnt = __popc(imp);
          const int ci = warp_incl_scan(cnt);
          const int ct = __shfl_sync(kFull, ci, 31);
          int bb = 0;
          if (ct > 0) {
            if (lane == 31) bb = atomicAdd(nB, ct);
            bb = __shfl_sync(kFull, bb, 31) + (ci - cnt);
          }
          glob = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if ((imp >> k) & 1u) {
              if (bb < P.cap_local) {
                LocalEntry& d = B[LCHK(bb, P.cap_local, 113)];
                d.start = rs[k];
                d.deg = rd[k];
                d.label = lab[k];
                d.u = v[k];
                d.n0 = r0[k];
                d.n1 = r1[k];
              } else {
                glob |= 1u << k;  // shared queue full: the vertex waits in the global queue
              }
              ++bb;
            }
        }
        append_global(P, s, v, glob);
      }
      done += take;
    }
  }
}

template <typename RP, bool STATS>
__global__ void __launch_bounds__(kLocalThreads, 1) bfs_local_kernel(LParams P) {
  extern __shared__ unsigned long long l_dyn_smem[];
  LocalEntry* QA = reinterpret_cast<LocalEntry*>(l_dyn_smem);
  LocalEntry* QB = QA + P.cap_local;
  __shared__ int s_n[2];
  __shared__ long long s_count;
  __shared__ unsigned long long s_t;
  unsigned epoch = 0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  // init: every label "unreached", the source 0; both queued bitmaps clear; queue 0 = {src}
  {
    const long long n4 = P.n >> 2;
    uint4* d4 = reinterpret_cast<uint4*>(P.dist);
    const bool al = (reinterpret_cast<uintptr_t>(P.dist) & 15u) == 0;
    const long long done = al ? n4 << 2 : 0;
    if (al)
      for (long long i = tid; i < n4; i += nth) d4[i] = make_uint4(kInf, kInf, kInf, kInf);
    for (long long i = done + tid; i < P.n; i += nth) P.dist[i] = kInf;
    for (long long w = tid; w < P.nw; w += nth) {
      P.qb0[w] = 0u;
      P.qb1[w] = 0u;
    }
  }
  if (!grid_barrier_ctl(P.ctrl, P.timeout_ns, P.barrier_extra, epoch)) return;
  if (tid == 0) {
    P.dist[P.src] = 0u;
    P.q0[0] = P.src;
    P.ctrl->slot[0].nv = 1ull;
  }
  if (!grid_barrier_ctl(P.ctrl, P.timeout_ns, P.barrier_extra, epoch)) return;
  if (threadIdx.x == 0) s_t = globaltimer_ns();
  LAcc acc;
  for (int s = 0;; ++s) {
    if (threadIdx.x == 0) s_count = (long long)ld_relaxed_u64(&P.ctrl->slot[s & 3].nv);
    __syncthreads();
    const long long count = s_count;
    if (count == 0) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      Slot* z = &P.ctrl->slot[(s + 2) & 3];
      z->items = 0; z->nv = 0; z->mf = 0; z->nq = 0; z->cursor = 0; z->mega = 0;
    }
    // This block's contiguous share of the global queue.
    const long long lo = count * (long long)blockIdx.x / gridDim.x;
    const long long hi = count * ((long long)blockIdx.x + 1) / gridDim.x;
    const int* gq = (s & 1) ? P.q1 : P.q0;
    if (threadIdx.x == 0) s_n[1] = 0;
    __syncthreads();
    LocalEntry* A = QA;
    LocalEntry* B = QB;
    int cur = 1;  // s_n[cur] counts the entries of B
    expand_local<RP, STATS>(P, s, true, gq, lo, hi - lo, nullptr, B, &s_n[cur], P.K > 1, acc);
    for (int k = 1; k < P.K; ++k) {
      __syncthreads();
      const int na = s_n[cur] < P.cap_local ? s_n[cur] : P.cap_local;
      if (na == 0) break;  // this block's wave is done (uniform: read after the barrier)
      LocalEntry* t = A; A = B; B = t;
      const int nxt = cur ^ 1;
      if (threadIdx.x == 0) s_n[nxt] = 0;
      __syncthreads();
      expand_local<RP, STATS>(P, s, false, nullptr, 0, na, A, B, &s_n[nxt], k + 1 < P.K, acc);
      cur = nxt;
    }
    if (!grid_barrier_ctl(P.ctrl, P.timeout_ns, P.barrier_extra, epoch)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.lst && s < P.lst_cap) {
      const unsigned long long t = globaltimer_ns();
      P.lst[s].direction = 2;
      P.lst[s].frontier = count;
      P.lst[s].found = (long long)ld_relaxed_u64(&P.ctrl->slot[(s + 1) & 3].nv);
      P.lst[s].ns = (long long)(t - s_t);
      s_t = t;
    }
    if (STATS) {
      // counters of the super-step: one atomic per warp
      const unsigned long long ex = warp_sum_u64(acc.examined), xp = warp_sum_u64(acc.expanded),
                               im = warp_sum_u64(acc.improved);
      if (lane_id() == 0) {
        if (ex) atomicAdd(&P.ctrl->td_edges, ex);
        if (xp) atomicAdd(&P.ctrl->td_frontier, xp);
        if (im) atomicAdd(&P.ctrl->improved, im);
        if (P.lst && s < P.lst_cap && ex) atomicAdd(reinterpret_cast<unsigned long long*>(&P.lst[s].edges), ex);
      }
      acc = LAcc();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl->supersteps = s + 1;
  }
  if (STATS) {
    // reached vertices, their degree sum and the eccentricity, from the final labels
    unsigned long long r = 0, ed = 0;
    unsigned mx = 0;
    for (long long v = tid; v < P.n; v += nth) {
      const unsigned d = P.dist[v];
      if (d != kInf) {
        ++r;
        ed += (unsigned long long)(rp_at<RP>(P.rp, v + 1) - rp_at<RP>(P.rp, v));
        mx = d > mx ? d : mx;
      }
    }
    r = warp_sum_u64(r);
    ed = warp_sum_u64(ed);
    mx = __reduce_max_sync(kFull, mx);
    if (lane_id() == 0) {
      if (r) atomicAdd(&P.ctrl->reached, r);
      if (ed) atomicAdd(&P.ctrl->edges_reached, ed);
      atomicMax(&P.ctrl->levels, (int)mx + 1);
    }
  }
}

template <typename RP, bool STATS>
void* local_kernel() {
  return reinterpret_cast<void*>(&bfs_local_kernel<RP, STATS>);
}

}  // namespace

// Shared memory of one block: two local queues.
static size_t local_smem(int cap_local) { return 2 * sizeof(LocalEntry) * (size_t)cap_local; }

int run_local(bfs_graph* g, int src, int* dist_dev, const bfs_params& p, bfs_stats* st, bfs_level_stat* levels,
              int level_cap, cudaStream_t stream) {
  SingleWs& ws = g->ws;
  LParams P{};
  P.rp = g->rp;
  P.col = g->col;
  P.head = g->head;
  P.n = g->n;
  P.m = g->m;
  P.nw = g->nw;
  P.src = src;
  P.dist = reinterpret_cast<unsigned*>(dist_dev);
  P.q0 = ws.qv[0];
  P.q1 = ws.qv[1];
  P.qb0 = ws.bm[0];
  P.qb1 = ws.bm[1];
  P.ctrl = ws.ctrl;
  P.K = p.local_levels;
  // Shared queue slots: 8 per thread (at least 256, at most 1024), so small
  // blocks stay small enough for many to share an SM.
  const int threads = p.local_threads;
  P.cap_local = 8 * threads < 256 ? 256 : (8 * threads > 1024 ? 1024 : 8 * threads);
  P.timeout_ns = (long long)p.timeout_ms * 1000000ll;
  P.barrier_extra = p.test_barrier_extra;
  const bool stats = st != nullptr;
  if (levels && level_cap > 0) {
    P.lst = ws.lst;
    P.lst_cap = level_cap;
  }
  void* fn = g->rp_bits == 32 ? (stats ? local_kernel<int, true>() : local_kernel<int, false>())
                              : (stats ? local_kernel<long long, true>() : local_kernel<long long, false>());
  const size_t smem = local_smem(P.cap_local);
  GBFS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  if (per_sm < 1) return BFS_EINVAL;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  dim3 grid((unsigned)(per_sm * g->num_sms)), block((unsigned)threads);
  void* args[] = {&P};
  GBFS_CUDA(enqueue_ctrl_reset(ws, stream));
  GBFS_CUDA(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, stream));
  return BFS_OK;
}

bool bounds_read_local(unsigned long long* first, bool reset) {
#ifdef GBFS_DEBUG_BOUNDS
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_local_bounds_err, sizeof(v)) != cudaSuccess) v = 0;
  if (reset) {
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_local_bounds_err, &z, sizeof(z));
  }
  *first = v;
  return true;
#else
  *first = 0;
  (void)reset;
  return false;
#endif
}

}  // namespace gbfs
