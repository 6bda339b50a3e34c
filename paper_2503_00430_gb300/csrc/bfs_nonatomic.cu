// bfs_single_nonatomic: the paper's BFS-NonAtomic top-down variant (Section 2),
// kept to measure its duplicate frontier entries on this GPU.
//
// Listing 1's relaxation without a claim: a thread that finds neighbour v
// unvisited marks it (visited byte, dist = L + 1) with plain stores and appends
// it to the next frontier.  Two threads that test v before either store is
// visible both append it, so the frontier can hold duplicates; every writer
// stores the same level, so dist is still exact.  The visited set is a byte
// per vertex: a bit-packed word written without atomics could lose bits and
// change distances, a byte cannot.
//
// The paper expands duplicates again at the next level (mode BFS_DUP_EXPAND
// here).  On this GPU a whole level's tests run nearly at once, so a vertex
// with many frontier neighbours is appended about once per neighbour, its
// copies re-read its list at the next level, and duplicates multiply from
// level to level (they overflowed an n + m entry queue on R-MAT scale 14 by
// the second level: BFS_ENOMEM, nothing written out of bounds).  So by default
// (BFS_DUP_DEDUP) the appended entries are reduced between levels to distinct
// vertices without atomics: every entry stores its index into owner[v] (plain
// 4-byte stores: one of them remains), and the entry whose index remained is
// the one kept.  Per level the library counts the appended entries
// (duplicates included), the distinct vertices among them and the list
// entries read.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "bfs_internal.cuh"

namespace gbfs {

struct NonAtomicWs {
  unsigned char* vis = nullptr;   // [n] visited bytes
  int* owner = nullptr;           // [n] index of the appended entry of v that is kept
  int* q[2] = {nullptr, nullptr}; // [0] distinct frontier, [1] appended entries; capacity cap each
  long long cap = 0;
  unsigned long long* heavy = nullptr;  // [hcap][2] long-list records: vertex, first chunk ticket
  long long hcap = 0;
  unsigned long long* ctr = nullptr;    // device counters (see k_na_* below)
  unsigned long long* h_ctr = nullptr;  // pinned mirror
};

namespace {

constexpr int kNaChunk = 256;  // entries per chunk ticket of a long list

// Device counters: new frontier length, overflow flag, list entries read,
// distinct new vertices, long-list records (low 32 bits) and chunk tickets
// (high 32 bits) handed out by one packed atomic, so records are in ticket order.
enum { C_NOUT = 0, C_OVER = 1, C_EDGES = 2, C_UNIQUE = 3, C_HEAVY = 4, C_COUNT = 8 };

template <typename RP>
__device__ __forceinline__ long long na_rp(const void* rp, long long i) {
  return (long long)__ldg(reinterpret_cast<const RP*>(rp) + i);
}

// Warp-aggregated append with a capacity check (an overflow is reported, the
// entry dropped; the host then returns BFS_ENOMEM).
__device__ __forceinline__ void na_append(bool flag, int v, int* q, long long cap, unsigned long long* ctr) {
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (!b) return;
  const unsigned lane = threadIdx.x & 31u;
  const int leader = __ffs(b) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(&ctr[C_NOUT], (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, leader);
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  if (flag) {
    const unsigned long long pos = base + __popc(b & lt);
    if ((long long)pos < cap) q[pos] = v;
    else atomicOr(&ctr[C_OVER], 1ull);
  }
}

// The unguarded test-and-set of Listing 1 (with the byte map of Listing 3).
// The byte is read through L2: an SM's L1 is not coherent within a kernel, so
// a plain load could keep returning a stale 0 after another SM stored 1 for
// as long as the line stays cached, and duplicates then multiply from level to
// level (a first version overflowed its n + m queue on R-MAT scale 14).  An L2
// read is the counterpart of the coherent plain load of the paper's multicore
// setting: a duplicate then needs two threads to test v before either store
// reaches L2.
__device__ __forceinline__ bool na_visit(int v, unsigned char* vis, int* dist, int L) {
  if (__ldcg(vis + v) != 0) return false;
  vis[v] = 1;
  dist[v] = L + 1;
  return true;
}

// Warp: entries [s, e) of one list, 32 at a time.
__device__ __forceinline__ void na_span(const int* col, long long s, long long e, unsigned char* vis, int* dist, int L,
                                        int* qout, long long cap, unsigned long long* ctr) {
  const unsigned lane = threadIdx.x & 31u;
  for (long long j0 = s; j0 < e; j0 += 32) {
    const long long j = j0 + lane;
    int v = 0;
    bool add = false;
    if (j < e) {
      v = __ldg(col + j);
      add = na_visit(v, vis, dist, L);
    }
    na_append(add, v, qout, cap, ctr);
  }
}

// Level L, pass 1: a warp per frontier entry with at most kNaChunk entries;
// longer lists get a record and chunk tickets (one packed atomic per warp).
template <typename RP>
__global__ void __launch_bounds__(256) k_na_level(const void* rp, const int* col, const int* qin, long long nq,
                                                  int* qout, long long cap, unsigned char* vis, int* dist, int L,
                                                  unsigned long long* heavy, long long hcap, unsigned long long* ctr) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long edges = 0;
  for (long long i = gw; i < nq; i += nwarps) {
    const int u = qin[i];
    const long long s = na_rp<RP>(rp, u), e = na_rp<RP>(rp, (long long)u + 1);
    if (e - s > kNaChunk) {
      if (lane == 0) {
        const unsigned long long nch = (unsigned long long)((e - s + kNaChunk - 1) / kNaChunk);
        const unsigned long long b = atomicAdd(&ctr[C_HEAVY], 1ull | (nch << 32));
        const unsigned long long r = b & 0xffffffffull;
        if ((long long)r < hcap) {
          heavy[2 * r] = (unsigned long long)u;
          heavy[2 * r + 1] = b >> 32;  // first ticket
        } else {
          atomicOr(&ctr[C_OVER], 1ull);
        }
      }
      continue;
    }
    if (lane == 0) edges += (unsigned long long)(e - s);
    na_span(col, s, e, vis, dist, L, qout, cap, ctr);
  }
  if (lane == 0 && edges) atomicAdd(&ctr[C_EDGES], edges);
}

// Level L, pass 2: a warp per chunk ticket of the long lists; ticket t
// belongs to the last record whose first ticket is <= t (32-way search).
template <typename RP>
__global__ void __launch_bounds__(256) k_na_chunks(const void* rp, const int* col, int* qout, long long cap,
                                                   unsigned char* vis, int* dist, int L,
                                                   const unsigned long long* heavy, long long hcap,
                                                   unsigned long long* ctr) {
  const unsigned long long hv = ctr[C_HEAVY];  // written by k_na_level earlier on this stream
  long long nrec = (long long)(hv & 0xffffffffull);
  const long long ntick = (long long)(hv >> 32);
  if (nrec > hcap) nrec = hcap;  // overflowed (reported): search the stored records only
  if (nrec == 0) return;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long edges = 0;
  for (long long t = gw; t < ntick; t += nwarps) {
    long long lo = 0, hi = nrec;
    while (hi - lo > 1) {
      const long long step = (hi - lo + 31) / 32;
      const long long idx = lo + (long long)lane * step;
      const bool ok = idx < hi && (long long)heavy[2 * idx + 1] <= t;
      const unsigned bm = __ballot_sync(0xffffffffu, ok);
      lo += (long long)(31 - __clz(bm)) * step;
      hi = lo + step < hi ? lo + step : hi;
    }
    const long long found = lo;
    const int u = (int)heavy[2 * found];
    const long long t0 = (long long)heavy[2 * found + 1];
    const long long s0 = na_rp<RP>(rp, u), e0 = na_rp<RP>(rp, (long long)u + 1);
    const long long cs = s0 + (t - t0) * kNaChunk, ce = cs + kNaChunk < e0 ? cs + kNaChunk : e0;
    if (lane == 0) edges += (unsigned long long)(ce - cs);
    na_span(col, cs, ce, vis, dist, L, qout, cap, ctr);
  }
  if (lane == 0 && edges) atomicAdd(&ctr[C_EDGES], edges);
}

// Duplicate removal, pass 1: every appended entry i of v stores i into owner[v].
__global__ void k_na_own(const int* q, long long nq, int* owner) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < nq; i += nth) owner[q[i]] = (int)i;
}

// Pass 2 (a later launch, so every store of pass 1 is visible): the entry
// whose index remained is appended to the next frontier, once per vertex
// (qnext null: the distinct vertices are only counted).
__global__ void k_na_keep(const int* q, long long nq, const int* owner, int* qnext, unsigned long long* ctr) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  for (long long base = tid - lane; base < nq; base += nth) {
    const long long i = base + lane;
    int v = 0;
    bool keep = false;
    if (i < nq) {
      v = q[i];
      keep = owner[v] == (int)i;
    }
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if (!b) continue;
    const int leader = __ffs(b) - 1;
    unsigned long long pos = 0;
    if ((int)lane == leader) pos = atomicAdd(&ctr[C_UNIQUE], (unsigned long long)__popc(b));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    if (keep && qnext) qnext[pos + __popc(b & lt)] = v;
  }
}

__global__ void k_na_init(unsigned char* vis, int* dist, long long n, int src, int* q0) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += nth) {
    vis[v] = v == src ? 1 : 0;
    dist[v] = v == src ? 0 : -1;
  }
  if (tid == 0) q0[0] = src;
}

// One BFS.  expand_dups = false: a level expands the distinct vertices of the
// appended entries; true (the paper's variant): it expands every appended
// entry, duplicates included, which can outgrow the queues (BFS_ENOMEM).
template <typename RP>
int run_na(bfs_graph* g, NonAtomicWs& ws, int src, int* dist, bool expand_dups, bfs_dup_stats* st,
           bfs_dup_level* lv, int lv_cap, cudaStream_t s) {
  const long long n = g->n;
  const int grid = g->num_sms * 8, block = 256;
  int* qin = ws.q[0];
  int* qout = ws.q[1];
  k_na_init<<<grid, block, 0, s>>>(ws.vis, dist, n, src, qin);
  GBFS_CUDA(cudaGetLastError());
  long long nq = 1, appended = 1, uniq = 1;  // the level-0 frontier {src}
  int L = 0;
  for (;;) {
    // Expand the nq entries of qin into qout (duplicates possible) ...
    GBFS_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(unsigned long long) * C_COUNT, s));
    k_na_level<RP><<<grid, block, 0, s>>>(g->rp, g->col, qin, nq, qout, ws.cap, ws.vis, dist, L, ws.heavy,
                                          ws.hcap, ws.ctr);
    k_na_chunks<RP><<<grid, block, 0, s>>>(g->rp, g->col, qout, ws.cap, ws.vis, dist, L, ws.heavy, ws.hcap,
                                           ws.ctr);
    GBFS_CUDA(cudaGetLastError());
    GBFS_CUDA(cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(unsigned long long) * C_COUNT, cudaMemcpyDeviceToHost, s));
    GBFS_CUDA(cudaStreamSynchronize(s));
    if (ws.h_ctr[C_OVER]) return BFS_ENOMEM;
    const long long nout = (long long)ws.h_ctr[C_NOUT];
    const long long edges = (long long)ws.h_ctr[C_EDGES];
    if (st) {
      st->levels = L + 1;
      st->frontier_entries += appended;
      st->unique += uniq;
      st->edges += edges;
    }
    if (lv && L < lv_cap) {
      lv[L].frontier = appended;
      lv[L].unique = uniq;
      lv[L].edges = edges;
    }
    if (nout == 0) break;
    // ... then count the distinct vertices of qout, and keep them in qin (or
    // keep every entry: the next level expands qout as it is).
    k_na_own<<<grid, block, 0, s>>>(qout, nout, ws.owner);
    k_na_keep<<<grid, block, 0, s>>>(qout, nout, ws.owner, expand_dups ? nullptr : qin, ws.ctr);
    GBFS_CUDA(cudaGetLastError());
    GBFS_CUDA(cudaMemcpyAsync(ws.h_ctr, ws.ctr, sizeof(unsigned long long) * C_COUNT, cudaMemcpyDeviceToHost, s));
    GBFS_CUDA(cudaStreamSynchronize(s));
    appended = nout;
    uniq = (long long)ws.h_ctr[C_UNIQUE];
    if (expand_dups) {
      int* t = qin;
      qin = qout;
      qout = t;
      nq = nout;
    } else {
      nq = uniq;
    }
    ++L;
  }
  return BFS_OK;
}

}  // namespace

void free_nonatomic_ws(NonAtomicWs* ws) {
  if (!ws) return;
  cudaFree(ws->vis);
  cudaFree(ws->owner);
  cudaFree(ws->q[0]);
  cudaFree(ws->q[1]);
  cudaFree(ws->heavy);
  cudaFree(ws->ctr);
  if (ws->h_ctr) cudaFreeHost(ws->h_ctr);
  delete ws;
}

int run_nonatomic(bfs_graph* g, int src, int* dist, int mode, bfs_dup_stats* st, bfs_dup_level* lv, int lv_cap,
                  cudaStream_t s) {
  if (!g->na) {
    NonAtomicWs* ws = new NonAtomicWs();
    const size_t n = (size_t)g->n;
    // A level expands distinct vertices, so it reads at most m list entries
    // and appends at most m entries (an overflow would still be reported as
    // BFS_ENOMEM, never written).  Entry indices are stored as int32.
    ws->cap = g->n + g->m + 1;
    if (ws->cap >= (1ll << 31)) {
      delete ws;
      return BFS_EINVAL;
    }
    cudaError_t e = cudaMalloc(&ws->vis, n);
    if (e == cudaSuccess) e = cudaMalloc(&ws->owner, sizeof(int) * n);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&ws->q[i], sizeof(int) * (size_t)ws->cap);
    // Long-list records: one per frontier entry of more than kNaChunk entries;
    // twice the number of such vertices leaves room for duplicated hubs.
    ws->hcap = 2 * (g->m / kNaChunk) + 4096;
    if (e == cudaSuccess) e = cudaMalloc(&ws->heavy, 2 * sizeof(unsigned long long) * (size_t)ws->hcap);
    if (e == cudaSuccess) e = cudaMalloc(&ws->ctr, sizeof(unsigned long long) * C_COUNT);
    if (e == cudaSuccess) e = cudaMallocHost(&ws->h_ctr, sizeof(unsigned long long) * C_COUNT);
    if (e != cudaSuccess) {
      free_nonatomic_ws(ws);
      return cuda_fail(e, "non-atomic workspace", __FILE__, __LINE__);
    }
    g->na = ws;
  }
  if (st) memset(st, 0, sizeof(*st));
  if (lv && lv_cap > 0) memset(lv, 0, sizeof(*lv) * (size_t)lv_cap);
  const bool expand = mode == BFS_DUP_EXPAND;
  return g->rp_bits == 32 ? run_na<int>(g, *g->na, src, dist, expand, st, lv, lv_cap, s)
                          : run_na<long long>(g, *g->na, src, dist, expand, st, lv, lv_cap, s);
}

}  // namespace gbfs
