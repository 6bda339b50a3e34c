// Multi-source BFS: up to 256 sources per group, one bit per source ("lane")
// in W = 1, 2 or 4 64-bit words per vertex.
//
// Per group and level L (the paper's level-synchronous loop, Section 2,
// applied to 64*W searches at once):
//   X[v]  lanes that have reached v;   F_L[v]  lanes that reached v at level L.
//   push (sparse levels, Listing 1's top-down form): every frontier vertex u
//     ORs F_L[u] & ~X[v] into an accumulator of each neighbour v; touched
//     vertices are then applied: F_{L+1}[v] = acc & ~X[v], X[v] |= F_{L+1}[v];
//   pull (dense levels, Listing 2's bottom-up form): every vertex not yet
//     reached by all lanes ORs F_L[u] over its neighbours u and stops as soon
//     as every lane is either known or found; F_{L+1}[v] = acc & ~X[v].
// The direction follows the same edge-count rule as the single-source path.
// Frontier masks of successive levels are kept in a ring of K arrays; a writer
// pass turns them into dist[source][vertex] rows with whole-sector stores
// (dist = the level whose frontier holds the lane's bit), so the output is
// written once instead of byte by byte at every level.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bfs_internal.cuh"

namespace gbfs {

struct MsCtrl {
  unsigned long long nf;        // vertices of the new frontier
  unsigned long long mf;        // their degree sum
  unsigned long long done_deg;  // degrees of vertices that became reached by every lane
  unsigned long long nq;        // new frontier queue length
  unsigned long long ntouch;    // push: touched vertices
  unsigned long long nheavy;    // pull: deferred high-degree vertices
  unsigned long long edges;     // entries examined (pull) or pushed (push)
  unsigned long long active;    // pull: vertices still missing an active lane (their lists are read)
  unsigned long long act[4];    // lanes present in the new frontier
};

// A pull vertex with more entries than ms_heavy_min: its adjacency is cut into
// chunks of kMsChunk entries, handed out as tickets base .. base+chunks-1.
struct MsHeavy {
  long long start;
  long long deg;
  unsigned long long base;
  long long v;
};
constexpr int kMsChunk = 2048;
constexpr int kMsCountBits = 32;

struct MultiWs {
  bool ready = false;
  int ring = 0;                        // K
  unsigned long long* X = nullptr;     // [n][4]
  unsigned long long* acc = nullptr;   // [n][4] push accumulator (kept zero between levels)
  unsigned long long* F = nullptr;     // [K][n][4]
  unsigned* touched_bm = nullptr;      // [nw] (kept zero between levels)
  int* q[2] = {nullptr, nullptr};      // frontier vertex queues
  int* touched = nullptr;              // push: touched vertices
  MsHeavy* heavy = nullptr;            // pull: deferred high-degree vertices
  int* d_src = nullptr;                // group sources
  int* order = nullptr;                // vertex ids by degree, highest first
  MsCtrl* ctrl = nullptr;
  MsCtrl* h_ctrl = nullptr;            // pinned
  void* staging = nullptr;             // host-output staging (one group)
  size_t staging_bytes = 0;
  cudaEvent_t done = nullptr;
};

namespace {

constexpr int kMsMaxRing = 16;
#ifndef GBFS_MS_PULL_MINB
#define GBFS_MS_PULL_MINB 3  // pull kernels: blocks of 256 per SM the register budget must allow
#endif

__device__ __forceinline__ unsigned ms_lane() { return threadIdx.x & 31u; }

template <typename RP>
__device__ __forceinline__ long long rpv(const void* rp, long long i) {
  return (long long)__ldg(reinterpret_cast<const RP*>(rp) + i);
}

template <int W>
struct Mask {
  unsigned long long w[W];
};

// A four-word mask is one 32-byte sector (every mask array is 32-byte aligned:
// 32 bytes per vertex from a cudaMalloc base), moved with one 256-bit access,
// so a scattered gather costs one L1 request instead of two.
// Masks that a kernel may have changed since it started (X, accumulators, the
// current frontier inside the persistent serving loop) are loaded through L2
// (.cg): another SM's atomics and stores are not visible in this SM's L1.
__device__ __forceinline__ void ld_v4_u64(const unsigned long long* p, Mask<4>& m) {
  asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(m.w[0]), "=l"(m.w[1]), "=l"(m.w[2]), "=l"(m.w[3]) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_nc_v4_u64(const unsigned long long* p, Mask<4>& m) {
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(m.w[0]), "=l"(m.w[1]), "=l"(m.w[2]), "=l"(m.w[3]) : "l"(p));
}
__device__ __forceinline__ void st_v4_u64(unsigned long long* p, const Mask<4>& m) {
  asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(m.w[0]), "l"(m.w[1]), "l"(m.w[2]),
               "l"(m.w[3]) : "memory");
}

template <int W>
__device__ __forceinline__ Mask<W> load_mask(const unsigned long long* p) {
  Mask<W> m;
  if constexpr (W == 4) {
    ld_v4_u64(p, m);
  } else if constexpr (W == 2) {
    const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2*>(p));
    m.w[0] = a.x; m.w[1] = a.y;
  } else {
    m.w[0] = __ldcg(p);
  }
  return m;
}

// Read-only gather of a frontier mask (the array was written by an earlier launch).
template <int W>
__device__ __forceinline__ Mask<W> ldg_mask(const unsigned long long* p) {
  Mask<W> m;
  if constexpr (W == 4) {
    ld_nc_v4_u64(p, m);
  } else if constexpr (W == 2) {
    const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(p));
    m.w[0] = a.x; m.w[1] = a.y;
  } else {
    m.w[0] = __ldg(p);
  }
  return m;
}

template <int W>
__device__ __forceinline__ void store_mask(unsigned long long* p, const Mask<W>& m) {
  if constexpr (W == 4) {
    st_v4_u64(p, m);
  } else if constexpr (W == 2) {
    reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(m.w[0], m.w[1]);
  } else {
    p[0] = m.w[0];
  }
}

struct MsArgs {
  const void* rp;
  const int* col;
  long long n;
  long long n_live;            // pull, dense apply, compact: vertices [0, n_live) (the rest have degree 0)
  int nw;
  unsigned long long full[4];   // lanes of the group
  unsigned long long act[4];    // lanes present in the current frontier (the only ones that can advance)
  unsigned long long* X;
  unsigned long long* acc;
  const unsigned long long* Fcur;
  unsigned long long* Fnext;
  unsigned* touched_bm;
  const int* qcur;
  int* qnext;
  int* touched;
  MsHeavy* heavy;
  const int* order;
  MsCtrl* ctrl;
  int heavy_min;               // pull: vertices with more entries go to the warp-cooperative pass
  int dense;                   // push: no touched list; the apply pass scans every vertex
  int want_queue;              // pull / dense apply: also append the new frontier's vertices to qnext
  // Serving groups that write distances as they are found (large-diameter
  // graphs): lane i's row is out[i], its level 0 is join[i]; out_level is the
  // level being found (L + 1).  Null out: rows are written from the ring.
  int* const* out;
  const int* join;
  int out_level;
};

template <int W>
__device__ __forceinline__ bool is_full(const Mask<W>& m, const unsigned long long* full) {
  bool f = true;
#pragma unroll
  for (int k = 0; k < W; ++k) f = f && (m.w[k] == full[k]);
  return f;
}

// Every lane of `act` is set in m (lanes outside act cannot change this level).
template <int W>
__device__ __forceinline__ bool covers(const Mask<W>& m, const unsigned long long* act) {
  bool f = true;
#pragma unroll
  for (int k = 0; k < W; ++k) f = f && ((m.w[k] & act[k]) == act[k]);
  return f;
}

// OR of the new frontier lanes into the level's active-lane record (one atomic per warp and word).
template <int W>
__device__ __forceinline__ void warp_or_active(const Mask<W>& nn, MsCtrl* ctrl) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    unsigned long long t = nn.w[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t |= __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31u) == 0 && t) atomicOr(&ctrl->act[k], t);
  }
}

// Lane i in nn found v at out_level: its distance is out_level - join[i].
template <int W>
__device__ __forceinline__ void direct_out(const MsArgs& A, long long v, const Mask<W>& nn) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    unsigned long long b = nn.w[k];
    while (b) {
      const int i = 64 * k + __ffsll((long long)b) - 1;
      b &= b - 1;
      A.out[i][v] = A.out_level - A.join[i];
    }
  }
}

template <int W>
__device__ __forceinline__ bool is_zero(const Mask<W>& m) {
  unsigned long long o = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) o |= m.w[k];
  return o == 0;
}

// Warp-aggregated append of v to a queue (flag: this lane appends).
__device__ __forceinline__ void warp_append(bool flag, int v, unsigned long long* counter, int* q) {
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (!b) return;
  const int leader = __ffs(b) - 1;
  unsigned long long base = 0;
  if ((int)ms_lane() == leader) base = atomicAdd(counter, (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, leader);
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  if (flag) q[base + __popc(b & lt)] = v;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// ---- seed: lanes' sources into X and F_0, unique sources into the queue ----
template <int W>
__global__ void k_ms_seed(MsArgs A, const int* src, int lanes) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < lanes; i += gridDim.x * blockDim.x) {
    const int s = src[i];
    atomicOr(A.X + (long long)s * W + (i >> 6), 1ull << (i & 63));
    atomicOr(const_cast<unsigned long long*>(A.Fcur) + (long long)s * W + (i >> 6), 1ull << (i & 63));
  }
}

// ---- push: frontier vertices OR their new lanes into neighbours' accumulators ----
// Vertices with more than kMsPushChunk entries are cut into chunks handed out
// as tickets (records planned first), so a hub's list is pushed by many warps.
constexpr int kMsPushChunk = 256;

// Plan: one record per frontier vertex with more than kMsPushChunk entries;
// one packed atomic per warp hands out record slots and chunk tickets in order.
// Counters another phase of the same level wrote: read through L2 (the
// persistent serving loop runs several levels in one launch).
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) { return __ldcg(p); }

template <typename RP>
__device__ __forceinline__ void ms_push_plan_body(const MsArgs& A, long long nq) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long base = tid - (tid & 31); base < nq; base += nth) {
    const long long i = base + ms_lane();
    long long s = 0, d = 0;
    int u = 0;
    if (i < nq) {
      u = __ldcg(A.qcur + i);
      s = rpv<RP>(A.rp, u);
      d = rpv<RP>(A.rp, (long long)u + 1) - s;
    }
    const bool big = d > kMsPushChunk;
    const int nch = big ? (int)((d + kMsPushChunk - 1) / kMsPushChunk) : 0;
    const unsigned bm = __ballot_sync(0xffffffffu, big);
    if (!bm) continue;
    int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)ms_lane() >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long b = 0;
    if (ms_lane() == 31)
      b = atomicAdd(&A.ctrl->nheavy, (unsigned long long)__popc(bm) | ((unsigned long long)tot << kMsCountBits));
    b = __shfl_sync(0xffffffffu, b, 31);
    if (big) {
      unsigned lt;
      asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
      MsHeavy& r = A.heavy[(b & ((1ull << kMsCountBits) - 1)) + __popc(bm & lt)];
      r.start = s;
      r.deg = d;
      r.base = (b >> kMsCountBits) + (unsigned long long)(incl - nch);
      r.v = u;
    }
  }
}

template <typename RP>
__global__ void __launch_bounds__(256) k_ms_push_plan(MsArgs A, long long nq) {
  ms_push_plan_body<RP>(A, nq);
}

// A chunk record the planning phase wrote (read through L2, see load_mask).
__device__ __forceinline__ MsHeavy ld_heavy(const MsHeavy* p) {
  MsHeavy r;
  r.start = __ldcg(&p->start);
  r.deg = __ldcg(&p->deg);
  r.base = __ldcg(&p->base);
  r.v = __ldcg(&p->v);
  return r;
}

// Warp-collective: push the lanes f of one vertex along entries [s, e), 32 per step.
template <int W>
__device__ __forceinline__ void ms_push_span(const MsArgs& A, const Mask<W>& f, long long s, long long e) {
  const unsigned lane = ms_lane();
  for (long long j0 = s; j0 < e; j0 += 32) {
    const long long j = j0 + lane;
    bool touch = false;
    int v = 0;
    if (j < e) {
      v = __ldg(A.col + j);
      const Mask<W> x = load_mask<W>(A.X + (long long)v * W);
      bool any = false;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const unsigned long long add = f.w[k] & ~x.w[k];
        if (add) {
          atomicOr(A.acc + (long long)v * W + k, add);
          any = true;
        }
      }
      if (any && !A.dense) {
        const unsigned bit = 1u << (v & 31);
        touch = !(atomicOr(A.touched_bm + (v >> 5), bit) & bit);
      }
    }
    if (!A.dense) warp_append(touch, v, &A.ctrl->ntouch, A.touched);
  }
}

// Frontier vertices with at most kMsThreadPush entries: a thread each, the
// warp stepping through entry k of its 32 vertices together (large-diameter
// graphs have thousands of levels of such vertices: a warp per vertex would
// leave most lanes idle).  Then a warp per frontier vertex of at most
// kMsPushChunk entries, then a warp per chunk ticket of the planned vertices
// (ticket t belongs to the last record whose base is <= t: 32-way search).
constexpr int kMsThreadPush = 8;

template <int W, typename RP>
__device__ __forceinline__ void ms_push_body(const MsArgs& A, long long nq) {
  const long long gw = (long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5);
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = ms_lane();
  const unsigned long long hv = ld_cg_u64(&A.ctrl->nheavy);  // written by the planning phase
  const long long nrec = (long long)(hv & ((1ull << kMsCountBits) - 1)), nch = (long long)(hv >> kMsCountBits);
  unsigned long long edges = 0;
  {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long base = tid - lane; base < nq; base += nth) {
      const long long i = base + lane;
      long long s = 0, d = 0;
      Mask<W> f;
      if (i < nq) {
        const int u = __ldcg(A.qcur + i);
        s = rpv<RP>(A.rp, u);
        d = rpv<RP>(A.rp, (long long)u + 1) - s;
        if (d > kMsThreadPush) d = 0;  // a warp pushes it below
        else f = load_mask<W>(A.Fcur + (long long)u * W);
      }
      edges += (unsigned long long)d;
      for (int k = 0; k < kMsThreadPush; ++k) {
        if (!__any_sync(0xffffffffu, k < d)) break;
        bool touch = false;
        int v = 0;
        if (k < d) {
          v = __ldg(A.col + s + k);
          const Mask<W> x = load_mask<W>(A.X + (long long)v * W);
          bool any = false;
#pragma unroll
          for (int w = 0; w < W; ++w) {
            const unsigned long long add = f.w[w] & ~x.w[w];
            if (add) {
              atomicOr(A.acc + (long long)v * W + w, add);
              any = true;
            }
          }
          if (any && !A.dense) {
            const unsigned bit = 1u << (v & 31);
            touch = !(atomicOr(A.touched_bm + (v >> 5), bit) & bit);
          }
        }
        if (!A.dense) warp_append(touch, v, &A.ctrl->ntouch, A.touched);
      }
    }
  }
  edges = warp_sum(edges);
  if (lane != 0) edges = 0;
  for (long long u0 = gw; u0 < nq + nch; u0 += nwarps) {
    if (u0 < nq) {
      const int u = __ldcg(A.qcur + u0);
      const long long s = rpv<RP>(A.rp, u), e = rpv<RP>(A.rp, (long long)u + 1);
      if (e - s <= kMsThreadPush) continue;  // pushed by its thread above
      if (e - s > kMsPushChunk) continue;    // pushed by chunk tickets
      if (lane == 0) edges += (unsigned long long)(e - s);
      ms_push_span<W>(A, load_mask<W>(A.Fcur + (long long)u * W), s, e);
    } else {
      const long long t = u0 - nq;
      long long lo = 0, hi = nrec;
      while (hi - lo > 1) {
        const long long step = (hi - lo + 31) / 32;
        const long long idx = lo + (long long)lane * step;
        const bool ok = idx < hi && (long long)__ldcg(&A.heavy[idx].base) <= t;
        const unsigned bm = __ballot_sync(0xffffffffu, ok);
        lo += (long long)(31 - __clz(bm)) * step;
        hi = lo + step < hi ? lo + step : hi;
      }
      const MsHeavy r = ld_heavy(A.heavy + lo);
      const long long cs = r.start + (t - (long long)r.base) * kMsPushChunk;
      const long long ce = cs + (r.deg - (cs - r.start) < kMsPushChunk ? r.deg - (cs - r.start) : kMsPushChunk);
      if (lane == 0) edges += (unsigned long long)(ce - cs);
      ms_push_span<W>(A, load_mask<W>(A.Fcur + r.v * W), cs, ce);
    }
  }
  if (lane == 0 && edges) atomicAdd(&A.ctrl->edges, edges);
}

template <int W, typename RP>
__global__ void __launch_bounds__(256) k_ms_push(MsArgs A, long long nq) {
  ms_push_body<W, RP>(A, nq);
}

// ---- apply after push: new lanes of touched vertices ----
template <int W, typename RP>
__device__ __forceinline__ void ms_apply_body(const MsArgs& A) {
  const long long nt = (long long)ld_cg_u64(&A.ctrl->ntouch);  // written by the push phase
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long nf = 0, mf = 0, dd = 0;
  Mask<W> act_acc;
#pragma unroll
  for (int k = 0; k < W; ++k) act_acc.w[k] = 0;
  for (long long base = tid - (tid & 31); base < nt; base += nth) {
    const long long i = base + ms_lane();
    bool in = i < nt;
    int v = 0;
    bool nz = false;
    Mask<W> nn;
#pragma unroll
    for (int k = 0; k < W; ++k) nn.w[k] = 0;
    if (in) {
      v = __ldcg(A.touched + i);
      Mask<W> a = load_mask<W>(A.acc + (long long)v * W);
      Mask<W> x = load_mask<W>(A.X + (long long)v * W);
      Mask<W> z;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        nn.w[k] = a.w[k] & ~x.w[k];
        x.w[k] |= nn.w[k];
        z.w[k] = 0;
      }
      store_mask<W>(A.acc + (long long)v * W, z);
      store_mask<W>(A.X + (long long)v * W, x);
      store_mask<W>(A.Fnext + (long long)v * W, nn);
      atomicAnd(A.touched_bm + (v >> 5), ~(1u << (v & 31)));
      nz = !is_zero<W>(nn);
      if (nz) {
        if (A.out) direct_out<W>(A, v, nn);
        const long long d = rpv<RP>(A.rp, (long long)v + 1) - rpv<RP>(A.rp, v);
        nf += 1;
        mf += (unsigned long long)d;
        if (is_full<W>(x, A.full)) dd += (unsigned long long)d;
      }
    }
    warp_append(nz, v, &A.ctrl->nq, A.qnext);
#pragma unroll
    for (int k = 0; k < W; ++k) act_acc.w[k] |= nn.w[k];
  }
  warp_or_active<W>(act_acc, A.ctrl);
  nf = warp_sum(nf);
  mf = warp_sum(mf);
  dd = warp_sum(dd);
  if (ms_lane() == 0) {
    if (nf) atomicAdd(&A.ctrl->nf, nf);
    if (mf) atomicAdd(&A.ctrl->mf, mf);
    if (dd) atomicAdd(&A.ctrl->done_deg, dd);
  }
}

template <int W, typename RP>
__global__ void __launch_bounds__(256) k_ms_apply(MsArgs A) {
  ms_apply_body<W, RP>(A);
}

// ---- apply after a dense push: every vertex, in id order (coalesced) ----
template <int W, typename RP>
__global__ void __launch_bounds__(256) k_ms_apply_dense(MsArgs A) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long nf = 0, mf = 0, dd = 0;
  Mask<W> act_acc;
#pragma unroll
  for (int k = 0; k < W; ++k) act_acc.w[k] = 0;
  for (long long base = tid - (tid & 31); base < A.n_live; base += nth) {
    const long long v = base + ms_lane();
    bool nz = false;
    Mask<W> nn;
#pragma unroll
    for (int k = 0; k < W; ++k) nn.w[k] = 0;
    if (v < A.n_live) {
      const Mask<W> a = load_mask<W>(A.acc + v * W);
      if (!is_zero<W>(a)) {
        Mask<W> x = load_mask<W>(A.X + v * W);
        Mask<W> z;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          nn.w[k] = a.w[k] & ~x.w[k];
          x.w[k] |= nn.w[k];
          z.w[k] = 0;
        }
        store_mask<W>(A.acc + v * W, z);
        nz = !is_zero<W>(nn);
        if (nz) {
          if (A.out) direct_out<W>(A, v, nn);
          store_mask<W>(A.X + v * W, x);
          store_mask<W>(A.Fnext + v * W, nn);  // Fnext was zeroed before the push
          const long long d = rpv<RP>(A.rp, v + 1) - rpv<RP>(A.rp, v);
          nf += 1;
          mf += (unsigned long long)d;
          if (is_full<W>(x, A.full)) dd += (unsigned long long)d;
        }
      }
    }
    if (A.want_queue) warp_append(nz, (int)v, &A.ctrl->nq, A.qnext);
#pragma unroll
    for (int k = 0; k < W; ++k) act_acc.w[k] |= nn.w[k];
  }
  warp_or_active<W>(act_acc, A.ctrl);
  nf = warp_sum(nf);
  mf = warp_sum(mf);
  dd = warp_sum(dd);
  if (ms_lane() == 0) {
    if (nf) atomicAdd(&A.ctrl->nf, nf);
    if (mf) atomicAdd(&A.ctrl->mf, mf);
    if (dd) atomicAdd(&A.ctrl->done_deg, dd);
  }
}

// ---- frontier queue from the frontier masks (before a push level that follows
// a level which kept no queue) ----
template <int W>
__global__ void __launch_bounds__(256) k_ms_compact(MsArgs A) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long base = tid - (tid & 31); base < A.n_live; base += nth) {
    const long long v = base + ms_lane();
    const bool nz = v < A.n_live && !is_zero<W>(load_mask<W>(A.Fcur + v * W));
    warp_append(nz, (int)v, &A.ctrl->nq, A.qnext);
  }
}

// ---- pull: thread per vertex; high-degree vertices deferred to the warp pass ----
template <int W, typename RP>
__global__ void __launch_bounds__(256, GBFS_MS_PULL_MINB) k_ms_pull(MsArgs A) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long nf = 0, mf = 0, dd = 0, edges = 0, nact = 0;
  Mask<W> act_acc;
#pragma unroll
  for (int k = 0; k < W; ++k) act_acc.w[k] = 0;
  for (long long base = tid - (tid & 31); base < A.n_live; base += nth) {
    const long long oi = base + ms_lane();
    const long long v = (A.order && oi < A.n_live) ? (long long)A.order[oi] : oi;
    bool nz = false, defer = false;
    long long sv = 0, dv = 0;
    Mask<W> nn;
#pragma unroll
    for (int k = 0; k < W; ++k) nn.w[k] = 0;
    if (v < A.n_live) {
      Mask<W> x = load_mask<W>(A.X + v * W);
      if (!covers<W>(x, A.act)) {
        ++nact;
        const long long s = rpv<RP>(A.rp, v), e = rpv<RP>(A.rp, v + 1);
        if (e - s > A.heavy_min) {
          defer = true;
          sv = s;
          dv = e - s;
        } else {
          Mask<W> acc;
#pragma unroll
          for (int k = 0; k < W; ++k) acc.w[k] = x.w[k];
          // Aligned groups of four entries: one 128-bit load, then the four
          // neighbours' masks are gathered together before they are combined;
          // the next group's entries are requested before this group's masks.
          long long j0 = s & ~3ll;
          int4 q = __ldg(reinterpret_cast<const int4*>(A.col + j0));
          for (; j0 < e; j0 += 4) {
            const int4 qn = j0 + 4 < e ? __ldg(reinterpret_cast<const int4*>(A.col + j0 + 4)) : make_int4(0, 0, 0, 0);
            const int c4[4] = {q.x, q.y, q.z, q.w};
            q = qn;
            Mask<W> f[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              if (j0 + t >= s && j0 + t < e) {
                f[t] = ldg_mask<W>(A.Fcur + (long long)c4[t] * W);
              } else {
#pragma unroll
                for (int k = 0; k < W; ++k) f[t].w[k] = 0;
              }
            }
#pragma unroll
            for (int k = 0; k < W; ++k) acc.w[k] |= f[0].w[k] | f[1].w[k] | f[2].w[k] | f[3].w[k];
            if (covers<W>(acc, A.act)) {
              j0 += 4;
              break;
            }
          }
          edges += (unsigned long long)((j0 < e ? j0 : e) - (s > (s & ~3ll) ? s : s));
#pragma unroll
          for (int k = 0; k < W; ++k) {
            nn.w[k] = acc.w[k] & ~x.w[k] & A.full[k];
            x.w[k] |= nn.w[k];
          }
          nz = !is_zero<W>(nn);
          if (nz) {
            if (A.out) direct_out<W>(A, v, nn);
            store_mask<W>(A.X + v * W, x);
            nf += 1;
            mf += (unsigned long long)(e - s);
            if (is_full<W>(x, A.full)) dd += (unsigned long long)(e - s);
          }
        }
      }
      if (!defer) store_mask<W>(A.Fnext + v * W, nn);
    }
    if (A.want_queue) warp_append(nz, (int)v, &A.ctrl->nq, A.qnext);
    {
      // Deferred vertices: one record each; one packed atomic per warp hands
      // out record slots and chunk tickets in the same order.
      const int nch = defer ? (int)((dv + kMsChunk - 1) / kMsChunk) : 0;
      const unsigned dm = __ballot_sync(0xffffffffu, defer);
      if (dm) {
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if ((int)ms_lane() >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long b = 0;
        if (ms_lane() == 31)
          b = atomicAdd(&A.ctrl->nheavy, (unsigned long long)__popc(dm) | ((unsigned long long)tot << kMsCountBits));
        b = __shfl_sync(0xffffffffu, b, 31);
        if (defer) {
          unsigned lt;
          asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
          MsHeavy& r = A.heavy[(b & ((1ull << kMsCountBits) - 1)) + __popc(dm & lt)];
          r.start = sv;
          r.deg = dv;
          r.base = (b >> kMsCountBits) + (unsigned long long)(incl - nch);
          r.v = v;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) act_acc.w[k] |= nn.w[k];
  }
  warp_or_active<W>(act_acc, A.ctrl);
  nf = warp_sum(nf);
  mf = warp_sum(mf);
  dd = warp_sum(dd);
  edges = warp_sum(edges);
  nact = warp_sum(nact);
  if (ms_lane() == 0) {
    if (nf) atomicAdd(&A.ctrl->nf, nf);
    if (mf) atomicAdd(&A.ctrl->mf, mf);
    if (dd) atomicAdd(&A.ctrl->done_deg, dd);
    if (edges) atomicAdd(&A.ctrl->edges, edges);
    if (nact) atomicAdd(&A.ctrl->active, nact);
  }
}

// ---- pull, deferred high-degree vertices: warp per chunk ticket ----
// Ticket t belongs to the last record whose base is <= t (32-way search).  The
// warp ORs the neighbours' frontier masks of its chunk, 128 entries per step
// (four gathers in flight per lane), stops once the vertex's pending active
// lanes are all covered, and ORs the new lanes into the vertex's accumulator.
template <int W, typename RP>
__global__ void __launch_bounds__(256, GBFS_MS_PULL_MINB) k_ms_heavy_chunks(MsArgs A) {
  const unsigned long long hv = A.ctrl->nheavy;  // written by k_ms_pull earlier on this stream
  const long long nrec = (long long)(hv & ((1ull << kMsCountBits) - 1)), nch = (long long)(hv >> kMsCountBits);
  const long long gw = (long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5);
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = ms_lane();
  unsigned long long edges = 0;
  for (long long t = gw; t < nch; t += nwarps) {
    long long lo = 0, hi = nrec;
    while (hi - lo > 1) {
      const long long step = (hi - lo + 31) / 32;
      const long long idx = lo + (long long)lane * step;
      const bool ok = idx < hi && (long long)A.heavy[idx].base <= t;
      const unsigned bm = __ballot_sync(0xffffffffu, ok);
      lo += (long long)(31 - __clz(bm)) * step;
      hi = lo + step < hi ? lo + step : hi;
    }
    const MsHeavy r = A.heavy[lo];
    const long long cs = r.start + (t - (long long)r.base) * kMsChunk;
    const long long ce = cs + (r.deg - (cs - r.start) < kMsChunk ? r.deg - (cs - r.start) : kMsChunk);
    const Mask<W> x = load_mask<W>(A.X + r.v * W);
    Mask<W> have = load_mask<W>(A.acc + r.v * W);
#pragma unroll
    for (int k = 0; k < W; ++k) have.w[k] |= x.w[k];
    if (covers<W>(have, A.act)) continue;
    // Lane-local OR over the chunk; the warp combines the lanes (and tests
    // whether the vertex's pending lanes are covered) every fourth step.  The
    // next step's entries are requested before this step's masks.
    Mask<W> la;
#pragma unroll
    for (int k = 0; k < W; ++k) la.w[k] = 0;
    long long base = cs & ~3ll;
    int4 q = base + 4 * (long long)lane < ce ? __ldg(reinterpret_cast<const int4*>(A.col + base + 4 * lane))
                                            : make_int4(0, 0, 0, 0);
    for (int step = 1; base < ce; base += 128, ++step) {
      const long long j = base + 4 * (long long)lane;
      const int c4[4] = {q.x, q.y, q.z, q.w};
      q = j + 128 < ce ? __ldg(reinterpret_cast<const int4*>(A.col + j + 128)) : make_int4(0, 0, 0, 0);
      Mask<W> f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (j + u >= cs && j + u < ce) {
          f[u] = ldg_mask<W>(A.Fcur + (long long)c4[u] * W);
        } else {
#pragma unroll
          for (int k = 0; k < W; ++k) f[u].w[k] = 0;
        }
      }
#pragma unroll
      for (int k = 0; k < W; ++k) la.w[k] |= f[0].w[k] | f[1].w[k] | f[2].w[k] | f[3].w[k];
      if ((step & 3) == 0) {
        Mask<W> tot;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          unsigned long long o = la.w[k];
#pragma unroll
          for (int sh = 16; sh > 0; sh >>= 1) o |= __shfl_xor_sync(0xffffffffu, o, sh);
          tot.w[k] = o | have.w[k];
        }
        if (covers<W>(tot, A.act)) {
          base += 128;
          break;
        }
      }
    }
    Mask<W> acc;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      unsigned long long o = la.w[k];
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) o |= __shfl_xor_sync(0xffffffffu, o, sh);
      acc.w[k] = o;
    }
    if (lane == 0) {
      edges += (unsigned long long)((base < ce ? base : ce) - cs);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const unsigned long long add = acc.w[k] & ~have.w[k];
        if (add) atomicOr(A.acc + r.v * W + k, add);
      }
    }
  }
  if (lane == 0 && edges) atomicAdd(&A.ctrl->edges, edges);
}

// ---- apply the deferred vertices' accumulators ----
template <int W, typename RP>
__global__ void __launch_bounds__(256) k_ms_heavy_apply(MsArgs A) {
  const long long nrec = (long long)(A.ctrl->nheavy & ((1ull << kMsCountBits) - 1));
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long nf = 0, mf = 0, dd = 0;
  Mask<W> act_acc;
#pragma unroll
  for (int k = 0; k < W; ++k) act_acc.w[k] = 0;
  for (long long base = tid - (tid & 31); base < nrec; base += nth) {
    const long long i = base + ms_lane();
    bool nz = false;
    long long v = 0;
    Mask<W> nn;
#pragma unroll
    for (int k = 0; k < W; ++k) nn.w[k] = 0;
    if (i < nrec) {
      const MsHeavy r = A.heavy[i];
      v = r.v;
      const Mask<W> a = load_mask<W>(A.acc + v * W);
      Mask<W> x = load_mask<W>(A.X + v * W);
      Mask<W> z;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        nn.w[k] = a.w[k] & ~x.w[k] & A.full[k];
        x.w[k] |= nn.w[k];
        z.w[k] = 0;
      }
      store_mask<W>(A.acc + v * W, z);
      store_mask<W>(A.Fnext + v * W, nn);
      nz = !is_zero<W>(nn);
      if (nz) {
        if (A.out) direct_out<W>(A, v, nn);
        store_mask<W>(A.X + v * W, x);
        nf += 1;
        mf += (unsigned long long)r.deg;
        if (is_full<W>(x, A.full)) dd += (unsigned long long)r.deg;
      }
    }
    if (A.want_queue) warp_append(nz, (int)v, &A.ctrl->nq, A.qnext);
#pragma unroll
    for (int k = 0; k < W; ++k) act_acc.w[k] |= nn.w[k];
  }
  warp_or_active<W>(act_acc, A.ctrl);
  nf = warp_sum(nf);
  mf = warp_sum(mf);
  dd = warp_sum(dd);
  if (ms_lane() == 0) {
    if (nf) atomicAdd(&A.ctrl->nf, nf);
    if (mf) atomicAdd(&A.ctrl->mf, mf);
    if (dd) atomicAdd(&A.ctrl->done_deg, dd);
  }
}

__device__ __forceinline__ void ms_zero_body(unsigned long long* p, long long count) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < count; i += nth) p[i] = 0ull;
}

__global__ void k_ms_zero(unsigned long long* p, long long count) { ms_zero_body(p, count); }

// ---- writer: ring levels [l0, l0 + nlev) into dist[i][v] ----
// A block owns a tile of 128 vertices (caller's ids).
// Phase 1, one thread per (vertex, word): the vertex's masks of the window's
// levels (coalesced reads; on a renumbered graph at its new id, and a vertex
// of degree 0 is reached only by the lanes it is the source of - level 0,
// first window - which X holds) become, per lane, the offset of the level
// that found it, bit-sliced over the 64 lanes of the word (four planes) plus
// the found mask.  Every group of four lanes (a nibble of each plane) then
// becomes one 32-bit word of four output bytes: spread4 moves bit i of a
// nibble to byte i, so byte i = found ? base + offset : 255, four lanes at a
// time without branches (base = l0 for uint8 rows, 0 for int32 rows, which add
// l0 when they widen).  The words go to shared memory as [word][nibble][vertex]
// (vertex index XOR-swizzled by the word, so the four threads of a vertex hit
// different banks).
// Phase 2, one thread per (word, nibble, four consecutive vertices): one
// 16-byte shared load, a 4x4 byte transpose (__byte_perm) gives the four rows'
// entries of those vertices, so a warp stores 128 consecutive entries of a row
// per instruction (4 bytes a lane for uint8, 16 for int32).  The first window
// writes every entry; later windows write only what they found and skip rows
// with nothing found in the tile.
constexpr int kWt = 128;

// Bit i of a nibble (x < 16) to bit 0 of byte i: the four shifted copies of x
// (by 0, 7, 14 and 21 bits) do not overlap, so the product has no carries.
__device__ __forceinline__ unsigned spread4(unsigned x) { return (x * 0x00204081u) & 0x01010101u; }

template <int W, typename T>
__global__ void __launch_bounds__(256) k_ms_write(const unsigned long long* F, const unsigned long long* X,
                                                  const int* new_of, long long n, long long n_live, int ring, int l0,
                                                  int nlev, int lanes, bool first, T* dist) {
  __shared__ __align__(16) unsigned code[W][16][kWt];
  __shared__ unsigned long long tile_or[W];
  const long long ntiles = (n + kWt - 1) / kWt;
  const unsigned base = sizeof(T) == 1 ? (unsigned)l0 : 0u;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long v0 = tile * kWt;
    if (threadIdx.x < W) tile_or[threadIdx.x] = 0ull;
    __syncthreads();
    for (int idx = threadIdx.x; idx < kWt * W; idx += blockDim.x) {
      const int j = idx / W, ww = idx % W;
      const long long v = v0 + j;
      unsigned long long f = 0, p0 = 0, p1 = 0, p2 = 0, p3 = 0;
      if (v < n) {
        const long long vv = new_of ? (long long)new_of[v] : v;
        if (vv < n_live) {
          unsigned long long m[kMsMaxRing];
#pragma unroll
          for (int l = 0; l < kMsMaxRing; ++l)
            m[l] = l < nlev ? F[(long long)((l0 + l) % ring) * n * W + vv * W + ww] : 0ull;
#pragma unroll
          for (int l = kMsMaxRing - 1; l >= 0; --l) {
            f |= m[l];
            p0 = (p0 & ~m[l]) | ((l & 1) ? m[l] : 0ull);
            p1 = (p1 & ~m[l]) | ((l & 2) ? m[l] : 0ull);
            p2 = (p2 & ~m[l]) | ((l & 4) ? m[l] : 0ull);
            p3 = (p3 & ~m[l]) | ((l & 8) ? m[l] : 0ull);
          }
        } else if (first) {
          f = X[vv * W + ww];
        }
      }
      if (!first && f) atomicOr(&tile_or[ww], f);
      const int js = j ^ (8 * ww);
      if (f == 0) {  // no lane found: every entry "unreached"
#pragma unroll
        for (int k = 0; k < 16; ++k) code[ww][k][js] = 0xffffffffu;
        continue;
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const unsigned sf = spread4((unsigned)(f >> (4 * k)) & 0xfu);
        const unsigned lv = spread4((unsigned)(p0 >> (4 * k)) & 0xfu) + 2u * spread4((unsigned)(p1 >> (4 * k)) & 0xfu) +
                            4u * spread4((unsigned)(p2 >> (4 * k)) & 0xfu) + 8u * spread4((unsigned)(p3 >> (4 * k)) & 0xfu);
        code[ww][k][js] = lv + base * sf + (sf ^ 0x01010101u) * 255u;
      }
    }
    __syncthreads();
    const bool full_tile = v0 + kWt <= n;
    for (int task = threadIdx.x; task < W * 16 * (kWt / 4); task += blockDim.x) {
      const int q = task % (kWt / 4), k = (task / (kWt / 4)) % 16, ww = task / (16 * (kWt / 4));
      const int r0 = 64 * ww + 4 * k;
      if (r0 >= lanes) continue;
      const uint4 c = *reinterpret_cast<const uint4*>(&code[ww][k][(4 * q) ^ (8 * ww)]);
      // c.x..c.w: vertices 4q..4q+3, byte i = row r0 + i.  Transpose to rows.
      const unsigned a = __byte_perm(c.x, c.y, 0x5140), b = __byte_perm(c.z, c.w, 0x5140);
      const unsigned d = __byte_perm(c.x, c.y, 0x7362), e = __byte_perm(c.z, c.w, 0x7362);
      const unsigned rowv[4] = {__byte_perm(a, b, 0x5410), __byte_perm(a, b, 0x7632), __byte_perm(d, e, 0x5410),
                                __byte_perm(d, e, 0x7632)};
      const long long va = v0 + 4 * q;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + i;
        if (r >= lanes) break;
        if (!first && !((tile_or[ww] >> (4 * k + i)) & 1ull)) continue;
        const unsigned w4 = rowv[i];
        if (!first && w4 == 0xffffffffu) continue;
        T* row = dist + (long long)r * n + va;
        if constexpr (sizeof(T) == 1) {
          if (first && full_tile && (reinterpret_cast<uintptr_t>(row) & 3u) == 0) {
            *reinterpret_cast<unsigned*>(row) = w4;
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const unsigned by = (w4 >> (8 * t)) & 0xffu;
              if (va + t < n && (first || by != 0xffu)) row[t] = (T)by;
            }
          }
        } else {
          int x[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const unsigned by = (w4 >> (8 * t)) & 0xffu;
            x[t] = by == 0xffu ? -1 : l0 + (int)by;
          }
          if (first && full_tile && (reinterpret_cast<uintptr_t>(row) & 15u) == 0) {
            *reinterpret_cast<int4*>(row) = make_int4(x[0], x[1], x[2], x[3]);
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (va + t < n && (first || x[t] >= 0)) row[t] = (T)x[t];
          }
        }
      }
    }
    __syncthreads();
  }
}

// Caller's vertex ids -> renumbered ids, in place.
__global__ void k_ms_map(int* ids, int count, const int* new_of) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) ids[i] = new_of[ids[i]];
}

template <typename RP>
__global__ void k_ms_degree_sum(const RP* rp, const int* src, int k, unsigned long long* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const int s = src[i];
    atomicAdd(out, (unsigned long long)(rp[s + 1] - rp[s]));
  }
}

}  // namespace

int ensure_multi_ws(bfs_graph* g, int ring) {
  if (!g->ms) g->ms = new MultiWs();
  MultiWs& ws = *g->ms;
  if (ws.ready && ws.ring == ring) return BFS_OK;
  if (ws.ready) free_multi_ws(g), g->ms = new MultiWs();
  MultiWs& w2 = *g->ms;
  const size_t n = (size_t)g->n;
  GBFS_CUDA(cudaMalloc(&w2.X, sizeof(unsigned long long) * 4 * n));
  GBFS_CUDA(cudaMalloc(&w2.acc, sizeof(unsigned long long) * 4 * n));
  GBFS_CUDA(cudaMemset(w2.acc, 0, sizeof(unsigned long long) * 4 * n));
  GBFS_CUDA(cudaMalloc(&w2.F, sizeof(unsigned long long) * 4 * n * (size_t)ring));
  GBFS_CUDA(cudaMalloc(&w2.touched_bm, sizeof(unsigned) * (size_t)g->nw));
  GBFS_CUDA(cudaMemset(w2.touched_bm, 0, sizeof(unsigned) * (size_t)g->nw));
  for (int i = 0; i < 2; ++i) GBFS_CUDA(cudaMalloc(&w2.q[i], sizeof(int) * n));
  GBFS_CUDA(cudaMalloc(&w2.touched, sizeof(int) * n));
  GBFS_CUDA(cudaMalloc(&w2.heavy, sizeof(MsHeavy) * (n + 2)));
  GBFS_CUDA(cudaMalloc(&w2.d_src, sizeof(int) * 256));
  GBFS_CUDA(cudaMalloc(&w2.order, sizeof(int) * n));
  {
    const int rc = vertices_by_degree(g, w2.order);
    if (rc != BFS_OK) return rc;
  }
  GBFS_CUDA(cudaMalloc(&w2.ctrl, sizeof(MsCtrl)));
  GBFS_CUDA(cudaMallocHost(&w2.h_ctrl, sizeof(MsCtrl)));
  GBFS_CUDA(cudaEventCreateWithFlags(&w2.done, cudaEventDisableTiming));
  w2.ring = ring;
  w2.ready = true;
  return BFS_OK;
}

void free_multi_ws(bfs_graph* g) {
  if (!g->ms) return;
  MultiWs& ws = *g->ms;
  if (ws.done) cudaEventSynchronize(ws.done);
  cudaFree(ws.X);
  cudaFree(ws.acc);
  cudaFree(ws.F);
  cudaFree(ws.touched_bm);
  cudaFree(ws.q[0]);
  cudaFree(ws.q[1]);
  cudaFree(ws.touched);
  cudaFree(ws.heavy);
  cudaFree(ws.d_src);
  cudaFree(ws.order);
  cudaFree(ws.ctrl);
  cudaFree(ws.staging);
  if (ws.h_ctrl) cudaFreeHost(ws.h_ctrl);
  if (ws.done) cudaEventDestroy(ws.done);
  delete g->ms;
  g->ms = nullptr;
}

namespace {

// One level of a lane group, launched asynchronously: every count a later
// kernel needs is read from the control block on the device.
// A push level whose frontier's degree sum exceeds n / 8 touches a large share
// of the vertices: it keeps no touched list and applies by a scan of all vertices.
// A push level's kernels get grids sized to the frontier: nf vertices whose
// degrees sum to mf (an upper bound is enough) need nf planning threads, at
// most nf + mf / kMsPushChunk pushing warps and mf applying threads.
template <int W, typename RP>
void ms_step(MsArgs A, bool push, bool dense, long long nf, long long mf, unsigned long long* Fn, long long n,
             int grid, cudaStream_t s) {
  cudaMemsetAsync(A.ctrl, 0, sizeof(MsCtrl), s);
  A.dense = push && dense ? 1 : 0;
  if (push) {
    auto fit = [grid](long long units, long long per_block) {
      const long long b = (units + per_block - 1) / per_block;
      return (int)(b < 1 ? 1 : (b > grid ? grid : b));
    };
    k_ms_zero<<<grid, 256, 0, s>>>(Fn, n * W);
    k_ms_push_plan<RP><<<fit(nf, 256), 256, 0, s>>>(A, nf);
    k_ms_push<W, RP><<<fit(nf + mf / kMsPushChunk + 1, 8), 256, 0, s>>>(A, nf);
    if (A.dense) k_ms_apply_dense<W, RP><<<grid, 256, 0, s>>>(A);
    else k_ms_apply<W, RP><<<fit(mf, 256), 256, 0, s>>>(A);
  } else {
    k_ms_pull<W, RP><<<grid, 256, 0, s>>>(A);
    k_ms_heavy_chunks<W, RP><<<grid, 256, 0, s>>>(A);
    k_ms_heavy_apply<W, RP><<<grid, 256, 0, s>>>(A);
  }
}

template <int W, typename RP, typename T>
int run_group(bfs_graph* g, const int* srcs, int lanes, T* dist, T unreached, int max_level, const bfs_params& p,
              bfs_multi_stats* st, cudaStream_t s) {
  MultiWs& ws = *g->ms;
  const long long n = g->n;
  const int grid = g->num_sms * 8, block = 256;
  const Relabel* rl = p.ms_relabel ? g->rl : nullptr;
  MsArgs A{};
  A.rp = rl ? rl->rp : g->rp;
  A.col = rl ? rl->col : g->col;
  A.n = n;
  A.n_live = rl ? rl->n_live : n;
  A.nw = g->nw;
  for (int k = 0; k < 4; ++k) {
    const int lo = 64 * k;
    A.full[k] = lanes >= lo + 64 ? ~0ull : (lanes > lo ? ((1ull << (lanes - lo)) - 1ull) : 0ull);
    A.act[k] = A.full[k];
  }
  A.X = ws.X;
  A.acc = ws.acc;
  A.touched_bm = ws.touched_bm;
  A.touched = ws.touched;
  A.heavy = ws.heavy;
  A.ctrl = ws.ctrl;
  A.heavy_min = p.ms_heavy_min;
  A.order = (!rl && p.ms_degree_order) ? ws.order : nullptr;
  A.want_queue = 0;
  const int K = ws.ring;
  auto slot = [&](int l) { return ws.F + (long long)(l % K) * n * W; };
  // Unique sources form the level-0 frontier queue.
  std::vector<int> uniq(srcs, srcs + lanes);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  GBFS_CUDA(cudaMemcpyAsync(ws.d_src, srcs, sizeof(int) * (size_t)lanes, cudaMemcpyHostToDevice, s));
  GBFS_CUDA(cudaMemcpyAsync(ws.q[0], uniq.data(), sizeof(int) * uniq.size(), cudaMemcpyHostToDevice, s));
  if (rl) {
    k_ms_map<<<1, 256, 0, s>>>(ws.d_src, lanes, rl->new_of);
    k_ms_map<<<1, 256, 0, s>>>(ws.q[0], (int)uniq.size(), rl->new_of);
  }
  k_ms_zero<<<grid, block, 0, s>>>(ws.X, n * W);
  k_ms_zero<<<grid, block, 0, s>>>(slot(0), n * W);
  A.Fcur = slot(0);
  k_ms_seed<W><<<1, 256, 0, s>>>(A, ws.d_src, lanes);
  GBFS_CUDA(cudaMemsetAsync(ws.ctrl, 0, sizeof(MsCtrl), s));
  k_ms_degree_sum<RP><<<1, 256, 0, s>>>(reinterpret_cast<const RP*>(A.rp), ws.q[0], (int)uniq.size(), &ws.ctrl->mf);
  GBFS_CUDA(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(MsCtrl), cudaMemcpyDeviceToHost, s));
  GBFS_CUDA(cudaStreamSynchronize(s));
  long long nf = (long long)uniq.size(), mf = (long long)ws.h_ctrl->mf, nf_prev = nf;
  long long m_unfinished = g->m;
  bool push = true;
  bool queue_ready = true;  // ws.q[qc] lists the current frontier (pull and dense push levels keep none)
  int L = 0, flushed = 0, qc = 0;
  bool first_flush = true;
  int rc = BFS_OK;
  auto flush = [&](int upto) -> int {  // write levels [flushed, upto]
    const int nlev = upto - flushed + 1;
    if (nlev <= 0) return BFS_OK;
    k_ms_write<W, T><<<g->num_sms * 16, 256, 0, s>>>(ws.F, ws.X, rl ? rl->new_of : nullptr, n, A.n_live, K, flushed,
                                                     nlev, lanes, first_flush, dist);
    GBFS_CUDA(cudaGetLastError());
    first_flush = false;
    flushed = upto + 1;
    if (st) st->output_bytes += (long long)sizeof(T) * (long long)lanes * n;
    return BFS_OK;
  };
  for (;;) {
    // Direction for this level (edge-count rule, Section 2's BFS-Hybrid-dagger).
    if (L > 0) {
      if (push) push = !((long long)p.ms_alpha * mf > m_unfinished);
      else push = (long long)p.beta * nf < n && nf < nf_prev;
    }
    if (L + 1 - flushed >= K) {
      rc = flush(L);
      if (rc != BFS_OK) return rc;
    }
    unsigned long long* Fn = slot(L + 1);
    A.Fcur = slot(L);
    if (push && !queue_ready) {
      MsArgs C = A;
      C.qnext = ws.q[qc];
      GBFS_CUDA(cudaMemsetAsync(&ws.ctrl->nq, 0, sizeof(unsigned long long), s));
      k_ms_compact<W><<<grid, block, 0, s>>>(C);
      GBFS_CUDA(cudaGetLastError());
    }
    A.Fnext = Fn;
    A.qcur = ws.q[qc];
    A.qnext = ws.q[qc ^ 1];
    const bool dense = mf > n / 8;
    ms_step<W, RP>(A, push, dense, nf, mf, Fn, A.n_live, grid, s);
    queue_ready = push && !dense;
    GBFS_CUDA(cudaGetLastError());
    GBFS_CUDA(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(MsCtrl), cudaMemcpyDeviceToHost, s));
    GBFS_CUDA(cudaStreamSynchronize(s));
    const MsCtrl c = *ws.h_ctrl;
    if (st) {
      if (push) {
        ++st->push_levels;
        st->pushed_edges += (long long)c.edges;
        st->push_frontier += nf;
      } else {
        ++st->pull_levels;
        st->pulled_edges += (long long)c.edges;
        st->pull_active += (long long)c.active;
      }
      st->found += (long long)c.nf;
    }
    for (int k = 0; k < 4; ++k) A.act[k] = c.act[k];
    nf_prev = nf;
    nf = (long long)c.nf;
    mf = (long long)c.mf;
    m_unfinished -= (long long)c.done_deg;
    if (nf == 0) break;
    if (L + 1 > max_level) return BFS_ERANGE;
    ++L;
    qc ^= 1;
  }
  if (st && L + 1 > st->levels) st->levels = L + 1;
  rc = flush(L);
  if (rc != BFS_OK) return rc;
  GBFS_CUDA(cudaEventRecord(ws.done, s));
  return BFS_OK;
}

template <int W>
int run_group_w(bfs_graph* g, const int* srcs, int lanes, void* dist, int bits, const bfs_params& p,
                bfs_multi_stats* st, cudaStream_t s) {
  if (bits == 8) {
    if (g->rp_bits == 32)
      return run_group<W, int, uint8_t>(g, srcs, lanes, (uint8_t*)dist, (uint8_t)255, 254, p, st, s);
    return run_group<W, long long, uint8_t>(g, srcs, lanes, (uint8_t*)dist, (uint8_t)255, 254, p, st, s);
  }
  if (g->rp_bits == 32)
    return run_group<W, int, int32_t>(g, srcs, lanes, (int32_t*)dist, -1, 0x7fffffff, p, st, s);
  return run_group<W, long long, int32_t>(g, srcs, lanes, (int32_t*)dist, -1, 0x7fffffff, p, st, s);
}

}  // namespace

int run_multi(bfs_graph* g, const int32_t* srcs, int k, void* dist, int bits, const bfs_params& p,
              bfs_multi_stats* st, cudaStream_t s) {
  int ring = p.ms_ring;
  if (ring < 2) ring = 2;
  if (ring > kMsMaxRing) ring = kMsMaxRing;
  int rc = ensure_multi_ws(g, ring);
  if (rc != BFS_OK) return rc;
  if (p.ms_relabel) {
    rc = ensure_relabel(g);
    if (rc != BFS_OK) return rc;
  }
  MultiWs& ws = *g->ms;
  GBFS_CUDA(cudaStreamWaitEvent(s, ws.done, 0));
  const bool host_out = !is_device_pointer(dist);
  const size_t esz = (size_t)bits / 8;
  const int per_group = p.ms_lanes;
  for (int g0 = 0; g0 < k; g0 += per_group) {
    const int lanes = std::min(per_group, k - g0);
    void* out = host_out ? nullptr : (void*)((char*)dist + (size_t)g0 * (size_t)g->n * esz);
    if (host_out) {
      const size_t need = (size_t)lanes * (size_t)g->n * esz;
      if (ws.staging_bytes < need) {
        cudaFree(ws.staging);
        ws.staging = nullptr;
        ws.staging_bytes = 0;
        GBFS_CUDA(cudaMalloc(&ws.staging, need));
        ws.staging_bytes = need;
      }
      out = ws.staging;
    }
    const int W = (lanes + 63) / 64;
    if (W == 1) rc = run_group_w<1>(g, srcs + g0, lanes, out, bits, p, st, s);
    else if (W == 2) rc = run_group_w<2>(g, srcs + g0, lanes, out, bits, p, st, s);
    else rc = run_group_w<4>(g, srcs + g0, lanes, out, bits, p, st, s);
    if (rc != BFS_OK) return rc;
    if (st) ++st->groups;
    if (host_out) {
      GBFS_CUDA(cudaMemcpyAsync((char*)dist + (size_t)g0 * (size_t)g->n * esz, out,
                                (size_t)lanes * (size_t)g->n * esz, cudaMemcpyDeviceToHost, s));
    }
  }
  GBFS_CUDA(cudaEventRecord(ws.done, s));
  GBFS_CUDA(cudaStreamSynchronize(s));
  return BFS_OK;
}

}  // namespace gbfs

// ============================================================================
// Serving support: one 64-lane group per resident graph.  Queries join free
// lanes at level boundaries (their own level 0 is the group's current level),
// run with the other lanes, and leave when their frontier empties; their rows
// are written from the frontier ring with per-lane offsets.
// ============================================================================
namespace gbfs {

// State of one persistent serving launch (zeroed before it starts).
struct ServeLoop {
  unsigned long long barrier;   // grid-barrier arrivals
  int status;                   // BFS_OK or BFS_ETIMEOUT
  int levels;                   // levels the launch completed
  MsCtrl ctrl[2];               // counters of the launch's even / odd levels
};

struct ServeGroup {
  bfs_graph* g = nullptr;
  int ring = 8;
  long long n = 0;
  int heavy_min = 256;
  unsigned long long* X = nullptr;
  unsigned long long* acc = nullptr;
  unsigned long long* F = nullptr;
  unsigned* touched_bm = nullptr;
  int* q[2] = {nullptr, nullptr};
  int* touched = nullptr;
  MsHeavy* heavy = nullptr;
  int* order = nullptr;
  MsCtrl* ctrl = nullptr;
  MsCtrl* h_ctrl = nullptr;
  int** d_out = nullptr;   // [64] output row per lane
  int* d_join = nullptr;   // [64] join level per lane
  int* d_new = nullptr;    // [64] sources of joining lanes
  int* d_newlane = nullptr;
  int** h_out = nullptr;   // pinned mirrors
  int* h_join = nullptr;
  int* h_new = nullptr;
  int* h_newlane = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_level = nullptr;
  // Blocks per launch.  A high-priority group gets the usual grid; the others
  // get about one block per 2048 vertices, so each block is short-lived and
  // the priority group's kernels find free SM slots between them instead of
  // waiting for a grid-stride kernel to end.
  int grid = 0, wgrid = 0;
  int L = 0, qc = 0, flushed = 0;
  long long nf = 0;
  long long mf = 0;        // degree sum of the current frontier (an upper bound after joins)
  unsigned long long lanes = 0, act = 0, first = 0;
  bool launched = false;
  // Large-diameter groups write distances as they are found (no ring flush)
  // and run consecutive push levels in one persistent launch.
  bool direct = false;
  bool use_loop = false;
  bool loop_launched = false;
  int loop_grid = 0;
  ServeLoop* SL = nullptr;      // device
  ServeLoop* h_SL = nullptr;    // pinned mirror
};

namespace {

__global__ void k_serve_clear(unsigned long long* X, long long n, unsigned long long keep) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < n; v += nth) X[v] &= keep;
}

__global__ void k_serve_seed(unsigned long long* X, unsigned long long* Fcur, int* q, long long nf, const int* src,
                             const int* lane, int count) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const int s = src[k];
    const unsigned long long bit = 1ull << lane[k];
    atomicOr(X + s, bit);
    atomicOr(Fcur + s, bit);
    q[nf + k] = s;
  }
}

// Direct-output groups: the joining lanes' rows start as "unreached" with 0
// at their sources.
__global__ void k_serve_init_rows(int* const* out, const int* lane, const int* src, int count, long long n) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long t = tid; t < (long long)count * n; t += nth) {
    const int k = (int)(t / n);
    const long long v = t - (long long)k * n;
    out[lane[k]][v] = v == (long long)src[k] ? 0 : -1;
  }
}

// Rows of the lanes in `lanes` from ring levels [l0, l0+nlev): lane i's value
// at a vertex is (level - join[i]) for the first level >= join[i] whose
// frontier holds bit i (levels below join[i] are masked by valid[]), else -1
// on the lane's first window.
__global__ void __launch_bounds__(256) k_serve_write(const unsigned long long* F, long long n, int ring, int l0,
                                                     int nlev, const unsigned long long* valid, unsigned long long lanes,
                                                     unsigned long long first, int* const* out, const int* join) {
  __shared__ unsigned long long pl[5][kWt];
  __shared__ unsigned long long vmask[kMsMaxRing];
  if (threadIdx.x < kMsMaxRing) vmask[threadIdx.x] = threadIdx.x < (unsigned)nlev ? valid[threadIdx.x] : 0ull;
  const long long ntiles = (n + kWt - 1) / kWt;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long v0 = tile * kWt;
    for (int j = threadIdx.x; j < kWt; j += blockDim.x) {
      const long long v = v0 + j;
      unsigned long long f = 0, p0 = 0, p1 = 0, p2 = 0, p3 = 0;
      if (v < n) {
        // All of the window's loads in flight at once, then the planes.
        unsigned long long mm[kMsMaxRing];
#pragma unroll
        for (int l = 0; l < kMsMaxRing; ++l) mm[l] = l < nlev ? F[(long long)((l0 + l) % ring) * n + v] & vmask[l] : 0ull;
#pragma unroll
        for (int l = kMsMaxRing - 1; l >= 0; --l) {
          const unsigned long long m = mm[l];
          f |= m;
          p0 = (p0 & ~m) | ((l & 1) ? m : 0ull);
          p1 = (p1 & ~m) | ((l & 2) ? m : 0ull);
          p2 = (p2 & ~m) | ((l & 4) ? m : 0ull);
          p3 = (p3 & ~m) | ((l & 8) ? m : 0ull);
        }
      }
      pl[0][j] = f;
      pl[1][j] = p0;
      pl[2][j] = p1;
      pl[3][j] = p2;
      pl[4][j] = p3;
    }
    __syncthreads();
    unsigned long long todo = lanes;
    for (int r = 0; todo; ++r) {
      const int i = __ffsll((long long)todo) - 1;
      todo &= todo - 1;
      if ((r % (int)nwarp) != (int)warp) continue;
      const bool fst = (first >> i) & 1ull;
      int* row = out[i] + v0;
      const int jn = join[i];
#pragma unroll
      for (int q = 0; q < kWt / 32; ++q) {
        const int j = (int)lane + 32 * q;
        if (v0 + j >= n) break;
        if ((pl[0][j] >> i) & 1ull) {
          const int lv = (int)(((pl[1][j] >> i) & 1ull) | (((pl[2][j] >> i) & 1ull) << 1) |
                               (((pl[3][j] >> i) & 1ull) << 2) | (((pl[4][j] >> i) & 1ull) << 3));
          row[j] = l0 + lv - jn;
        } else if (fst) {
          row[j] = -1;
        }
      }
    }
    __syncthreads();
  }
}

MsArgs serve_args(const ServeGroup* G) {
  MsArgs A{};
  A.rp = G->g->rp;
  A.col = G->g->col;
  A.n = G->n;
  A.n_live = G->n;
  A.nw = G->g->nw;
  A.full[0] = G->lanes;
  A.act[0] = G->act;
  for (int k = 1; k < 4; ++k) A.full[k] = A.act[k] = 0;
  A.X = G->X;
  A.acc = G->acc;
  A.Fcur = G->F + (long long)(G->L % G->ring) * G->n;
  A.Fnext = G->F + (long long)((G->L + 1) % G->ring) * G->n;
  A.touched_bm = G->touched_bm;
  A.qcur = G->q[G->qc];
  A.qnext = G->q[G->qc ^ 1];
  A.touched = G->touched;
  A.heavy = G->heavy;
  A.order = G->order;
  A.ctrl = G->ctrl;
  A.heavy_min = G->heavy_min;
  A.want_queue = 1;
  if (G->direct) {
    A.out = G->d_out;
    A.join = G->d_join;
    A.out_level = G->L + 1;
  }
  return A;
}

template <typename RP>
void serve_step(ServeGroup* G, bool push) {
  const MsArgs A = serve_args(G);
  ms_step<1, RP>(A, push, false, G->nf, G->mf, A.Fnext, G->n, G->grid, G->stream);
}

// Grid barrier of the persistent serving launch: arrival with a release add,
// a bounded acquire spin; on timeout the status is set and every block returns.
// `extra` (testing) makes it wait for that many blocks more than were launched.
__device__ bool loop_barrier(ServeLoop* SL, unsigned& epoch, long long timeout_ns, int extra) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned long long target = (unsigned long long)epoch * ((unsigned long long)gridDim.x + (unsigned)extra);
    __threadfence();
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&SL->barrier) : "memory");
    int ok = 1;
    unsigned long long t0 = 0;
    unsigned spins = 0;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&SL->barrier) : "memory");
      if (v >= target) break;
      if (*reinterpret_cast<volatile int*>(&SL->status) != 0) {
        ok = 0;
        break;
      }
      if ((++spins & 63u) == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t0 == 0) {
          t0 = t;
        } else if ((long long)(t - t0) > timeout_ns) {
          atomicCAS(&SL->status, 0, BFS_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && *reinterpret_cast<volatile int*>(&SL->status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Consecutive push levels of a 64-lane serving group in one cooperative
// launch (the same phases as the per-level launches, grid barriers between
// them).  It stops after the level at which a lane's frontier empties (the
// host retires it), when the frontier is empty or dense enough for a pull,
// or after max_levels levels (the frontier ring must be flushed).  Frontier
// masks change between levels of the launch, so they are read with coherent
// loads only.
template <typename RP>
__global__ void __launch_bounds__(256) k_serve_loop(MsArgs A, unsigned long long* F, int ring, int L0, int* q0,
                                                    int* q1, int qc0, long long nf0, long long mf0, int max_levels,
                                                    int tau_inv, long long timeout_ns, int need_plan, ServeLoop* SL,
                                                    int barrier_extra) {
  unsigned epoch = 0;
  const unsigned long long lanes = A.full[0];
  unsigned long long act = A.act[0];
  long long nf = nf0;
  int L = L0, qc = qc0;
  (void)mf0;
  for (int it = 0;;) {
    MsCtrl* C = &SL->ctrl[it & 1];
    A.ctrl = C;
    A.Fcur = F + (long long)(L % ring) * A.n;
    A.Fnext = F + (long long)((L + 1) % ring) * A.n;
    A.qcur = qc ? q1 : q0;
    A.qnext = qc ? q0 : q1;
    A.act[0] = act;
    A.out_level = L + 1;
    ms_zero_body(A.Fnext, A.n);
    if (need_plan) ms_push_plan_body<RP>(A, nf);  // only vertices of more than kMsPushChunk entries
    if (!loop_barrier(SL, epoch, timeout_ns, barrier_extra)) return;
    ms_push_body<1, RP>(A, nf);
    if (!loop_barrier(SL, epoch, timeout_ns, barrier_extra)) return;
    ms_apply_body<1, RP>(A);
    if (!loop_barrier(SL, epoch, timeout_ns, barrier_extra)) return;
    const long long nf2 = (long long)ld_cg_u64(&C->nf);
    const unsigned long long act2 = ld_cg_u64(&C->act[0]) & lanes;
    ++it;
    if (nf2 == 0 || act2 != lanes || it >= max_levels || !((long long)tau_inv * nf2 < A.n)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) SL->levels = it;
      return;
    }
    // Counters of the next level: the slot used two levels ago, which every
    // block has finished reading (they all passed this level's barriers).
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      unsigned long long* z = reinterpret_cast<unsigned long long*>(&SL->ctrl[it & 1]);
      for (int k = 0; k < (int)(sizeof(MsCtrl) / sizeof(unsigned long long)); ++k) z[k] = 0ull;
    }
    L += 1;
    qc ^= 1;
    nf = nf2;
    act = act2;
  }
}

int serve_flush(ServeGroup* G, int upto) {
  if (G->direct) {  // rows were written as the levels ran
    G->flushed = upto + 1;
    return BFS_OK;
  }
  const int nlev = upto - G->flushed + 1;
  if (nlev <= 0 || !G->lanes) {
    G->flushed = upto + 1;
    return BFS_OK;
  }
  unsigned long long valid[kMsMaxRing] = {0};
  for (int l = 0; l < nlev; ++l)
    for (int i = 0; i < 64; ++i)
      if (((G->lanes >> i) & 1ull) && G->h_join[i] <= G->flushed + l) valid[l] |= 1ull << i;
  unsigned long long* d_valid = reinterpret_cast<unsigned long long*>(G->ctrl + 1);
  GBFS_CUDA(cudaMemcpyAsync(d_valid, valid, sizeof(valid), cudaMemcpyHostToDevice, G->stream));
  k_serve_write<<<G->wgrid, 256, 0, G->stream>>>(G->F, G->n, G->ring, G->flushed, nlev, d_valid, G->lanes,
                                                           G->first, G->d_out, G->d_join);
  GBFS_CUDA(cudaGetLastError());
  G->first &= ~G->lanes;
  G->flushed = upto + 1;
  return BFS_OK;
}

}  // namespace

size_t serve_group_bytes(const bfs_graph* g, int ring) {
  const size_t n = (size_t)g->n;
  const size_t heavy = (std::min(n, (size_t)g->m / 9) + 2) * sizeof(MsHeavy);
  return n * 8 * (2 + (size_t)ring) + n * 4 * 4 + heavy + (size_t)g->nw * 4 + 4096;
}

int serve_group_create(bfs_graph* g, int ring, int heavy_min, int high_priority, ServeGroup** out) {
  ServeGroup* G = new ServeGroup();
  G->g = g;
  G->ring = ring < 2 ? 2 : (ring > kMsMaxRing ? kMsMaxRing : ring);
  G->n = g->n;
  G->heavy_min = heavy_min;
  const size_t n = (size_t)g->n;
  {
    const long long base = (long long)g->num_sms * 8;
    const long long many = ((long long)n + 2047) / 2048, tiles = ((long long)n + kWt - 1) / kWt / 4;
    G->grid = (int)(high_priority ? base : std::min(std::max(base, many), 1ll << 20));
    G->wgrid = (int)(high_priority ? base : std::min(std::max(base, tiles), 1ll << 20));
  }
  int rc = BFS_OK;
  do {
    cudaError_t e = cudaMalloc(&G->X, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&G->acc, 8 * n);
    if (e == cudaSuccess) e = cudaMemset(G->acc, 0, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&G->F, 8 * n * (size_t)G->ring);
    if (e == cudaSuccess) e = cudaMalloc(&G->touched_bm, 4 * (size_t)g->nw);
    if (e == cudaSuccess) e = cudaMemset(G->touched_bm, 0, 4 * (size_t)g->nw);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&G->q[i], 4 * n + 4 * 64);
    if (e == cudaSuccess) e = cudaMalloc(&G->touched, 4 * n);
    if (G->heavy_min < 8) G->heavy_min = 8;
    const size_t heavy_cap = std::min(n, (size_t)g->m / (size_t)(G->heavy_min + 1)) + 2;
    if (e == cudaSuccess) e = cudaMalloc(&G->heavy, sizeof(MsHeavy) * heavy_cap);
    if (e == cudaSuccess) e = cudaMalloc(&G->order, 4 * n);
    // The control block, then the per-level lane masks of a flush (serve_flush).
    if (e == cudaSuccess) e = cudaMalloc(&G->ctrl, sizeof(MsCtrl) + sizeof(unsigned long long) * kMsMaxRing);
    if (e == cudaSuccess) e = cudaMallocHost(&G->h_ctrl, sizeof(MsCtrl));
    if (e == cudaSuccess) e = cudaMalloc(&G->d_out, sizeof(int*) * 64);
    if (e == cudaSuccess) e = cudaMalloc(&G->d_join, sizeof(int) * 64);
    if (e == cudaSuccess) e = cudaMalloc(&G->d_new, sizeof(int) * 64);
    if (e == cudaSuccess) e = cudaMalloc(&G->d_newlane, sizeof(int) * 64);
    if (e == cudaSuccess) e = cudaMallocHost(&G->h_out, sizeof(int*) * 64);
    if (e == cudaSuccess) e = cudaMallocHost(&G->h_join, sizeof(int) * 64);
    if (e == cudaSuccess) e = cudaMallocHost(&G->h_new, sizeof(int) * 64);
    if (e == cudaSuccess) e = cudaMallocHost(&G->h_newlane, sizeof(int) * 64);
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&G->stream, cudaStreamNonBlocking, high_priority ? prio_hi : prio_lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->ev_level, cudaEventDisableTiming);
    if (e == cudaSuccess && high_priority) {
      // Persistent push levels: all blocks must be resident at once (cooperative launch).
      e = cudaMalloc(&G->SL, sizeof(ServeLoop));
      if (e == cudaSuccess) e = cudaMallocHost(&G->h_SL, sizeof(ServeLoop));
      int per_sm = 0;
      const void* fn = g->rp_bits == 32 ? reinterpret_cast<const void*>(&k_serve_loop<int>)
                                        : reinterpret_cast<const void*>(&k_serve_loop<long long>);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
      if (e == cudaSuccess && per_sm >= 1) {
        G->loop_grid = std::min(per_sm, 2) * g->num_sms;
        G->use_loop = true;
      }
      G->direct = true;
    }
    if (e != cudaSuccess) { rc = cuda_fail(e, "serving group allocation", __FILE__, __LINE__); break; }
    rc = vertices_by_degree(g, G->order);
  } while (0);
  if (rc != BFS_OK) {
    serve_group_destroy(G);
    return rc;
  }
  *out = G;
  return BFS_OK;
}

void serve_group_destroy(ServeGroup* G) {
  if (!G) return;
  if (G->stream) cudaStreamSynchronize(G->stream);
  cudaFree(G->X);
  cudaFree(G->acc);
  cudaFree(G->F);
  cudaFree(G->touched_bm);
  cudaFree(G->q[0]);
  cudaFree(G->q[1]);
  cudaFree(G->touched);
  cudaFree(G->heavy);
  cudaFree(G->order);
  cudaFree(G->ctrl);
  cudaFree(G->d_out);
  cudaFree(G->d_join);
  cudaFree(G->d_new);
  cudaFree(G->d_newlane);
  if (G->h_ctrl) cudaFreeHost(G->h_ctrl);
  if (G->h_out) cudaFreeHost(G->h_out);
  if (G->h_join) cudaFreeHost(G->h_join);
  if (G->h_new) cudaFreeHost(G->h_new);
  if (G->h_newlane) cudaFreeHost(G->h_newlane);
  if (G->ev_level) cudaEventDestroy(G->ev_level);
  cudaFree(G->SL);
  if (G->h_SL) cudaFreeHost(G->h_SL);
  if (G->stream) cudaStreamDestroy(G->stream);
  delete G;
}

cudaStream_t serve_group_stream(ServeGroup* G) { return G->stream; }
unsigned long long serve_group_lanes(const ServeGroup* G) { return G->lanes; }
int serve_group_level(const ServeGroup* G) { return G->L; }

int serve_group_join(ServeGroup* G, int count, const int* lanes_idx, const int* srcs, int* const* outs) {
  if (count <= 0) return BFS_OK;
  const int grid = G->grid;
  unsigned long long mask = 0;
  for (int k = 0; k < count; ++k) mask |= 1ull << lanes_idx[k];
  if (G->lanes == 0) {
    // Idle group: start a new timeline at level 0.
    G->L = 0;
    G->qc = 0;
    G->flushed = 0;
    G->nf = 0;
    G->mf = 0;
    G->act = 0;
    k_ms_zero<<<grid, 256, 0, G->stream>>>(G->X, G->n);
    k_ms_zero<<<grid, 256, 0, G->stream>>>(G->F, G->n);
  } else {
    k_serve_clear<<<grid, 256, 0, G->stream>>>(G->X, G->n, ~mask);
  }
  // A joining lane's level 0 is level L: it must lie in the next flushed window.
  if (G->flushed > G->L) G->flushed = G->L;
  for (int k = 0; k < count; ++k) {
    G->h_new[k] = srcs[k];
    G->h_newlane[k] = lanes_idx[k];
    G->h_join[lanes_idx[k]] = G->L;
    G->h_out[lanes_idx[k]] = outs[k];
  }
  GBFS_CUDA(cudaMemcpyAsync(G->d_new, G->h_new, sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, G->stream));
  GBFS_CUDA(cudaMemcpyAsync(G->d_newlane, G->h_newlane, sizeof(int) * (size_t)count, cudaMemcpyHostToDevice,
                            G->stream));
  GBFS_CUDA(cudaMemcpyAsync(G->d_join, G->h_join, sizeof(int) * 64, cudaMemcpyHostToDevice, G->stream));
  GBFS_CUDA(cudaMemcpyAsync(G->d_out, G->h_out, sizeof(int*) * 64, cudaMemcpyHostToDevice, G->stream));
  if (G->direct) {
    const long long total = (long long)count * G->n;
    const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)G->g->num_sms * 32);
    k_serve_init_rows<<<blocks, 256, 0, G->stream>>>(G->d_out, G->d_newlane, G->d_new, count, G->n);
  }
  k_serve_seed<<<1, 64, 0, G->stream>>>(G->X, G->F + (long long)(G->L % G->ring) * G->n, G->q[G->qc], G->nf, G->d_new,
                                        G->d_newlane, count);
  GBFS_CUDA(cudaGetLastError());
  G->nf += count;
  G->mf += (long long)count * G->g->max_deg;  // the sources' degrees are not known on the host
  G->lanes |= mask;
  G->act |= mask;
  G->first |= mask;
  return BFS_OK;
}

int serve_group_launch(ServeGroup* G, int tau_inv, long long timeout_ns, int barrier_extra) {
  if (!G->lanes || G->launched) return BFS_OK;
  if (!G->direct && G->L + 1 - G->flushed >= G->ring) {
    const int rc = serve_flush(G, G->L);
    if (rc != BFS_OK) return rc;
  }
  const bool push = (long long)tau_inv * G->nf < G->n;
  if (G->use_loop && push) {
    // As many push levels as the ring has room for, in one launch.
    MsArgs A = serve_args(G);
    unsigned long long* F = G->F;
    // Ring-writer groups stop when the ring is full; direct-output groups stop
    // at a retirement, or after 64 levels while lanes are free (queries that
    // arrive meanwhile join at the next launch).
    int ring = G->ring, L0 = G->L, qc0 = G->qc;
    int max_levels = G->direct ? (G->lanes == ~0ull ? 4096 : 64) : G->ring - 1 - (G->L - G->flushed);
    int* q0 = G->q[0];
    int* q1 = G->q[1];
    long long nf0 = G->nf, mf0 = G->mf;
    ServeLoop* SL = G->SL;
    int need_plan = G->g->max_deg > kMsPushChunk ? 1 : 0;
    void* args[] = {&A,  &F,          &ring,    &L0,         &q0,        &q1, &qc0,
                    &nf0, &mf0,       &max_levels, &tau_inv, &timeout_ns, &need_plan, &SL, &barrier_extra};
    GBFS_CUDA(cudaMemsetAsync(G->SL, 0, sizeof(ServeLoop), G->stream));
    const void* fn = G->g->rp_bits == 32 ? reinterpret_cast<const void*>(&k_serve_loop<int>)
                                         : reinterpret_cast<const void*>(&k_serve_loop<long long>);
    GBFS_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)G->loop_grid), dim3(256), args, 0, G->stream));
    GBFS_CUDA(cudaMemcpyAsync(G->h_SL, G->SL, sizeof(ServeLoop), cudaMemcpyDeviceToHost, G->stream));
    G->loop_launched = true;
  } else {
    if (G->g->rp_bits == 32) serve_step<int>(G, push); else serve_step<long long>(G, push);
    GBFS_CUDA(cudaGetLastError());
    GBFS_CUDA(cudaMemcpyAsync(G->h_ctrl, G->ctrl, sizeof(MsCtrl), cudaMemcpyDeviceToHost, G->stream));
  }
  GBFS_CUDA(cudaEventRecord(G->ev_level, G->stream));
  G->launched = true;
  return BFS_OK;
}

// 1: a launched level has completed, 0: still running, -1: nothing launched.
int serve_group_ready(ServeGroup* G) {
  if (!G->launched) return -1;
  const cudaError_t e = cudaEventQuery(G->ev_level);
  if (e == cudaErrorNotReady) return 0;
  return 1;  // errors surface in serve_group_finish's synchronize
}

int serve_group_finish(ServeGroup* G, unsigned long long* retired) {
  *retired = 0;
  if (!G->launched) return BFS_OK;
  GBFS_CUDA(cudaEventSynchronize(G->ev_level));
  G->launched = false;
  MsCtrl c = *G->h_ctrl;
  if (G->loop_launched) {
    // The launch ran levels L .. L+k-1; continue as after a single step at L+k-1.
    G->loop_launched = false;
    if (G->h_SL->status != BFS_OK) return G->h_SL->status;
    const int k = G->h_SL->levels;
    if (k < 1) return BFS_ECUDA;
    c = G->h_SL->ctrl[(k - 1) & 1];
    G->L += k - 1;
    G->qc ^= (k - 1) & 1;
  }
  const unsigned long long act_next = c.act[0] & G->lanes;
  const unsigned long long done = G->lanes & ~act_next;
  G->nf = (long long)c.nf;
  G->mf = (long long)c.mf;
  G->act = act_next;
  if (done) {
    // The finished lanes' last frontier is level L (their level L+1 is empty);
    // level L+1 stays unflushed, so lanes that join there are written later.
    const int rc = serve_flush(G, G->L);
    if (rc != BFS_OK) return rc;
    G->lanes &= ~done;
  }
  G->L += 1;
  G->qc ^= 1;
  *retired = done;
  return BFS_OK;
}

}  // namespace gbfs
