// Single-source hybrid BFS on sm_103a.
//
// One query runs either as ONE persistent cooperative launch (every level,
// grid barrier between phases) or as one launch per phase with the host
// reading the frontier size after each level.  Both use the same device phase
// functions below.
//
// Paper mapping (Section 2):
//   * top-down level  = Listing 1's frontier loop with the visited test of
//     Listing 3: a neighbour whose visited bit is clear is claimed with one
//     atomicOr on its bitmap word (a bit-packed set cannot take the paper's
//     plain `visited_bm[dst] = true`: two plain read-modify-writes of one word
//     can lose a bit), then dist is written with a plain store;
//   * bottom-up level = Listing 2/3: every unvisited vertex scans its
//     adjacency in CSR order and stops at the first neighbour in the frontier
//     bitmap; one warp owns 32 consecutive vertices, so the new frontier and
//     visited words are built with a ballot and stored plainly;
//   * direction switch = Listing 2's rule (or the edge-count rule it cites),
//     queue <-> bitmap conversion on a change of direction.
// GPU-specific pieces: the frontier is stored as edge-range work items binned
// by degree when a vertex is discovered (small vertices 32 per warp, larger
// ones one warp per <= chunk edges), neighbour lists are read with 128-bit
// loads, and queue appends are aggregated per warp.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "bfs_device.cuh"
#include "bfs_internal.cuh"

namespace gbfs {

namespace {

using namespace dev;

// Bounds-checked build (GBFS_DEBUG_BOUNDS, the stand-in for a memory checker):
// every data-dependent global index of the kernels below is checked against
// its array; the first out-of-range index is recorded in a device word
// (bit 63, site << 48, low 48 bits of the index) and the access goes to element
// 0 instead, so the kernel still completes.  Release builds compile the
// checks away (the macros are the index itself).
#ifdef GBFS_DEBUG_BOUNDS
__device__ unsigned long long g_bounds_err;
__device__ __forceinline__ long long bchk(long long i, long long lim, int site) {
  if (i >= 0 && i < lim) return i;
  atomicCAS(&g_bounds_err, 0ull,
            (1ull << 63) | ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
  return 0;
}
#define GBFS_CHK(i, lim, site) bchk((long long)(i), (long long)(lim), (site))
#else
#define GBFS_CHK(i, lim, site) (i)
#endif
#define BV(i, site) GBFS_CHK(i, P.n, site)          // per-vertex arrays (head, dist, level bytes, id maps)
#define BRP(i, site) GBFS_CHK(i, P.n + 1, site)     // row pointers
#define BW(i, site) GBFS_CHK(i, P.nw, site)         // bitmap words (visited, next frontier, mask)
#define BWF(i, site) GBFS_CHK(i, P.nw, site)        // frontier bitmap words
#define BQ(i, site) GBFS_CHK(i, P.n, site)          // vertex queues
#define BIT(i, site) GBFS_CHK(i, P.cap, site)       // work items
#define BMG(i, site) GBFS_CHK(i, P.mg_cap, site)    // hub records
#define BCOL(i, site) GBFS_CHK(i, P.col_cap, site)  // one neighbour id
#define BCOL4(i, site) GBFS_CHK(i, P.col_cap - 3, site)  // four neighbour ids from index i


// The level of vertex v is L + 1: a level byte while the search keeps them
// (direct = false), else its int32 distance.
__device__ __forceinline__ void mark_level(const KParams& P, bool direct, int v, int L) {
  if (direct) P.dist[BV(P.old_of ? P.old_of[BV(v, 1)] : v, 2)] = L + 1;
  else st_u8_last(P.lv8 + BV(v, 3), (unsigned)(L + 1));
}

__device__ __forceinline__ unsigned long long pack_item(long long start, int len) {
  return ((unsigned long long)start << 16) | (unsigned long long)(unsigned)len;
}

// Bounded grid barrier of the query's control block.
__device__ __forceinline__ bool grid_barrier(const KParams& P, unsigned& epoch) {
  return grid_barrier_ctl(P.ctrl, P.timeout_ns, P.barrier_extra, epoch);
}

// Per-thread work counters of one phase.
struct Acc {
  unsigned long long found = 0, mf = 0;        // bottom-up discoveries
  unsigned long long edges = 0, unvisited = 0;  // statistics
};

// Block-reduce (found, mf, edges, unvisited) and add them to the level's
// counters with one atomic per block.
template <bool STATS>
__device__ void flush_acc(const KParams& P, int L, Acc& a, Slot* out, bool bottom_up) {
  __shared__ unsigned long long s_red[4][32];
  unsigned long long v0 = warp_sum_u64(a.found), v1 = warp_sum_u64(a.mf);
  unsigned long long v2 = STATS ? warp_sum_u64(a.edges) : 0ull;
  unsigned long long v3 = STATS ? warp_sum_u64(a.unvisited) : 0ull;
  const unsigned w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  if (lane_id() == 0) {
    s_red[0][w] = v0;
    s_red[1][w] = v1;
    s_red[2][w] = v2;
    s_red[3][w] = v3;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = warp_sum_u64(threadIdx.x < nwb ? s_red[k][threadIdx.x] : 0ull);
    if (threadIdx.x == 0) {
      if (bottom_up) {
        if (r[0]) atomicAdd(&out->nv, r[0]);
        if (r[1]) atomicAdd(&out->mf, r[1]);
      }
      if (STATS) {
        if (bottom_up) {
          atomicAdd(&P.ctrl->bu_edges, r[2]);
          atomicAdd(&P.ctrl->bu_unvisited, r[3]);
        } else {
          atomicAdd(&P.ctrl->td_edges, r[2]);
        }
        if (P.lst && L < P.lst_cap) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&P.lst[L].edges), r[2]);
          atomicAdd(reinterpret_cast<unsigned long long*>(&P.lst[L].unvisited), r[3]);
        }
      }
    }
  }
  __syncthreads();
  a = Acc();
}

// ---------------------------------------------------------------- init

// dist[:] = -1 except dist[src] = 0; visited = degree-0/padding mask | src bit.
template <typename RP>
__device__ __noinline__ void init_phase(const KParams& P) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long n = P.n;
  if (P.lv8) {
    // Level bytes: 255 everywhere (the allocation is rounded up to 16 bytes), 0 at src.
    const long long n16 = (n + 15) >> 4;
    for (long long i = tid; i < n16; i += nth) {
      unsigned w[4] = {kFull, kFull, kFull, kFull};
      if ((long long)(P.src >> 4) == i) w[(P.src >> 2) & 3] &= ~(0xffu << (8 * (P.src & 3)));
      st_v4_last(P.lv8 + 16 * i, w[0], w[1], w[2], w[3]);
    }
  } else if ((reinterpret_cast<uintptr_t>(P.dist) & 15u) == 0) {
    int4* d4 = reinterpret_cast<int4*>(P.dist);
    const long long n4 = n >> 2;
    for (long long i = tid; i < n4; i += nth) {
      int4 v = make_int4(-1, -1, -1, -1);
      if ((long long)(P.src >> 2) == i) {
        int k = P.src & 3;
        if (k == 0) v.x = 0;
        if (k == 1) v.y = 0;
        if (k == 2) v.z = 0;
        if (k == 3) v.w = 0;
      }
      d4[i] = v;
    }
    for (long long i = (n4 << 2) + tid; i < n; i += nth) P.dist[i] = (i == P.src) ? 0 : -1;
  } else {
    for (long long i = tid; i < n; i += nth) P.dist[i] = (i == P.src) ? 0 : -1;
  }
  const int sw = P.src >> 5;
  for (long long w = tid; w < P.nw; w += nth) {
    unsigned x = __ldg(P.init_vis + BW(w, 4));
    if (w == sw) x |= 1u << (P.src & 31);
    P.vis[BW(w, 5)] = x;
  }
}

// dist[v] = level byte of v, or -1 where it is 255 (every vertex written).
// On a renumbered graph the byte of caller vertex v is at new_of[v]; a
// vertex of degree 0 (new id >= n_live) other than the source is unreached.
// Each thread takes kExpandBatch groups of four vertices at once (all loads
// issued before the first use), so that a thread has several stream loads and
// level-byte gathers in flight instead of one dependent chain per group.
constexpr int kExpandBatch = 4;

__device__ __noinline__ void expand_phase(const KParams& P) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long n = P.n;
  long long done = 0;
  if (P.new_of) {
    auto level_at = [&](int nv) -> int {
      const bool live = (long long)nv < P.n_live || nv == P.src;
      const int t = live ? (int)P.lv8[BV(nv, 6)] : 255;
      return t == 255 ? -1 : t;
    };
    if ((reinterpret_cast<uintptr_t>(P.dist) & 15u) == 0) {
      const long long n4 = n >> 2;
      const int4* m4 = reinterpret_cast<const int4*>(P.new_of);
      int4* d4 = reinterpret_cast<int4*>(P.dist);
      for (long long i0 = tid; i0 < n4; i0 += nth * kExpandBatch) {
        int4 a[kExpandBatch];
#pragma unroll
        for (int u = 0; u < kExpandBatch; ++u) {
          const long long i = i0 + u * nth;
          a[u] = i < n4 ? __ldcs(m4 + i) : make_int4(0, 0, 0, 0);
        }
        int4 r[kExpandBatch];
#pragma unroll
        for (int u = 0; u < kExpandBatch; ++u)
          r[u] = make_int4(level_at(a[u].x), level_at(a[u].y), level_at(a[u].z), level_at(a[u].w));
#pragma unroll
        for (int u = 0; u < kExpandBatch; ++u) {
          const long long i = i0 + u * nth;
          if (i < n4) __stcs(d4 + i, r[u]);
        }
      }
      done = n4 << 2;
    }
    for (long long i = done + tid; i < n; i += nth) P.dist[i] = level_at(P.new_of[BV(i, 7)]);
    return;
  }
  if ((reinterpret_cast<uintptr_t>(P.dist) & 15u) == 0) {
    const long long n4 = n >> 2;
    const unsigned* l4 = reinterpret_cast<const unsigned*>(P.lv8);
    int4* d4 = reinterpret_cast<int4*>(P.dist);
    for (long long i0 = tid; i0 < n4; i0 += nth * kExpandBatch) {
      unsigned b[kExpandBatch];
#pragma unroll
      for (int u = 0; u < kExpandBatch; ++u) {
        const long long i = i0 + u * nth;
        b[u] = i < n4 ? l4[i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kExpandBatch; ++u) {
        const long long i = i0 + u * nth;
        int x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int t = (int)((b[u] >> (8 * k)) & 0xffu);
          x[k] = t == 255 ? -1 : t;
        }
        if (i < n4) __stcs(d4 + i, make_int4(x[0], x[1], x[2], x[3]));
      }
    }
    done = n4 << 2;
  }
  for (long long i = done + tid; i < n; i += nth) {
    const int t = P.lv8[i];
    P.dist[i] = t == 255 ? -1 : t;
  }
}

// Level-0 frontier {src}: vertex queue, work items and counters of slot 0.
template <typename RP>
__device__ __noinline__ void seed_phase(const KParams& P) {
  const long long s = rp_at<RP>(P.rp, BRP(P.src, 8));
  const long long d = rp_at<RP>(P.rp, BRP((long long)P.src + 1, 9)) - s;
  Slot* sl = &P.ctrl->slot[0];
  P.qv0[0] = P.src;
  unsigned long long nsm = 0, nlg = 0;
  if (d > 0 && d < P.small_max) {
    P.it0[0] = pack_item(s, (int)d);
    nsm = 1;
  } else if (d >= P.small_max && (d + P.chunk - 1) / P.chunk > 32) {
    P.mg0[0].start = s;
    P.mg0[0].deg = d;
    P.mg0[0].base = 0;
    sl->mega = 1ull | ((unsigned long long)((d + P.chunk - 1) / P.chunk) << kMegaCountBits);
  } else if (d >= P.small_max) {
    for (long long c = 0; c * P.chunk < d; ++c) {
      long long len = d - c * P.chunk;
      if (len > P.chunk) len = P.chunk;
      P.it0[BIT(P.cap - 1 - nlg, 10)] = pack_item(s + c * P.chunk, (int)len);
      ++nlg;
    }
  }
  sl->items = nsm | (nlg << 32);
  sl->nv = 1;
  sl->mf = (unsigned long long)d;
}

// ---------------------------------------------------------------- top-down

// Warp-collective: append hub records (vertices needing more than 32 chunks).
// Lane-local candidates k with (mask >> k) & 1 get a record; one packed
// atomic per warp hands out record slots and chunk tickets in the same order.
__device__ __forceinline__ void append_hubs(const KParams& P, unsigned mask, const long long (&s)[4],
                                            const int (&d)[4], Slot* out, MegaRec* mgn) {
  int nrec = 0, nch = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((mask >> k) & 1u) {
      ++nrec;
      nch += (d[k] + P.chunk - 1) / P.chunk;
    }
  if (__ballot_sync(kFull, nrec != 0) == 0) return;
  const int r_incl = warp_incl_scan(nrec), c_incl = warp_incl_scan(nch);
  const int r_tot = __shfl_sync(kFull, r_incl, 31), c_tot = __shfl_sync(kFull, c_incl, 31);
  unsigned long long b = 0;
  if (lane_id() == 31)
    b = atomicAdd(&out->mega, (unsigned long long)r_tot | ((unsigned long long)c_tot << kMegaCountBits));
  b = __shfl_sync(kFull, b, 31);
  unsigned long long r = (b & ((1ull << kMegaCountBits) - 1)) + (unsigned long long)(r_incl - nrec);
  unsigned long long c = (b >> kMegaCountBits) + (unsigned long long)(c_incl - nch);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((mask >> k) & 1u) {
      const long long rr = BMG(r, 11);
      mgn[rr].start = s[k];
      mgn[rr].deg = d[k];
      mgn[rr].base = c;
      ++r;
      c += (unsigned long long)((d[k] + P.chunk - 1) / P.chunk);
    }
}

// Warp-collective: visit up to four neighbours per lane (c[k] < 0: none) at
// level L.  All four visited words are read before any is claimed, all claims
// (atomicOr on the bitmap word) are issued before any result is used, and the
// degrees of the claimed vertices are fetched together, so one lane keeps
// several memory requests in flight.  The lane that set a bit is the only
// writer of that vertex's dist (a plain store) and appends it to the next
// frontier: vertex queue and degree-binned work items, one set of atomics per
// warp.
template <typename RP>
__device__ __forceinline__ void td_visit4(const KParams& P, int L, bool direct, const int (&c)[4], Slot* out, int* qvn,
                                          unsigned long long* itn, MegaRec* mgn) {
  unsigned cur[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) cur[k] = c[k] >= 0 ? ld_relaxed_u32(P.vis + BW(c[k] >> 5, 12)) : kFull;
  unsigned old[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned bit = 1u << (c[k] & 31);
    old[k] = (c[k] >= 0 && !(cur[k] & bit)) ? atomicOr(P.vis + BW(c[k] >> 5, 13), bit) : kFull;
  }
  unsigned cl = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!(old[k] & (1u << (c[k] & 31)))) cl |= 1u << k;
  if (__ballot_sync(kFull, cl != 0) == 0) return;
  long long s[4];
  int d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s[k] = 0;
    d[k] = 0;
    if ((cl >> k) & 1u) {
      mark_level(P, direct, c[k], L);
      if (P.head) {
        const int4 h = __ldg(P.head + BV(c[k], 14));
        s[k] = h.z;
        d[k] = h.w;
      } else {
        s[k] = rp_at<RP>(P.rp, BRP(c[k], 15));
        d[k] = (int)(rp_at<RP>(P.rp, BRP((long long)c[k] + 1, 16)) - s[k]);
      }
    }
  }
  const int ncl = __popc(cl);
  int nsm = 0, nlg = 0;
  unsigned long long dsum = 0;
  unsigned hubs = 0;  // bit k: candidate k needs more than 32 chunks and gets a hub record
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if ((cl >> k) & 1u) {
      const int ni = (d[k] + P.chunk - 1) / P.chunk;
      if (d[k] > 0 && d[k] < P.small_max) ++nsm;
      else if (d[k] >= P.small_max && ni > 32) hubs |= 1u << k;
      else if (d[k] >= P.small_max) nlg += ni;
      dsum += (unsigned long long)d[k];
    }
  }
  const int q_incl = warp_incl_scan(ncl), sm_incl = warp_incl_scan(nsm), lg_incl = warp_incl_scan(nlg);
  const int q_tot = __shfl_sync(kFull, q_incl, 31), sm_tot = __shfl_sync(kFull, sm_incl, 31),
            lg_tot = __shfl_sync(kFull, lg_incl, 31);
  const unsigned long long dsum_tot = warp_sum_u64(dsum);
  unsigned long long b_items = 0, b_q = 0;
  if (lane_id() == 0) {
    b_items = atomicAdd(&out->items, (unsigned long long)sm_tot | ((unsigned long long)lg_tot << 32));
    b_q = atomicAdd(&out->nv, (unsigned long long)q_tot);
    atomicAdd(&out->mf, dsum_tot);
  }
  b_items = __shfl_sync(kFull, b_items, 0);
  b_q = __shfl_sync(kFull, b_q, 0);
  unsigned long long qi = b_q + (unsigned long long)(q_incl - ncl);
  unsigned long long si = (b_items & 0xffffffffull) + (unsigned long long)(sm_incl - nsm);
  unsigned long long li = (b_items >> 32) + (unsigned long long)(lg_incl - nlg);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!((cl >> k) & 1u)) continue;
    if (P.need_qv) qvn[BQ(qi++, 17)] = c[k];
    if (d[k] > 0 && d[k] < P.small_max) {
      itn[BIT(si++, 18)] = pack_item(s[k], d[k]);
    } else if (d[k] >= P.small_max && !((hubs >> k) & 1u)) {
      for (int o = 0; o < d[k]; o += P.chunk) {
        const int len = d[k] - o < P.chunk ? d[k] - o : P.chunk;
        itn[BIT(P.cap - 1 - (long long)(li++), 19)] = pack_item(s[k] + o, len);
      }
    }
  }
  append_hubs(P, hubs, s, d, out, mgn);
}

// Warp-collective: visit the entries [s, e) of one adjacency span, 128 per
// step through aligned 128-bit loads (four candidates per lane).
template <typename RP>
__device__ __forceinline__ void td_span(const KParams& P, int L, bool direct, long long s, long long e, Slot* out, int* qvn,
                                        unsigned long long* itn, MegaRec* mgn) {
  const unsigned lane = lane_id();
  for (long long base = s & ~3ll; base < e; base += 128) {
    const long long j = base + 4 * (long long)lane;
    int4 q = make_int4(-1, -1, -1, -1);
    if (j < e) q = ldg4_first(P.col + BCOL4(j, 20));
    const int c[4] = {(j >= s && j < e) ? q.x : -1, (j + 1 >= s && j + 1 < e) ? q.y : -1,
                      (j + 2 >= s && j + 2 < e) ? q.z : -1, (j + 3 >= s && j + 3 < e) ? q.w : -1};
    td_visit4<RP>(P, L, direct, c, out, qvn, itn, mgn);
  }
}

// Top-down level.  The level's work is one index space: groups of 32 small
// items, then large items (<= chunk entries each), then hub chunk tickets;
// warps take indices in block-major order (consecutive indices go to
// different blocks), so no warp holds work of two kinds while others idle.
template <typename RP, bool STATS>
__device__ void td_phase(const KParams& P, int L, bool direct, unsigned long long items_cur, unsigned long long mega_cur) {
  const unsigned long long nsmall = items_cur & 0xffffffffull, nlarge = items_cur >> 32;
  const unsigned long long* it = (L & 1) ? P.it1 : P.it0;
  unsigned long long* itn = (L & 1) ? P.it0 : P.it1;
  const MegaRec* mg = (L & 1) ? P.mg1 : P.mg0;
  MegaRec* mgn = (L & 1) ? P.mg0 : P.mg1;
  int* qvn = (L & 1) ? P.qv0 : P.qv1;
  Slot* out = &P.ctrl->slot[(L + 1) & 3];
  const unsigned lane = lane_id();
  const long long gw = (long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5);
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long ngroups = (long long)((nsmall + 31ull) / 32ull);
  const long long nrec = (long long)(mega_cur & ((1ull << kMegaCountBits) - 1));
  const long long nch = (long long)(mega_cur >> kMegaCountBits);
  const long long nwork = ngroups + (long long)nlarge + nch;
  Acc acc;
  for (long long u = gw; u < nwork; u += nwarps) {
    if (u < ngroups) {
      // 32 small items; their entries are dealt to the lanes through an
      // exclusive scan of the lengths, 128 per step (four per lane).
      const unsigned long long i = (unsigned long long)u * 32ull + lane;
      const unsigned long long item = i < nsmall ? it[BIT(i, 21)] : 0ull;
      const long long s = (long long)(item >> 16);
      const int len = (int)(item & 0xffffull);
      const int incl = warp_incl_scan(len);
      const int excl = incl - len;
      const int total = __shfl_sync(kFull, incl, 31);
      if (STATS) acc.edges += (unsigned long long)len;
      for (int base = 0; base < total; base += 128) {
        int c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = base + 32 * k + (int)lane;
          const int o = owner_of(excl, e);
          const long long so = __shfl_sync(kFull, s, o);
          const int exo = __shfl_sync(kFull, excl, o);
          c[k] = e < total ? __ldg(P.col + BCOL(so + (e - exo), 22)) : -1;
        }
        td_visit4<RP>(P, L, direct, c, out, qvn, itn, mgn);
      }
    } else if (u < ngroups + (long long)nlarge) {
      const unsigned long long item = it[BIT(P.cap - 1 - (u - ngroups), 23)];
      const long long s = (long long)(item >> 16);
      const int len = (int)(item & 0xffffull);
      if (STATS && lane == 0) acc.edges += (unsigned long long)len;
      td_span<RP>(P, L, direct, s, s + len, out, qvn, itn, mgn);
    } else {
      // Hub chunk ticket t belongs to the last record whose base is <= t (a
      // 32-way search over the records, which are ordered by base).
      const long long t = u - ngroups - (long long)nlarge;
      long long lo = 0, hi = nrec;
      while (hi - lo > 1) {
        const long long step = (hi - lo + 31) / 32;
        const long long idx = lo + (long long)lane * step;
        const bool ok = idx < hi && (long long)mg[BMG(idx, 24)].base <= t;
        const unsigned bm = __ballot_sync(kFull, ok);
        const long long k = 31 - __clz(bm);
        lo = lo + k * step;
        hi = lo + step < hi ? lo + step : hi;
      }
      const long long lr = BMG(lo, 25);
      const long long o = (t - (long long)mg[lr].base) * P.chunk;
      const long long hd = mg[lr].deg;
      const long long s = mg[lr].start + o;
      const long long e = s + (hd - o < P.chunk ? hd - o : P.chunk);
      if (STATS && lane == 0) acc.edges += (unsigned long long)(e - s);
      td_span<RP>(P, L, direct, s, e, out, qvn, itn, mgn);
    }
  }
  if (STATS) flush_acc<STATS>(P, L, acc, out, false);
}

// ---------------------------------------------------------------- bottom-up

#define in_frontier(front, u) ((((front)[BWF((u) >> 5, 26)]) >> ((u) & 31)) & 1u)

// Shared-memory staging of one warp in a bottom-up batch.
#ifndef GBFS_DRAIN_MIN
#define GBFS_DRAIN_MIN 32
#endif
constexpr int kBuU = 1;  // unvisited vertices per lane in a bottom-up round
constexpr int kDrainMin = GBFS_DRAIN_MIN;  // deferred scans that trigger a drain within a batch
constexpr int kPendCap = 32 * kBuU + kDrainMin - 1;  // deferred long scans per warp
static_assert(kDrainMin <= 32, "a drain of one group leaves fewer than 32 scans behind");
constexpr int kNBuf = 3;  // ring slots of head records in flight
struct BuWarpSmem {
  int4 hbuf[kNBuf][32 * kBuU];   // head records of the rounds in flight (lane-private slots)
  int vbuf[kNBuf][32 * kBuU];    // their vertices
  unsigned next[32];             // new-frontier bits of the batch's 32 words
  long long pstart[kPendCap];    // deferred scan: next entry to examine
  int plen[kPendCap];            // entries left
  int pv[kPendCap];              // vertex
  int pd[kPendCap];              // its degree
  int pex[kPendCap];             // entries examined so far (statistics)
  int npend;
};

__device__ __forceinline__ void bu_mark_found(const KParams& P, int L, bool direct, BuWarpSmem& sm, long long w0, int v, int d,
                                              Acc& acc) {
  atomicOr(&sm.next[(int)((long long)v / 32 - w0)], 1u << (v & 31));
  mark_level(P, direct, v, L);
  acc.found += 1;
  acc.mf += (unsigned long long)d;
}

// Warp-collective: finish this warp's deferred scans.  The remaining
// adjacency ranges are scanned as one concatenation, four entries per lane per
// step (four column loads, then four frontier probes, in flight together); a
// vertex's remaining entries are skipped once it has found a parent.  Ranges
// longer than bu_warp_min are scanned one at a time by the whole warp.
template <bool STATS>
__device__ void bu_drain(const KParams& P, int L, bool direct, const unsigned* front, BuWarpSmem& sm, long long w0, Acc& acc,
                         bool one_group = false) {
  const unsigned lane = lane_id();
  __syncwarp();
  const int np_all = sm.npend;
  // one_group: only the first 32 are scanned (a full group of lanes); the
  // rest move to the front of the queue and wait for the next drain.
  const int np = one_group && np_all > 32 ? 32 : np_all;
  for (int g0 = 0; g0 < np; g0 += 32) {
    const int j = g0 + (int)lane;
    const bool have = j < np;
    long long ps = have ? sm.pstart[j] : 0;
    int pl = have ? sm.plen[j] : 0;
    const int pv = have ? sm.pv[j] : 0;
    const int pdeg = have ? sm.pd[j] : 0;
    int ex = have ? sm.pex[j] : 0;
    // Each lane first continues its own vertex for up to bu_thread_max entries,
    // two aligned 128-bit groups (up to eight probes in flight) at a time; the
    // first group masks the entries before ps.
    bool tfound = false;
    for (int done = 0; pl > 0 && done < P.bu_thread_max;) {
      const long long a = ps & ~3ll;
      const int off = (int)(ps - a);
      const int4 q0 = ldg4_first(P.col + BCOL4(a, 27));
      const int4 q1 = pl > 4 - off ? ldg4_first(P.col + BCOL4(a + 4, 28)) : make_int4(0, 0, 0, 0);
      const int c8[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      bool h[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) h[t] = t >= off && t - off < pl && in_frontier(front, c8[t]);
      int ft = -1;
#pragma unroll
      for (int t = 7; t >= 0; --t)
        if (h[t]) ft = t;
      if (ft >= 0) {
        tfound = true;
        ex += ft - off + 1;
        pl = 0;
        break;
      }
      const int step = pl < 8 - off ? pl : 8 - off;
      ex += step;
      pl -= step;
      ps += step;
      done += step;
    }
    const bool heavy = pl > P.bu_warp_min;
    const int len = heavy ? 0 : pl;
    const int incl = warp_incl_scan(len);
    const int excl = incl - len;
    const int total = __shfl_sync(kFull, incl, 31);
    unsigned pend = __ballot_sync(kFull, len > 0);
    unsigned fnd = 0;
    int last = (int)__reduce_max_sync(kFull, (unsigned)(((pend >> lane) & 1u) ? incl : 0));
    for (int base = 0; base < last; base += 128) {
      int o[4], u[4];
      bool want[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ei = base + 32 * k + (int)lane;
        o[k] = owner_of(excl, ei);
        const long long so = __shfl_sync(kFull, ps, o[k]);
        const int exo = __shfl_sync(kFull, excl, o[k]);
        want[k] = ei < total && ((pend >> o[k]) & 1u);
        u[k] = want[k] ? __ldg(P.col + BCOL(so + (ei - exo), 29)) : 0;
      }
      bool hk[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned fw = want[k] ? front[BWF(u[k] >> 5, 30)] : 0u;
        hk[k] = (fw >> (u[k] & 31)) & 1u;
      }
      unsigned mine = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (hk[k]) mine |= 1u << o[k];
      const unsigned hm = __reduce_or_sync(kFull, mine) & pend;
      if (STATS && hm) {
        unsigned t = hm;
        while (t) {
          const int oo = __ffs(t) - 1;
          t &= t - 1;
          unsigned best = 0xffffffffu;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (hk[k] && o[k] == oo) best = min(best, (unsigned)(base + 32 * k + (int)lane));
          const unsigned mn = __reduce_min_sync(kFull, best);
          if ((int)lane == oo) ex += (int)mn - excl + 1;
        }
      }
      pend &= ~hm;
      fnd |= hm;
      if (!pend) break;
      last = (int)__reduce_max_sync(kFull, (unsigned)(((pend >> lane) & 1u) ? incl : 0));
    }
    bool found = tfound || ((fnd >> lane) & 1u);
    if (STATS && len > 0 && !((fnd >> lane) & 1u)) ex += len;
    unsigned hv = __ballot_sync(kFull, heavy);
    while (hv) {
      const int h = __ffs(hv) - 1;
      hv &= hv - 1;
      const long long hs = __shfl_sync(kFull, ps, h);
      const long long he = hs + __shfl_sync(kFull, pl, h);
      bool hf = false;
      long long hx = he - hs;
      // 256 entries per step: two aligned 128-bit loads and eight probes in
      // flight per lane; the first hit in list order is the warp minimum.
      for (long long a = hs & ~3ll; a < he; a += 256) {
        const long long j0 = a + 8 * (long long)lane;
        int4 q0 = make_int4(0, 0, 0, 0), q1 = make_int4(0, 0, 0, 0);
        if (j0 < he) q0 = ldg4_first(P.col + BCOL4(j0, 31));
        if (j0 + 4 < he) q1 = ldg4_first(P.col + BCOL4(j0 + 4, 32));
        const int c8[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        bool h8[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) h8[t] = j0 + t >= hs && j0 + t < he && in_frontier(front, c8[t]);
        unsigned first = 0xffffffffu;
#pragma unroll
        for (int t = 7; t >= 0; --t)
          if (h8[t]) first = (unsigned)(j0 + t - hs);
        const unsigned mn = __reduce_min_sync(kFull, first);
        if (mn != 0xffffffffu) {
          hf = true;
          hx = (long long)mn + 1;
          break;
        }
      }
      if ((int)lane == h) {
        found = hf;
        ex += (int)hx;
      }
    }
    if (found) bu_mark_found(P, L, direct, sm, w0, pv, pdeg, acc);
    if (STATS && have) acc.edges += (unsigned long long)ex;
  }
  __syncwarp();
  const int rest = np_all - np;  // < 32: records np .. np_all-1 move to 0 .. rest-1 (no overlap)
  if ((int)lane < rest) {
    sm.pstart[lane] = sm.pstart[np + lane];
    sm.plen[lane] = sm.plen[np + lane];
    sm.pv[lane] = sm.pv[np + lane];
    sm.pd[lane] = sm.pd[np + lane];
    sm.pex[lane] = sm.pex[np + lane];
  }
  if (lane == 0) sm.npend = rest;
  __syncwarp();
}

// Warp-collective: the unvisited vertices r0 + 32k + lane (k < kBuU) of a batch
// whose 32 words have active masks `act` (one per lane) and exclusive prefix
// counts `excl`; -1 past the end.
__device__ __forceinline__ void round_vertices(unsigned act, int excl, int total, long long w0, int r0,
                                               int (&v)[kBuU]) {
  const unsigned lane = lane_id();
  if (total > 32 * 32 - 32) {
    // Nearly every vertex of the batch is unvisited: packing would give the
    // same 32 rounds, so round r takes word r as it is (lane i = bit i; -1
    // where the vertex is visited) and skips the search for each lane's vertex.
#pragma unroll
    for (int k = 0; k < kBuU; ++k) {
      const int wi = r0 / 32 + k;
      const unsigned aw = __shfl_sync(kFull, act, wi & 31);
      v[k] = (wi < 32 && ((aw >> lane) & 1u)) ? (int)((w0 + wi) * 32 + (long long)lane) : -1;
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < kBuU; ++k) {
    const int kk = r0 + 32 * k + (int)lane;
    const int wo = owner_of(excl, kk);
    const unsigned aw = __shfl_sync(kFull, act, wo);
    const int ew = __shfl_sync(kFull, excl, wo);
    v[k] = -1;
    if (kk < total) v[k] = (int)((w0 + wo) * 32 + (long long)nth_set_bit(aw, kk - ew));
  }
}

#ifndef GBFS_BU_HEAD_DEPTH
#define GBFS_BU_HEAD_DEPTH 2
#endif
constexpr int kHeadDepth = GBFS_BU_HEAD_DEPTH;  // rounds of head records in flight (2 or 3)

// Warp-collective: the rounds of a batch on the head table.  A dense batch
// (nearly every vertex unvisited) takes word r as round r, lane i its bit i;
// otherwise the unvisited vertices are packed onto the lanes
// (round_vertices).  An idle lane (-1) gets a zero-filled head record: degree
// 0, which no unvisited vertex has (degree-0 vertices are visited from the
// start).  Pipeline: round r + kHeadDepth's records are requested, round
// r + 1's frontier words are loaded (its record and vertex are then kept in
// registers, which frees the ring slot), round r is decided.  Deferred scans
// are drained here once kDrainMin are pending; the rest are left in sm.npend.
template <bool STATS>
__device__ __forceinline__ void bu_head_batch(const KParams& P, int L, bool direct, const unsigned* front,
                                              long long w0, unsigned act, int excl, int total, BuWarpSmem& sm,
                                              Acc& acc) {
  static_assert(kNBuf == 3 && kBuU == 1 && (kHeadDepth == 2 || kHeadDepth == 3), "head pipeline layout");
  const unsigned lane = lane_id();
  const bool dense = total > 32 * 32 - 32;
  const int nrounds = dense ? 32 : (total + 31) / 32;
  auto issue = [&](int r, int b) {
    int v;
    if (dense) {
      v = (__shfl_sync(kFull, act, r) >> lane) & 1u ? (int)((w0 + r) * 32 + (long long)lane) : -1;
    } else {
      int vv[1];
      round_vertices(act, excl, total, w0, 32 * r, vv);
      v = vv[0];
    }
    sm.vbuf[b][lane] = v;
    cp_async16_first(&sm.hbuf[b][lane], v >= 0 ? P.head + BV(v, 33) : P.head, v >= 0 ? 16 : 0);
  };
  auto probe = [&](int b, int4& h, int& v, unsigned& x0, unsigned& x1) {
    h = sm.hbuf[b][lane];
    v = sm.vbuf[b][lane];
    x0 = h.w > 0 ? front[BWF(h.x >> 5, 34)] : 0u;  // a vertex of degree > 0 has a first neighbour
    x1 = h.w > 0 && h.y >= 0 ? front[BWF(h.y >> 5, 35)] : 0u;
  };
#pragma unroll
  for (int r = 0; r < kHeadDepth; ++r) {
    if (r < nrounds) issue(r, r);
    cp_async_commit();
  }
  int4 h = make_int4(0, 0, 0, 0);
  int v = -1;
  unsigned p0 = 0, p1 = 0;
  if (nrounds > 0) {
    cp_async_wait<kHeadDepth - 1>();
    probe(0, h, v, p0, p1);
  }
  int np = 0;  // deferred scans pending (sm.npend is written before a drain)
  int bi = kHeadDepth % 3, bp = 1;  // ring slots of the round to request and of the round to probe
#pragma unroll 1
  for (int r = 0; r < nrounds; ++r) {
    if (r + kHeadDepth < nrounds) issue(r + kHeadDepth, bi);
    cp_async_commit();
    bi = bi == 2 ? 0 : bi + 1;
    int4 hn = make_int4(0, 0, 0, 0);
    int vn = -1;
    unsigned n0 = 0, n1 = 0;
    if (r + 1 < nrounds) {
      cp_async_wait<kHeadDepth - 1>();
      probe(bp, hn, vn, n0, n1);
    }
    bp = bp == 2 ? 0 : bp + 1;
    // Decide round r: p0/p1 are 0 for idle lanes and a missing second
    // neighbour (id -1), so no bit of them is found there.
    const int d = h.w;
    const unsigned f0 = (p0 >> (h.x & 31)) & 1u, f1 = (p1 >> (h.y & 31)) & 1u;
    const bool fnd = (f0 | f1) != 0u;
    const bool enq = !fnd && d > 2;
    if (dense) {
      const unsigned fm = __ballot_sync(kFull, fnd);
      if (lane == 0) sm.next[r] = fm;  // word r is this round's alone until the drains
    } else if (fnd) {
      atomicOr(&sm.next[(int)((long long)v / 32 - w0)], 1u << (v & 31));
    }
    if (fnd) {
      mark_level(P, direct, v, L);
      acc.found += 1;
      acc.mf += (unsigned long long)d;
    }
    if (STATS) {
      if (fnd) acc.edges += f0 ? 1ull : 2ull;
      else if (!enq) acc.edges += (unsigned long long)d;
    }
    const unsigned em = __ballot_sync(kFull, enq);
    if (enq) {
      const int slot = np + __popc(em & lanemask_lt());
      sm.pstart[slot] = (long long)h.z + 2;
      sm.plen[slot] = d - 2;
      sm.pv[slot] = v;
      sm.pd[slot] = d;
      sm.pex[slot] = 2;
    }
    np += __popc(em);
    h = hn;
    v = vn;
    p0 = n0;
    p1 = n1;
    if (np >= kDrainMin) {
      __syncwarp();
      if (lane == 0) sm.npend = np;
      bu_drain<STATS>(P, L, direct, front, sm, w0, acc, true);
      np = sm.npend;
    }
  }
  __syncwarp();
  if (lane == 0) sm.npend = np;
  __syncwarp();
}

// One batch of 32 bitmap words (1024 vertices) of a bottom-up level, by one
// warp.  Each unvisited vertex looks for a frontier neighbour among its first
// entries - the two of its head record (bu_head_batch), else the aligned four
// of one 128-bit load - and, if it has more entries, becomes a deferred scan,
// drained by the warp 32 at a time (bu_drain).  New-frontier bits are gathered
// in shared memory and stored once per word, together with the updated
// visited word.
template <typename RP, bool STATS>
__device__ void bu_batch(const KParams& P, int L, bool direct, const unsigned* front, unsigned* next, long long w0,
                         unsigned vw, BuWarpSmem& sm, Acc& acc) {
  const unsigned lane = lane_id();
  const long long w = w0 + lane;
  const unsigned act = ~vw;  // padding bits past n are set in vis, so act holds vertices < n only
  sm.next[lane] = 0u;
  const int cnt = __popc(act);
  const int incl = warp_incl_scan(cnt);
  const int excl = incl - cnt;
  const int total = __shfl_sync(kFull, incl, 31);
  if (STATS) acc.unvisited += (unsigned long long)cnt;
  __syncwarp();
  if (P.head) {
    bu_head_batch<STATS>(P, L, direct, front, w0, act, excl, total, sm, acc);
  } else {
    // Row pointers and the aligned first four entries, one vertex per lane per round.
    const int nrounds = (total + 31) / 32;
    for (int r = 0; r < nrounds; ++r) {
      int v[kBuU];
      round_vertices(act, excl, total, w0, 32 * r, v);
      long long s[kBuU], e[kBuU];
#pragma unroll
      for (int k = 0; k < kBuU; ++k) {
        s[k] = 0;
        e[k] = 0;
        if (v[k] >= 0) {
          s[k] = rp_at<RP>(P.rp, BRP(v[k], 36));
          e[k] = rp_at<RP>(P.rp, BRP((long long)v[k] + 1, 37));
        }
      }
      int4 q[kBuU];
#pragma unroll
      for (int k = 0; k < kBuU; ++k) {
        q[k] = make_int4(0, 0, 0, 0);
        if (e[k] > s[k]) q[k] = __ldg(reinterpret_cast<const int4*>(P.col + BCOL4(s[k] & ~3ll, 38)));
      }
      unsigned f[kBuU][4];
#pragma unroll
      for (int k = 0; k < kBuU; ++k) {
        const long long a0 = s[k] & ~3ll;
        const int c4[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const bool ok = a0 + t >= s[k] && a0 + t < e[k];
          f[k][t] = ok ? in_frontier(front, c4[t]) : 0u;
        }
      }
#pragma unroll
      for (int k = 0; k < kBuU; ++k) {
        if (v[k] < 0) continue;
        const long long a0 = s[k] & ~3ll;
        long long hit = -1;
#pragma unroll
        for (int t = 3; t >= 0; --t)
          if (f[k][t]) hit = a0 + t;
        const int d = (int)(e[k] - s[k]);
        const long long rest = a0 + 4;
        if (hit >= 0) {
          bu_mark_found(P, L, direct, sm, w0, v[k], d, acc);
          if (STATS) acc.edges += (unsigned long long)(hit - s[k] + 1);
        } else if (rest < e[k]) {
          const int slot = atomicAdd(&sm.npend, 1);
          sm.pstart[slot] = rest;
          sm.plen[slot] = (int)(e[k] - rest);
          sm.pv[slot] = v[k];
          sm.pd[slot] = d;
          sm.pex[slot] = (int)(rest - s[k]);
        } else if (STATS) {
          acc.edges += (unsigned long long)d;
        }
      }
      __syncwarp();
      if (sm.npend >= kDrainMin) bu_drain<STATS>(P, L, direct, front, sm, w0, acc, true);
    }
  }
  __syncwarp();
  if (sm.npend > 0) bu_drain<STATS>(P, L, direct, front, sm, w0, acc);
  __syncwarp();
  const unsigned nx = sm.next[lane];
  if (w < P.nw) {
    next[BW(w, 39)] = nx;
    if (nx) P.vis[BW(w, 40)] = vw | nx;  // this warp is the only writer of its batch's words
  }
  __syncwarp();
}

// Bitmap words that can hold a vertex of degree > 0: on a renumbered copy the
// words of ids below n_live, else every word.  Degree-0 vertices are set in the
// visited mask from the start and are no vertex's neighbour, so bottom-up
// levels and conversions never need the words past these: the frontier bits
// there are neither written nor read.
__device__ __forceinline__ long long live_words(const KParams& P) {
  const long long lw = P.new_of ? (P.n_live + 31) >> 5 : (long long)P.nw;
  return lw < (long long)P.nw ? lw : (long long)P.nw;
}

// Visited word of lane `lane` in the batch starting at word w0 (all-set past the end).
__device__ __forceinline__ unsigned batch_word(const KParams& P, long long w0) {
  const long long w = w0 + lane_id();
  return w < P.nw ? P.vis[BW(w, 48)] : kFull;
}

// Bottom-up level, over the live words.  Batches of 32 words go to warps
// statically (interleaved: bu_chunk = 0, or a level with fewer unvisited
// vertices than bitmap words, where most batches are empty and a shared cursor
// would only add atomics) or bu_chunk batches at a time from a shared cursor.  A warp requests its next
// grab (and loads the visited words of its next batch) before it processes
// the current batch, so neither latency sits between two batches.
template <typename RP, bool STATS>
__device__ void bu_phase(const KParams& P, int L, bool direct, const unsigned* front, unsigned* next, bool dyn) {
  extern __shared__ unsigned long long g_dyn_smem[];  // blockDim.x / 32 BuWarpSmem records
  BuWarpSmem& sm = reinterpret_cast<BuWarpSmem*>(g_dyn_smem)[threadIdx.x >> 5];
  Slot* out = &P.ctrl->slot[(L + 1) & 3];
  const unsigned lane = lane_id();
  const long long nbatch = (live_words(P) + 31) / 32;
  if (lane == 0) sm.npend = 0;
  __syncwarp();
  Acc acc;
  if (P.bu_chunk <= 0 || !dyn) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long b = gw;
    unsigned vw = b < nbatch ? batch_word(P, b * 32) : kFull;
    while (b < nbatch) {
      const long long bn = b + nwarps;
      const unsigned vwn = bn < nbatch ? batch_word(P, bn * 32) : kFull;
      bu_batch<RP, STATS>(P, L, direct, front, next, b * 32, vw, sm, acc);
      b = bn;
      vw = vwn;
    }
  } else {
    unsigned long long* cur = &P.ctrl->slot[L & 3].cursor;
    const long long ch = P.bu_chunk;
    // Grabs of ch consecutive batches; `g1` is requested one grab ahead.
    long long g0 = 0, g1 = 0;
    if (lane == 0) {
      g0 = (long long)atomicAdd(cur, (unsigned long long)ch);
      g1 = (long long)atomicAdd(cur, (unsigned long long)ch);
    }
    g0 = __shfl_sync(kFull, g0, 0);
    g1 = __shfl_sync(kFull, g1, 0);
    unsigned vw = g0 < nbatch ? batch_word(P, g0 * 32) : kFull;
    while (g0 < nbatch) {
      long long g2 = 0;
      if (lane == 0) g2 = (long long)atomicAdd(cur, (unsigned long long)ch);
      const long long gend = g0 + ch < nbatch ? g0 + ch : nbatch;
      for (long long b = g0; b < gend; ++b) {
        // Next batch: the following one of this grab, else the first of the next grab.
        const long long bn = b + 1 < gend ? b + 1 : g1;
        const unsigned vwn = bn < nbatch ? batch_word(P, bn * 32) : kFull;
        bu_batch<RP, STATS>(P, L, direct, front, next, b * 32, vw, sm, acc);
        vw = vwn;
      }
      g0 = g1;
      g1 = __shfl_sync(kFull, g2, 0);
    }
  }
  flush_acc<STATS>(P, L, acc, out, true);
}

// ---------------------------------------------------------------- conversions

__device__ void zero_words(unsigned* p, long long nw) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long w = tid; w < nw; w += nth) p[w] = 0u;
}

// Queue -> bitmap: set the bit of every vertex of F (nv entries of qv).
__device__ void scatter_phase(const KParams& P, const int* qv, long long nv, unsigned* bm) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < nv; i += nth) {
    const int v = qv[BQ(i, 41)];
    atomicOr(bm + BW(v >> 5, 42), 1u << (v & 31));
  }
}

// Bottom-up -> top-down: the work items of F_{L+1} from its bitmap `fbm` (the
// new-frontier bitmap of the last bottom-up level).  A warp scans 256 words per
// step (eight per lane) and packs their set bits onto the lanes, one vertex per
// lane per round, so a sparse frontier costs one round (and one atomic) per
// 8192 vertices scanned.
template <typename RP>
__device__ __noinline__ void convert_phase(const KParams& P, int L, const unsigned* fbm) {
  const int Ln = L + 1;
  unsigned long long* itn = (Ln & 1) ? P.it1 : P.it0;
  Slot* out = &P.ctrl->slot[Ln & 3];
  const unsigned lane = lane_id();
  const unsigned lt = lanemask_lt();
  const long long gw = (long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5);
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  constexpr int kW = 8;  // bitmap words per lane: 8192 vertices per warp step (frontiers here are sparse)
  const long long nwl = live_words(P);
  const long long nstep = (nwl + 32 * kW - 1) / (32 * kW);
  for (long long bt = gw; bt < nstep; bt += nwarps) {
    const long long w0 = bt * 32 * kW + (long long)lane * kW;
    unsigned x[kW];
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < kW; ++j) {
      x[j] = w0 + j < nwl ? fbm[w0 + j] : 0u;
      cnt += __popc(x[j]);
    }
    const int incl = warp_incl_scan(cnt);
    const int excl = incl - cnt;
    const int total = __shfl_sync(kFull, incl, 31);
    for (int r0 = 0; r0 < total; r0 += 32) {
      const int kk = r0 + (int)lane;
      const int wo = owner_of(excl, kk);
      int r = kk - __shfl_sync(kFull, excl, wo);
      long long vw = -1;  // word of this lane's vertex
      unsigned aw = 0;
#pragma unroll
      for (int j = 0; j < kW; ++j) {
        const unsigned xj = __shfl_sync(kFull, x[j], wo);
        const int c = __popc(xj);
        if (kk < total && vw < 0) {
          if (r < c) {
            vw = bt * 32 * kW + (long long)wo * kW + j;
            aw = xj;
          } else {
            r -= c;
          }
        }
      }
      long long s = 0;
      int d = 0;
      if (vw >= 0) {
        const int v = (int)(vw * 32 + (long long)nth_set_bit(aw, r));
        if (P.head) {
          const int4 h = __ldg(P.head + BV(v, 43));
          s = h.z;
          d = h.w;
        } else {
          s = rp_at<RP>(P.rp, BRP(v, 44));
          d = (int)(rp_at<RP>(P.rp, BRP((long long)v + 1, 45)) - s);
        }
      }
      const int ni = (d + P.chunk - 1) / P.chunk;
      const bool hub = d >= P.small_max && ni > 32;
      const int nsm = (d > 0 && d < P.small_max) ? 1 : 0;
      const int nlg = (d >= P.small_max && !hub) ? ni : 0;
      {
        const long long hs[4] = {s, 0, 0, 0};
        const int hd[4] = {d, 0, 0, 0};
        append_hubs(P, hub ? 1u : 0u, hs, hd, out, (Ln & 1) ? P.mg1 : P.mg0);
      }
      const unsigned smask = __ballot_sync(kFull, nsm);
      const int lg_incl = warp_incl_scan(nlg);
      const int lg_tot = __shfl_sync(kFull, lg_incl, 31);
      unsigned long long b_items = 0;
      if (lane == 0)
        b_items = atomicAdd(&out->items, (unsigned long long)__popc(smask) | ((unsigned long long)lg_tot << 32));
      b_items = __shfl_sync(kFull, b_items, 0);
      if (nsm) itn[BIT((b_items & 0xffffffffull) + __popc(smask & lt), 46)] = pack_item(s, d);
      if (nlg) {
        unsigned long long bb = (b_items >> 32) + (unsigned long long)(lg_incl - nlg);
        for (int o = 0; o < d; o += P.chunk) {
          const int len = d - o < P.chunk ? d - o : P.chunk;
          itn[BIT(P.cap - 1 - (long long)(bb++), 47)] = pack_item(s + o, len);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- level loop

// Dynamic batch assignment for a bottom-up level only while at least one
// unvisited vertex of degree > 0 per bitmap word remains.
__host__ __device__ inline bool bu_dynamic(const KParams& P, long long reached) {
  return P.n_live - reached >= (long long)P.nw;
}

struct LoopState {
  int L = 0;
  bool td = true;
  int fb = 0;                   // bitmap index holding the frontier in bottom-up mode
  long long nf_cur = 1;         // |F_L|
  long long edges_visited = 0;  // degrees of all visited vertices
  long long reached = 1;
};

template <bool STATS>
__device__ void record_level(const KParams& P, const LoopState& st, long long found, int converted,
                             unsigned long long& t_mark) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && (STATS || P.lst)) {
    const unsigned long long t = globaltimer_ns();
    if (P.lst && st.L < P.lst_cap) {
      P.lst[st.L].direction = st.td ? 0 : 1;
      P.lst[st.L].converted = converted;
      P.lst[st.L].frontier = st.nf_cur;
      P.lst[st.L].found = found;
      P.lst[st.L].ns = (long long)(t - t_mark);
    }
    t_mark = t;
    if (STATS && st.td) {
      P.ctrl->td_frontier += (unsigned long long)st.nf_cur;
    } else if (STATS) {
      P.ctrl->bu_found += (unsigned long long)found;
    }
  }
}

template <typename RP, bool STATS>
__global__ void __launch_bounds__(1024) bfs_persistent_kernel(KParams P) {
  // Loop state lives in shared memory: thread 0 of every block reads the level
  // counters after the barrier and decides (all blocks decide identically),
  // so the phases run with no loop state held in registers.
  struct LoopShared {
    LoopState st;
    unsigned long long items, mega, t_mark;
    long long nf;
    int action;  // 0 next level, 1 top-down -> bottom-up conversion, 2 bottom-up -> top-down, 3 done
    int converted, conversions, tdl, bul;
    int direct;  // levels are written to dist directly (no level bytes, or past level 254)
  };
  __shared__ LoopShared S;
  unsigned epoch = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl->t_begin = globaltimer_ns();
  init_phase<RP>(P);
  if (blockIdx.x == 0 && threadIdx.x == 0) seed_phase<RP>(P);
  if (!grid_barrier(P, epoch)) return;
  if (threadIdx.x == 0) {
    S.st = LoopState();
    S.st.edges_visited = (long long)ld_relaxed_u64(&P.ctrl->slot[0].mf);
    S.items = ld_relaxed_u64(&P.ctrl->slot[0].items);
    S.mega = ld_relaxed_u64(&P.ctrl->slot[0].mega);
    S.t_mark = globaltimer_ns();
    if (blockIdx.x == 0) P.ctrl->t_levels = S.t_mark;
    S.converted = S.conversions = S.tdl = S.bul = 0;
    S.direct = P.lv8 == nullptr;
  }
  __syncthreads();
  for (;;) {
    const int L = S.st.L;
    if (!S.direct && L >= 254) {
      // Level bytes hold levels up to 254: from here on dist is written directly.
      expand_phase(P);
      if (!grid_barrier(P, epoch)) return;
      if (threadIdx.x == 0) S.direct = 1;
      __syncthreads();
    }
    const bool direct = S.direct != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      Slot* z = &P.ctrl->slot[(L + 2) & 3];
      z->items = 0; z->nv = 0; z->mf = 0; z->nq = 0; z->cursor = 0; z->mega = 0;
    }
    if (S.st.td) {
      td_phase<RP, STATS>(P, L, direct, S.items, S.mega);
    } else {
      const int fb = S.st.fb;
      bu_phase<RP, STATS>(P, L, direct, fb ? P.bm1 : P.bm0, fb ? P.bm0 : P.bm1, bu_dynamic(P, S.st.reached));
    }
    if (!grid_barrier(P, epoch)) return;
    if (threadIdx.x == 0) {
      LoopState st = S.st;
      if (st.td) ++S.tdl; else ++S.bul;
      Slot* nx = &P.ctrl->slot[(L + 1) & 3];
      const long long nf = (long long)ld_relaxed_u64(&nx->nv);
      const long long mf = (long long)ld_relaxed_u64(&nx->mf);
      unsigned long long t_mark = S.t_mark;
      record_level<STATS>(P, st, nf, S.converted, t_mark);
      S.t_mark = t_mark;
      int action = 3;
      if (nf != 0) {
        st.edges_visited += mf;
        st.reached += nf;
        const bool ntd = next_is_top_down(P.policy, P.alpha, P.beta, P.tau_inv, P.script, L + 1, st.td, nf,
                                          st.nf_cur, mf, P.m - st.edges_visited, P.n);
        action = 0;
        if (st.td && !ntd) {
          action = 1;
          st.fb = 0;
        } else if (!st.td && ntd) {
          action = 2;
        } else if (!st.td && !ntd) {
          st.fb ^= 1;
        }
        S.converted = action == 1 || action == 2;
        if (S.converted) {
          ++S.conversions;
          if (STATS && blockIdx.x == 0) P.ctrl->conv_frontier += (unsigned long long)nf;
        }
        if (ntd && action == 0) {  // after a conversion they are read once it has run
          S.items = ld_relaxed_u64(&nx->items);
          S.mega = ld_relaxed_u64(&nx->mega);
        }
        st.td = ntd;
        st.nf_cur = nf;
        st.L = L + 1;
      }
      S.st = st;
      S.nf = nf;
      S.action = action;
    }
    __syncthreads();
    const int action = S.action;
    if (action == 3) {
      if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl->t_levels_end = globaltimer_ns();
      if (!direct) expand_phase(P);
      if (blockIdx.x == 0) {
        __syncthreads();
        if (threadIdx.x == 0) P.ctrl->t_end = globaltimer_ns();
      }
      break;
    }
    const long long nf = S.nf;
    if (action == 1) {
      // top-down -> bottom-up: the new frontier's vertex queue becomes bitmap bm0
      zero_words(P.bm0, P.nw);
      if (!grid_barrier(P, epoch)) return;
      scatter_phase(P, ((L + 1) & 1) ? P.qv1 : P.qv0, nf, P.bm0);
      if (!grid_barrier(P, epoch)) return;
    } else if (action == 2) {
      // bottom-up -> top-down: work items from the new frontier's bitmap
      convert_phase<RP>(P, L, S.st.fb ? P.bm0 : P.bm1);
      if (!grid_barrier(P, epoch)) return;
      if (threadIdx.x == 0) {
        const Slot* nx = &P.ctrl->slot[(L + 1) & 3];
        S.items = ld_relaxed_u64(&nx->items);
        S.mega = ld_relaxed_u64(&nx->mega);
      }
      __syncthreads();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.ctrl->levels = S.st.L + 1;
    P.ctrl->td_levels = S.tdl;
    P.ctrl->bu_levels = S.bul;
    P.ctrl->conversions = S.conversions;
    P.ctrl->reached = (unsigned long long)S.st.reached;
    P.ctrl->edges_reached = (unsigned long long)S.st.edges_visited;
  }
}

// ---- per-phase kernels (BFS_LAUNCH_PER_LEVEL) ----

template <typename RP>
__global__ void __launch_bounds__(1024) k_init_seed(KParams P) {
  init_phase<RP>(P);
  if (blockIdx.x == 0 && threadIdx.x == 0) seed_phase<RP>(P);
}

#ifndef GBFS_KLEVEL_THREADS
#define GBFS_KLEVEL_THREADS 1024
#define GBFS_KLEVEL_MINB 1
#endif
template <typename RP, bool STATS>
__global__ void __launch_bounds__(GBFS_KLEVEL_THREADS, GBFS_KLEVEL_MINB) k_level(KParams P, int L, int direct, int td, int fb,
                                                unsigned long long items, unsigned long long mega,
                                                long long reached) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Slot* z = &P.ctrl->slot[(L + 2) & 3];
    z->items = 0; z->nv = 0; z->mf = 0; z->nq = 0; z->cursor = 0; z->mega = 0;
  }
  if (td) {
    td_phase<RP, STATS>(P, L, direct != 0, items, mega);
  } else {
    bu_phase<RP, STATS>(P, L, direct != 0, fb ? P.bm1 : P.bm0, fb ? P.bm0 : P.bm1, bu_dynamic(P, reached));
  }
}

__global__ void __launch_bounds__(1024) k_zero_words(unsigned* p, long long nw) { zero_words(p, nw); }

__global__ void __launch_bounds__(1024) k_expand(KParams P) { expand_phase(P); }

__global__ void __launch_bounds__(1024) k_scatter(KParams P, const int* qv, long long nv, unsigned* bm) {
  scatter_phase(P, qv, nv, bm);
}

template <typename RP>
__global__ void __launch_bounds__(1024) k_convert(KParams P, int L, const unsigned* fbm) {
  convert_phase<RP>(P, L, fbm);
}

template <typename RP, bool STATS>
struct Kernels {
  static void* persistent() { return reinterpret_cast<void*>(&bfs_persistent_kernel<RP, STATS>); }
};

}  // namespace

// ------------------------------------------------------------------ host side

// Dynamic shared memory of every kernel that can run a bottom-up level.
static size_t dyn_smem_bytes(int threads_per_block) {
  return sizeof(BuWarpSmem) * (size_t)(threads_per_block / 32);
}

static cudaError_t prepare_kernel(const void* fn, int threads_per_block) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dyn_smem_bytes(threads_per_block));
}

// Resident blocks per SM of a kernel at a block size, with the kernel's
// dynamic shared-memory limit set to what that block size uses.  The
// occupancy is computed once per (device, kernel, block size) and the limit is
// set only when it changes: these host calls would otherwise run before every
// launch, while the stream idles.
static cudaError_t resident_blocks(const void* fn, int threads_per_block, int* per_sm) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int>, int> occ;   // (device, kernel, threads) -> blocks per SM
  static std::map<std::pair<int, const void*>, int> limit;       // (device, kernel) -> shared-memory limit set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int smem = (int)dyn_smem_bytes(threads_per_block);
  std::lock_guard<std::mutex> lock(mu);
  auto lit = limit.find({dev, fn});
  if (lit == limit.end() || lit->second != smem) {
    e = prepare_kernel(fn, threads_per_block);
    if (e != cudaSuccess) return e;
    limit[{dev, fn}] = smem;
  }
  auto it = occ.find({dev, fn, threads_per_block});
  if (it != occ.end()) {
    *per_sm = it->second;
    return cudaSuccess;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads_per_block, (size_t)smem);
  if (e != cudaSuccess) return e;
  occ[{dev, fn, threads_per_block}] = *per_sm;
  return cudaSuccess;
}

static int resolve_policy(const bfs_graph* g, const bfs_params& p) {
  if (p.policy != BFS_POLICY_AUTO) return p.policy;
  // Section 3: average degree below 7 marks a large-diameter graph -> top-down only; several
  // levels per grid barrier unless a long list would hold up one warp of the local kernel.
  if ((double)g->m < (double)p.large_diameter_degree * (double)g->n)
    return g->max_deg <= kLocalAutoMaxDegree && p.launch != BFS_LAUNCH_PER_LEVEL ? BFS_POLICY_LOCAL
                                                                                 : BFS_POLICY_TD_ONLY;
  return BFS_POLICY_EDGES;
}

bool uses_local_kernel(const bfs_graph* g, const bfs_params& p) { return resolve_policy(g, p) == BFS_POLICY_LOCAL; }

static void fill_kparams(bfs_graph* g, int src, int* dist, const bfs_params& p, KParams& K) {
  SingleWs& ws = g->ws;
  const Relabel* rl = (p.relabel && g->rl && g->rl->h_new_of) ? g->rl : nullptr;
  K.rp = rl ? rl->rp : g->rp;
  K.col = rl ? rl->col : g->col;
  K.n = g->n;
  K.m = g->m;
  K.nw = g->nw;
  K.src = rl ? rl->h_new_of[src] : src;
  K.init_vis = rl ? rl->init_vis : g->init_vis;
  K.head = rl ? rl->head : g->head;
  K.new_of = rl ? rl->new_of : nullptr;
  K.old_of = rl ? rl->old_of : nullptr;
  K.lv8 = ws.lv8;
  K.n_live = g->n - g->isolated;
  K.dist = dist;
  K.vis = ws.vis;
  K.bm0 = ws.bm[0];
  K.bm1 = ws.bm[1];
  K.qv0 = ws.qv[0];
  K.qv1 = ws.qv[1];
  K.it0 = ws.it[0];
  K.it1 = ws.it[1];
  K.cap = ws.cap;
  K.mg0 = ws.mg[0];
  K.mg1 = ws.mg[1];
  K.ctrl = ws.ctrl;
  K.lst = nullptr;
  K.lst_cap = 0;
  K.policy = resolve_policy(g, p);
  K.alpha = p.alpha;
  K.beta = p.beta;
  K.tau_inv = p.tau_inv;
  K.script = p.script;
  K.small_max = p.small_max;
  K.chunk = p.chunk;
  K.bu_warp_min = p.bu_warp_min;
  K.bu_chunk = p.bu_chunk;
  K.bu_thread_max = p.bu_thread_max;
  K.need_qv = K.policy != BFS_POLICY_TD_ONLY;
  K.timeout_ns = (long long)p.timeout_ms * 1000000ll;
  K.barrier_extra = p.test_barrier_extra;
  K.col_cap = g->m + 4;  // both the uploaded lists and the renumbered copy carry >= 4 spare entries
  K.mg_cap = g->m / 8192 + 2;
}

template <typename RP, bool STATS>
static int launch_persistent(bfs_graph* g, KParams& K, const bfs_params& p, cudaStream_t stream) {
  void* fn = Kernels<RP, STATS>::persistent();
  const size_t smem = dyn_smem_bytes(p.threads_per_block);
  int per_sm = 0;
  GBFS_CUDA(resident_blocks(fn, p.threads_per_block, &per_sm));
  if (per_sm < 1) return BFS_EINVAL;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  dim3 grid((unsigned)(per_sm * g->num_sms)), block((unsigned)p.threads_per_block);
  void* args[] = {&K};
  GBFS_CUDA(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, stream));
  return BFS_OK;
}

template <typename RP, bool STATS>
static int launch_per_level(bfs_graph* g, KParams& K, const bfs_params& p, cudaStream_t stream) {
  SingleWs& ws = g->ws;
  const size_t smem = dyn_smem_bytes(p.threads_per_block);
  GBFS_CUDA(prepare_kernel(reinterpret_cast<void*>(&k_level<RP, STATS>), p.threads_per_block));
  int per_sm = 0;
  GBFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, reinterpret_cast<void*>(&k_level<RP, STATS>), p.threads_per_block, smem));
  if (per_sm < 1) return BFS_EINVAL;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  dim3 grid((unsigned)(per_sm * g->num_sms)), block((unsigned)p.threads_per_block);
  k_init_seed<RP><<<grid, block, 0, stream>>>(K);
  GBFS_CUDA(cudaGetLastError());
  GBFS_CUDA(cudaMemcpyAsync(ws.h_slot, &ws.ctrl->slot[0], sizeof(Slot), cudaMemcpyDeviceToHost, stream));
  GBFS_CUDA(cudaStreamSynchronize(stream));
  long long edges_visited = (long long)ws.h_slot->mf;
  unsigned long long items = ws.h_slot->items, mega = ws.h_slot->mega;
  long long nf_cur = 1, reached = 1;
  int L = 0, fb = 0, tdl = 0, bul = 0, conversions = 0, converted = 0;
  bool td = true;
  Ctrl host_tot{};
  int direct = K.lv8 == nullptr;
  for (;;) {
    if (!direct && L >= 254) {
      k_expand<<<grid, block, 0, stream>>>(K);
      direct = 1;
    }
    k_level<RP, STATS><<<grid, block, smem, stream>>>(K, L, direct, td ? 1 : 0, fb, items, mega, reached);
    GBFS_CUDA(cudaGetLastError());
    if (td) ++tdl; else ++bul;
    GBFS_CUDA(cudaMemcpyAsync(ws.h_slot, &ws.ctrl->slot[(L + 1) & 3], sizeof(Slot), cudaMemcpyDeviceToHost,
                              stream));
    GBFS_CUDA(cudaStreamSynchronize(stream));
    const long long nf = (long long)ws.h_slot->nv, mf = (long long)ws.h_slot->mf;
    if (K.lst && L < K.lst_cap) {
      bfs_level_stat ls{};
      GBFS_CUDA(cudaMemcpy(&ls, &K.lst[L], sizeof(ls), cudaMemcpyDeviceToHost));
      ls.direction = td ? 0 : 1;
      ls.converted = converted;
      ls.frontier = nf_cur;
      ls.found = nf;
      GBFS_CUDA(cudaMemcpy(&K.lst[L], &ls, sizeof(ls), cudaMemcpyHostToDevice));
    }
    if (STATS) {
      if (td) host_tot.td_frontier += (unsigned long long)nf_cur; else host_tot.bu_found += (unsigned long long)nf;
    }
    if (nf == 0) break;
    edges_visited += mf;
    reached += nf;
    const bool ntd = next_is_top_down(K.policy, K.alpha, K.beta, K.tau_inv, K.script, L + 1, td, nf, nf_cur, mf,
                                      K.m - edges_visited, K.n);
    converted = 0;
    if (td && !ntd) {
      k_zero_words<<<grid, block, 0, stream>>>(K.bm0, K.nw);
      k_scatter<<<grid, block, 0, stream>>>(K, ((L + 1) & 1) ? K.qv1 : K.qv0, nf, K.bm0);
      GBFS_CUDA(cudaGetLastError());
      fb = 0;
      converted = 1;
    } else if (!td && ntd) {
      k_convert<RP><<<grid, block, 0, stream>>>(K, L, fb ? K.bm0 : K.bm1);
      GBFS_CUDA(cudaGetLastError());
      GBFS_CUDA(cudaMemcpyAsync(ws.h_slot, &ws.ctrl->slot[(L + 1) & 3], sizeof(Slot), cudaMemcpyDeviceToHost,
                                stream));
      GBFS_CUDA(cudaStreamSynchronize(stream));
      converted = 1;
    } else if (!td && !ntd) {
      fb ^= 1;
    }
    if (converted) {
      ++conversions;
      host_tot.conv_frontier += (unsigned long long)nf;
    }
    if (ntd) {
      items = ws.h_slot->items;
      mega = ws.h_slot->mega;
    }
    td = ntd;
    nf_cur = nf;
    ++L;
  }
  if (!direct) k_expand<<<grid, block, 0, stream>>>(K);
  GBFS_CUDA(cudaGetLastError());
  // Write the loop's totals where the persistent kernel would have left them.
  GBFS_CUDA(cudaStreamSynchronize(stream));
  Ctrl c{};
  GBFS_CUDA(cudaMemcpy(&c, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  c.levels = L + 1;
  c.td_levels = tdl;
  c.bu_levels = bul;
  c.conversions = conversions;
  c.reached = (unsigned long long)reached;
  c.edges_reached = (unsigned long long)edges_visited;
  c.td_frontier = host_tot.td_frontier;
  c.bu_found = host_tot.bu_found;
  c.conv_frontier = host_tot.conv_frontier;
  GBFS_CUDA(cudaMemcpy(ws.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice));
  return BFS_OK;
}

// Control-block reset before a query: the previous query's status (still in
// the block) is kept in *sticky if no earlier failure is, then the block is
// zeroed.  One block; the status is read before any word is cleared.
__global__ void __launch_bounds__(128) k_ctrl_reset(Ctrl* c, int* sticky) {
  static_assert(sizeof(Ctrl) % sizeof(unsigned long long) == 0, "control block of whole words");
  constexpr int kWords = (int)(sizeof(Ctrl) / sizeof(unsigned long long));
  if (threadIdx.x == 0) {
    const int s = c->status;
    if (s != 0 && *sticky == 0) *sticky = s;
  }
  __syncthreads();
  unsigned long long* w = reinterpret_cast<unsigned long long*>(c);
  for (int i = threadIdx.x; i < kWords; i += blockDim.x) w[i] = 0ull;
}

cudaError_t enqueue_ctrl_reset(SingleWs& ws, cudaStream_t stream) {
  k_ctrl_reset<<<1, 128, 0, stream>>>(ws.ctrl, ws.sticky);
  return cudaGetLastError();
}

// The persistent launch (control-block reset + cooperative kernel) captured
// once as a CUDA graph per workspace and replayed with refreshed arguments.
template <typename RP>
static int launch_graph(bfs_graph* g, KParams& K, const bfs_params& p, cudaStream_t stream) {
  SingleWs& ws = g->ws;
  void* fn = Kernels<RP, false>::persistent();
  const size_t smem = dyn_smem_bytes(p.threads_per_block);
  int per_sm = 0;
  GBFS_CUDA(resident_blocks(fn, p.threads_per_block, &per_sm));
  if (per_sm < 1) return BFS_EINVAL;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  cudaKernelNodeParams kp{};
  kp.func = fn;
  kp.gridDim = dim3((unsigned)(per_sm * g->num_sms));
  kp.blockDim = dim3((unsigned)p.threads_per_block);
  kp.sharedMemBytes = (unsigned)smem;
  void* args[] = {&K};
  kp.kernelParams = args;
  const int key = (per_sm * 4096 + p.threads_per_block) * 2 + (g->rp_bits == 32 ? 1 : 0);
  if (ws.gexec == nullptr || ws.gkey != key) {
    if (ws.gexec) cudaGraphExecDestroy(ws.gexec);
    if (ws.graph) cudaGraphDestroy(ws.graph);
    ws.gexec = nullptr;
    ws.graph = nullptr;
    GBFS_CUDA(cudaGraphCreate(&ws.graph, 0));
    cudaGraphNode_t reset_node;
    cudaKernelNodeParams rp{};
    rp.func = reinterpret_cast<void*>(&k_ctrl_reset);
    rp.gridDim = dim3(1);
    rp.blockDim = dim3(128);
    void* rargs[] = {&ws.ctrl, &ws.sticky};
    rp.kernelParams = rargs;
    GBFS_CUDA(cudaGraphAddKernelNode(&reset_node, ws.graph, nullptr, 0, &rp));
    GBFS_CUDA(cudaGraphAddKernelNode(&ws.knode, ws.graph, &reset_node, 1, &kp));
    cudaLaunchAttributeValue coop{};
    coop.cooperative = 1;
    GBFS_CUDA(cudaGraphKernelNodeSetAttribute(ws.knode, cudaLaunchAttributeCooperative, &coop));
    GBFS_CUDA(cudaGraphInstantiate(&ws.gexec, ws.graph, 0));
    ws.gkey = key;
  } else {
    GBFS_CUDA(cudaGraphExecKernelNodeSetParams(ws.gexec, ws.knode, &kp));
  }
  GBFS_CUDA(cudaGraphLaunch(ws.gexec, stream));
  return BFS_OK;
}

// Launch the persistent kernel (no statistics) on prepared arguments, with the
// default block shape: used by the entry point whose scratch lives in a static
// device array and that therefore has no bfs_graph object.
int launch_persistent_prepared(KParams& K, int rp_bits, int num_sms, int threads_per_block,
                               cudaStream_t stream) {
  void* fn = rp_bits == 32 ? Kernels<int, false>::persistent() : Kernels<long long, false>::persistent();
  const size_t smem = dyn_smem_bytes(threads_per_block);
  int per_sm = 0;
  GBFS_CUDA(resident_blocks(fn, threads_per_block, &per_sm));
  if (per_sm < 1) return BFS_EINVAL;
  dim3 grid((unsigned)(per_sm * num_sms)), block((unsigned)threads_per_block);
  void* args[] = {&K};
  GBFS_CUDA(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, stream));
  return BFS_OK;
}

int run_single(bfs_graph* g, int src, int* dist_dev, const bfs_params& p, bfs_stats* st,
               bfs_level_stat* levels, int level_cap, cudaStream_t stream, bool wait) {
  SingleWs& ws = g->ws;
  KParams K;
  fill_kparams(g, src, dist_dev, p, K);
  const bool stats = st != nullptr;
  if (levels && level_cap > 0) {
    if (ws.lst_cap < level_cap) {
      if (ws.lst) cudaFree(ws.lst);
      ws.lst = nullptr;
      ws.lst_cap = 0;
      GBFS_CUDA(cudaMalloc(&ws.lst, sizeof(bfs_level_stat) * (size_t)level_cap));
      ws.lst_cap = level_cap;
    }
    GBFS_CUDA(cudaMemsetAsync(ws.lst, 0, sizeof(bfs_level_stat) * (size_t)level_cap, stream));
    K.lst = ws.lst;
    K.lst_cap = level_cap;
  }
  GBFS_CUDA(cudaStreamWaitEvent(stream, ws.done, 0));
  int rc;
  int launch = p.launch;
  const bool local = K.policy == BFS_POLICY_LOCAL;
  if (local && launch == BFS_LAUNCH_PER_LEVEL) return BFS_EINVAL;
  if (launch == BFS_LAUNCH_GRAPH && stats) launch = BFS_LAUNCH_PERSISTENT;
  if (launch != BFS_LAUNCH_GRAPH && !local) GBFS_CUDA(enqueue_ctrl_reset(ws, stream));
  if (local) {
    rc = run_local(g, src, dist_dev, p, st, levels, level_cap, stream);
  } else if (launch == BFS_LAUNCH_GRAPH) {
    rc = g->rp_bits == 32 ? launch_graph<int>(g, K, p, stream) : launch_graph<long long>(g, K, p, stream);
  } else if (launch == BFS_LAUNCH_PER_LEVEL) {
    if (g->rp_bits == 32)
      rc = stats ? launch_per_level<int, true>(g, K, p, stream) : launch_per_level<int, false>(g, K, p, stream);
    else
      rc = stats ? launch_per_level<long long, true>(g, K, p, stream)
                 : launch_per_level<long long, false>(g, K, p, stream);
  } else {
    if (g->rp_bits == 32)
      rc = stats ? launch_persistent<int, true>(g, K, p, stream) : launch_persistent<int, false>(g, K, p, stream);
    else
      rc = stats ? launch_persistent<long long, true>(g, K, p, stream)
                 : launch_persistent<long long, false>(g, K, p, stream);
  }
  if (rc != BFS_OK) return rc;
  if (!wait) {
    GBFS_CUDA(cudaEventRecord(ws.done, stream));
    return BFS_OK;
  }
  GBFS_CUDA(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream));
  GBFS_CUDA(cudaEventRecord(ws.done, stream));
  GBFS_CUDA(cudaStreamSynchronize(stream));
  const Ctrl& c = *ws.h_ctrl;
  if (c.status != 0) {
    // Returned here: cleared, so that the next query's reset does not keep it
    // for bfs_single_wait as well.
    GBFS_CUDA(cudaMemset(&ws.ctrl->status, 0, sizeof(int)));
    return c.status;
  }
  if (st) {
    st->levels = c.levels;
    st->td_levels = c.td_levels;
    st->bu_levels = c.bu_levels;
    st->conversions = c.conversions;
    st->reached = (int64_t)c.reached;
    st->edges_reached = (int64_t)c.edges_reached;
    st->td_frontier = (int64_t)c.td_frontier;
    st->td_edges = (int64_t)c.td_edges;
    st->bu_unvisited = (int64_t)c.bu_unvisited;
    st->bu_edges = (int64_t)c.bu_edges;
    st->bu_found = (int64_t)c.bu_found;
    st->conv_frontier = (int64_t)c.conv_frontier;
    st->init_ns = c.t_levels > c.t_begin ? (int64_t)(c.t_levels - c.t_begin) : 0;
    st->finish_ns = c.t_end > c.t_levels_end ? (int64_t)(c.t_end - c.t_levels_end) : 0;
    st->supersteps = local ? c.supersteps : 0;
    st->improved = local ? (int64_t)c.improved : 0;
    if (local) st->td_levels = c.levels;
  }
  if (levels && level_cap > 0) {
    const int nrec = local ? c.supersteps : c.levels;
    int nl = nrec < level_cap ? nrec : level_cap;
    GBFS_CUDA(cudaMemcpy(levels, ws.lst, sizeof(bfs_level_stat) * (size_t)nl, cudaMemcpyDeviceToHost));
  }
  return BFS_OK;
}

bool bounds_read_single(unsigned long long* first, bool reset) {
#ifdef GBFS_DEBUG_BOUNDS
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_err, sizeof(v)) != cudaSuccess) v = 0;
  if (reset) {
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_bounds_err, &z, sizeof(z));
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
