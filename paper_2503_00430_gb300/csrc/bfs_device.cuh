// Device helpers shared by the single-source kernels (bfs_single.cu, bfs_local.cu):
// memory-ordering loads and reductions, L2 cache hints, warp scans and
// searches, and the bounded grid barrier of the persistent launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bfs_internal.cuh"

namespace gbfs {
namespace dev {

static __device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
static __device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}
static __device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
static __device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
static __device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
static __device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
static __device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
static __device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
static __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// L2 eviction-priority policies: data read once per level (adjacency, head
// records) is marked evict-first, the small per-vertex state that every level
// updates (level bytes) evict-last, so the streaming reads do not push it out.
// A policy is a plain value (no side effect), so the compiler may compute it
// once outside a loop.
static __device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
static __device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
static __device__ __forceinline__ void st_u8_last(unsigned char* p, unsigned v) {
  asm volatile("st.global.L2::cache_hint.u8 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(policy_evict_last()) : "memory");
}
static __device__ __forceinline__ void st_v4_last(void* p, unsigned a, unsigned b, unsigned c, unsigned d) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(a), "r"(b), "r"(c),
               "r"(d), "l"(policy_evict_last())
               : "memory");
}
// Asynchronous 16-byte global -> shared copy, evict-first in L2 (zero-filled
// when src_bytes is 0).
static __device__ __forceinline__ void cp_async16_first(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(sa), "l"(gmem),
               "r"(src_bytes), "l"(policy_evict_first())
               : "memory");
}
static __device__ __forceinline__ int4 ldg4_first(const int* p) {
  int4 q;
  asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(q.x), "=r"(q.y), "=r"(q.z), "=r"(q.w)
               : "l"(p), "l"(policy_evict_first()));
  return q;
}

template <typename RP>
static __device__ __forceinline__ long long rp_at(const void* rp, long long i) {
  return (long long)__ldg(reinterpret_cast<const RP*>(rp) + i);
}

static __device__ __forceinline__ int warp_incl_scan(int x) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(kFull, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  return x;
}

static __device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Position of the n-th (0-based) set bit of mask, by halving the window with
// population counts; always in [0, 31].
static __device__ __forceinline__ int nth_set_bit(unsigned mask, int n) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const int c = __popc(mask & ((1u << w) - 1u));
    if (n >= c) {
      n -= c;
      mask >>= w;
      pos += w;
    }
  }
  return pos;
}

// Lane holding entry e of the concatenation described by the exclusive scan
// `excl` of 32 lengths (largest lane whose start is <= e).
static __device__ __forceinline__ int owner_of(int excl, int e) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int ex = __shfl_sync(kFull, excl, lo + step);
    if (ex <= e) lo += step;
  }
  return lo;
}

// Bounded grid barrier over the blocks of a cooperative launch (every block's
// thread 0 arrives on one counter and spins until all have).  `extra` makes it
// wait for that many blocks more than were launched (a test of the limit).
// Returns false when the launch must stop (a wait ran out of time here or
// elsewhere); then ctrl->status holds BFS_ETIMEOUT.
static __device__ bool grid_barrier_ctl(Ctrl* ctrl, long long timeout_ns, int extra, unsigned& epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned long long nb = (unsigned long long)gridDim.x + (unsigned long long)extra;
    const unsigned long long target = (unsigned long long)epoch * nb;
    red_release_add(&ctrl->barrier, 1ull);
    int ok = 1;
    unsigned long long t0 = 0;
    unsigned spins = 0;
    while (ld_acquire_u64(&ctrl->barrier) < target) {
      if (ld_relaxed_s32(&ctrl->status) != 0) {
        ok = 0;
        break;
      }
      if ((++spins & 63u) == 0) {
        unsigned long long t = globaltimer_ns();
        if (t0 == 0) {
          t0 = t;
        } else if ((long long)(t - t0) > timeout_ns) {
          atomicCAS(&ctrl->status, 0, BFS_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && ld_relaxed_s32(&ctrl->status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace dev
}  // namespace gbfs
