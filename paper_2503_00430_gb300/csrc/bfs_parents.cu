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

#include <mutex>
#include <unordered_map>

#include "bfs_internal.cuh"

namespace gbfs {

// Long lists: a vertex still open after its lane's scan with more than
// kParLong entries left is cut into kParLong-entry chunk tickets scanned by
// many warps; the smallest hit offset (atomicMin) gives the same first-in-list
// parent.  rec holds {vertex, first ticket, first entry} per such vertex.
struct ParentWs {
  unsigned long long* rec = nullptr;
  int* best = nullptr;                 // smallest hit offset from the record's first entry
  unsigned long long* ctr = nullptr;   // records (low 32 bits) and tickets (high 32 bits)
  long long cap = 0;
};

namespace {

constexpr int kParLane = 32;    // entries a lane scans on its own before the warp takes over
constexpr int kParLong = 1024;  // remaining entries above which a list is scanned in chunks

template <typename RP>
__device__ __forceinline__ long long par_rp(const void* rp, long long i) {
  return (long long)__ldg(reinterpret_cast<const RP*>(rp) + i);
}

// A warp takes 32 consecutive vertices: each lane scans the first kParLane
// entries of its vertex; vertices still unresolved with longer lists are then
// scanned by the whole warp, 32 entries per step, one vertex at a time.
template <typename RP>
__global__ void __launch_bounds__(256) k_parents(const void* rp, const int* col, const int* dist, long long n,
                                                 int* parent, ParentWs W) {
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
        if (open && e - j > kParLong) {
          // Chunked below; its parent is written by k_parents_finish.
          const unsigned long long nch = (unsigned long long)((e - j + kParLong - 1) / kParLong);
          const unsigned long long b = atomicAdd(W.ctr, 1ull | (nch << 32));
          const long long r = (long long)(b & 0xffffffffull);
          if (r < W.cap) {  // always: at most m / (kParLong + kParLane) such vertices
            W.rec[3 * r] = (unsigned long long)v;
            W.rec[3 * r + 1] = b >> 32;
            W.rec[3 * r + 2] = (unsigned long long)j;
            W.best[r] = 0x7fffffff;
          }
          open = false;
          p = -2;  // written later
        }
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
    if (v < n && p != -2) parent[v] = p;
  }
}

// A warp per chunk ticket: ticket t belongs to the last record whose first
// ticket is <= t (32-way search); the first hit of the chunk lowers best[r].
template <typename RP>
__global__ void __launch_bounds__(256) k_parents_chunks(const void* rp, const int* col, const int* dist,
                                                        ParentWs W) {
  const unsigned long long hv = *W.ctr;  // written by k_parents earlier on this stream
  long long nrec = (long long)(hv & 0xffffffffull);
  const long long ntick = (long long)(hv >> 32);
  if (nrec > W.cap) nrec = W.cap;
  if (nrec == 0) return;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  for (long long t = gw; t < ntick; t += nwarps) {
    long long lo = 0, hi = nrec;
    while (hi - lo > 1) {
      const long long step = (hi - lo + 31) / 32;
      const long long idx = lo + (long long)lane * step;
      const bool ok = idx < hi && (long long)W.rec[3 * idx + 1] <= t;
      const unsigned bm = __ballot_sync(0xffffffffu, ok);
      lo += (long long)(31 - __clz(bm)) * step;
      hi = lo + step < hi ? lo + step : hi;
    }
    const long long v = (long long)W.rec[3 * lo], t0 = (long long)W.rec[3 * lo + 1];
    const long long js = (long long)W.rec[3 * lo + 2], e = par_rp<RP>(rp, v + 1);
    const long long off0 = (t - t0) * kParLong;
    if (js + off0 >= e) continue;
    if ((long long)__ldcg(W.best + lo) < off0) continue;  // an earlier chunk already has a hit
    const int d = __ldg(dist + v);
    const long long ce = js + off0 + kParLong < e ? js + off0 + kParLong : e;
    for (long long k0 = js + off0; k0 < ce; k0 += 32) {
      const long long k = k0 + lane;
      const bool hit = k < ce && __ldg(dist + __ldg(col + k)) == d - 1;
      const unsigned b = __ballot_sync(0xffffffffu, hit);
      if (b) {
        if ((int)lane == __ffs(b) - 1) atomicMin(W.best + lo, (int)(k - js));
        break;
      }
    }
  }
}

// Parents of the chunked vertices (-1 if no entry qualified).
__global__ void k_parents_finish(const int* col, int* parent, ParentWs W) {
  long long nrec = (long long)(*W.ctr & 0xffffffffull);
  if (nrec > W.cap) nrec = W.cap;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += (long long)gridDim.x * blockDim.x) {
    const long long v = (long long)W.rec[3 * r], js = (long long)W.rec[3 * r + 2];
    const int b = W.best[r];
    parent[v] = b == 0x7fffffff ? -1 : col[js + b];
  }
}

}  // namespace

namespace {

// Host side of a graph's parent workspace.  Every call on the graph uses the
// same device buffers, so calls are ordered on the device: each one waits for
// the previous call's completion event before it touches the buffers, and
// records its own (calls from different streams then run one after another).
struct ParentHost {
  ParentWs W;
  cudaEvent_t done = nullptr;
  std::mutex mu;  // makes wait-on-previous + enqueue + record one step per call
};

void free_ws(ParentHost* w) {
  if (!w) return;
  cudaFree(w->W.rec);
  cudaFree(w->W.best);
  cudaFree(w->W.ctr);
  if (w->done) cudaEventDestroy(w->done);
  delete w;
}

// Workspace per graph, created on the graph's first parent array.
std::mutex g_par_mu;
std::unordered_map<const bfs_graph*, ParentHost*> g_par;

}  // namespace

// Called by bfs_graph_free.
void free_parent_ws_of(const bfs_graph* g) {
  std::lock_guard<std::mutex> lock(g_par_mu);
  auto it = g_par.find(g);
  if (it == g_par.end()) return;
  free_ws(it->second);
  g_par.erase(it);
}

int run_parents(bfs_graph* g, const int* dist, int* parent, cudaStream_t s) {
  ParentHost* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_par_mu);
    auto it = g_par.find(g);
    if (it != g_par.end()) ws = it->second;
    if (!ws) {
      ParentHost* w = new ParentHost();
      w->W.cap = g->m / (kParLong + kParLane) + 2;
      cudaError_t e = cudaMalloc(&w->W.rec, 3 * sizeof(unsigned long long) * (size_t)w->W.cap);
      if (e == cudaSuccess) e = cudaMalloc(&w->W.best, sizeof(int) * (size_t)w->W.cap);
      if (e == cudaSuccess) e = cudaMalloc(&w->W.ctr, sizeof(unsigned long long));
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        free_ws(w);
        return cuda_fail(e, "parent workspace", __FILE__, __LINE__);
      }
      g_par[g] = w;
      ws = w;
    }
  }
  std::lock_guard<std::mutex> order(ws->mu);
  const ParentWs W = ws->W;
  const int grid = g->num_sms * 8, block = 256;
  // The previous call on this graph (any stream) must be done with W first.
  GBFS_CUDA(cudaStreamWaitEvent(s, ws->done, 0));
  GBFS_CUDA(cudaMemsetAsync(W.ctr, 0, sizeof(unsigned long long), s));
  if (g->rp_bits == 32) {
    k_parents<int><<<grid, block, 0, s>>>(g->rp, g->col, dist, g->n, parent, W);
    k_parents_chunks<int><<<grid, block, 0, s>>>(g->rp, g->col, dist, W);
  } else {
    k_parents<long long><<<grid, block, 0, s>>>(g->rp, g->col, dist, g->n, parent, W);
    k_parents_chunks<long long><<<grid, block, 0, s>>>(g->rp, g->col, dist, W);
  }
  k_parents_finish<<<g->num_sms, 256, 0, s>>>(g->col, parent, W);
  GBFS_CUDA(cudaGetLastError());
  GBFS_CUDA(cudaEventRecord(ws->done, s));
  return BFS_OK;
}

}  // namespace gbfs
