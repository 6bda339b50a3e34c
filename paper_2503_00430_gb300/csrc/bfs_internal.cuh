// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "bfs.h"

namespace gbfs {

// An NVTX range around one API call, so profiler timelines name the library's
// work (a no-op unless a profiling tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GBFS_NVTX(name) ::gbfs::NvtxRange gbfs_nvtx_range_(name)

constexpr unsigned kFull = 0xffffffffu;

// Counters of one frontier F_L, kept in a ring of four slots indexed by L & 3.
struct Slot {
  unsigned long long items;  // low 32 bits: small work items, high 32 bits: large work items
  unsigned long long nv;     // |F_L|
  unsigned long long mf;     // sum of degrees over F_L
  unsigned long long nq;     // reserved (zeroed with the slot)
  unsigned long long cursor; // bottom-up: next bitmap word to hand out (dynamic assignment)
  unsigned long long mega;   // hub records: low 26 bits record count, high 38 bits chunk count
};

// A vertex whose adjacency spans more than 32 chunks ("hub"): one record, its
// chunks handed out at the next top-down level as tickets base .. base+nch-1.
struct MegaRec {
  long long start;
  long long deg;
  unsigned long long base;
};
constexpr int kMegaCountBits = 26;

// Device control block of one single-source query (zeroed before each launch).
struct Ctrl {
  unsigned long long barrier;  // grid-barrier arrival counter
  int status;                  // BFS_OK or BFS_ETIMEOUT
  int levels, td_levels, bu_levels, conversions;
  int supersteps;              // BFS_POLICY_LOCAL
  int pad[2];
  unsigned long long reached, edges_reached;
  unsigned long long td_frontier, td_edges, bu_unvisited, bu_edges, bu_found, conv_frontier;
  unsigned long long improved;  // BFS_POLICY_LOCAL: labels lowered
  unsigned long long t_begin, t_levels, t_levels_end, t_end;  // device clock: kernel entry, end of init,
                                                              // end of the last level, end of the final
                                                              // expansion (block 0's view)
  Slot slot[4];
};

// Arguments of the single-source kernels (passed by value).
struct KParams {
  const void* rp;            // int32 or int64 row pointers [n+1]
  const int* col;            // neighbour ids, padded with >= 4 spare entries
  long long n, m;
  int nw;                    // bitmap words = ceil(n / 32)
  int src;
  const unsigned* init_vis;  // degree-0 vertices and padding bits set
  const int4* head;          // per vertex {first neighbour, second neighbour, list start, degree}
                             // (-1 for a missing neighbour), or null: read rp / col instead
  long long n_live;          // vertices of degree > 0 (n when unknown)
  int* dist;
  unsigned char* lv8;        // per-vertex level bytes (255 = not reached) while the search runs, or
                             // null: levels go straight to dist
  unsigned* vis;
  unsigned* bm0;
  unsigned* bm1;
  int* qv0;
  int* qv1;
  unsigned long long* it0;
  unsigned long long* it1;
  long long cap;             // entries of it0 / it1
  MegaRec* mg0;
  MegaRec* mg1;
  Ctrl* ctrl;
  bfs_level_stat* lst;
  int lst_cap;
  int policy, alpha, beta, tau_inv;
  unsigned long long script;
  int small_max, chunk, bu_warp_min, bu_chunk, bu_thread_max;
  int need_qv;
  long long timeout_ns;
  int barrier_extra;
  // Degree-renumbered graph (single-source queries with params->relabel): the
  // search runs in new ids; dist is written in the caller's ids through these
  // maps.  Null: the graph as uploaded.
  const int* new_of = nullptr;   // [n] caller id -> new id (expansion of the level bytes)
  const int* old_of = nullptr;   // [n] new id -> caller id (direct int32 writes past level 254)
  long long col_cap = 0;         // readable entries of col (bounds-checked build)
  long long mg_cap = 0;          // entries of mg0 / mg1 (bounds-checked build)
};

// Direction of level `next_level` (true = top-down), from the counters of the
// frontier F_{next} that level next_level-1 produced.  Used identically by the
// device (persistent kernel) and the host (per-level launches).
//   nf_next   |F_next|          nf_cur  |F_{next-1}|
//   mf_next   degrees in F_next m_unvisited  entries of vertices not yet visited
__host__ __device__ inline bool next_is_top_down(int policy, int alpha, int beta, int tau_inv,
                                                 unsigned long long script, int next_level,
                                                 bool cur_td, long long nf_next, long long nf_cur,
                                                 long long mf_next, long long m_unvisited,
                                                 long long n) {
  if (next_level == 0) return true;
  switch (policy) {
    case BFS_POLICY_TD_ONLY:
      return true;
    case BFS_POLICY_BU_FROM_1:
      return false;
    case BFS_POLICY_SCRIPT: {
      int b = next_level < 63 ? next_level : 63;
      return ((script >> b) & 1ull) == 0;
    }
    case BFS_POLICY_FRONTIER:
      // Section 2's frontier-size rule (Listing 2: top-down while |F| is below 5 % of n), taken
      // as the exact integer test tau_inv*|F| < n.
      return (long long)tau_inv * nf_next < n;
    case BFS_POLICY_EDGES:
    default:
      if (cur_td) return !((long long)alpha * mf_next > m_unvisited);
      return (long long)beta * nf_next < n && nf_next < nf_cur;
  }
}

// Host-side graph object.
struct SingleWs {
  bool ready = false;
  unsigned* vis = nullptr;
  unsigned char* lv8 = nullptr;  // n bytes (rounded up to 16)
  unsigned* bm[2] = {nullptr, nullptr};
  int* qv[2] = {nullptr, nullptr};
  unsigned long long* it[2] = {nullptr, nullptr};
  long long cap = 0;
  MegaRec* mg[2] = {nullptr, nullptr};
  Ctrl* ctrl = nullptr;       // device
  Ctrl* h_ctrl = nullptr;     // pinned host mirror
  Slot* h_slot = nullptr;     // pinned, per-level launch mode
  int* dist_tmp = nullptr;    // device staging for host-memory output
  bfs_level_stat* lst = nullptr;
  int lst_cap = 0;
  cudaEvent_t done = nullptr;  // last query's completion on the device
  int* sticky = nullptr;       // device: first failed status of a query since the last bfs_single_wait
  cudaGraph_t graph = nullptr;     // captured persistent launch (BFS_LAUNCH_GRAPH)
  cudaGraphNode_t knode = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gkey = -1;
};

}  // namespace gbfs

namespace gbfs {
struct MultiWs;
struct NonAtomicWs;

// A copy of the graph with the vertices renumbered by decreasing degree (ties
// by id): new id i is the i-th vertex of that order.  Multi-source levels run
// on it, so the frontier masks of the high-degree vertices, which most
// neighbour lists point to, share cache lines, and the degree-0 vertices
// (ids >= n_live) are never scanned.  Lists are sorted by new id, i.e. highest
// degree first.  Built once per graph, on first use.
struct Relabel {
  void* rp = nullptr;      // row pointers of the renumbered graph, same width as the graph's
  int* col = nullptr;      // renumbered neighbour ids (m entries + 4 zero pads)
  int* new_of = nullptr;   // [n] new id of every original vertex
  int* old_of = nullptr;   // [n] original id of every new id
  long long n_live = 0;    // vertices of degree > 0 (they take ids 0 .. n_live-1)
  // Single-source queries on the copy (built on first use): its head table and
  // visited mask, and new_of on the host (to map the source).
  int4* head = nullptr;
  unsigned* init_vis = nullptr;
  int* h_new_of = nullptr;
};
}

struct bfs_graph {
  long long n = 0, m = 0;
  int rp_bits = 64;
  int nw = 0;
  int device = 0;
  int num_sms = 0;
  void* rp = nullptr;         // device row pointers
  int* col = nullptr;         // device neighbour ids (padded)
  unsigned* init_vis = nullptr;
  int4* head = nullptr;       // per-vertex head table (null with BFS_NO_HEAD or m >= 2^31)
  long long max_deg = 0, isolated = 0;
  std::mutex mu;
  gbfs::SingleWs ws;
  gbfs::MultiWs* ms = nullptr;  // multi-source workspace (bfs_multi.cu)
  gbfs::Relabel* rl = nullptr;  // degree-renumbered copy (bfs_reorder.cu), built on first use
  gbfs::NonAtomicWs* na = nullptr;  // bfs_single_nonatomic workspace (bfs_nonatomic.cu)
  bool deg_ordered = false;     // lists were sorted highest degree first at upload
};

namespace gbfs {

int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
#define GBFS_CUDA(call)                                                           \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return ::gbfs::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

bool is_device_pointer(const void* p);
void* pinned_device_alias(const void* p);
bool uses_local_kernel(const bfs_graph* g, const bfs_params& p);  // the query runs bfs_local.cu's kernel
int reorder_by_degree(bfs_graph* g);
int build_head(bfs_graph* g);
int vertices_by_degree(bfs_graph* g, int* order);
int ensure_relabel(bfs_graph* g);  // builds g->rl once (caller holds g->mu)
int ensure_relabel_single(bfs_graph* g);  // + head table, visited mask, host new_of
void free_relabel(bfs_graph* g);
int ensure_single_ws(bfs_graph* g);
void free_single_ws(bfs_graph* g);
// One single-source query on the graph's workspace.  wait = false enqueues it
// and returns (no statistics, no level records); its status then reaches the
// workspace's sticky status when the next query is enqueued, or the next
// bfs_single_wait reads it.
int run_single(bfs_graph* g, int src, int* dist_dev, const bfs_params& p, bfs_stats* st,
               bfs_level_stat* levels, int level_cap, cudaStream_t stream, bool wait = true);
// Control-block reset before a single-source query (replaces a memset): the
// previous query's status is folded into ws.sticky, then the block is zeroed.
cudaError_t enqueue_ctrl_reset(SingleWs& ws, cudaStream_t stream);
int run_nonatomic(bfs_graph* g, int src, int* dist, int mode, bfs_dup_stats* st, bfs_dup_level* lv, int lv_cap,
                  cudaStream_t s);
void free_nonatomic_ws(NonAtomicWs* ws);
int ensure_multi_ws(bfs_graph* g, int ring);
void free_multi_ws(bfs_graph* g);
int run_multi(bfs_graph* g, const int32_t* srcs, int k, void* dist, int bits, const bfs_params& p,
              bfs_multi_stats* st, cudaStream_t s);
// Serving groups (bfs_multi.cu): 64 lanes on one graph, lanes joining at level boundaries.
struct ServeGroup;
size_t serve_group_bytes(const bfs_graph* g, int ring);
int serve_group_create(bfs_graph* g, int ring, int heavy_min, int high_priority, ServeGroup** out);
void serve_group_destroy(ServeGroup* G);
cudaStream_t serve_group_stream(ServeGroup* G);
unsigned long long serve_group_lanes(const ServeGroup* G);
int serve_group_level(const ServeGroup* G);
int serve_group_join(ServeGroup* G, int count, const int* lanes_idx, const int* srcs, int* const* outs);
int serve_group_launch(ServeGroup* G, int tau_inv, long long timeout_ns, int barrier_extra);
int serve_group_ready(ServeGroup* G);
int serve_group_finish(ServeGroup* G, unsigned long long* retired);
// Bounds-checked build (GBFS_DEBUG_BOUNDS): first recorded violation of each
// kernel file (bit 63 set, site << 48 | low 48 bits of the index; 0 = none),
// optionally cleared.  Both return false when the file was built without checks.
bool bounds_read_single(unsigned long long* first, bool reset);
bool bounds_read_local(unsigned long long* first, bool reset);
// Graph-set facts for the tuner (bfs_graphset.cu).
long long graphset_total_vertices(const bfs_graphset* s);
int graphset_count(const bfs_graphset* s);
// BFS_POLICY_AUTO picks BFS_POLICY_LOCAL for large-diameter graphs whose longest list is at most
// this long (the local kernel scans a list with one warp).
constexpr long long kLocalAutoMaxDegree = 4096;
// Multi-level local expansion (bfs_local.cu): launches the BFS_POLICY_LOCAL kernel.
int run_local(bfs_graph* g, int src, int* dist_dev, const bfs_params& p, bfs_stats* st, bfs_level_stat* levels,
              int level_cap, cudaStream_t stream);
int launch_persistent_prepared(KParams& K, int rp_bits, int num_sms, int threads_per_block,
                               cudaStream_t stream);

}  // namespace gbfs
