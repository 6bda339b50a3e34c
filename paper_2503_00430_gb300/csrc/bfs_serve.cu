// Serving loop: resident graphs, a stream of (graph, source) queries, and
// continuous batching into 64-lane multi-source groups.
//
// Every registered graph has one lane group (created on its first query if
// the device-memory budget allows) and one worker thread that drives it, so
// groups on different graphs advance independently, each on its own stream.
// A worker loops: (1) waits for its group's launched level and retires lanes
// whose frontier emptied (their rows are written and, for host outputs,
// copied back; a query is done when its copy is); (2) admits queued queries
// into free lanes - a query needs a free lane and, if its output is host
// memory, a device staging buffer of 4n bytes within the budget - where they
// join the running group at its next level; (3) launches the next level.
// Large-diameter graphs (average degree below the paper's threshold of
// Section 3) run thousands of short levels: their group's stream gets the
// highest priority, so its small kernels are scheduled ahead of the dense
// levels of other groups instead of queueing behind them.
//
// Memory pressure: a graph whose group (or a query's staging buffer) does not
// fit the budget registers as blocked.  While any graph is blocked, every
// other worker stops admitting, lets its running queries finish and then
// releases its group and staging buffers, so the blocked graph gets the
// memory; the released graph's own queries then wait their turn the same way.
// A device wait that runs out in a group fails that group's running queries
// (status BFS_ETIMEOUT) and frees the group; the server keeps serving.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bfs_internal.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Query {
  uint64_t ticket = 0;
  int graph = 0;
  int src = 0;
  int32_t* user_out = nullptr;
  bool host_out = false;
  int32_t* dev_out = nullptr;
  int lane = -1;
  int join = 0;
  int levels = 0;
  int status = BFS_OK;
  bool done = false;
  int64_t t_submit = 0, t_start = 0, t_done = 0;
  cudaEvent_t ev = nullptr;
};

struct GraphEntry {
  bfs_graph* g = nullptr;
  gbfs::ServeGroup* grp = nullptr;
  size_t grp_bytes = 0;               // budget bytes the group holds
  bool mem_blocked = false;           // counted in bfs_server::mem_blocked (guarded by the server mutex)
  std::deque<Query*> pending;         // submitted, not yet taken by the worker (guarded by the server mutex)
  std::condition_variable cv;         // wakes the worker (with the server mutex)
  // Owned by the worker thread:
  std::deque<Query*> waiting;         // taken, waiting for a lane or memory
  Query* lane_q[64] = {};
  std::vector<int32_t*> staging_free;
  std::vector<int32_t*> staging_all;
  std::vector<Query*> completing;
  std::thread th;
};

}  // namespace

struct bfs_server {
  size_t budget = 0;
  size_t used = 0;                    // guarded by mu
  bfs_params p{};
  int device = 0;
  std::vector<GraphEntry*> graphs;    // entries never move once added (guarded by mu)
  std::mutex mu;
  std::condition_variable cv_done;
  size_t queued = 0;                  // submitted, not yet admitted
  size_t queue_cap = (size_t)1 << 20;
  int mem_blocked = 0;                // graphs waiting for budget memory (guarded by mu)
  std::unordered_map<uint64_t, Query*> tickets;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::atomic<int> error{BFS_OK};
};

namespace {

void fill_stats(const Query* q, bfs_query_stats* st) {
  if (!st) return;
  memset(st, 0, sizeof(*st));
  st->submit_ns = q->t_submit;
  st->start_ns = q->t_start;
  st->done_ns = q->t_done;
  st->levels = q->levels;
  st->lane = q->lane;
  st->graph_id = q->graph;
  st->status = q->status;
}

void complete(bfs_server* S, GraphEntry* ge);

// Takes `bytes` of the budget; false if they do not fit.
bool reserve(bfs_server* S, size_t bytes) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->used + bytes > S->budget) return false;
  S->used += bytes;
  return true;
}

void unreserve(bfs_server* S, size_t bytes) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->used -= bytes;
}

void set_blocked(bfs_server* S, GraphEntry* ge, bool blocked) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (ge->mem_blocked == blocked) return;
  ge->mem_blocked = blocked;
  S->mem_blocked += blocked ? 1 : -1;
}

// Another graph waits for budget memory that this one holds.
bool others_blocked(bfs_server* S, GraphEntry* ge) {
  std::lock_guard<std::mutex> lk(S->mu);
  return S->mem_blocked > (ge->mem_blocked ? 1 : 0);
}

void mark_done(bfs_server* S, Query* q, int status) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->status = status;
    q->t_done = now_ns();
    q->done = true;
  }
  S->cv_done.notify_all();
}

// Frees the group and the staging buffers (none may be in use) and returns
// their bytes to the budget.
void release_memory(bfs_server* S, GraphEntry* ge) {
  if (ge->grp) {
    gbfs::serve_group_destroy(ge->grp);
    ge->grp = nullptr;
    unreserve(S, ge->grp_bytes);
    ge->grp_bytes = 0;
  }
  const size_t nbytes = sizeof(int32_t) * (size_t)ge->g->n;
  for (int32_t* b : ge->staging_all) {
    cudaFree(b);
    unreserve(S, nbytes);
  }
  ge->staging_all.clear();
  ge->staging_free.clear();
}

// A device-side failure of the group's launched levels: its running queries
// end with that status, the group is freed (rebuilt by the next admission).
// Only a CUDA error stays with the server.
void fail_group(bfs_server* S, GraphEntry* ge, int rc) {
  if (rc == BFS_ECUDA) S->error = rc;
  for (int i = 0; i < 64; ++i) {
    Query* q = ge->lane_q[i];
    if (!q) continue;
    ge->lane_q[i] = nullptr;
    if (q->host_out) ge->staging_free.push_back(q->dev_out);
    q->levels = 0;
    mark_done(S, q, rc);
  }
  if (ge->grp) cudaStreamSynchronize(gbfs::serve_group_stream(ge->grp));
  complete(S, ge);
  if (ge->grp) {
    gbfs::serve_group_destroy(ge->grp);
    ge->grp = nullptr;
    unreserve(S, ge->grp_bytes);
    ge->grp_bytes = 0;
  }
}

// The group's launched level is done: retire lanes whose frontier emptied.
void finish_level(bfs_server* S, GraphEntry* ge) {
  unsigned long long retired = 0;
  const int rc = gbfs::serve_group_finish(ge->grp, &retired);
  if (rc != BFS_OK) {
    fail_group(S, ge, rc);
    return;
  }
  while (retired) {
    const int i = __builtin_ctzll(retired);
    retired &= retired - 1;
    Query* q = ge->lane_q[i];
    ge->lane_q[i] = nullptr;
    if (!q) continue;
    q->levels = gbfs::serve_group_level(ge->grp) - q->join;
    cudaStream_t st = gbfs::serve_group_stream(ge->grp);
    if (q->host_out)
      cudaMemcpyAsync(q->user_out, q->dev_out, sizeof(int32_t) * (size_t)ge->g->n, cudaMemcpyDeviceToHost, st);
    cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    cudaEventRecord(q->ev, st);
    ge->completing.push_back(q);
  }
}

// Queries whose results (and host copies) are complete.
void complete(bfs_server* S, GraphEntry* ge) {
  std::vector<Query*> still;
  bool any = false;
  for (Query* q : ge->completing) {
    const cudaError_t e = cudaEventQuery(q->ev);
    if (e == cudaErrorNotReady) {
      still.push_back(q);
      continue;
    }
    cudaEventDestroy(q->ev);
    q->ev = nullptr;
    if (e != cudaSuccess) q->status = BFS_ECUDA;
    if (q->host_out) ge->staging_free.push_back(q->dev_out);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      q->t_done = now_ns();
      q->done = true;
    }
    any = true;
  }
  ge->completing.swap(still);
  if (any) S->cv_done.notify_all();
}

// Waiting queries into free lanes (they join at the group's next level).
void admit(bfs_server* S, GraphEntry* ge) {
  const unsigned long long in_use = ge->grp ? gbfs::serve_group_lanes(ge->grp) : 0ull;
  std::vector<int> lanes, srcs;
  std::vector<int*> outs;
  int next_lane = 0;
  while (!ge->waiting.empty()) {
    int lane = -1;
    for (; next_lane < 64; ++next_lane)
      if (!((in_use >> next_lane) & 1ull) && ge->lane_q[next_lane] == nullptr) {
        lane = next_lane++;
        break;
      }
    if (lane < 0) break;
    Query* q = ge->waiting.front();
    const size_t nbytes = sizeof(int32_t) * (size_t)ge->g->n;
    if (!ge->grp) {
      const size_t need = gbfs::serve_group_bytes(ge->g, S->p.ms_ring);
      if (need + (q->host_out ? nbytes : 0) > S->budget) {
        // This graph's group can never fit the budget: the query fails instead of waiting forever.
        ge->waiting.pop_front();
        {
          std::lock_guard<std::mutex> lk(S->mu);
          S->queued -= 1;
        }
        mark_done(S, q, BFS_ENOMEM);
        --next_lane;
        continue;
      }
      if (!reserve(S, need)) {
        set_blocked(S, ge, true);  // other groups release memory once they drain
        break;
      }
      const int prio = ge->g->m < (long long)S->p.large_diameter_degree * ge->g->n ? 1 : 0;
      const int rc = gbfs::serve_group_create(ge->g, S->p.ms_ring, S->p.ms_heavy_min, prio, &ge->grp);
      if (rc != BFS_OK) {
        unreserve(S, need);
        S->error = rc;
        break;
      }
      ge->grp_bytes = need;
    }
    if (q->host_out) {
      if (ge->staging_free.empty()) {
        if (!reserve(S, nbytes)) {
          // No staging memory: wait for this group's running queries, or, with none running, for
          // other groups to release theirs.
          if (!gbfs::serve_group_lanes(ge->grp) && ge->completing.empty()) set_blocked(S, ge, true);
          break;
        }
        int32_t* buf = nullptr;
        if (cudaMalloc(&buf, nbytes) != cudaSuccess) {
          cudaGetLastError();
          unreserve(S, nbytes);
          break;
        }
        ge->staging_free.push_back(buf);
        ge->staging_all.push_back(buf);
      }
      q->dev_out = ge->staging_free.back();
      ge->staging_free.pop_back();
    } else {
      q->dev_out = q->user_out;
    }
    ge->waiting.pop_front();
    set_blocked(S, ge, false);
    q->lane = lane;
    q->t_start = now_ns();
    q->join = gbfs::serve_group_lanes(ge->grp) ? gbfs::serve_group_level(ge->grp) : 0;
    ge->lane_q[lane] = q;
    lanes.push_back(lane);
    srcs.push_back(q->src);
    outs.push_back(q->dev_out);
  }
  if (!lanes.empty()) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->queued -= lanes.size();
    }
    const int rc = gbfs::serve_group_join(ge->grp, (int)lanes.size(), lanes.data(), srcs.data(), outs.data());
    if (rc != BFS_OK) S->error = rc;
  }
}

void graph_worker(bfs_server* S, GraphEntry* ge) {
  cudaSetDevice(S->device);
  for (;;) {
    bool stopping;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      while (!ge->pending.empty()) {
        ge->waiting.push_back(ge->pending.front());
        ge->pending.pop_front();
      }
      stopping = S->stop;
    }
    if (ge->grp && gbfs::serve_group_ready(ge->grp) >= 0) finish_level(S, ge);  // blocks until the level is done
    complete(S, ge);
    // While another graph waits for memory this one holds, admit nothing and
    // release the memory once the running queries are done.
    const bool yield = others_blocked(S, ge);
    if (!stopping && !yield) admit(S, ge);
    const bool running = ge->grp && gbfs::serve_group_lanes(ge->grp);
    if (running) {
      const int rc = gbfs::serve_group_launch(ge->grp, S->p.tau_inv, (long long)S->p.timeout_ms * 1000000ll,
                                              S->p.test_barrier_extra);
      if (rc != BFS_OK) fail_group(S, ge, rc);
      continue;
    }
    if (yield && ge->completing.empty() && (ge->grp || !ge->staging_all.empty())) release_memory(S, ge);
    if (!ge->completing.empty()) {
      std::this_thread::yield();
      continue;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop) break;
    // Nothing running: sleep until a query arrives (or 1 ms, to retry admission).
    if (ge->pending.empty()) ge->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
}

}  // namespace

extern "C" {

int bfs_serve_create(size_t mem_budget, const bfs_params* params, bfs_server** out) {
  GBFS_NVTX("bfs_serve_create");
  if (!out) return BFS_EINVAL;
  *out = nullptr;
  bfs_server* S = new bfs_server();
  S->budget = mem_budget;
  if (params) S->p = *params; else bfs_params_default(&S->p);
  if (S->p.ms_ring < 2 || S->p.ms_ring > 16 || S->p.tau_inv < 1 || S->p.timeout_ms < 1 ||
      S->p.test_barrier_extra < 0 || S->p.serve_queue < 0) {
    delete S;
    return BFS_EINVAL;
  }
  if (S->p.serve_queue > 0) S->queue_cap = (size_t)S->p.serve_queue;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return BFS_ECUDA;
  }
  *out = S;
  return BFS_OK;
}

int bfs_serve_add_graph(bfs_server* S, bfs_graph* g, int32_t* graph_id) {
  GBFS_NVTX("bfs_serve_add_graph");
  if (!S || !g || !graph_id) return BFS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return BFS_EINVAL;
  GraphEntry* ge = new GraphEntry();
  ge->g = g;
  S->graphs.push_back(ge);
  *graph_id = (int32_t)S->graphs.size() - 1;
  ge->th = std::thread(graph_worker, S, ge);
  return BFS_OK;
}

int bfs_serve_submit(bfs_server* S, int32_t graph_id, int32_t src, int32_t* dist_out, uint64_t* ticket) {
  GBFS_NVTX("bfs_serve_submit");
  if (!S || !dist_out || !ticket) return BFS_EINVAL;
  const bool host_out = !gbfs::is_device_pointer(dist_out);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->error.load() != BFS_OK) return S->error.load();
  if (graph_id < 0 || graph_id >= (int32_t)S->graphs.size()) return BFS_ENOTFOUND;
  GraphEntry* ge = S->graphs[graph_id];
  if (src < 0 || (int64_t)src >= ge->g->n) return BFS_EINVAL;
  if (S->queued >= S->queue_cap) return BFS_EAGAIN;
  Query* q = new Query();
  q->ticket = S->next_ticket++;
  q->graph = graph_id;
  q->src = src;
  q->user_out = dist_out;
  q->host_out = host_out;
  q->t_submit = now_ns();
  S->tickets[q->ticket] = q;
  ge->pending.push_back(q);
  ++S->queued;
  *ticket = q->ticket;
  ge->cv.notify_one();
  return BFS_OK;
}

int bfs_serve_poll(bfs_server* S, uint64_t ticket, int* done, bfs_query_stats* stats) {
  if (!S || !done) return BFS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return BFS_ENOTFOUND;
  Query* q = it->second;
  *done = q->done ? 1 : 0;
  if (!q->done) return BFS_OK;
  fill_stats(q, stats);
  const int status = q->status;
  S->tickets.erase(it);
  delete q;
  return status;
}

int bfs_serve_wait(bfs_server* S, uint64_t ticket, int64_t timeout_us, bfs_query_stats* stats) {
  GBFS_NVTX("bfs_serve_wait");
  if (!S) return BFS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return BFS_ENOTFOUND;
  Query* q = it->second;
  auto pred = [&] { return q->done || S->error.load() != BFS_OK; };
  if (timeout_us < 0) {
    S->cv_done.wait(lk, pred);
  } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
    return BFS_ETIMEOUT;
  }
  if (!q->done) return S->error;
  fill_stats(q, stats);
  const int status = q->status;
  S->tickets.erase(ticket);
  delete q;
  return status;
}

void bfs_serve_destroy(bfs_server* S) {
  GBFS_NVTX("bfs_serve_destroy");
  if (!S) return;
  std::vector<GraphEntry*> ges;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    ges = S->graphs;
  }
  // Workers finish their running lanes, then exit.
  for (GraphEntry* ge : ges) ge->cv.notify_all();
  for (GraphEntry* ge : ges)
    if (ge->th.joinable()) ge->th.join();
  cudaSetDevice(S->device);
  // Queries never admitted (still queued at shutdown) and completed ones not yet
  // reported are all still registered under their tickets.
  for (GraphEntry* ge : ges) {
    release_memory(S, ge);
    delete ge;
  }
  for (auto& kv : S->tickets) delete kv.second;
  delete S;
}

}  // extern "C"
