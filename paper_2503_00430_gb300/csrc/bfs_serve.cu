// Serving loop: resident graphs, a stream of (graph, source) queries, and
// continuous batching into 64-lane multi-source groups.
//
// A server thread owns one lane group per graph (created on first use if the
// device-memory budget allows).  Each pass it (1) moves submitted queries to
// their graph's queue, (2) admits queued queries into free lanes - a query
// needs a free lane and, if its output is host memory, a device staging
// buffer of 4n bytes within the budget - where they join the running group at
// its next level, (3) launches one level of every busy group (each on its own
// stream, so groups on different graphs overlap on the GPU); each group moves
// on to its next level as soon as its own level has finished (groups are not
// in lockstep), retiring lanes whose frontier emptied: their rows are written
// and, for host outputs, copied back; a query is done when its copy is.
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
  std::deque<Query*> pending;
  Query* lane_q[64] = {};
  std::vector<int32_t*> staging_free;
};

}  // namespace

struct bfs_server {
  size_t budget = 0;
  size_t used = 0;
  bfs_params p{};
  int device = 0;
  std::vector<GraphEntry*> graphs;  // entries never move once added
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Query*> inbox;
  size_t inbox_cap = (size_t)1 << 20;
  std::unordered_map<uint64_t, Query*> tickets;
  std::vector<Query*> completing;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::atomic<int> error{BFS_OK};
  std::thread th;
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

// One pass of the server; returns true if any work is in flight or queued.
bool server_pass(bfs_server* S) {
  std::vector<GraphEntry*> ges;
  bool admit = true;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    while (!S->inbox.empty()) {
      Query* q = S->inbox.front();
      S->inbox.pop_front();
      S->graphs[q->graph]->pending.push_back(q);
    }
    ges = S->graphs;
    admit = !S->stop;
  }
  bool busy = false;
  for (GraphEntry* ge : ges) {
    // A group advances as soon as its own level is done, independently of the others.
    if (ge->grp) {
      const int r = gbfs::serve_group_ready(ge->grp);
      if (r == 0) {
        busy = true;
        continue;
      }
      if (r == 1) {
        unsigned long long retired = 0;
        const int rc = gbfs::serve_group_finish(ge->grp, &retired);
        if (rc != BFS_OK) S->error = rc;
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
          S->completing.push_back(q);
        }
      }
    }
    // Admission into free lanes, then the next level.
    const unsigned long long in_use = ge->grp ? gbfs::serve_group_lanes(ge->grp) : 0ull;
    std::vector<int> lanes, srcs;
    std::vector<int*> outs;
    while (admit && !ge->pending.empty()) {
      int lane = -1;
      for (int i = 0; i < 64; ++i)
        if (!((in_use >> i) & 1ull) && ge->lane_q[i] == nullptr) {
          bool taken = false;
          for (int l : lanes) taken |= (l == i);
          if (!taken) {
            lane = i;
            break;
          }
        }
      if (lane < 0) break;
      Query* q = ge->pending.front();
      const size_t nbytes = sizeof(int32_t) * (size_t)ge->g->n;
      if (!ge->grp) {
        const size_t need = gbfs::serve_group_bytes(ge->g, S->p.ms_ring);
        if (S->used + need > S->budget) break;
        int rc = gbfs::serve_group_create(ge->g, S->p.ms_ring, S->p.ms_heavy_min, &ge->grp);
        if (rc != BFS_OK) {
          S->error = rc;
          break;
        }
        S->used += need;
      }
      if (q->host_out) {
        if (ge->staging_free.empty()) {
          if (S->used + nbytes > S->budget) break;
          int32_t* buf = nullptr;
          if (cudaMalloc(&buf, nbytes) != cudaSuccess) {
            cudaGetLastError();
            break;
          }
          S->used += nbytes;
          ge->staging_free.push_back(buf);
        }
        q->dev_out = ge->staging_free.back();
        ge->staging_free.pop_back();
      } else {
        q->dev_out = q->user_out;
      }
      ge->pending.pop_front();
      q->lane = lane;
      q->t_start = now_ns();
      q->join = gbfs::serve_group_lanes(ge->grp) ? gbfs::serve_group_level(ge->grp) : 0;
      ge->lane_q[lane] = q;
      lanes.push_back(lane);
      srcs.push_back(q->src);
      outs.push_back(q->dev_out);
    }
    if (!lanes.empty()) {
      const int rc = gbfs::serve_group_join(ge->grp, (int)lanes.size(), lanes.data(), srcs.data(), outs.data());
      if (rc != BFS_OK) S->error = rc;
    }
    if (ge->grp && gbfs::serve_group_lanes(ge->grp)) {
      const int rc = gbfs::serve_group_launch(ge->grp, S->p.tau_inv);
      if (rc != BFS_OK) S->error = rc;
      busy = true;
    }
    if (admit && !ge->pending.empty()) busy = true;
  }
  // Completions.
  std::vector<Query*> still;
  for (Query* q : S->completing) {
    const cudaError_t e = cudaEventQuery(q->ev);
    if (e == cudaErrorNotReady) {
      still.push_back(q);
      continue;
    }
    cudaEventDestroy(q->ev);
    q->ev = nullptr;
    if (e != cudaSuccess) q->status = BFS_ECUDA;
    if (q->host_out) ges[q->graph]->staging_free.push_back(q->dev_out);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      q->t_done = now_ns();
      q->done = true;
    }
    S->cv_done.notify_all();
  }
  S->completing.swap(still);
  return busy || !S->completing.empty();
}

void server_main(bfs_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    const bool busy = server_pass(S);
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop && !busy && S->inbox.empty()) break;
    if (!busy && S->inbox.empty()) S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
    else if (busy) {
      lk.unlock();
      std::this_thread::yield();
    }
  }
}

}  // namespace

extern "C" {

int bfs_serve_create(size_t mem_budget, const bfs_params* params, bfs_server** out) {
  if (!out) return BFS_EINVAL;
  *out = nullptr;
  bfs_server* S = new bfs_server();
  S->budget = mem_budget;
  if (params) S->p = *params; else bfs_params_default(&S->p);
  if (S->p.ms_ring < 2 || S->p.ms_ring > 8 || S->p.tau_inv < 1) {
    delete S;
    return BFS_EINVAL;
  }
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return BFS_ECUDA;
  }
  S->th = std::thread(server_main, S);
  *out = S;
  return BFS_OK;
}

int bfs_serve_add_graph(bfs_server* S, bfs_graph* g, int32_t* graph_id) {
  if (!S || !g || !graph_id) return BFS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  GraphEntry* ge = new GraphEntry();
  ge->g = g;
  S->graphs.push_back(ge);
  *graph_id = (int32_t)S->graphs.size() - 1;
  return BFS_OK;
}

int bfs_serve_submit(bfs_server* S, int32_t graph_id, int32_t src, int32_t* dist_out, uint64_t* ticket) {
  if (!S || !dist_out || !ticket) return BFS_EINVAL;
  const bool host_out = !gbfs::is_device_pointer(dist_out);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->error.load() != BFS_OK) return S->error.load();
  if (graph_id < 0 || graph_id >= (int32_t)S->graphs.size()) return BFS_ENOTFOUND;
  if (src < 0 || (int64_t)src >= S->graphs[graph_id]->g->n) return BFS_EINVAL;
  if (S->inbox.size() >= S->inbox_cap) return BFS_EAGAIN;
  Query* q = new Query();
  q->ticket = S->next_ticket++;
  q->graph = graph_id;
  q->src = src;
  q->user_out = dist_out;
  q->host_out = host_out;
  q->t_submit = now_ns();
  S->tickets[q->ticket] = q;
  S->inbox.push_back(q);
  *ticket = q->ticket;
  S->cv_work.notify_one();
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
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  cudaSetDevice(S->device);
  // Queries never admitted (still queued at shutdown) and completed ones not yet
  // reported are all still registered under their tickets.
  for (GraphEntry* ge : S->graphs) {
    gbfs::serve_group_destroy(ge->grp);
    for (int32_t* b : ge->staging_free) cudaFree(b);
    delete ge;
  }
  for (auto& kv : S->tickets) delete kv.second;
  delete S;
}

}  // extern "C"
