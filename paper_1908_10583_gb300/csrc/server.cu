// Serving runtime: continuous batching of SSPPR queries over resident graphs.
//
// Each graph gets `lanes_per_graph` lanes.  A lane owns a workspace sized for its slot
// capacity (the HBM budget divided over the lanes, by the workspace's own buffer sizes
// per query slot: residue, reserve, walk tallies, frontiers), a CUDA stream and a host
// thread.  Requests queue per graph; a free lane admits as many compatible queued
// requests as it has slots (after a short batching window when fewer are waiting) and
// runs them as one batched query on its stream.  While that batch is in its push rounds,
// requests that arrive take the batch's free slots between two rounds (admit_during_push)
// and share its walk phase; while one lane's batch is on the GPU the next arrivals are
// also admitted by another lane, so batches overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fora.h"
#include "fora_engine.cuh"
#include "runtime.h"

using namespace fora;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int graph = 0;
  int32_t source = 0;
  fora_params params{};
  int status = 0;  // 0 queued, 1 running, 2 done, < 0 error code
  std::vector<int32_t> ids;
  std::vector<double> vals;
  fora_request_info info{};
  std::string err;
};

// Requests can share a batch when everything but k agrees (the batch runs with the
// largest k; a smaller k is a prefix of the same order).
bool compatible(const fora_params& a, const fora_params& b) {
  return a.alpha == b.alpha && a.eps == b.eps && a.delta == b.delta && a.pf == b.pf &&
         a.rmax == b.rmax && a.seed == b.seed && a.flags == b.flags;
}

// The most query slots whose workspace (the same buffer sizes the workspace allocates)
// fits `share` bytes, at most `cap`; 0 if not even one fits.
int slots_within(const fora_graph* g, size_t share, int cap) {
  const size_t one = workspace_sizes(g->n, g->hub_chunks, 1).total();
  if (one > share) return 0;
  const size_t per = workspace_sizes(g->n, g->hub_chunks, 2).total() - one;  // linear in slots
  const size_t more = per ? (share - one) / per : (size_t)cap;
  return (int)std::min<size_t>((size_t)cap, 1 + more);
}

}  // namespace

struct Lane {
  int graph = 0;
  int index = 0;
  int cap = 1;
  Workspace ws;
  cudaStream_t stream = nullptr;
  std::thread th;
};

struct fora_server {
  std::vector<fora_graph*> graphs;
  fora_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::deque<uint64_t>> queue;  // per graph
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  std::vector<std::unique_ptr<Lane>> lanes;
  bool stop = false;
  Clock::time_point t0 = Clock::now();
  uint64_t batches = 0, completed = 0, batched_queries = 0, joined = 0;
  int lanes_busy = 0, max_lanes_busy = 0;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }

  void lane_loop(Lane* L) {
    fora_graph* g = graphs[L->graph];
    cudaSetDevice(g->device);
    std::vector<uint64_t> batch;
    std::vector<int32_t> src, ids;
    std::vector<double> vals;
    std::vector<fora_stats> st;
    for (;;) {
      std::unique_lock<std::mutex> lk(mu);
      auto& q = queue[L->graph];
      cv_work.wait(lk, [&] { return stop || !q.empty(); });
      if (stop) return;
      if ((int)q.size() < L->cap && cfg.batch_window_ms > 0)
        cv_work.wait_for(lk, std::chrono::duration<double, std::milli>(cfg.batch_window_ms),
                         [&] { return stop || (int)q.size() >= L->cap; });
      if (stop) return;
      if (q.empty()) continue;
      // admit up to cap compatible requests, oldest first
      batch.clear();
      const fora_params first = reqs[q.front()].params;
      uint32_t kmax = 0;
      for (auto it = q.begin(); it != q.end() && (int)batch.size() < L->cap;) {
        Request& r = reqs[*it];
        if (compatible(r.params, first)) {
          batch.push_back(*it);
          kmax = r.params.k > kmax ? r.params.k : kmax;
          it = q.erase(it);
        } else {
          ++it;
        }
      }
      const double t_start = now_ms();
      src.resize(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) {
        Request& r = reqs[batch[i]];
        r.status = 1;
        r.info.start_ms = t_start;
        src[i] = r.source;
      }
      ++lanes_busy;
      if (lanes_busy > max_lanes_busy) max_lanes_busy = lanes_busy;
      lk.unlock();

      fora_params p = first;
      p.k = kmax;
      p.flags &= ~(FORA_OUT_DEVICE | FORA_ASYNC);
      int nb = (int)batch.size();
      ids.resize((size_t)L->cap * kmax);
      vals.resize((size_t)L->cap * kmax);
      st.resize(L->cap);
      // continuous admission: between two push rounds, compatible requests that arrived
      // meanwhile (k <= the batch's k) take free slots of this batch
      JoinHook hook;
      hook.cap = L->cap;
      hook.nsrc_final = &nb;
      hook.poll = [&](int32_t* dst, int room) {
        std::lock_guard<std::mutex> g2(mu);
        int added = 0;
        const double t_join = now_ms();
        for (auto it = q.begin(); it != q.end() && added < room;) {
          Request& r = reqs[*it];
          if (compatible(r.params, first) && r.params.k <= kmax) {
            r.status = 1;
            r.info.start_ms = t_join;
            r.info.joined = 1;
            dst[added++] = r.source;
            batch.push_back(*it);
            it = q.erase(it);
          } else {
            ++it;
          }
        }
        joined += (uint64_t)added;
        return added;
      };
      const bool admit = cfg.admit_during_push != 0;
      const int rc = run_batch_ws(g, &L->ws, &p, src.data(), nb, ids.data(), vals.data(), st.data(),
                                  nullptr, 0, L->stream, RmaxSource(), nullptr, nullptr,
                                  admit ? &hook : nullptr);
      const std::string err = rc ? fora_last_error() : "";
      const double t_end = now_ms();
      nb = (int)batch.size();

      lk.lock();
      --lanes_busy;
      ++batches;
      batched_queries += nb;
      for (int i = 0; i < nb; ++i) {
        Request& r = reqs[batch[i]];
        r.status = rc ? rc : 2;
        r.info.end_ms = t_end;
        r.info.batch_size = (uint32_t)nb;
        r.info.lane = L->index;
        if (rc) r.err = err;
        if (!rc) {
          const uint32_t k = r.params.k;
          r.ids.assign(ids.begin() + (size_t)i * kmax, ids.begin() + (size_t)i * kmax + k);
          r.vals.assign(vals.begin() + (size_t)i * kmax, vals.begin() + (size_t)i * kmax + k);
          r.info.stats = st[i];
        }
        ++completed;
      }
      cv_done.notify_all();
    }
  }
};

extern "C" {

int fora_server_create(fora_graph* const* graphs, int32_t ngraphs, const fora_server_config* cfg,
                       fora_server** out) {
  if (!out || !graphs || ngraphs < 1 || !cfg) return report_error(FORA_ERR_BAD_ARG, "bad arguments");
  *out = nullptr;
  if (cfg->lanes_per_graph < 1 || cfg->max_batch < 1 || cfg->max_batch > 65535)
    return report_error(FORA_ERR_BAD_ARG, "lanes_per_graph and max_batch must be >= 1");
  for (int i = 0; i < ngraphs; ++i)
    if (!graphs[i]) return report_error(FORA_ERR_BAD_ARG, "null graph %d", i);
  auto s = std::make_unique<fora_server>();
  s->graphs.assign(graphs, graphs + ngraphs);
  s->cfg = *cfg;
  s->queue.resize(ngraphs);
  size_t budget = cfg->memory_budget_bytes;
  if (budget == 0) {  // 80% of the free device memory
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
      return report_error(FORA_ERR_CUDA, "cannot query free device memory");
    budget = free_b / 10 * 8;
  }
  // admission by HBM footprint: each lane gets an equal share of the budget and as many
  // query slots as that share holds
  const size_t share = budget / ((size_t)ngraphs * cfg->lanes_per_graph);
  for (int gi = 0; gi < ngraphs; ++gi) {
    const int slots = slots_within(graphs[gi], share, cfg->max_batch);
    if (slots < 1)
      return report_error(FORA_ERR_OOM, "memory budget too small for one query of graph %d", gi);
    for (int l = 0; l < cfg->lanes_per_graph; ++l) {
      auto L = std::make_unique<Lane>();
      L->graph = gi;
      L->index = (int)s->lanes.size();
      L->cap = slots;
      if (cudaSetDevice(graphs[gi]->device) != cudaSuccess ||
          cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess)
        return report_error(FORA_ERR_CUDA, "cannot create a lane stream");
      const int rc = reserve_workspace(graphs[gi], &L->ws, L->cap);  // the lane's HBM, up front
      if (rc) {
        cudaStreamDestroy(L->stream);
        for (auto& M : s->lanes) cudaStreamDestroy(M->stream);
        return rc;
      }
      s->lanes.push_back(std::move(L));
    }
  }
  fora_server* srv = s.release();
  for (auto& L : srv->lanes) {
    Lane* lp = L.get();
    lp->th = std::thread([srv, lp] { srv->lane_loop(lp); });
  }
  *out = srv;
  return FORA_OK;
}

void fora_server_destroy(fora_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& L : s->lanes) {
    if (L->th.joinable()) L->th.join();
    cudaSetDevice(s->graphs[L->graph]->device);
    {
      std::lock_guard<std::mutex> wl(L->ws.mu);
      L->ws.release();
    }
    if (L->stream) cudaStreamDestroy(L->stream);
  }
  delete s;
}

int fora_server_lane_capacity(const fora_server* s, int32_t lane, int32_t* graph, int32_t* slots) {
  if (!s || lane < 0 || lane >= (int32_t)s->lanes.size()) return report_error(FORA_ERR_BAD_ARG, "bad lane");
  if (graph) *graph = s->lanes[lane]->graph;
  if (slots) *slots = s->lanes[lane]->cap;
  return FORA_OK;
}

int fora_server_submit(fora_server* s, int32_t graph, int32_t source, const fora_params* params,
                       uint64_t* ticket) {
  if (!s || !params || !ticket) return report_error(FORA_ERR_BAD_ARG, "bad arguments");
  if (graph < 0 || graph >= (int32_t)s->graphs.size()) return report_error(FORA_ERR_BAD_ARG, "bad graph index");
  const fora_graph* g = s->graphs[graph];
  if (source < 0 || source >= g->n) return report_error(FORA_ERR_BAD_ARG, "source out of range");
  if (params->k < 1 || params->k > FORA_MAX_K || (int64_t)params->k > g->n)
    return report_error(FORA_ERR_BAD_ARG, "k out of range");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.graph = graph;
    r.source = source;
    r.params = *params;
    r.info.submit_ms = s->now_ms();
    s->queue[graph].push_back(t);
    *ticket = t;
  }
  s->cv_work.notify_all();
  return FORA_OK;
}

int fora_server_wait(fora_server* s, uint64_t ticket, double timeout_ms, int32_t* out_ids,
                     double* out_vals, fora_request_info* info) {
  if (!s) return report_error(FORA_ERR_BAD_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return report_error(FORA_ERR_BAD_ARG, "unknown ticket");
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] {
    auto jt = s->reqs.find(ticket);
    return jt->second.status == 2 || jt->second.status < 0;
  });
  if (!ok) return report_error(FORA_ERR_TIMEOUT, "request %llu not finished within %.1f ms",
                               (unsigned long long)ticket, timeout_ms);
  Request& r = s->reqs.find(ticket)->second;
  const int status = r.status;
  const std::string err = r.err;
  if (status == 2) {
    if (out_ids) memcpy(out_ids, r.ids.data(), r.ids.size() * sizeof(int32_t));
    if (out_vals) memcpy(out_vals, r.vals.data(), r.vals.size() * sizeof(double));
    if (info) *info = r.info;
  }
  s->reqs.erase(ticket);
  if (status < 0) return report_error(status, "request failed: %s", err.c_str());
  return FORA_OK;
}

int fora_server_stats(fora_server* s, uint64_t* completed, uint64_t* batches, int32_t* max_concurrent,
                      uint64_t* joined) {
  if (!s) return report_error(FORA_ERR_BAD_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (batches) *batches = s->batches;
  if (max_concurrent) *max_concurrent = s->max_lanes_busy;
  if (joined) *joined = s->joined;
  return FORA_OK;
}

}  // extern "C"
