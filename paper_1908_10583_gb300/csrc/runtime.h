// Host-side state of the query engine, shared by capi.cu and server.cu.
#pragma once

#include <cuda_runtime.h>

#include <condition_variable>
#include <functional>
#include <mutex>

#include "fora.h"
#include "fora_engine.cuh"

namespace fora {

// The residual kernels run at most this many blocks (8 per SM on up to 512 SMs), so the
// per-block scan buffers have a size that does not depend on the device.
constexpr int kMaxResidualGrid = 4096;

// Device bytes of every buffer of a query workspace for nsrc sources of a graph with n
// nodes and hub_chunks hub items (workspace_sizes).  The workspace allocates exactly
// these; the server's admission and fora_workspace_bytes count them.
struct WorkspaceSizes {
  size_t N = 0;  // nsrc * n
  size_t r = 0, res = 0, tally = 0, q = 0, fa = 0, hub = 0, small = 0, work = 0, alist = 0,
         slot_cnt = 0, pre = 0, ps = 0, err = 0, sources = 0, rmax = 0, stats = 0, stopped = 0,
         light = 0, tile_dirty = 0, last_edges = 0, blk = 0,
         topk = 0, feat = 0, pred = 0, rmax_learned = 0, out_ids = 0, out_vals = 0;
  size_t total() const;  // q and hub count twice (two parities)
};
WorkspaceSizes workspace_sizes(int64_t n, uint64_t hub_chunks, int nsrc);

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// What an instantiated push-loop graph was built for.
struct PushGraphKey {
  uint64_t generation = 0;
  int nsrc = 0;
  double alpha = 0.0;
  int spread_width = 0;
  int spread_hot = 0;
  uint32_t max_rounds = 0;
  int balance = 0;
  double bal[4] = {0, 0, 0, 0};  // C', cost_edge, cost_push, cost_walk (balanced push)
  bool operator==(const PushGraphKey& o) const {
    return generation == o.generation && nsrc == o.nsrc && alpha == o.alpha &&
           spread_width == o.spread_width && spread_hot == o.spread_hot &&
           max_rounds == o.max_rounds &&
           balance == o.balance && bal[0] == o.bal[0] && bal[1] == o.bal[1] &&
           bal[2] == o.bal[2] && bal[3] == o.bal[3];
  }
};

// Device and pinned host buffers of one in-flight batched query (up to `cap` sources).
// A graph owns one for its own entry points; the server owns one per lane.  A
// workspace serves one call at a time (its mutex).
struct Workspace {
  // workspace for up to `cap` sources
  int cap = 0;
  double* r = nullptr;
  double* res = nullptr;
  Tally* tally = nullptr;
  unsigned long long* q[2] = {nullptr, nullptr};
  unsigned long long* hub[2] = {nullptr, nullptr};
  double* fa = nullptr;
  unsigned long long* small = nullptr;  // counters[4] totals[2]
  unsigned long long* work = nullptr;
  uint32_t* alist = nullptr;      // [nsrc] sources with a non-empty frontier
  uint32_t* slot_cnt = nullptr;   // [4][nsrc] per-source frontier entries and hub items
  unsigned long long* pre = nullptr;  // [2][nsrc + 1] group and hub-item prefixes
  uint32_t* err = nullptr;
  int32_t* sources = nullptr;
  double* rmax = nullptr;
  SlotStats* stats = nullptr;
  uint32_t* stopped = nullptr;        // [nsrc] balanced push: the cost rule stopped the source
  uint8_t* light = nullptr;           // [nsrc] light-round flags of the push take
  uint8_t* tile_dirty = nullptr;      // [nsrc][tiles] tiles a light round's spread touched
  unsigned long long* last_edges = nullptr;  // [nsrc]
  unsigned long long* blk = nullptr;  // [2][residual_grid]
  int residual_grid = 0;
  void* topk_scratch = nullptr;
  float* feat = nullptr;        // learned r_max: features [cap][16], predictions, r_max
  float* pred = nullptr;
  double* rmax_learned = nullptr;
  int32_t* out_ids = nullptr;  // device staging of host-bound results [cap][FORA_MAX_K]
  double* out_vals = nullptr;
  // pinned host mirrors
  unsigned long long* h_counters = nullptr;
  SlotStats* h_stats = nullptr;
  uint32_t* h_err = nullptr;
  int32_t* h_sources = nullptr;
  double* h_rmax = nullptr;
  uint32_t* go_host = nullptr;  // PushState::go of the host-driven push loop
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

  PushState* ps = nullptr;
  uint64_t generation = 0;               // bumped whenever the buffers are reallocated
  cudaGraphExec_t push_exec = nullptr;   // the push rounds as a device-side loop
  PushGraphKey push_key;
  cudaStream_t capture_stream = nullptr; // for capturing the loop body
  std::mutex mu;

  void release() {
    if (push_exec) cudaGraphExecDestroy(push_exec);
    push_exec = nullptr;
    dfree(ps);
    dfree(r); dfree(res); dfree(tally);
    dfree(q[0]); dfree(q[1]); dfree(hub[0]); dfree(hub[1]); dfree(fa);
    dfree(small); dfree(work); dfree(alist); dfree(slot_cnt); dfree(pre); dfree(err); dfree(sources); dfree(rmax); dfree(stats); dfree(stopped); dfree(light); dfree(tile_dirty); dfree(last_edges); dfree(blk);
    if (topk_scratch) cudaFree(topk_scratch);
    topk_scratch = nullptr;
    dfree(out_ids); dfree(out_vals); dfree(feat); dfree(pred); dfree(rmax_learned);
    if (h_counters) cudaFreeHost(h_counters);
    if (h_stats) cudaFreeHost(h_stats);
    if (h_err) cudaFreeHost(h_err);
    if (h_sources) cudaFreeHost(h_sources);
    if (h_rmax) cudaFreeHost(h_rmax);
    if (go_host) cudaFreeHost(go_host);
    h_counters = nullptr; h_stats = nullptr; h_err = nullptr; h_sources = nullptr; h_rmax = nullptr;
    go_host = nullptr;
    cap = 0;
  }
  ~Workspace() {
    release();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    for (int i = 0; i < 5; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
  }
};

}  // namespace fora

namespace fora {

// Ordering between consecutive parts of a pipelined batch: the later part's push waits
// on the device until the earlier part's push is done (so the earlier part's walks run
// beside the later part's push).  The earlier part's host thread records `ev` after
// enqueueing its push and signals; it signals without recording if it stops early.
struct PipeLink {
  std::mutex m;
  std::condition_variable cv;
  bool signalled = false;
  bool recorded = false;
  cudaEvent_t ev = nullptr;
  void signal(bool rec) {
    {
      std::lock_guard<std::mutex> lk(m);
      if (signalled) return;
      signalled = true;
      recorded = rec;
    }
    cv.notify_all();
  }
  bool wait() {  // true if ev was recorded
    std::unique_lock<std::mutex> lk(m);
    cv.wait(lk, [&] { return signalled; });
    return recorded;
  }
};
struct PipeHook {
  PipeLink* before = nullptr;  // wait for this one before the push
  PipeLink* after = nullptr;   // signal this one after enqueueing the push
};
constexpr int kMaxPipeline = 4;

// Admission of further sources while a batch is in its push rounds (the serving lanes):
// the rounds run from a host loop, and after each round `poll` may write up to `room`
// sources to `dst` (HOST) and returns how many; they join the batch as its next slots and
// their queries run exactly as they would alone.  The batch then has *nsrc_final sources
// (outputs and stats are sized for `cap`).
struct JoinHook {
  int cap = 0;
  std::function<int(int32_t* dst, int room)> poll;
  int* nsrc_final = nullptr;
};

}  // namespace fora

struct fora_graph {
  int64_t n = 0, m = 0, max_deg = 0;
  uint64_t hub_chunks = 0;  // sum over nodes with d > kHubChunk of ceil(d / kHubChunk)
  uint32_t* row = nullptr;
  int32_t* col = nullptr;
  uint32_t* colp = nullptr;   // col bit-packed to colbits bits per target (0: not packed)
  int colbits = 0;
  uint32_t* indeg = nullptr;  // in-degrees (features of the learned r_max)
  double* invd = nullptr;     // RN(1 / d(v)) per node
  uint2* rd = nullptr;        // {row[v], d(v)} per node (the walks' node record)
  uint32_t* scol = nullptr;   // the spread's target codes (GraphDev::scol), or null
  uint32_t* hot_node = nullptr;
  int nhot = 0;
  // FORA+ walk index (Section 3.3): ends of omega_max(v) walks from every v
  unsigned long long* idx_off = nullptr;  // [n + 1] exclusive prefix of omega_max
  uint32_t* idx_dest = nullptr;           // [idx_entries] walk ends
  int64_t idx_entries = 0;
  double idx_rmax = 0.0, idx_scale = 0.0, idx_alpha = 0.0;
  uint64_t idx_seed = 0;
  bool idx_zero_hop = false;  // the stored walks are zero-hop walks (Section 4.1)
  int device = 0;
  int num_sms = 0;
  fora::Tuning tune;
  std::mutex mu;              // guards `tune`
  fora::Workspace ws;         // the graph's own entry points
  // parts of a pipelined batch: a workspace and a stream each
  fora::Workspace pipe_ws[fora::kMaxPipeline];
  cudaStream_t pipe_stream[fora::kMaxPipeline] = {};
  fora::GraphDev dev() const {
    return fora::GraphDev{n, m, row, col, colp, colbits, invd, rd, scol, hot_node, nhot};
  }
};

namespace fora {

// Engine entry points (capi.cu).
int report_error(int code, const char* fmt, ...);
struct RmaxSource {
  const double* host = nullptr;
  const double* device = nullptr;
};
// Allocate w for nsrc queries of g now (under w's lock).
int reserve_workspace(fora_graph* g, Workspace* w, int nsrc);
int run_batch_ws(fora_graph* g, Workspace* w, const fora_params* p, const int32_t* sources,
                 int nsrc, int32_t* out_ids, double* out_vals, fora_stats* st,
                 const fora_debug_io* dbg, uint32_t dbg_flags, cudaStream_t stream,
                 RmaxSource rsrc, const PipeHook* hook = nullptr,
                 const fora_balance* bal = nullptr, const JoinHook* join = nullptr);

}  // namespace fora
