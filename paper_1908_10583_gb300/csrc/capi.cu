// C ABI (include/fora.h) and the host side of the query engine: graph residency,
// the per-graph workspace, and the phase sequence of a (batched) query.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fora.h"
#include "fora_engine.cuh"
#include "runtime.h"

using namespace fora;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? FORA_ERR_OOM : FORA_ERR_CUDA,        \
                  "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,      \
                  __LINE__);                                                             \
  } while (0)

}  // namespace

int fora::report_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

namespace {

std::mutex g_occ_mu;
std::map<std::pair<int, const void*>, int> g_occ;  // (device, kernel) -> blocks per SM

// fora_debug_fail_alloc: allocations left before the one that is made to fail (0: off)
std::atomic<long long> g_fail_alloc_in{0};

}  // namespace

int fora::resident_blocks(const void* kernel, int threads) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(g_occ_mu);
  const auto key = std::make_pair(dev, kernel);
  const auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
    return 0;
  if (per_sm < 1) per_sm = 1;
  g_occ[key] = per_sm;
  return per_sm;
}

cudaError_t fora::device_alloc(void** p, size_t bytes) {
  long long left = g_fail_alloc_in.load();
  while (left > 0) {
    if (g_fail_alloc_in.compare_exchange_weak(left, left - 1)) {
      if (left == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

fora::WorkspaceSizes fora::workspace_sizes(int64_t n, uint64_t hub_chunks, int nsrc) {
  WorkspaceSizes z;
  const size_t S = (size_t)nsrc;
  z.N = S * (size_t)n;
  const size_t H = S * hub_chunks + 1;
  z.r = z.N * sizeof(double);
  z.res = z.N * sizeof(double);
  z.tally = z.N * sizeof(Tally);
  z.q = (z.N + 1) * sizeof(unsigned long long);
  z.fa = (z.N + 1) * sizeof(double);
  z.hub = H * sizeof(unsigned long long);
  z.small = 8 * sizeof(unsigned long long);
  z.work = 32 * sizeof(unsigned long long);
  z.alist = S * sizeof(uint32_t);
  z.slot_cnt = 4 * S * sizeof(uint32_t);
  z.pre = 2 * (S + 1) * sizeof(unsigned long long);
  z.ps = sizeof(PushState);
  z.err = sizeof(uint32_t);
  z.sources = S * sizeof(int32_t);
  z.rmax = S * sizeof(double);
  z.stats = S * sizeof(SlotStats);
  z.stopped = S * sizeof(uint32_t);
  z.light = S;
  z.tile_dirty = S * (((size_t)n + kTakeTile - 1) / kTakeTile);
  z.last_edges = S * sizeof(unsigned long long);
  z.blk = 2 * (size_t)kMaxResidualGrid * sizeof(unsigned long long);
  z.topk = topk_scratch_bytes(nsrc);
  z.feat = S * FORA_NUM_FEATURES * sizeof(float);
  z.pred = S * sizeof(float);
  z.rmax_learned = S * sizeof(double);
  z.out_ids = S * FORA_MAX_K * sizeof(int32_t);
  z.out_vals = S * FORA_MAX_K * sizeof(double);
  return z;
}

size_t fora::WorkspaceSizes::total() const {
  return r + res + tally + 2 * q + fa + 2 * hub + small + work + alist + slot_cnt + pre + ps +
         err + sources + rmax + stats + stopped + light + tile_dirty + last_edges + blk + topk +
         feat + pred + rmax_learned + out_ids + out_vals;
}

namespace {

// NVTX ranges (shown by profilers that record them, no effect otherwise): one per batched
// call, and one per phase inside it; `next` closes the open phase and opens another.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
struct NvtxPhases {
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhases() {
    if (open) nvtxRangePop();
  }
};

template <typename T>
cudaError_t dalloc(T** p, size_t bytes) {
  return device_alloc(reinterpret_cast<void**>(p), bytes);
}

int ensure_workspace(fora_graph* g, Workspace* w, int nsrc) {
  if (nsrc <= w->cap) return FORA_OK;
  w->release();
  const WorkspaceSizes z = workspace_sizes(g->n, g->hub_chunks, nsrc);
  // hub items hold a queue index in their upper 64 - kHubChunkBits bits
  if (z.N >= (1ull << (64 - kHubChunkBits)))
    return fail(FORA_ERR_BAD_ARG, "%d sources x %lld nodes exceed the queue index range", nsrc,
                (long long)g->n);
  w->residual_grid = std::min(g->num_sms * 8, kMaxResidualGrid);
  CUDA_TRY(dalloc(&w->r, z.r));
  CUDA_TRY(dalloc(&w->res, z.res));
  CUDA_TRY(dalloc(&w->tally, z.tally));
  CUDA_TRY(dalloc(&w->q[0], z.q));
  CUDA_TRY(dalloc(&w->q[1], z.q));
  CUDA_TRY(dalloc(&w->fa, z.fa));
  CUDA_TRY(dalloc(&w->hub[0], z.hub));
  CUDA_TRY(dalloc(&w->hub[1], z.hub));
  CUDA_TRY(dalloc(&w->small, z.small));
  CUDA_TRY(dalloc(&w->work, z.work));
  CUDA_TRY(dalloc(&w->alist, z.alist));
  CUDA_TRY(dalloc(&w->slot_cnt, z.slot_cnt));
  CUDA_TRY(dalloc(&w->pre, z.pre));
  CUDA_TRY(dalloc(&w->ps, z.ps));
  if (!w->capture_stream) CUDA_TRY(cudaStreamCreateWithFlags(&w->capture_stream, cudaStreamNonBlocking));
  CUDA_TRY(dalloc(&w->err, z.err));
  CUDA_TRY(dalloc(&w->sources, z.sources));
  CUDA_TRY(dalloc(&w->rmax, z.rmax));
  CUDA_TRY(dalloc(&w->stats, z.stats));
  CUDA_TRY(dalloc(&w->stopped, z.stopped));
  CUDA_TRY(dalloc(&w->light, z.light));
  CUDA_TRY(dalloc(&w->tile_dirty, z.tile_dirty));
  CUDA_TRY(dalloc(&w->last_edges, z.last_edges));
  CUDA_TRY(dalloc(&w->blk, z.blk));
  CUDA_TRY(dalloc(&w->topk_scratch, z.topk));
  CUDA_TRY(dalloc(&w->feat, z.feat));
  CUDA_TRY(dalloc(&w->pred, z.pred));
  CUDA_TRY(dalloc(&w->rmax_learned, z.rmax_learned));
  CUDA_TRY(dalloc(&w->out_ids, z.out_ids));
  CUDA_TRY(dalloc(&w->out_vals, z.out_vals));
  CUDA_TRY(cudaMallocHost(&w->h_counters, 8 * sizeof(unsigned long long)));
  CUDA_TRY(cudaMallocHost(&w->h_stats, nsrc * sizeof(SlotStats)));
  CUDA_TRY(cudaMallocHost(&w->h_err, sizeof(uint32_t)));
  CUDA_TRY(cudaMallocHost(&w->h_sources, nsrc * sizeof(int32_t)));
  CUDA_TRY(cudaMallocHost(&w->h_rmax, nsrc * sizeof(double)));
  CUDA_TRY(cudaMallocHost(&w->go_host, sizeof(uint32_t)));
  for (int i = 0; i < 5; ++i)
    if (!w->ev[i]) CUDA_TRY(cudaEventCreate(&w->ev[i]));
  w->cap = nsrc;
  ++w->generation;
  return FORA_OK;
}

// The ten Philox4x32-10 round keys of a 64-bit seed (Salmon et al.: the key (lo, hi) is
// bumped by (0x9E3779B9, 0xBB67AE85) after every round), kept in the kernel parameters so
// that the walk kernels read them as constants.
void set_round_keys(BatchDev* b, uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int i = 0; i < 10; ++i) {
    b->round_key[i] = make_uint2(k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Parameters as a query resolves them (Alg. 2; Eq. rmax and Case 2, Section 3.2).
struct Resolved {
  double alpha, eps, delta, pf, rmax, walk_scale;
  uint32_t alpha_threshold;
};

int resolve(const fora_graph* g, const fora_params* p, Resolved* out) {
  if (!g || !p) return fail(FORA_ERR_BAD_ARG, "null graph or params");
  Resolved r;
  r.alpha = p->alpha;
  r.eps = p->eps;
  r.delta = p->delta > 0 ? p->delta : 1.0 / (double)g->n;
  r.pf = p->pf > 0 ? p->pf : 1.0 / (double)g->n;
  if (!(r.alpha > 0.0 && r.alpha < 1.0)) return fail(FORA_ERR_BAD_ARG, "alpha must be in (0,1)");
  if (!(r.eps > 0.0) || !std::isfinite(r.eps)) return fail(FORA_ERR_BAD_ARG, "eps must be > 0");
  if (!(r.delta <= 1.0)) return fail(FORA_ERR_BAD_ARG, "delta must be in (0,1]");
  if (!(r.pf < 1.0)) return fail(FORA_ERR_BAD_ARG, "pf must be in (0,1)");
  const double m = (double)g->m;
  // C = omega / r_sum = (2 eps/3 + 2) log(2/p_f) / (eps^2 delta)
  r.walk_scale = ((2.0 * r.eps / 3.0 + 2.0) * log(2.0 / r.pf)) / (r.eps * r.eps * r.delta);
  if (p->rmax > 0.0) {
    r.rmax = p->rmax;
  } else {
    r.rmax = (r.eps / sqrt(m)) * sqrt(r.delta / ((2.0 * r.eps / 3.0 + 2.0) * log(2.0 / r.pf)));
    if (m * r.rmax > 1.0)
      r.rmax = (r.eps * r.eps * r.delta) / ((2.0 * r.eps / 3.0 + 2.0) * log(2.0 / r.pf));
  }
  if (!std::isfinite(r.walk_scale) || !std::isfinite(r.rmax))
    return fail(FORA_ERR_BAD_ARG, "parameters give a non-finite r_max or walk count");
  r.alpha_threshold = (uint32_t)floor(r.alpha * 4294967296.0);
  *out = r;
  return FORA_OK;
}

}  // namespace

namespace {

// The push rounds as a CUDA graph: one conditional while-node whose body is a round
// (spread, detect, scan, emit, advance); the advance kernel sets the loop condition.
// The instantiated graph is kept in the workspace and rebuilt when the workspace, the
// number of sources, alpha or the launch shape change.
int push_loop_graph(fora_graph* g, Workspace* w, const GraphDev& gd, const BatchDev& b) {
  PushGraphKey key;
  key.generation = w->generation;
  key.nsrc = b.nsrc;
  key.alpha = b.alpha;
  key.spread_width = b.spread_width;
  key.spread_hot = b.spread_hot;
  key.max_rounds = b.max_rounds;
  key.balance = b.balance;
  key.bal[0] = b.bal_scale;
  key.bal[1] = b.cost_edge;
  key.bal[2] = b.cost_push;
  key.bal[3] = b.cost_walk;
  if (w->push_exec && key == w->push_key) return FORA_OK;
  if (w->push_exec) {
    cudaGraphExecDestroy(w->push_exec);
    w->push_exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle loop;
  cudaGraphNode_t node;
  cudaGraphNodeParams np{};
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(w->capture_stream, np.conditional.phGraph_out[0], nullptr,
                                      nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const cudaError_t le = launch_push_body(gd, b, g->num_sms, loop, true, w->capture_stream);
    e = cudaStreamEndCapture(w->capture_stream, &captured);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&w->push_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    w->push_exec = nullptr;
    return fail(FORA_ERR_CUDA, "push loop graph: %s", cudaGetErrorString(e));
  }
  w->push_key = key;
  return FORA_OK;
}

}  // namespace

int fora::reserve_workspace(fora_graph* g, Workspace* w, int nsrc) {
  std::lock_guard<std::mutex> lock(w->mu);
  CUDA_TRY(cudaSetDevice(g->device));
  return ensure_workspace(g, w, nsrc);
}

// One batched query on workspace w (the whole phase sequence of include/fora.h).
int fora::run_batch_ws(fora_graph* g, Workspace* w, const fora_params* p,
                       const int32_t* sources, int nsrc, int32_t* out_ids, double* out_vals,
                       fora_stats* st, const fora_debug_io* dbg, uint32_t dbg_flags,
                       cudaStream_t stream, RmaxSource rsrc, const PipeHook* hook,
                       const fora_balance* bal, const JoinHook* join) {
  // a pipelined part always signals the next part, also when it stops early
  struct SignalOnExit {
    PipeLink* link;
    ~SignalOnExit() {
      if (link) link->signal(false);
    }
  } signal_on_exit{hook ? hook->after : nullptr};
  Resolved rp;
  int rc = resolve(g, p, &rp);
  if (rc) return rc;
  if (nsrc < 1 || !sources) return fail(FORA_ERR_BAD_ARG, "need at least one source");
  if (nsrc > 65535) return fail(FORA_ERR_BAD_ARG, "at most 65535 sources per call");
  if (p->k > FORA_MAX_K || (int64_t)p->k > g->n) return fail(FORA_ERR_BAD_ARG, "k out of range");
  if (p->k > 0 && (!out_ids || !out_vals)) return fail(FORA_ERR_BAD_ARG, "null output");
  const bool out_dev = (p->flags & FORA_OUT_DEVICE) != 0;
  const bool async = (p->flags & FORA_ASYNC) != 0;
  if (async && (!out_dev || st)) return fail(FORA_ERR_BAD_ARG, "FORA_ASYNC needs FORA_OUT_DEVICE and no stats");
  const bool indexed = (p->flags & FORA_USE_INDEX) != 0;
  if (indexed) {
    if (!g->idx_dest) return fail(FORA_ERR_BAD_ARG, "FORA_USE_INDEX without a walk index (fora_index_build)");
    if (((p->flags & FORA_ZERO_HOP) != 0) != g->idx_zero_hop)
      return fail(FORA_ERR_BAD_ARG, g->idx_zero_hop ? "the walk index holds zero-hop walks: FORA_USE_INDEX needs FORA_ZERO_HOP"
                                                    : "the walk index holds plain walks: FORA_USE_INDEX excludes FORA_ZERO_HOP");
    if (rp.walk_scale != g->idx_scale || rp.alpha != g->idx_alpha)
      return fail(FORA_ERR_BAD_ARG, "the walk index was built for other alpha / eps / delta / p_f");
  }
  if (!bal && dbg) bal = dbg->balance;
  if (join && (join->cap < nsrc || join->cap > 65535 || bal || dbg || !join->poll))
    return fail(FORA_ERR_BAD_ARG, "a joining batch needs cap >= nsrc and no balance or debug");
  if (bal) {
    if (!(bal->edge_push >= 0.0) || !(bal->push >= 0.0) || !(bal->walk >= 0.0) ||
        !std::isfinite(bal->edge_push) || !std::isfinite(bal->push) || !std::isfinite(bal->walk))
      return fail(FORA_ERR_BAD_ARG, "balance costs must be finite and >= 0");
    if (indexed) return fail(FORA_ERR_BAD_ARG, "FORA_USE_INDEX cannot serve the balanced push");
  }
  const bool given = (dbg_flags & FORA_DBG_GIVEN_PUSH) != 0;
  if (given && (!dbg || !dbg->reserve || !dbg->residue))
    return fail(FORA_ERR_BAD_ARG, "FORA_DBG_GIVEN_PUSH needs reserve and residue arrays");
  for (int i = 0; i < nsrc; ++i)
    if (sources[i] < 0 || sources[i] >= g->n) return fail(FORA_ERR_BAD_ARG, "source %d out of range", i);

  std::lock_guard<std::mutex> lock(w->mu);
  CUDA_TRY(cudaSetDevice(g->device));
  rc = ensure_workspace(g, w, join ? join->cap : nsrc);
  if (rc) return rc;
  size_t N = (size_t)nsrc * (size_t)g->n;
  for (int i = 0; i < nsrc; ++i) {
    w->h_sources[i] = sources[i];
    w->h_rmax[i] = bal ? 1.0 : rsrc.host ? rsrc.host[i] : rp.rmax;
    if (!(w->h_rmax[i] > 0.0) || !std::isfinite(w->h_rmax[i]))
      return fail(FORA_ERR_BAD_ARG, "r_max of source %d must be positive and finite", i);
    if (indexed && !rsrc.device && w->h_rmax[i] > g->idx_rmax)
      return fail(FORA_ERR_BAD_ARG, "r_max of source %d is above the walk index's r_max", i);
  }
  CUDA_TRY(cudaMemcpyAsync(w->sources, w->h_sources, nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  if (rsrc.device)
    CUDA_TRY(cudaMemcpyAsync(w->rmax, rsrc.device, nsrc * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  else
    CUDA_TRY(cudaMemcpyAsync(w->rmax, w->h_rmax, nsrc * sizeof(double), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemsetAsync(w->tally, 0, N * sizeof(Tally), stream));
  CUDA_TRY(cudaMemsetAsync(w->small, 0, 8 * sizeof(unsigned long long), stream));
  CUDA_TRY(cudaMemsetAsync(w->err, 0, sizeof(uint32_t), stream));
  CUDA_TRY(cudaMemsetAsync(w->stats, 0, nsrc * sizeof(SlotStats), stream));

  const GraphDev gd = g->dev();
  const size_t n64 = (size_t)g->n;
  BatchDev b{};
  b.nsrc = nsrc;
  b.alpha = rp.alpha;
  b.walk_scale = rp.walk_scale;
  b.alpha_threshold = rp.alpha_threshold;
  b.seed = p->seed;
  set_round_keys(&b, p->seed);
  b.zero_hop = (p->flags & FORA_ZERO_HOP) != 0;
  b.want_count = dbg && dbg->count;
  b.r = w->r; b.res = w->res; b.tally = w->tally;
  b.q[0] = w->q[0]; b.q[1] = w->q[1]; b.fa = w->fa;
  b.hub[0] = w->hub[0]; b.hub[1] = w->hub[1];
  b.hub_stride = g->hub_chunks;
  b.slot_cnt = w->slot_cnt;
  b.cnt_stride = w->cap;
  b.gpre = w->pre;
  b.hpre = w->pre + (w->cap + 1);
  b.alist = w->alist;
  b.work = w->work;
  b.ps = w->ps;
  b.totals = w->small + 4;
  b.sources = w->sources; b.rmax = w->rmax; b.stats = w->stats; b.err = w->err;
  b.wr_entry = w->q[0];
  b.wr_offset = w->q[1];
  b.wr_weight = reinterpret_cast<unsigned long long*>(w->fa);
  b.blk_cnt = w->blk;
  b.blk_walks = w->blk + w->residual_grid;
  b.residual_grid = w->residual_grid;
  b.theta = w->rmax;
  b.stopped = w->stopped;
  b.light = w->light;
  b.tile_dirty = w->tile_dirty;
  b.last_edges = w->last_edges;
  b.tiles = ((unsigned long long)g->n + kTakeTile - 1) / kTakeTile;
  // a frontier whose spread touches at most about half of a source's tiles
  b.light_edges = b.tiles / 2;
  if (bal) {
    b.balance = 1;
    b.bal_scale = b.zero_hop ? (1.0 - rp.alpha) * rp.walk_scale : rp.walk_scale;
    b.cost_edge = bal->edge_push;
    b.cost_push = bal->push;
    b.cost_walk = bal->walk;
  }
  bool host_loop;
  {
    std::lock_guard<std::mutex> tlock(g->mu);
    b.spread_width = g->tune.spread_width;
    b.spread_hot = (g->tune.spread_hot != 0 && g->nhot > 0) ? 1 : 0;
    b.walk_blocks = g->tune.walk_blocks;
    b.max_rounds = g->tune.max_push_rounds;
    host_loop = g->tune.push_host_loop != 0;
  }

  if (hook && hook->before && hook->before->wait())  // the earlier part's push is done
    CUDA_TRY(cudaStreamWaitEvent(stream, hook->before->ev, 0));
  NvtxRange nvtx_call("fora: batched query");
  NvtxPhases nvtx_phase;
  nvtx_phase.next("fora: push");
  const bool timed = st != nullptr;
  if (timed) CUDA_TRY(cudaEventRecord(w->ev[0], stream));

  // ---- push (Alg. 1) ----
  if (given) {
    CUDA_TRY(cudaMemcpyAsync(w->res, dbg->reserve, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    CUDA_TRY(cudaMemcpyAsync(w->r, dbg->residue, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  } else {
    CUDA_TRY(cudaMemsetAsync(w->r, 0, N * sizeof(double), stream));
    CUDA_TRY(cudaMemsetAsync(w->res, 0, N * sizeof(double), stream));
    CUDA_TRY(cudaMemsetAsync(w->work, 0, 32 * sizeof(unsigned long long), stream));
    CUDA_TRY(cudaMemsetAsync(w->slot_cnt, 0, 4 * (size_t)w->cap * sizeof(uint32_t), stream));
    CUDA_TRY(cudaMemsetAsync(w->tile_dirty, 0, (size_t)w->cap * b.tiles, stream));
    CUDA_TRY(cudaMemsetAsync(w->last_edges, 0, (size_t)w->cap * sizeof(unsigned long long), stream));
    CUDA_TRY(launch_push_seed(gd, b, stream));
    if (join) {
      // rounds from a host loop; after each round further sources may join as new slots
      uint32_t go = 1;
      while (go) {
        CUDA_TRY(launch_push_body(gd, b, g->num_sms, 0, false, stream));
        CUDA_TRY(cudaMemcpyAsync(w->go_host, &w->ps->go, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                 stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        go = *w->go_host;
        const int room = join->cap - b.nsrc;
        const int k = room > 0 ? join->poll(w->h_sources + b.nsrc, room) : 0;
        if (k <= 0) continue;
        const int first = b.nsrc;
        for (int i = first; i < first + k; ++i) w->h_rmax[i] = rp.rmax;
        CUDA_TRY(cudaMemcpyAsync(w->sources + first, w->h_sources + first, k * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(w->rmax + first, w->h_rmax + first, k * sizeof(double),
                                 cudaMemcpyHostToDevice, stream));
        const size_t off = (size_t)first * n64, len = (size_t)k * n64;
        CUDA_TRY(cudaMemsetAsync(w->r + off, 0, len * sizeof(double), stream));
        CUDA_TRY(cudaMemsetAsync(w->res + off, 0, len * sizeof(double), stream));
        CUDA_TRY(cudaMemsetAsync(w->tally + off, 0, len * sizeof(Tally), stream));
        CUDA_TRY(cudaMemsetAsync(w->stats + first, 0, k * sizeof(SlotStats), stream));
        b.nsrc = first + k;
        CUDA_TRY(launch_push_join(gd, b, first, k, stream));
        go = 1;
      }
      nsrc = b.nsrc;
      N = (size_t)nsrc * n64;
      if (join->nsrc_final) *join->nsrc_final = nsrc;
    } else if (host_loop) {
      // the same round kernels launched one round at a time from the host (for profilers
      // that cannot look inside conditional graph nodes); one host round trip per round
      uint32_t go = 1;
      while (go) {
        CUDA_TRY(launch_push_body(gd, b, g->num_sms, 0, false, stream));
        CUDA_TRY(cudaMemcpyAsync(w->go_host, &w->ps->go, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                 stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        go = *w->go_host;
      }
    } else {
      // the rounds run as a device-side while loop (no host round trip per round)
      rc = push_loop_graph(g, w, gd, b);
      if (rc) return rc;
      CUDA_TRY(cudaGraphLaunch(w->push_exec, stream));
    }
    if (dbg && dbg->reserve)
      CUDA_TRY(cudaMemcpyAsync(dbg->reserve, w->res, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    if (dbg && dbg->residue)
      CUDA_TRY(cudaMemcpyAsync(dbg->residue, w->r, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  }
  if (timed) CUDA_TRY(cudaEventRecord(w->ev[1], stream));
  if (hook && hook->after) {
    CUDA_TRY(cudaEventRecord(hook->after->ev, stream));
    hook->after->signal(true);
  }

  // ---- walks (Alg. 2) ----
  nvtx_phase.next("fora: walks");
  CUDA_TRY(launch_residuals(gd, b, stream));
  if (timed) CUDA_TRY(cudaEventRecord(w->ev[2], stream));
  if (indexed)
    CUDA_TRY(launch_walks_indexed(gd, b, g->num_sms, g->idx_off, g->idx_dest, stream));
  else
    CUDA_TRY(launch_walks(gd, b, g->num_sms, stream));
  if (timed) CUDA_TRY(cudaEventRecord(w->ev[3], stream));
  if (dbg && (dbg->count || dbg->acc))
    CUDA_TRY(launch_unpack_tally(w->tally, dbg->count, reinterpret_cast<unsigned long long*>(dbg->acc), N,
                                 g->num_sms, stream));

  // ---- estimate and top-k (the residue array becomes the estimate) ----
  nvtx_phase.next("fora: estimate and top-k");
  CUDA_TRY(launch_estimate(w->res, w->tally, w->r, w->r, rp.alpha, b.zero_hop, N, g->num_sms, stream));
  if (dbg && dbg->estimate)
    CUDA_TRY(cudaMemcpyAsync(dbg->estimate, w->r, N * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  int32_t* ids_dev = out_dev ? out_ids : w->out_ids;
  double* vals_dev = out_dev ? out_vals : w->out_vals;
  CUDA_TRY(launch_topk(w->r, g->n, nsrc, p->k, ids_dev, vals_dev,
                       topk_scratch_carve(w->topk_scratch, nsrc), g->num_sms, stream));
  if (timed) CUDA_TRY(cudaEventRecord(w->ev[4], stream));
  if (!out_dev && p->k > 0) {
    CUDA_TRY(cudaMemcpyAsync(out_ids, w->out_ids, (size_t)nsrc * p->k * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(out_vals, w->out_vals, (size_t)nsrc * p->k * sizeof(double), cudaMemcpyDeviceToHost, stream));
  }
  if (async) return FORA_OK;
  CUDA_TRY(cudaMemcpyAsync(w->h_err, w->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  if (st) CUDA_TRY(cudaMemcpyAsync(w->h_stats, w->stats, nsrc * sizeof(SlotStats), cudaMemcpyDeviceToHost, stream));
  if (st && (rsrc.device || bal))  // the thresholds used were set on the device
    CUDA_TRY(cudaMemcpyAsync(w->h_rmax, w->rmax, nsrc * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (*w->h_err & kErrPushNotConverged)
    return fail(FORA_ERR_PUSH_NOT_CONVERGED, "push did not converge in %u rounds", b.max_rounds);
  if (*w->h_err & kErrWalkOverflow) return fail(FORA_ERR_WALK_OVERFLOW, "a source needs 2^32 or more walks");
  if (*w->h_err & kErrWalkCap) return fail(FORA_ERR_WALK_CAP, "a walk exceeded %d moves", FORA_MAX_WALK_STEPS);
  if (*w->h_err & kErrBounds)
    return fail(FORA_ERR_BOUNDS, "a device index check failed (this is a FORA_DEBUG build)");
  if (*w->h_err & kErrIndexRange)
    return fail(FORA_ERR_BAD_ARG, "a residue needs more walks than the walk index holds (r_max above the index's)");
  if (st) {
    float ms[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) CUDA_TRY(cudaEventElapsedTime(&ms[i], w->ev[i], w->ev[i + 1]));
    for (int i = 0; i < nsrc; ++i) {
      const SlotStats& s = w->h_stats[i];
      fora_stats& o = st[i];
      o.rmax = w->h_rmax[i];
      o.rsum = s.rsum;
      o.pushes = s.pushes;
      o.edge_pushes = s.edge_pushes;
      o.residual_nodes = s.residual_nodes;
      o.walks = s.walks;
      o.walk_steps = s.walk_steps;
      o.push_rounds = s.rounds;
      o.source = w->h_sources[i];
      o.ms_push = ms[0];
      o.ms_residual = ms[1];
      o.ms_walk = ms[2];
      o.ms_topk = ms[3];
    }
  }
  return FORA_OK;
}

namespace {

// A batch in `parts` parts, each on its own workspace and stream, driven by its own host
// thread; part k's push waits for part k-1's push to finish, so part k-1's walks (bound
// by instruction issue) run beside part k's push (bound by L2 reductions).  The caller's
// stream waits for every part, so work queued on it afterwards sees the results.
constexpr int kMinPartSources = 32;

int run_batch_pipelined(fora_graph* g, const fora_params* p, const int32_t* sources, int nsrc,
                        int32_t* out_ids, double* out_vals, fora_stats* st, cudaStream_t stream,
                        RmaxSource rsrc, int parts, const fora_balance* bal) {
  CUDA_TRY(cudaSetDevice(g->device));
  {
    std::lock_guard<std::mutex> lock(g->mu);
    for (int k = 0; k < parts; ++k)
      if (!g->pipe_stream[k])
        CUDA_TRY(cudaStreamCreateWithFlags(&g->pipe_stream[k], cudaStreamNonBlocking));
  }
  cudaEvent_t start = nullptr;
  CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  std::vector<PipeLink> links(parts);
  std::vector<cudaEvent_t> ends(parts, nullptr);
  cudaError_t e = cudaEventRecord(start, stream);
  for (int k = 0; k < parts && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&links[k].ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ends[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->pipe_stream[k], start, 0);
  }
  std::vector<int> rcs(parts, FORA_OK);
  std::vector<std::string> errs(parts);
  if (e == cudaSuccess) {
    std::vector<std::thread> th;
    const int k_out = p->k;
    for (int k = 0; k < parts; ++k) {
      const int lo = (int)((int64_t)nsrc * k / parts), hi = (int)((int64_t)nsrc * (k + 1) / parts);
      try {
        th.emplace_back([&, k, lo, hi] {
          PipeHook hook{k > 0 ? &links[k - 1] : nullptr, k + 1 < parts ? &links[k] : nullptr};
          RmaxSource rs;
          rs.host = rsrc.host ? rsrc.host + lo : nullptr;
          rs.device = rsrc.device ? rsrc.device + lo : nullptr;
          if (cudaSetDevice(g->device) != cudaSuccess) {
            if (hook.after) hook.after->signal(false);
            rcs[k] = FORA_ERR_CUDA;
            errs[k] = "cudaSetDevice failed in a pipeline part";
            return;
          }
          rcs[k] = run_batch_ws(g, &g->pipe_ws[k], p, sources + lo, hi - lo,
                                out_ids ? out_ids + (size_t)lo * k_out : nullptr,
                                out_vals ? out_vals + (size_t)lo * k_out : nullptr,
                                st ? st + lo : nullptr, nullptr, 0, g->pipe_stream[k], rs, &hook,
                                bal);
          if (rcs[k]) errs[k] = g_err;
        });
      } catch (...) {  // no thread for part k: release every waiter, run no further part
        for (auto& l : links) l.signal(false);
        rcs[k] = FORA_ERR_CUDA;
        errs[k] = "could not start a host thread for a pipeline part";
        break;
      }
    }
    for (auto& t : th) t.join();
    for (int k = 0; k < parts && e == cudaSuccess; ++k) {
      e = cudaEventRecord(ends[k], g->pipe_stream[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ends[k], 0);
    }
  }
  cudaEventDestroy(start);
  for (int k = 0; k < parts; ++k) {
    if (links[k].ev) cudaEventDestroy(links[k].ev);
    if (ends[k]) cudaEventDestroy(ends[k]);
  }
  for (int k = 0; k < parts; ++k)
    if (rcs[k]) return fail(rcs[k], "%s", errs[k].c_str());
  CUDA_TRY(e);
  return FORA_OK;
}

// The hot nodes of the spread, ascending: the kHotSlots nodes of highest in-degree (ties
// at the cut leave all tied nodes out), each with in-degree >= kHotMinIndeg.  col holds m
// ids in [0, n).
std::vector<uint32_t> hot_nodes_of(int64_t n, const int32_t* col, int64_t m) {
  std::vector<uint32_t> indeg((size_t)n, 0u);
  for (int64_t k = 0; k < m; ++k) ++indeg[(size_t)col[k]];
  std::vector<uint32_t> sorted(indeg);
  uint32_t cut = kHotMinIndeg;  // hot: in-degree >= cut
  if ((int64_t)sorted.size() > kHotSlots) {
    std::nth_element(sorted.begin(), sorted.end() - (kHotSlots + 1), sorted.end());
    cut = std::max(cut, sorted[sorted.size() - (kHotSlots + 1)] + 1u);
  }
  std::vector<uint32_t> hot;
  for (int64_t v = 0; v < n; ++v)
    if (indeg[v] >= cut) hot.push_back((uint32_t)v);
  return hot;
}

int run_batch(fora_graph* g, const fora_params* p, const int32_t* sources, int nsrc,
              int32_t* out_ids, double* out_vals, fora_stats* st, const fora_debug_io* dbg,
              uint32_t dbg_flags, cudaStream_t stream, RmaxSource rsrc = RmaxSource(),
              const fora_balance* bal = nullptr) {
  int parts;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    parts = g->tune.pipeline;
  }
  parts = std::min(parts, nsrc / kMinPartSources);
  if (!dbg && parts > 1)
    return run_batch_pipelined(g, p, sources, nsrc, out_ids, out_vals, st, stream, rsrc, parts,
                               bal);
  return run_batch_ws(g, &g->ws, p, sources, nsrc, out_ids, out_vals, st, dbg, dbg_flags, stream,
                      rsrc, nullptr, bal);
}

}  // namespace

extern "C" {

int fora_graph_create(int64_t n, const int64_t* row_ptr, const int32_t* col, uint32_t flags,
                      fora_graph** out) {
  if (!out) return fail(FORA_ERR_BAD_ARG, "null output handle");
  *out = nullptr;
  if (flags != 0) return fail(FORA_ERR_BAD_ARG, "unknown flags");
  if (n < 1 || n > 0x7FFFFFFF || !row_ptr || !col) return fail(FORA_ERR_BAD_ARG, "bad n or null arrays");
  if (row_ptr[0] != 0) return fail(FORA_ERR_BAD_ARG, "row_ptr[0] must be 0");
  const int64_t m = row_ptr[n];
  if (m < 1 || m > 0xFFFFFFFFll) return fail(FORA_ERR_BAD_ARG, "m must be in [1, 2^32)");
  std::vector<uint32_t> row((size_t)n + 1);
  int64_t max_deg = 0;
  uint64_t hub_chunks = 0;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (d < 0 || row_ptr[v + 1] > m) return fail(FORA_ERR_BAD_ARG, "row_ptr not monotone at %lld", (long long)v);
    if (d == 0) return fail(FORA_ERR_DANGLING, "node %lld has no out-edge", (long long)v);
    if (d > max_deg) max_deg = d;
    if ((uint64_t)d > kHubChunk) hub_chunks += ((uint64_t)d + kHubChunk - 1) / kHubChunk;
    row[v] = (uint32_t)row_ptr[v];
  }
  row[n] = (uint32_t)m;
  for (int64_t e = 0; e < m; ++e)
    if (col[e] < 0 || col[e] >= n) return fail(FORA_ERR_BAD_ARG, "col[%lld] out of range", (long long)e);

  fora_graph* g = new fora_graph();
  g->n = n;
  g->m = m;
  g->max_deg = max_deg;
  g->hub_chunks = hub_chunks;
  auto bail = [&](int code) {
    fora_graph_destroy(g);
    return code;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) return bail(fail(FORA_ERR_CUDA, "no CUDA device"));
  if (cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
    return bail(fail(FORA_ERR_CUDA, "cannot query the SM count"));
  cudaError_t e = dalloc(&g->row, ((size_t)n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = dalloc(&g->col, (size_t)m * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(g->row, row.data(), ((size_t)n + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->col, col, (size_t)m * sizeof(int32_t), cudaMemcpyHostToDevice);
  // walk copy of col: ceil(log2 n) bits per target when that saves at least a quarter
  int bits = 1;
  while (bits < 31 && (1ll << bits) < n) ++bits;
  if (e == cudaSuccess && bits <= 24) {
    const size_t words = ((size_t)m * bits + 31) / 32 + 2;
    std::vector<uint32_t> packed(words, 0u);
    for (int64_t k = 0; k < m; ++k) {
      const uint64_t bit = (uint64_t)k * bits;
      const uint64_t w = bit >> 5;
      const uint32_t off = (uint32_t)(bit & 31);
      const uint64_t v = (uint64_t)(uint32_t)col[k] << off;
      packed[w] |= (uint32_t)v;
      packed[w + 1] |= (uint32_t)(v >> 32);
    }
    e = dalloc(&g->colp, words * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(g->colp, packed.data(), words * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) g->colbits = bits;
  }
  if (e == cudaSuccess) {  // reciprocal out-degrees (every d >= 1 here)
    std::vector<double> invd((size_t)n);
    for (int64_t v = 0; v < n; ++v) invd[v] = 1.0 / (double)(row[v + 1] - row[v]);
    e = dalloc(&g->invd, (size_t)n * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpy(g->invd, invd.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {  // the walks' node records {first edge, out-degree}
    std::vector<uint2> rd((size_t)n);
    for (int64_t v = 0; v < n; ++v) rd[v] = make_uint2(row[v], row[v + 1] - row[v]);
    e = dalloc(&g->rd, (size_t)n * sizeof(uint2));
    if (e == cudaSuccess)
      e = cudaMemcpy(g->rd, rd.data(), (size_t)n * sizeof(uint2), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    // hot targets of the spread, and the target codes that mark them
    const std::vector<uint32_t> hot = hot_nodes_of(n, col, m);
    std::vector<uint32_t> code((size_t)n);
    for (int64_t v = 0; v < n; ++v) code[v] = (uint32_t)v;
    for (size_t h = 0; h < hot.size(); ++h) code[hot[h]] = kHotBit | (uint32_t)h;
    if (!hot.empty()) {
      std::vector<uint32_t> sc((size_t)m);
      for (int64_t k = 0; k < m; ++k) sc[k] = code[(size_t)col[k]];
      e = dalloc(&g->scol, (size_t)m * sizeof(uint32_t));
      if (e == cudaSuccess) e = dalloc(&g->hot_node, hot.size() * sizeof(uint32_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(g->scol, sc.data(), (size_t)m * sizeof(uint32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(g->hot_node, hot.data(), hot.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) g->nhot = (int)hot.size();
    }
  }
  if (e == cudaSuccess) e = dalloc(&g->indeg, (size_t)n * sizeof(uint32_t));
  if (e == cudaSuccess) {
    const GraphDev gd = g->dev();
    e = launch_indegree(gd, g->indeg, g->num_sms, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess)
    return bail(fail(e == cudaErrorMemoryAllocation ? FORA_ERR_OOM : FORA_ERR_CUDA, "graph upload: %s",
                     cudaGetErrorString(e)));
  *out = g;
  return FORA_OK;
}

int fora_hot_nodes(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* out,
                   int32_t capacity, int32_t* count) {
  if (n < 1 || n > 0x7FFFFFFF || !row_ptr || !col || capacity < 0 || (capacity > 0 && !out) ||
      !count)
    return fail(FORA_ERR_BAD_ARG, "bad arguments");
  const int64_t m = row_ptr[n];
  if (row_ptr[0] != 0 || m < 0 || m > 0xFFFFFFFFll)
    return fail(FORA_ERR_BAD_ARG, "row_ptr must start at 0 and end below 2^32");
  for (int64_t k = 0; k < m; ++k)
    if (col[k] < 0 || col[k] >= n) return fail(FORA_ERR_BAD_ARG, "col[%lld] out of range", (long long)k);
  const std::vector<uint32_t> hot = hot_nodes_of(n, col, m);
  for (size_t h = 0; h < hot.size() && (int64_t)h < capacity; ++h) out[h] = (int32_t)hot[h];
  *count = (int32_t)hot.size();
  return FORA_OK;
}

void fora_graph_destroy(fora_graph* g) {
  if (!g) return;
  {
    std::lock_guard<std::mutex> lock(g->ws.mu);
    cudaSetDevice(g->device);
    g->ws.release();
    for (int k = 0; k < kMaxPipeline; ++k) {
      std::lock_guard<std::mutex> plock(g->pipe_ws[k].mu);
      g->pipe_ws[k].release();
      if (g->pipe_stream[k]) cudaStreamDestroy(g->pipe_stream[k]);
    }
    dfree(g->row);
    dfree(g->col);
    dfree(g->colp);
    dfree(g->indeg);
    dfree(g->invd);
    dfree(g->rd);
    dfree(g->scol);
    dfree(g->hot_node);
    dfree(g->idx_off);
    dfree(g->idx_dest);
  }
  delete g;
}

int fora_index_build(fora_graph* g, const fora_params* params, void* stream_) {
  if (!g || !params) return fail(FORA_ERR_BAD_ARG, "null graph or params");
  const bool zero_hop = (params->flags & FORA_ZERO_HOP) != 0;
  Resolved rp;
  int rc = resolve(g, params, &rp);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)stream_;
  Workspace* w = &g->ws;
  std::lock_guard<std::mutex> lock(w->mu);
  CUDA_TRY(cudaSetDevice(g->device));
  rc = ensure_workspace(g, w, 1);
  if (rc) return rc;
  // one slot: residues r(v) = RN(r_max d(v)), whose walk counts are omega_max(v); the
  // walks' Philox counters carry the source id 2^32 - 1
  w->h_sources[0] = -1;
  w->h_rmax[0] = rp.rmax;
  CUDA_TRY(cudaMemcpyAsync(w->sources, w->h_sources, sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(w->rmax, w->h_rmax, sizeof(double), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemsetAsync(w->small, 0, 8 * sizeof(unsigned long long), stream));
  CUDA_TRY(cudaMemsetAsync(w->err, 0, sizeof(uint32_t), stream));
  CUDA_TRY(cudaMemsetAsync(w->stats, 0, sizeof(SlotStats), stream));
  const GraphDev gd = g->dev();
  BatchDev b{};
  b.nsrc = 1;
  b.alpha = rp.alpha;
  b.walk_scale = rp.walk_scale;
  b.alpha_threshold = rp.alpha_threshold;
  b.seed = params->seed;
  set_round_keys(&b, params->seed);
  // zero-hop: omega_max from (1 - alpha) RN(r_max d(v)) and walks with a forced first move
  b.zero_hop = zero_hop ? 1 : 0;
  b.r = w->r; b.res = w->res; b.tally = w->tally;
  b.q[0] = w->q[0]; b.q[1] = w->q[1]; b.fa = w->fa;
  b.hub[0] = w->hub[0]; b.hub[1] = w->hub[1];
  b.hub_stride = g->hub_chunks;
  b.slot_cnt = w->slot_cnt;
  b.cnt_stride = w->cap;
  b.gpre = w->pre;
  b.hpre = w->pre + (w->cap + 1);
  b.alist = w->alist;
  b.work = w->work;
  b.ps = w->ps;
  b.totals = w->small + 4;
  b.sources = w->sources; b.rmax = w->rmax; b.stats = w->stats; b.err = w->err;
  b.wr_entry = w->q[0];
  b.wr_offset = w->q[1];
  b.wr_weight = reinterpret_cast<unsigned long long*>(w->fa);
  b.blk_cnt = w->blk;
  b.blk_walks = w->blk + w->residual_grid;
  b.residual_grid = w->residual_grid;
  {
    std::lock_guard<std::mutex> tlock(g->mu);
    b.spread_width = g->tune.spread_width;
    b.walk_blocks = g->tune.walk_blocks;
    b.max_rounds = g->tune.max_push_rounds;
  }
  CUDA_TRY(launch_index_residue(gd, w->r, rp.rmax, stream));
  CUDA_TRY(launch_residuals(gd, b, stream));
  CUDA_TRY(cudaMemcpyAsync(w->h_counters, w->small + 4, 2 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaMemcpyAsync(w->h_err, w->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (*w->h_err & kErrWalkOverflow) return fail(FORA_ERR_WALK_OVERFLOW, "the index would need 2^32 or more walks");
  const unsigned long long nR = w->h_counters[0], W = w->h_counters[1];
  if (nR != (unsigned long long)g->n)
    return fail(FORA_ERR_BAD_ARG, "r_max too small for a walk index: a node would get no stored walk");
  dfree(g->idx_off);
  dfree(g->idx_dest);
  g->idx_entries = 0;
  CUDA_TRY(dalloc(&g->idx_off, ((size_t)g->n + 1) * sizeof(unsigned long long)));
  CUDA_TRY(dalloc(&g->idx_dest, (size_t)(W ? W : 1) * sizeof(uint32_t)));
  b.walk_dest = g->idx_dest;
  cudaError_t e = launch_walks(gd, b, g->num_sms, stream);
  // the residual offsets of the nodes 0 .. n-1 (every node is an entry), then W
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->idx_off, w->q[1], ((size_t)g->n + 1) * sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->h_err, w->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess || (*w->h_err & kErrWalkCap)) {
    dfree(g->idx_off);
    dfree(g->idx_dest);
    if (e != cudaSuccess) return fail(FORA_ERR_CUDA, "index walks: %s", cudaGetErrorString(e));
    return fail(FORA_ERR_WALK_CAP, "an index walk exceeded %d moves", FORA_MAX_WALK_STEPS);
  }
  g->idx_entries = (int64_t)W;
  g->idx_rmax = rp.rmax;
  g->idx_scale = rp.walk_scale;
  g->idx_alpha = rp.alpha;
  g->idx_seed = params->seed;
  g->idx_zero_hop = zero_hop;
  return FORA_OK;
}

int fora_index_info(const fora_graph* g, double* rmax, double* walk_scale, int64_t* entries) {
  if (!g) return fail(FORA_ERR_BAD_ARG, "null graph");
  if (rmax) *rmax = g->idx_dest ? g->idx_rmax : 0.0;
  if (walk_scale) *walk_scale = g->idx_dest ? g->idx_scale : 0.0;
  if (entries) *entries = g->idx_dest ? g->idx_entries : 0;
  return FORA_OK;
}

int fora_index_export(const fora_graph* g, int64_t* off, uint32_t* dest) {
  if (!g || !off || !dest) return fail(FORA_ERR_BAD_ARG, "null graph or output");
  if (!g->idx_dest) return fail(FORA_ERR_BAD_ARG, "the graph has no walk index");
  CUDA_TRY(cudaSetDevice(g->device));
  CUDA_TRY(cudaMemcpy(off, g->idx_off, ((size_t)g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (g->idx_entries > 0)
    CUDA_TRY(cudaMemcpy(dest, g->idx_dest, (size_t)g->idx_entries * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost));
  return FORA_OK;
}

int fora_index_destroy(fora_graph* g) {
  if (!g) return fail(FORA_ERR_BAD_ARG, "null graph");
  std::lock_guard<std::mutex> lock(g->ws.mu);
  CUDA_TRY(cudaSetDevice(g->device));
  dfree(g->idx_off);
  dfree(g->idx_dest);
  g->idx_entries = 0;
  return FORA_OK;
}

int fora_graph_info(const fora_graph* g, int64_t* n, int64_t* m, int64_t* max_degree) {
  if (!g) return fail(FORA_ERR_BAD_ARG, "null graph");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (max_degree) *max_degree = g->max_deg;
  return FORA_OK;
}

int fora_resolve_params(const fora_graph* g, const fora_params* params, double* rmax,
                        double* walk_scale, uint32_t* alpha_threshold) {
  Resolved r;
  const int rc = resolve(g, params, &r);
  if (rc) return rc;
  if (rmax) *rmax = r.rmax;
  if (walk_scale) *walk_scale = r.walk_scale;
  if (alpha_threshold) *alpha_threshold = r.alpha_threshold;
  return FORA_OK;
}

int fora_ssppr(fora_graph* g, const fora_params* params, int32_t source, int32_t* out_ids,
               double* out_vals, fora_stats* stats, void* stream) {
  return run_batch(g, params, &source, 1, out_ids, out_vals, stats, nullptr, 0, (cudaStream_t)stream);
}

int fora_ssppr_batch(fora_graph* g, const fora_params* params, const int32_t* sources, int32_t nsrc,
                     int32_t* out_ids, double* out_vals, fora_stats* stats, void* stream) {
  return run_batch(g, params, sources, nsrc, out_ids, out_vals, stats, nullptr, 0, (cudaStream_t)stream);
}

int fora_ssppr_batch_rmax(fora_graph* g, const fora_params* params, const int32_t* sources,
                          const double* rmax, int32_t nsrc, int32_t* out_ids, double* out_vals,
                          fora_stats* stats, void* stream) {
  if (!rmax) return fail(FORA_ERR_BAD_ARG, "null r_max array");
  RmaxSource rs;
  rs.host = rmax;
  return run_batch(g, params, sources, nsrc, out_ids, out_vals, stats, nullptr, 0,
                   (cudaStream_t)stream, rs);
}

int fora_ssppr_batch_balanced(fora_graph* g, const fora_params* params, const fora_balance* costs,
                              const int32_t* sources, int32_t nsrc, int32_t* out_ids,
                              double* out_vals, fora_stats* stats, void* stream) {
  if (!costs) return fail(FORA_ERR_BAD_ARG, "null balance costs");
  return run_batch(g, params, sources, nsrc, out_ids, out_vals, stats, nullptr, 0,
                   (cudaStream_t)stream, RmaxSource(), costs);
}

int fora_ssppr_batch_debug(fora_graph* g, const fora_params* params, const int32_t* sources,
                           int32_t nsrc, int32_t* out_ids, double* out_vals, fora_stats* stats,
                           const fora_debug_io* dbg, uint32_t dbg_flags, void* stream) {
  return run_batch(g, params, sources, nsrc, out_ids, out_vals, stats, dbg, dbg_flags,
                   (cudaStream_t)stream);
}

int fora_topk_ssppr_batch(fora_graph* g, const fora_params* params, const int32_t* sources,
                          int32_t nsrc, int32_t* out_ids, double* out_vals, fora_stats* stats,
                          uint32_t* iterations, void* stream) {
  if (!g || !params || !sources || nsrc < 1) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  const uint32_t k = params->k;
  if (k < 1 || k > FORA_MAX_K || (int64_t)k > g->n) return fail(FORA_ERR_BAD_ARG, "k out of range");
  if (!out_ids || !out_vals) return fail(FORA_ERR_BAD_ARG, "null output");
  if (params->flags & (FORA_OUT_DEVICE | FORA_ASYNC))
    return fail(FORA_ERR_BAD_ARG, "top-k FORA writes host outputs and runs synchronously");
  const double n = (double)g->n;
  // rounds i < I use delta = 1/(k 2^i), round I uses 1/n (Alg. 5)
  int32_t last = 0;
  while ((double)k * ldexp(1.0, last) < n) ++last;
  double lg = log2(n / (double)k);
  if (lg < 1.0) lg = 1.0;
  const double pf = params->pf > 0 ? params->pf : 1.0 / n;
  const double pf_round = pf / (n * lg);  // p_f' = p_f / (n log2(n/k))
  std::vector<int32_t> active(nsrc), src(nsrc);
  for (int i = 0; i < nsrc; ++i) active[i] = i;
  std::vector<int32_t> ids((size_t)nsrc * k);
  std::vector<double> vals((size_t)nsrc * k);
  std::vector<fora_stats> st(nsrc);
  for (int32_t round = 0; round <= last && !active.empty(); ++round) {
    fora_params pr = *params;
    pr.eps = params->eps / 2.0;  // eps' = eps / 2 (Alg. 5)
    pr.delta = round < last ? 1.0 / ((double)k * ldexp(1.0, round)) : 1.0 / n;
    pr.pf = pf_round;
    pr.seed = params->seed + (uint64_t)round;
    pr.flags = params->flags & ~(FORA_OUT_DEVICE | FORA_ASYNC);
    const int na = (int)active.size();
    for (int i = 0; i < na; ++i) src[i] = sources[active[i]];
    const int rc = run_batch(g, &pr, src.data(), na, ids.data(), vals.data(), st.data(), nullptr, 0,
                             (cudaStream_t)stream);
    if (rc) return rc;
    std::vector<int32_t> still;
    for (int i = 0; i < na; ++i) {
      const int j = active[i];
      // stop once the k-th estimate is at least (1 + eps) delta (Alg. 5)
      if (vals[(size_t)i * k + k - 1] >= (1.0 + params->eps) * pr.delta || round == last) {
        memcpy(out_ids + (size_t)j * k, ids.data() + (size_t)i * k, k * sizeof(int32_t));
        memcpy(out_vals + (size_t)j * k, vals.data() + (size_t)i * k, k * sizeof(double));
        if (stats) stats[j] = st[i];
        if (iterations) iterations[j] = (uint32_t)round + 1;
      } else {
        still.push_back(j);
      }
    }
    active.swap(still);
  }
  return FORA_OK;
}

int fora_topk(const double* est, int64_t n, int32_t nrows, uint32_t k, int32_t* out_ids,
              double* out_vals, void* stream) {
  if (!est || n < 1 || n > 0x7FFFFFFF || nrows < 1) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  if (k > FORA_MAX_K || (int64_t)k > n) return fail(FORA_ERR_BAD_ARG, "k out of range");
  if (k == 0) return FORA_OK;
  if (!out_ids || !out_vals) return fail(FORA_ERR_BAD_ARG, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* scratch = nullptr;
  CUDA_TRY(cudaMallocAsync(&scratch, topk_scratch_bytes(nrows), st));
  const cudaError_t e = launch_topk(est, n, nrows, k, out_ids, out_vals, topk_scratch_carve(scratch, nrows),
                                    sms, st);
  cudaFreeAsync(scratch, st);
  CUDA_TRY(e);
  CUDA_TRY(cudaStreamSynchronize(st));
  return FORA_OK;
}

int fora_philox_debug(const uint32_t* ctr_key, uint32_t* out, int32_t count) {
  if (count < 0 || (count > 0 && (!ctr_key || !out))) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  if (count == 0) return FORA_OK;
  uint32_t *d_in = nullptr, *d_out = nullptr;
  CUDA_TRY(cudaMalloc(&d_in, (size_t)count * 6 * sizeof(uint32_t)));
  cudaError_t e = cudaMalloc(&d_out, (size_t)count * 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, ctr_key, (size_t)count * 6 * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox_table(d_in, d_out, count, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, (size_t)count * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_out);
  CUDA_TRY(e);
  return FORA_OK;
}

int fora_threshold_debug(const double* r, const double* rmax, const uint32_t* d, uint8_t* out,
                         int32_t count) {
  if (count < 0 || (count > 0 && (!r || !rmax || !d || !out))) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  if (count == 0) return FORA_OK;
  const size_t c = (size_t)count;
  char* buf = nullptr;  // r [c] | rmax [c] | d [c] | out [c]
  CUDA_TRY(cudaMalloc(&buf, c * (2 * sizeof(double) + sizeof(uint32_t) + 1)));
  double* dr = reinterpret_cast<double*>(buf);
  double* drm = dr + c;
  uint32_t* dd = reinterpret_cast<uint32_t*>(drm + c);
  uint8_t* dout = reinterpret_cast<uint8_t*>(dd + c);
  cudaError_t e = cudaMemcpy(dr, r, c * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(drm, rmax, c * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dd, d, c * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_threshold_table(dr, drm, dd, dout, count, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, c, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  CUDA_TRY(e);
  return FORA_OK;
}

int fora_graph_tune(fora_graph* g, const char* key, int64_t value) {
  if (!g || !key) return fail(FORA_ERR_BAD_ARG, "null graph or key");
  std::lock_guard<std::mutex> lock(g->mu);
  if (strcmp(key, "spread_width") == 0) {
    if (value < 1 || value > 4096) return fail(FORA_ERR_BAD_ARG, "spread_width must be in [1, 4096]");
    g->tune.spread_width = (int)value;
    return FORA_OK;
  }
  if (strcmp(key, "spread_hot") == 0) {
    if (value != 0 && value != 1) return fail(FORA_ERR_BAD_ARG, "spread_hot must be 0 or 1");
    g->tune.spread_hot = (int)value;
    return FORA_OK;
  }
  if (strcmp(key, "walk_blocks") == 0) {
    if (value < 3 || value > 5) return fail(FORA_ERR_BAD_ARG, "walk_blocks must be 3, 4 or 5");
    g->tune.walk_blocks = (int)value;
    return FORA_OK;
  }
  if (strcmp(key, "pipeline") == 0) {
    if (value < 1 || value > kMaxPipeline) return fail(FORA_ERR_BAD_ARG, "pipeline must be in [1, %d]", kMaxPipeline);
    g->tune.pipeline = (int)value;
    return FORA_OK;
  }
  if (strcmp(key, "push_host_loop") == 0) {
    if (value != 0 && value != 1) return fail(FORA_ERR_BAD_ARG, "push_host_loop must be 0 or 1");
    g->tune.push_host_loop = (int)value;
    return FORA_OK;
  }
  if (strcmp(key, "max_push_rounds") == 0) {
    if (value < 1 || value > (int64_t)kMaxPushRounds)
      return fail(FORA_ERR_BAD_ARG, "max_push_rounds must be in [1, %u]", kMaxPushRounds);
    g->tune.max_push_rounds = (uint32_t)value;
    return FORA_OK;
  }
  return fail(FORA_ERR_BAD_ARG, "unknown tuning key '%s'", key);
}

}  // extern "C"

struct fora_model {
  int device = 0;
  float* master = nullptr;  // FORA_MODEL_PARAMS
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;
  float* norm = nullptr;    // mu[16], sigma[16]
  int step = 0;
  std::mutex mu;
};

namespace {

uint64_t splitmix(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Device buffers of one model call (inputs, targets, partials) on the default stream.
struct ModelScratch {
  float* x = nullptr;
  float* t = nullptr;
  float* y = nullptr;
  float* partial = nullptr;
  float* loss = nullptr;
  int32_t* idx = nullptr;
  ~ModelScratch() {
    dfree(x); dfree(t); dfree(y); dfree(partial); dfree(loss); dfree(idx);
  }
};

}  // namespace

extern "C" {

int fora_model_create(uint64_t seed, fora_model** out) {
  if (!out) return fail(FORA_ERR_BAD_ARG, "null output handle");
  *out = nullptr;
  fora_model* m = new fora_model();
  std::vector<float> p(FORA_MODEL_PARAMS, 0.0f), norm(2 * FORA_NUM_FEATURES, 0.0f);
  uint64_t st = seed;
  auto uni = [&](float bound) {
    return (float)(((double)(splitmix(&st) >> 11) * 0x1p-53 * 2.0 - 1.0) * bound);
  };
  const int in = FORA_NUM_FEATURES, hid = 64;
  for (int i = 0; i < hid * in; ++i) p[i] = uni(sqrtf(6.0f / in));                      // W1
  for (int i = 0; i < hid * hid; ++i) p[hid * in + hid + i] = uni(sqrtf(6.0f / hid));   // W2
  for (int i = 0; i < hid; ++i) p[hid * in + hid + hid * hid + hid + i] = uni(sqrtf(6.0f / hid));  // W3
  for (int i = 0; i < FORA_NUM_FEATURES; ++i) norm[FORA_NUM_FEATURES + i] = 1.0f;
  auto bail = [&](cudaError_t e) {
    fora_model_destroy(m);
    return fail(e == cudaErrorMemoryAllocation ? FORA_ERR_OOM : FORA_ERR_CUDA, "model: %s",
                cudaGetErrorString(e));
  };
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaMalloc(&m->master, FORA_MODEL_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, FORA_MODEL_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, FORA_MODEL_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, FORA_MODEL_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->norm, 2 * FORA_NUM_FEATURES * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(m->master, p.data(), FORA_MODEL_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->norm, norm.data(), 2 * FORA_NUM_FEATURES * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, FORA_MODEL_PARAMS * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, FORA_MODEL_PARAMS * sizeof(float));
  if (e != cudaSuccess) return bail(e);
  *out = m;
  return FORA_OK;
}

void fora_model_destroy(fora_model* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  dfree(m->master); dfree(m->adam_m); dfree(m->adam_v); dfree(m->grad); dfree(m->norm);
  delete m;
}

int fora_model_get(const fora_model* m, float* params, float* norm) {
  if (!m) return fail(FORA_ERR_BAD_ARG, "null model");
  CUDA_TRY(cudaSetDevice(m->device));
  if (params) CUDA_TRY(cudaMemcpy(params, m->master, FORA_MODEL_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
  if (norm) CUDA_TRY(cudaMemcpy(norm, m->norm, 2 * FORA_NUM_FEATURES * sizeof(float), cudaMemcpyDeviceToHost));
  return FORA_OK;
}

int fora_model_set(fora_model* m, const float* params, const float* norm) {
  if (!m) return fail(FORA_ERR_BAD_ARG, "null model");
  std::lock_guard<std::mutex> lock(m->mu);
  CUDA_TRY(cudaSetDevice(m->device));
  if (params) CUDA_TRY(cudaMemcpy(m->master, params, FORA_MODEL_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
  if (norm) CUDA_TRY(cudaMemcpy(m->norm, norm, 2 * FORA_NUM_FEATURES * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(m->adam_m, 0, FORA_MODEL_PARAMS * sizeof(float)));
  CUDA_TRY(cudaMemset(m->adam_v, 0, FORA_MODEL_PARAMS * sizeof(float)));
  m->step = 0;
  return FORA_OK;
}

int fora_model_predict(fora_model* m, const float* x, int32_t n, float* y) {
  if (!m || !x || !y || n < 1) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  std::lock_guard<std::mutex> lock(m->mu);
  CUDA_TRY(cudaSetDevice(m->device));
  ModelScratch s;
  CUDA_TRY(cudaMalloc(&s.x, (size_t)n * FORA_NUM_FEATURES * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.y, (size_t)n * sizeof(float)));
  CUDA_TRY(cudaMemcpy(s.x, x, (size_t)n * FORA_NUM_FEATURES * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(launch_mlp_forward(m->master, m->norm, s.x, n, s.y, 0));
  CUDA_TRY(cudaMemcpy(y, s.y, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
  return FORA_OK;
}

int fora_model_gradient(fora_model* m, const float* x, const float* t, int32_t n, float* grad,
                        float* loss) {
  if (!m || !x || !t || !grad || n < 1) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  std::lock_guard<std::mutex> lock(m->mu);
  CUDA_TRY(cudaSetDevice(m->device));
  ModelScratch s;
  const int tiles = (n + mlp_tile() - 1) / mlp_tile();
  CUDA_TRY(cudaMalloc(&s.x, (size_t)n * FORA_NUM_FEATURES * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.t, (size_t)n * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.partial, (size_t)tiles * FORA_MODEL_PARAMS * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.loss, (size_t)n * sizeof(float)));
  CUDA_TRY(cudaMemcpy(s.x, x, (size_t)n * FORA_NUM_FEATURES * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s.t, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(launch_mlp_grad(m->master, m->norm, s.x, s.t, nullptr, n, s.partial, s.loss, m->grad, 0));
  CUDA_TRY(cudaMemcpy(grad, m->grad, FORA_MODEL_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
  if (loss) {
    std::vector<float> l(n);
    CUDA_TRY(cudaMemcpy(l.data(), s.loss, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
    double sum = 0.0;
    for (int i = 0; i < n; ++i) sum += l[i];
    *loss = (float)(sum / n);
  }
  return FORA_OK;
}

int fora_model_train(fora_model* m, const float* x, const float* t, int32_t n, int32_t epochs,
                     int32_t batch, float lr, uint64_t seed, float* loss_per_epoch) {
  if (!m || !x || !t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
    return fail(FORA_ERR_BAD_ARG, "bad arguments");
  std::lock_guard<std::mutex> lock(m->mu);
  CUDA_TRY(cudaSetDevice(m->device));
  // feature normalisation from the training inputs
  const int F = FORA_NUM_FEATURES;
  std::vector<float> norm(2 * F);
  for (int i = 0; i < F; ++i) {
    double s1 = 0, s2 = 0;
    for (int r = 0; r < n; ++r) { s1 += x[(size_t)r * F + i]; s2 += (double)x[(size_t)r * F + i] * x[(size_t)r * F + i]; }
    const double mean = s1 / n, var = s2 / n - mean * mean;
    norm[i] = (float)mean;
    norm[F + i] = var > 1e-12 ? (float)sqrt(var) : 1.0f;
  }
  CUDA_TRY(cudaMemcpy(m->norm, norm.data(), 2 * F * sizeof(float), cudaMemcpyHostToDevice));
  ModelScratch s;
  const int b = batch < n ? batch : n;
  const int tiles = (b + mlp_tile() - 1) / mlp_tile();
  CUDA_TRY(cudaMalloc(&s.x, (size_t)n * F * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.t, (size_t)n * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.idx, (size_t)n * sizeof(int32_t)));
  CUDA_TRY(cudaMalloc(&s.partial, (size_t)tiles * FORA_MODEL_PARAMS * sizeof(float)));
  CUDA_TRY(cudaMalloc(&s.loss, (size_t)n * sizeof(float)));
  CUDA_TRY(cudaMemcpy(s.x, x, (size_t)n * F * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s.t, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
  std::vector<int32_t> perm(n);
  std::vector<float> l(n);
  uint64_t st = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {  // seeded Fisher-Yates
      const int j = (int)(splitmix(&st) % (uint64_t)(i + 1));
      const int32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
    CUDA_TRY(cudaMemcpy(s.idx, perm.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice));
    for (int off = 0; off < n; off += b) {
      const int cnt = (n - off) < b ? (n - off) : b;
      CUDA_TRY(launch_mlp_grad(m->master, m->norm, s.x, s.t, s.idx + off, cnt, s.partial,
                               s.loss + off, m->grad, 0));
      CUDA_TRY(launch_adam(m->master, m->adam_m, m->adam_v, m->grad, ++m->step, lr, 0));
    }
    if (loss_per_epoch) {
      CUDA_TRY(cudaMemcpy(l.data(), s.loss, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
      double sum = 0.0;
      for (int i = 0; i < n; ++i) sum += l[i];
      loss_per_epoch[ep] = (float)(sum / n);
    }
  }
  CUDA_TRY(cudaDeviceSynchronize());
  return FORA_OK;
}

int fora_source_features(fora_graph* g, const fora_params* params, const int32_t* sources,
                         int32_t nsrc, float* out) {
  Resolved rp;
  int rc = resolve(g, params, &rp);
  if (rc) return rc;
  if (!sources || nsrc < 1 || !out) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  for (int i = 0; i < nsrc; ++i)
    if (sources[i] < 0 || sources[i] >= g->n) return fail(FORA_ERR_BAD_ARG, "source %d out of range", i);
  CUDA_TRY(cudaSetDevice(g->device));
  // features need no query workspace: two small buffers of their own
  int32_t* d_src = nullptr;
  float* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_src, (size_t)nsrc * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)nsrc * FORA_NUM_FEATURES * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d_src, sources, (size_t)nsrc * sizeof(int32_t), cudaMemcpyHostToDevice);
  const GraphDev gd = g->dev();
  if (e == cudaSuccess) e = launch_features(gd, g->indeg, d_src, nsrc, rp.alpha, rp.rmax, d_out, 0);
  if (e == cudaSuccess)
    e = cudaMemcpy(out, d_out, (size_t)nsrc * FORA_NUM_FEATURES * sizeof(float), cudaMemcpyDeviceToHost);
  dfree(d_src);
  dfree(d_out);
  CUDA_TRY(e);
  return FORA_OK;
}

int fora_ssppr_batch_learned(fora_graph* g, const fora_params* params, fora_model* model,
                             const int32_t* sources, int32_t nsrc, int32_t* out_ids,
                             double* out_vals, fora_stats* stats, void* stream) {
  if (!model) return fail(FORA_ERR_BAD_ARG, "null model");
  Resolved rp;
  int rc = resolve(g, params, &rp);
  if (rc) return rc;
  if (!sources || nsrc < 1 || nsrc > 65535) return fail(FORA_ERR_BAD_ARG, "bad sources");
  for (int i = 0; i < nsrc; ++i)
    if (sources[i] < 0 || sources[i] >= g->n) return fail(FORA_ERR_BAD_ARG, "source %d out of range", i);
  cudaStream_t st = (cudaStream_t)stream;
  {
    Workspace* w = &g->ws;
    std::lock_guard<std::mutex> lock(w->mu);
    CUDA_TRY(cudaSetDevice(g->device));
    rc = ensure_workspace(g, w, nsrc);
    if (rc) return rc;
    memcpy(w->h_sources, sources, nsrc * sizeof(int32_t));
    CUDA_TRY(cudaMemcpyAsync(w->sources, w->h_sources, nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const GraphDev gd = g->dev();
    // r_rule of these parameters (params->rmax is not used here)
    fora_params pr = *params;
    pr.rmax = 0.0;
    Resolved rule;
    rc = resolve(g, &pr, &rule);
    if (rc) return rc;
    CUDA_TRY(launch_features(gd, g->indeg, w->sources, nsrc, rule.alpha, rule.rmax, w->feat, st));
    std::lock_guard<std::mutex> mlock(model->mu);
    CUDA_TRY(launch_mlp_forward(model->master, model->norm, w->feat, nsrc, w->pred, st));
    CUDA_TRY(launch_pred_to_rmax(w->pred, nsrc, rule.rmax, -3.0f, 3.0f, w->rmax_learned, st));
  }
  RmaxSource rs;
  rs.device = g->ws.rmax_learned;
  return run_batch(g, params, sources, nsrc, out_ids, out_vals, stats, nullptr, 0, st, rs);
}

int fora_graph_autotune(fora_graph* g, const fora_params* params, const int32_t* sources,
                        int32_t nsrc, int32_t* spread_width, int32_t* walk_blocks, void* stream) {
  if (!g || !params || !sources || nsrc < 1) return fail(FORA_ERR_BAD_ARG, "bad arguments");
  fora_params p = *params;
  p.flags &= ~(FORA_OUT_DEVICE | FORA_ASYNC);
  const uint32_t k = p.k;
  std::vector<int32_t> ids((size_t)nsrc * (k ? k : 1));
  std::vector<double> vals((size_t)nsrc * (k ? k : 1));
  std::vector<fora_stats> st(nsrc);
  auto run = [&](float* push_ms, float* walk_ms) {
    const int rc = run_batch(g, &p, sources, nsrc, ids.data(), vals.data(), st.data(), nullptr, 0,
                             (cudaStream_t)stream);
    if (rc) return rc;
    *push_ms = st[0].ms_push;
    *walk_ms = st[0].ms_walk;
    return FORA_OK;
  };
  int parts_asked;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    parts_asked = g->tune.pipeline;
    g->tune.pipeline = 1;  // phase times below are those of the whole batch
  }
  float pm = 0, wm = 0;
  int rc = run(&pm, &wm);  // warm-up: workspace and push-loop graph
  if (rc) return rc;
  // the push depends on spread_width only, the walk kernel on walk_blocks only
  int best_sw = 1, best_wb = 3;
  float best = 0;
  const int widths[] = {1, 2, 4, 8, 16};
  for (int i = 0; i < 5; ++i) {
    {
      std::lock_guard<std::mutex> lock(g->mu);
      g->tune.spread_width = widths[i];
    }
    rc = run(&pm, &wm);
    if (rc) return rc;
    if (i == 0 || pm < best) { best = pm; best_sw = widths[i]; }
  }
  {
    std::lock_guard<std::mutex> lock(g->mu);
    g->tune.spread_width = best_sw;
  }
  // the hot-node sums of the spread against one reduction per push, at that width
  if (g->nhot > 0) {
    float hot_ms[2] = {0, 0};
    for (int h = 0; h <= 1; ++h) {
      {
        std::lock_guard<std::mutex> lock(g->mu);
        g->tune.spread_hot = h;
      }
      rc = run(&pm, &wm);
      if (rc) return rc;
      hot_ms[h] = pm;
    }
    std::lock_guard<std::mutex> lock(g->mu);
    g->tune.spread_hot = hot_ms[1] <= hot_ms[0] ? 1 : 0;
  }
  for (int wb = 3; wb <= 5; ++wb) {
    {
      std::lock_guard<std::mutex> lock(g->mu);
      g->tune.walk_blocks = wb;
    }
    rc = run(&pm, &wm);
    if (rc) return rc;
    if (wb == 3 || wm < best) { best = wm; best_wb = wb; }
  }
  {
    std::lock_guard<std::mutex> lock(g->mu);
    g->tune.walk_blocks = best_wb;
  }
  // pipeline: 1 or 2 parts (when the batch allows two), by the whole batch's time
  int best_parts = 1;
  if (nsrc >= 2 * kMinPartSources || parts_asked > 1) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best_total = 0;
    for (int parts = 1; parts <= 2 && rc == FORA_OK; ++parts) {
      {
        std::lock_guard<std::mutex> lock(g->mu);
        g->tune.pipeline = parts;
      }
      float t = 0;
      for (int rep = 0; rep < 2 && rc == FORA_OK; ++rep) {  // the faster of two runs
        cudaEventRecord(e0, (cudaStream_t)stream);
        rc = run(&pm, &wm);
        cudaEventRecord(e1, (cudaStream_t)stream);
        float ms = 0;
        if (rc == FORA_OK && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (rep == 0 || ms < t))
          t = ms;
      }
      if (parts == 1 || t < best_total) { best_total = t; best_parts = parts; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
  }
  {
    std::lock_guard<std::mutex> lock(g->mu);
    g->tune.pipeline = best_parts;
  }
  if (spread_width) *spread_width = best_sw;
  if (walk_blocks) *walk_blocks = best_wb;
  return FORA_OK;
}

int fora_graph_tuning(fora_graph* g, const char* key, int64_t* value) {
  if (!g || !key || !value) return fail(FORA_ERR_BAD_ARG, "null graph, key or value");
  std::lock_guard<std::mutex> lock(g->mu);
  if (strcmp(key, "spread_width") == 0) { *value = g->tune.spread_width; return FORA_OK; }
  if (strcmp(key, "spread_hot") == 0) { *value = g->tune.spread_hot; return FORA_OK; }
  if (strcmp(key, "hot_nodes") == 0) { *value = g->nhot; return FORA_OK; }
  if (strcmp(key, "walk_blocks") == 0) { *value = g->tune.walk_blocks; return FORA_OK; }
  if (strcmp(key, "pipeline") == 0) { *value = g->tune.pipeline; return FORA_OK; }
  if (strcmp(key, "push_host_loop") == 0) { *value = g->tune.push_host_loop; return FORA_OK; }
  if (strcmp(key, "max_push_rounds") == 0) { *value = g->tune.max_push_rounds; return FORA_OK; }
  return fail(FORA_ERR_BAD_ARG, "unknown tuning key '%s'", key);
}

int fora_workspace_bytes(int64_t n, const int64_t* row_ptr, int32_t nsrc, uint64_t* bytes) {
  if (n < 1 || n > 0x7FFFFFFF || !row_ptr || nsrc < 1 || nsrc > 65535 || !bytes)
    return fail(FORA_ERR_BAD_ARG, "bad arguments");
  uint64_t hub_chunks = 0;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (d < 0) return fail(FORA_ERR_BAD_ARG, "row_ptr not monotone at %lld", (long long)v);
    if ((uint64_t)d > kHubChunk) hub_chunks += ((uint64_t)d + kHubChunk - 1) / kHubChunk;
  }
  *bytes = (uint64_t)workspace_sizes(n, hub_chunks, nsrc).total();
  return FORA_OK;
}

int fora_debug_checks(void) {
#ifdef FORA_DEBUG
  return 1;
#else
  return 0;
#endif
}

int fora_debug_fail_alloc(int64_t nth) {
  if (nth < 0) return fail(FORA_ERR_BAD_ARG, "nth must be >= 0");
  g_fail_alloc_in.store((long long)nth);
  return FORA_OK;
}

const char* fora_last_error(void) { return g_err.c_str(); }

}  // extern "C"
