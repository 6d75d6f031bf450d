// Internal declarations of the FORA query engine (device state and kernel
// launchers).  Not part of the C ABI (include/fora.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fora {

// Nodes with more out-edges than this are pushed in chunks of this many edges,
// one warp per chunk, so that a hub never serialises a round on one warp.
constexpr uint32_t kHubChunk = 256;

// Nodes of one source a warp of the push take scans as one tile.
constexpr uint32_t kTakeTile = 1024;
constexpr int kHubChunkBits = 24;  // hub item = (frontier index << 24) | chunk

// Top-k radix select: 96-bit keys (estimate bits : ~id), 12-bit digits.
constexpr int kDigitBits = 12;
constexpr int kBins = 1 << kDigitBits;
constexpr int kLevels = 96 / kDigitBits;
constexpr uint32_t kSortCap = 8192;  // candidates sorted in shared memory at the end

// Device error bits (ORed into BatchDev::err).
constexpr uint32_t kErrWalkCap = 1u;
constexpr uint32_t kErrWalkOverflow = 2u;
constexpr uint32_t kErrPushNotConverged = 4u;
constexpr uint32_t kErrIndexRange = 8u;  // a residue needs more walks than the index holds
constexpr uint32_t kErrBounds = 16u;     // a device index check failed (FORA_DEBUG builds)

// Device index checks of the FORA_DEBUG build: FORA_IN_RANGE(err, i, n) is true when
// i < n; otherwise it records kErrBounds in *err and is false, and the caller skips the
// access (the query then fails with FORA_ERR_BOUNDS).  In other builds it is `true` and
// costs nothing.
#ifdef FORA_DEBUG
__device__ __forceinline__ bool in_range_checked(uint32_t* err, unsigned long long i,
                                                 unsigned long long n) {
  if (i < n) return true;
  atomicOr(err, kErrBounds);
  return false;
}
#define FORA_IN_RANGE(err, i, n) \
  ::fora::in_range_checked((err), (unsigned long long)(i), (unsigned long long)(n))
#else
#define FORA_IN_RANGE(err, i, n) true
#endif
constexpr uint32_t kMaxPushRounds = 100000u;  // default cap of the push rounds

// Where the push loop stands: the parity of the current frontier queue, the number of
// rounds done, and the shape of the current frontier.  Kept on the device so the loop
// runs without the host.
struct PushState {
  int cur;
  uint32_t round;
  uint32_t go;    // the loop condition of the last round (read by the host-driven loop)
  uint32_t nact;  // sources with a non-empty current frontier (listed in BatchDev::alist)
  unsigned long long ngroups;  // 32-entry groups of the current frontier, over all sources
  unsigned long long nhub;     // hub items of the current frontier, over all sources
};

struct GraphDev {
  int64_t n;
  int64_t m;
  const uint32_t* row;  // [n+1] edge offsets (m < 2^32)
  const int32_t* col;   // [m]
  // The same targets bit-packed, colbits bits each (0 = not packed), for the walks: a
  // smaller footprint keeps more of the graph in L2 beside the walk tallies.
  const uint32_t* colp;
  int colbits;
  const double* invd;   // [n] RN(1 / d(v)): the push increment is a product, not a quotient
  const uint2* rd;      // [n] {row[v], d(v)}: a walk's move reads one aligned 8-byte record
  // The spread's copy of the targets (null when the graph has no hot nodes): the target
  // id, or kHotBit | h for the h-th hot node (a node of high in-degree, hot_node[h]), whose
  // increments a block sums in shared memory before one reduction reaches L2.
  const uint32_t* scol;
  const uint32_t* hot_node;  // [nhot] ascending ids
  int nhot;
};

// Hot targets of the spread: at most kHotSlots nodes, each of in-degree >= kHotMinIndeg.
// (2^20 R-MAT graph, 256 sources, push of the rule's / half the rule's r_max: 2048 hot
// nodes 100.5 / 151.8 ms, 1024: 98.6 / 146.6, 256: 97.1 / 140.5, 128: 97.3 / 138.1,
// 16: 98.7 / 138.6, one atomic per push 116.9 / 168.6; what the sums remove is mostly
// the queueing of reductions on the same few addresses at L2.)
#ifndef FORA_HOT_SLOTS
#define FORA_HOT_SLOTS 128
#endif
constexpr int kHotSlots = FORA_HOT_SLOTS;
constexpr uint32_t kHotMinIndeg = 64;
constexpr uint32_t kHotBit = 0x80000000u;

// Target e of a bit-packed column array (two 32-bit words always readable).
__device__ __forceinline__ uint32_t packed_target(const uint32_t* colp, int bits, uint32_t e) {
  const unsigned long long bit = (unsigned long long)e * (unsigned long long)bits;
  const unsigned long long w = bit >> 5;
  const unsigned long long two = (unsigned long long)colp[w] | ((unsigned long long)colp[w + 1] << 32);
  return (uint32_t)(two >> (bit & 31)) & ((1u << bits) - 1u);
}

// Walk end tally of one (source, node): fixed-point weight and count share one
// 16-byte record, so a walk's end touches a single L2 sector.
struct __align__(16) Tally {
  unsigned long long acc;  // sum of walk weights, 2^-63 units
  uint32_t cnt;            // number of walks
  uint32_t pad;
};

// Per-source counters kept on the device during a call.
struct SlotStats {
  unsigned long long pushes;
  unsigned long long edge_pushes;
  unsigned long long residual_nodes;
  unsigned long long walks;
  unsigned long long walk_steps;
  double rsum;
  double moved;    // sum of alpha r(v) over the pushes (balanced push: r_sum = 1 - moved)
  uint32_t rounds;
  uint32_t pad;
};

// Top-k select state of one row.
struct TopkSlot {
  unsigned long long pa;  // known bits of the key's upper 64 bits (estimate bits)
  uint32_t pb;            // known bits of the key's lower 32 bits (~id)
  uint32_t plen;          // number of leading key bits fixed so far
  uint32_t kk;            // how many keys still to take from the current bucket
  uint32_t done;
  uint32_t ncand;
  uint32_t pad;
};

// Pointers into a call's workspace; all arrays source-major ([slot][n]).
struct BatchDev {
  int32_t nsrc;
  double alpha;
  double walk_scale;         // C = omega / r_sum
  uint32_t alpha_threshold;  // floor(alpha * 2^32)
  uint64_t seed;
  uint2 round_key[10];       // Philox round keys of `seed` (key + i * (0x9E3779B9, 0xBB67AE85))
  int zero_hop;              // walk phase with zero-hop pruning (Section 4.1)
  int want_count;            // tally walk counts too (only a debug output reads them)
  uint32_t* walk_dest;       // non-null: k_walks stores walk g's end in walk_dest[g]
                             // (building a walk index) instead of tallying it
  double* r;                 // residue, later the estimate
  double* res;               // reserve
  Tally* tally;              // walk ends per (source, node)
  // Frontier of source `slot`: entries (slot << 32) | v at q[par][slot * n + j],
  // j < slot_cnt[par][slot], with increments fa[slot * n + j]; its hub items at
  // hub[par][slot * hub_stride + j], j < slot_cnt[2 + par][slot].
  unsigned long long* q[2];
  double* fa;                // per frontier entry: (1 - alpha) r(v) / d(v)
  unsigned long long* hub[2];  // hub chunk items: (q index << kHubChunkBits) | chunk
  unsigned long long hub_stride;
  uint32_t* slot_cnt;        // [4][cnt_stride]: entries of parity 0, 1; hub items of parity 0, 1
  int cnt_stride;            // slots per row of slot_cnt (the workspace's capacity)
  unsigned long long* gpre;  // [nsrc + 1]: exclusive prefix of ceil(entries / 32), current
  unsigned long long* hpre;  // [nsrc + 1]: exclusive prefix of hub items, current
  uint32_t* alist;           // [nsrc]: the sources with a non-empty current frontier
  unsigned long long* work;  // dynamic work counters of the spread ([0] and [16])
  PushState* ps;
  const int32_t* sources;    // [nsrc]
  const double* rmax;        // [nsrc]
  SlotStats* stats;          // [nsrc]
  uint32_t* err;
  // walk phase
  unsigned long long* wr_entry;   // residual list: (slot << 32) | v   (aliases q[0])
  unsigned long long* wr_offset;  // exclusive walk offsets, [|R| + 1]  (aliases q[1])
  unsigned long long* wr_weight;  // fixed-point weight per walk        (aliases fa)
  unsigned long long* blk_cnt;    // [grid] per-block counts, then block offsets
  unsigned long long* blk_walks;  // [grid] per-block counts, then block offsets
  unsigned long long* totals;     // [2]: |R|, W
  int residual_grid;
  int spread_width;  // interleaved segments of the frontier the spread visits at once
  int spread_hot;    // the spread sums hot targets per block (GraphDev::scol is set)
  int walk_blocks;   // resident walk blocks per SM (3, 4 or 5)
  uint32_t max_rounds;  // push rounds allowed before kErrPushNotConverged
  // Balanced push (Section 4.2, Alg. 3): balance != 0 makes rmax the per-source threshold
  // theta (halved on the device when no node is above it) and stops a source's push before
  // a round once cost_edge * edge pushes + cost_push * pushes >= ((1 - moved) * bal_scale)
  // * cost_walk, with bal_scale = C' (C, or (1 - alpha) C with zero-hop pruning).
  int balance;
  double bal_scale, cost_edge, cost_push, cost_walk;
  double* theta;       // [nsrc] the thresholds (the same array as rmax)
  uint32_t* stopped;   // [nsrc] 1 once the cost rule stopped the source's push
  // Light rounds: after every take each node of an active source is at or below its
  // threshold, so only nodes the next spread adds to can cross.  When a source's new
  // frontier spreads fewer than light_edges edges, light[s] = 1: its spread marks the
  // kTakeTile-node tiles it touches in tile_dirty and its take scans only those (clearing
  // them); otherwise the take scans every tile.
  uint8_t* light;                  // [nsrc]
  uint8_t* tile_dirty;             // [nsrc][tiles]
  unsigned long long* last_edges;  // [nsrc] the source's edge pushes at the last advance
  unsigned long long tiles;        // tiles per source, ceil(n / kTakeTile)
  unsigned long long light_edges;
};

// Launch-shape parameters of a graph (set through fora_graph_tune or the autotuner).
struct Tuning {
  int spread_width = 1;
  int spread_hot = 1;      // 1: heavy spread rounds sum hot targets' increments per block
  int walk_blocks = 4;
  int push_host_loop = 0;  // 1: rounds launched from a host loop instead of the graph
  int pipeline = 1;        // parts of a batch run on their own streams, pushes staggered
  uint32_t max_push_rounds = kMaxPushRounds;
};

// capi.cu: record a failure for fora_last_error() and return `code`.
int report_error(int code, const char* fmt, ...);
// capi.cu: resident blocks per SM of `kernel` launched with `threads` threads and no
// dynamic shared memory on the current device (at least 1; 0 if the query fails).
// Cached per (device, kernel) under a lock, so concurrent host threads may call it.
int resident_blocks(const void* kernel, int threads);
// capi.cu: cudaMalloc through the library's allocation hook (fora_debug_fail_alloc):
// returns cudaErrorMemoryAllocation without allocating when the hook says so.
cudaError_t device_alloc(void** p, size_t bytes);

// push.cu: r(s) = 1 and the loop state; then the rounds, each launched by the body of a
// conditional while-node of a CUDA graph (the body sets the loop condition itself), or,
// with in_graph false, from a host loop that reads PushState::go after each round.
cudaError_t launch_push_seed(const GraphDev& g, const BatchDev& b, cudaStream_t st);
cudaError_t launch_push_body(const GraphDev& g, const BatchDev& b, int num_sms,
                             cudaGraphConditionalHandle loop, bool in_graph, cudaStream_t st);
// push.cu: slots [first, first + k) join a batch between two push rounds (host loop only).
cudaError_t launch_push_join(const GraphDev& g, const BatchDev& b, int first, int k,
                             cudaStream_t st);
// push.cu: the frontier test r > RN(r_max * d) of the take, on given triples.
cudaError_t launch_threshold_table(const double* r, const double* rm, const uint32_t* d,
                                   uint8_t* out, int count, cudaStream_t st);

// walk.cu
cudaError_t launch_residuals(const GraphDev& g, const BatchDev& b, cudaStream_t st);
cudaError_t launch_walks(const GraphDev& g, const BatchDev& b, int num_sms, cudaStream_t st);
// walk.cu, FORA+ (Section 3.3): r[v] = RN(rmax * d(v)) for one slot (the residues whose
// omega_v are the index's omega_max(v)), and the walk phase served from an index.
cudaError_t launch_index_residue(const GraphDev& g, double* r, double rmax, cudaStream_t st);
cudaError_t launch_walks_indexed(const GraphDev& g, const BatchDev& b, int num_sms,
                                 const unsigned long long* idx_off, const uint32_t* idx_dest,
                                 cudaStream_t st);
cudaError_t launch_unpack_tally(const Tally* t, uint32_t* cnt, unsigned long long* acc,
                                uint64_t count, int num_sms, cudaStream_t st);
cudaError_t launch_philox_table(const uint32_t* ctr_key, uint32_t* out, int count,
                                cudaStream_t st);

// learn.cu
cudaError_t launch_indegree(const GraphDev& g, uint32_t* indeg, int num_sms, cudaStream_t st);
cudaError_t launch_features(const GraphDev& g, const uint32_t* indeg, const int32_t* sources,
                            int nsrc, double alpha, double rmax_rule, float* out, cudaStream_t st);
cudaError_t launch_mlp_forward(const float* master, const float* norm, const float* X, int n,
                               float* Y, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* master, const float* norm, const float* X,
                            const float* T, const int32_t* idx, int n, float* partial,
                            float* loss_partial, float* grad, cudaStream_t st);
cudaError_t launch_adam(float* master, float* m, float* v, const float* grad, int step, float lr,
                        cudaStream_t st);
cudaError_t launch_pred_to_rmax(const float* pred, int n, double rmax_rule, float lo, float hi,
                                double* rmax, cudaStream_t st);
int mlp_tile();

// topk.cu
// est may alias r (the residue array becomes the estimate); with zero_hop the estimate
// also takes alpha * r.
cudaError_t launch_estimate(const double* res, const Tally* tally, double* est, const double* r,
                            double alpha, int zero_hop, uint64_t count, int num_sms,
                            cudaStream_t st);
// Scratch of the top-k select: hist [nrows][kBins], slots [nrows], cand [nrows][kSortCap].
struct TopkScratch {
  uint32_t* hist;
  TopkSlot* slots;
  unsigned long long* cand_key;  // estimate bits
  uint32_t* cand_id;
};
size_t topk_scratch_bytes(int nrows);
TopkScratch topk_scratch_carve(void* base, int nrows);
cudaError_t launch_topk(const double* est, int64_t n, int nrows, uint32_t k, int32_t* out_ids,
                        double* out_vals, const TopkScratch& s, int num_sms, cudaStream_t st);

}  // namespace fora
