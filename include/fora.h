/*
 * fora.h -- C ABI of the GB300 (sm_103a) implementation of the index-free
 * FORA single-source Personalized PageRank (SSPPR) query (and of its FORA+ walk
 * index, Section 3.3) of Wang et al.,
 * "Efficient Algorithms for Approximate Single-Source Personalized PageRank
 * Queries" (TODS 2019).
 *
 * A query from source s (Section 2.1, Def. 1 and Def. 2) runs:
 *   1. Forward Push (Alg. 1) with residue threshold r_max, as synchronous
 *      rounds: round t takes every node v with r(v) > r_max * d_out(v),
 *      moves alpha * r(v) into its reserve, zeroes r(v), then adds
 *      (1 - alpha) * r(v) / d_out(v) to the residue of every out-neighbour
 *      (edges counted with multiplicity); residue that reaches a node of
 *      round t during round t waits for round t + 1;
 *   2. the walk phase of Alg. 2: omega_v = ceil(r(v) * C) alpha-terminating
 *      random walks from every v with r(v) > 0, where
 *      C = omega / r_sum = (2 eps/3 + 2) ln(2/p_f) / (eps^2 delta), each walk
 *      adding r(v)/omega_v to the estimate of the node where it stops;
 *   3. the estimate pi_hat(t) = reserve(t) + sum of walk weights ending at t,
 *      and the k nodes with the largest pi_hat (ties: smaller id first).
 * r_max defaults to the rule of Section 3.2 (Eq. rmax, with the Case 2
 * fallback when m * r_max > 1).
 *
 * Random numbers: walk j from node v of source s reads the 32-bit words of
 * Philox4x32-10 (Salmon et al., SC'11) blocks with counter (c, j, v, s),
 * c = 0, 1, 2, ..., and key (seed & 0xffffffff, seed >> 32), in order.  At
 * each node the walk takes one word u and stops if u < floor(alpha * 2^32);
 * otherwise it draws a neighbour index in [0, d_out) by Lemire's
 * multiply-and-reject method (one word per try).  Walk weights r(v)/omega_v
 * are summed as unsigned 64-bit fixed point with 63 fractional bits
 * (W_v = rint(r(v)/omega_v * 2^63)), so results do not depend on the order
 * in which walks finish; pi_hat(t) = reserve(t) + acc(t) * 2^-63.
 *
 * Conventions for every entry point:
 *   - return FORA_OK (0) or a negative FORA_ERR_* code; nothing is thrown
 *     across the ABI; fora_last_error() gives a message for the calling
 *     thread's last failure;
 *   - output buffers are allocated by the caller;
 *   - `stream` is a cudaStream_t owned by the caller (NULL = legacy default
 *     stream); unless FORA_ASYNC is set the call returns after the stream
 *     has finished the query;
 *   - a graph handle serialises the queries issued on it (one workspace per
 *     handle; concurrent calls on the same handle wait for each other).
 *
 * Differences from the minimal boundary this library started from (graph create /
 * destroy, fora_ssppr, fora_ssppr_batch, fora_last_error, with fora_params fields
 * k, seed, flags in that order and one stats struct of r_max, r_sum, walks, walk steps,
 * edge pushes, rounds and three phase times):
 *   - fora_params orders its fields k, flags, seed, so that the two 32-bit fields share
 *     one 8-byte slot and the struct has no padding hole (same size on every ABI);
 *   - fora_ssppr takes a `stream` argument like fora_ssppr_batch, so a single query can
 *     run on the caller's stream;
 *   - fora_stats also carries the node pushes, residual nodes and source id and splits
 *     the walk phase into residual compaction and walk kernel time (four phase times).
 */
#ifndef FORA_H_
#define FORA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FORA_OK 0
#define FORA_ERR_BAD_ARG (-1)            /* invalid argument or CSR */
#define FORA_ERR_DANGLING (-2)           /* a node with d_out = 0 (walks need d_out >= 1) */
#define FORA_ERR_OOM (-3)                /* device allocation failed */
#define FORA_ERR_WALK_OVERFLOW (-4)      /* a source needs >= 2^32 walks */
#define FORA_ERR_PUSH_NOT_CONVERGED (-5) /* push exceeded FORA_MAX_PUSH_ROUNDS rounds */
#define FORA_ERR_WALK_CAP (-6)           /* a walk exceeded FORA_MAX_WALK_STEPS moves */
#define FORA_ERR_CUDA (-7)               /* a CUDA runtime call failed */
#define FORA_ERR_TIMEOUT (-8)            /* a bounded wait ran out (serving) */
#define FORA_ERR_BOUNDS (-9)             /* a device index check failed (FORA_DEBUG builds) */

#define FORA_MAX_PUSH_ROUNDS 100000
#define FORA_MAX_WALK_STEPS 16384
#define FORA_MAX_K 4096

/* ---- flags of fora_params.flags ---- */
#define FORA_OUT_DEVICE 0x1u /* out_ids / out_vals are device pointers (else host) */
#define FORA_ASYNC 0x2u      /* return without synchronising (needs FORA_OUT_DEVICE and
                                no stats); errors found on the device are then not reported */
#define FORA_ZERO_HOP 0x4u   /* walk phase with zero-hop pruning (Section 4.1): alpha r(v)
                                goes to the estimate directly and omega_v = ceil((1-alpha)
                                r(v) C) walks each first move to a uniform out-neighbour of
                                v (no stop test at v), carrying (1-alpha) r(v) / omega_v */
#define FORA_USE_INDEX 0x8u  /* FORA+ (Section 3.3): walk j from v is the j-th walk stored
                                for v in the graph's walk index (fora_index_build) instead of
                                a walk simulated on the fly; needs the index's alpha, eps,
                                delta, p_f, every source's r_max <= the index's, and
                                FORA_ZERO_HOP exactly when the index was built with it
                                (else FORA_ERR_BAD_ARG) */

typedef struct fora_graph fora_graph; /* opaque: device copy of the CSR + query workspace */

/* Query parameters (Def. 1; Alg. 2; Section 3.2). */
typedef struct {
  double alpha;  /* stop probability of a walk, 0 < alpha < 1 */
  double eps;    /* relative error bound, > 0 */
  double delta;  /* PPR threshold of Def. 1; <= 0 selects 1/n */
  double pf;     /* failure probability, 0 < pf < 1; <= 0 selects 1/n */
  double rmax;   /* residue threshold of Alg. 1; <= 0 selects the rule of Section 3.2 */
  uint32_t k;    /* top-k size, 0 <= k <= min(n, FORA_MAX_K) */
  uint32_t flags;
  uint64_t seed; /* Philox key of the walk phase */
} fora_params;

/* Per-source counters of one query. */
typedef struct {
  double rmax;             /* residue threshold used */
  double rsum;             /* sum of residues after the push */
  uint64_t pushes;         /* node pushes over all rounds */
  uint64_t edge_pushes;    /* sum of d_out over pushed nodes */
  uint64_t residual_nodes; /* nodes with r(v) > 0 after the push */
  uint64_t walks;          /* sum of omega_v */
  uint64_t walk_steps;     /* moves over all walks (0 when walks come from a walk index) */
  uint32_t push_rounds;    /* rounds in which this source pushed at least one node */
  int32_t source;
  /* phase times of the call (the same for every source of a batch; for a batch run as
     pipeline parts, those of the source's part): push rounds, residual compaction + walk
     offsets, walk kernel, estimate + top-k */
  float ms_push, ms_residual, ms_walk, ms_topk;
} fora_stats;

/*
 * Copy a CSR graph to the device.  The graph is the directed G = (V, E) of Section 2.1
 * with n = |V| and m = |E|, stored as out-adjacency lists (the only direction Forward
 * Push and the walks of Alg. 2 follow: N_out(v) and d_out(v)).  row_ptr (n+1 entries,
 * row_ptr[0] = 0, non-decreasing) and col (row_ptr[n] entries in [0, n)) are HOST
 * arrays; they are copied and stay owned by the caller.  Requires 1 <= n < 2^31,
 * m = row_ptr[n] < 2^32 and d_out(v) >= 1 for every v (FORA_ERR_DANGLING: a walk of
 * Section 2.1 needs an out-neighbour at every node).  Edges are taken with
 * multiplicity; self-loops are allowed.  flags: 0.  Device memory: about
 * 4 (n + 1) + 4 m + 20 n bytes, plus a bit-packed copy of col for the walks when
 * ceil(log2 n) <= 24, plus 4 m bytes of target codes for the push when some node has
 * in-degree >= 64 (the up to 128 nodes of highest in-degree are marked in them, see
 * "spread_hot").  Errors: FORA_ERR_BAD_ARG, FORA_ERR_DANGLING, FORA_ERR_OOM,
 * FORA_ERR_CUDA (no device); *out is NULL on any error.
 */
int fora_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col, uint32_t flags,
                      fora_graph **out);

/*
 * The hot nodes of a CSR graph, as fora_graph_create marks them for the push (host
 * arithmetic only, no device): the up to 128 nodes of highest in-degree, each of
 * in-degree >= 64, where nodes tied at the cut are all left out; ascending ids.
 * row_ptr (n+1 entries, row_ptr[0] = 0) and col (row_ptr[n] ids in [0, n)) are HOST
 * arrays, read only.  Writes the first min(count, capacity) ids to out (capacity may be
 * 0, out then may be NULL) and the number of hot nodes to *count.  Errors:
 * FORA_ERR_BAD_ARG for bad sizes, null pointers or an id out of range.
 */
int fora_hot_nodes(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t *out,
                   int32_t capacity, int32_t *count);

/* Release the graph and its workspace.  NULL is accepted. */
void fora_graph_destroy(fora_graph *g);

/* n, m and the largest out-degree of a graph. */
int fora_graph_info(const fora_graph *g, int64_t *n, int64_t *m, int64_t *max_degree);

/*
 * Resolve the parameters as a query would: the r_max in use (rule of
 * Section 3.2 when params->rmax <= 0), C = omega / r_sum of Alg. 2,
 * and the walk stop threshold floor(alpha * 2^32).  Any output may be NULL.
 */
int fora_resolve_params(const fora_graph *g, const fora_params *params, double *rmax,
                        double *walk_scale, uint32_t *alpha_threshold);

/*
 * One SSPPR query from `source`: writes the top-k ids (int32) and
 * estimates (double) to out_ids[k] / out_vals[k] (host pointers, or device
 * pointers with FORA_OUT_DEVICE).  stats may be NULL.
 */
int fora_ssppr(fora_graph *g, const fora_params *params, int32_t source, int32_t *out_ids,
               double *out_vals, fora_stats *stats, void *stream);

/*
 * nsrc independent queries in one launch sequence (all sources advance the
 * push rounds together; the walks of all sources share one flat index space).
 * sources: HOST array of nsrc ids.  out_ids / out_vals: [nsrc][k] row-major.
 * stats: NULL or [nsrc].  Every source gives bit for bit the walk counts and
 * top-k it would give alone (same Philox counters), up to the FP64 rounding
 * order of the push.  The workspace for nsrc sources (about 56 bytes per
 * source and node; fora_workspace_bytes gives the exact size) is allocated on the
 * first call that needs it and kept.
 */
int fora_ssppr_batch(fora_graph *g, const fora_params *params, const int32_t *sources,
                     int32_t nsrc, int32_t *out_ids, double *out_vals, fora_stats *stats,
                     void *stream);

/*
 * fora_ssppr_batch with one residue threshold per source: rmax is a HOST array of nsrc
 * values > 0 (params->rmax is not used).  The accuracy guarantee of Lemma
 * (layerppr-conc) holds for any r_max, since omega scales with r_sum; r_max only moves
 * work between the push and the walks.  stats[i].rmax reports the value used.
 */
int fora_ssppr_batch_rmax(fora_graph *g, const fora_params *params, const int32_t *sources,
                          const double *rmax, int32_t nsrc, int32_t *out_ids, double *out_vals,
                          fora_stats *stats, void *stream);

/*
 * Push/walk balancing of Section 4.2 (Alg. 3): the push of each source stops, before a
 * round, as soon as its cost so far reaches the estimated cost of the walks that would
 * follow: FC = edge_push * (edge pushes) + push * (node pushes) against
 * (r_sum * C') * walk, with r_sum the residue left (1 minus the mass moved to reserves),
 * C' = C = omega / r_sum of Alg. 2 ((1 - alpha) C with FORA_ZERO_HOP) and `walk` the cost
 * of one walk.  The costs are in any one unit (for instance milliseconds measured on this
 * device); all three are finite and >= 0.  Alg. 3 starts from r_max = 1, under which no
 * node is above the threshold (r <= 1 <= d_out); this library reads it as a threshold
 * theta that starts at 1 and halves whenever no node of the source is above it, so the
 * threshold falls until the cost rule stops the push.  Pushes are otherwise the
 * synchronous rounds of Alg. 1, and the walks and estimate are those of Alg. 2 on the
 * residues the push leaves (the accuracy guarantee holds for any residues, Lemma
 * (layerppr-conc)).
 */
typedef struct {
  double edge_push; /* cost of pushing along one edge (with multiplicity) */
  double push;      /* cost of taking one node */
  double walk;      /* cost of one random walk */
} fora_balance;

/*
 * fora_ssppr_batch with the balanced push (fora_balance) per source instead of a fixed
 * r_max (params->rmax is not used); stats[i].rmax reports the final threshold theta of
 * source i.  FORA_USE_INDEX is refused (FORA_ERR_BAD_ARG: theta is not bounded by an
 * index's r_max).  Same outputs, conventions and errors as fora_ssppr_batch.
 */
int fora_ssppr_batch_balanced(fora_graph *g, const fora_params *params, const fora_balance *costs,
                              const int32_t *sources, int32_t nsrc, int32_t *out_ids,
                              double *out_vals, fora_stats *stats, void *stream);

/*
 * Top-k FORA (Alg. 5, Section 5.2) for nsrc sources: for delta = 1/k, 1/(2k), ...
 * and finally 1/n, run the query with eps' = eps/2, failure probability
 * p_f' = p_f / (n log2(n/k)) (log2 taken as at least 1) and r_max by the rule for these
 * values (or params->rmax if > 0); a source stops at the first round whose k-th
 * largest estimate is >= (1 + eps) delta.  Round i draws its walks with key seed + i.
 * params->delta is not used; params->pf is the overall p_f (<= 0 selects 1/n);
 * FORA_ZERO_HOP is honoured; FORA_USE_INDEX is not (every round has its own C, so a walk
 * index built for one round's parameters cannot serve the others: FORA_ERR_BAD_ARG).
 * Outputs are HOST arrays: out_ids / out_vals [nsrc][k],
 * stats [nsrc] (the stopping round's counters) and iterations [nsrc] (rounds run);
 * stats and iterations may be NULL.  1 <= k <= min(n, FORA_MAX_K).
 */
int fora_topk_ssppr_batch(fora_graph *g, const fora_params *params, const int32_t *sources,
                          int32_t nsrc, int32_t *out_ids, double *out_vals, fora_stats *stats,
                          uint32_t *iterations, void *stream);

/* ---- learned r_max ---- */

/*
 * A 16-64-64-1 MLP with BF16 weights and activations and FP32 accumulation that predicts
 * log2(r_max / r_rule) for a source from its features; the query then runs with
 * r_max = r_rule * 2^clamp(prediction, -3, 3).  Any r_max keeps the accuracy guarantee
 * of Lemma (layerppr-conc); the network only trades push work against walk work (the
 * role of the balancing of Section 4.2).  Parameters: FP32 masters, layout
 * W1[64][16] | b1[64] | W2[64][64] | b2[64] | W3[64] | b3; the forward rounds the weights
 * and every activation (inputs (f - mu)/sigma, hidden layers after ReLU) to BF16.
 */
#define FORA_NUM_FEATURES 16
#define FORA_MODEL_PARAMS 5313
typedef struct fora_model fora_model;

/* New model on the current device, weights drawn uniformly in +-sqrt(6/fan_in) from `seed`,
 * biases 0, normalisation mu = 0, sigma = 1. */
int fora_model_create(uint64_t seed, fora_model **out);
void fora_model_destroy(fora_model *m);
/* Host copies of the FP32 parameters [FORA_MODEL_PARAMS] and normalisation
 * [2 * FORA_NUM_FEATURES] (mu then sigma).  Either pointer may be NULL. */
int fora_model_get(const fora_model *m, float *params, float *norm);
int fora_model_set(fora_model *m, const float *params, const float *norm);
/* Forward pass on host arrays: x [n][16] -> y [n]. */
int fora_model_predict(fora_model *m, const float *x, int32_t n, float *y);
/* Gradient of 0.5 mean (y - t)^2 w.r.t. the parameters (host arrays, grad
 * [FORA_MODEL_PARAMS]) and the loss. */
int fora_model_gradient(fora_model *m, const float *x, const float *t, int32_t n, float *grad,
                        float *loss);
/* Adam training on the device (lr, beta 0.9/0.999): mu/sigma are first set from x
 * (sigma 1 where a feature is constant); each epoch visits the samples in a seeded
 * shuffled order in mini-batches of `batch`.  loss_per_epoch [epochs] (may be NULL). */
int fora_model_train(fora_model *m, const float *x, const float *t, int32_t n, int32_t epochs,
                     int32_t batch, float lr, uint64_t seed, float *loss_per_epoch);

/*
 * Features of each source (host output [nsrc][16] float), with r_rule the rule's r_max
 * for params: log1p d_out(s), log1p d_in(s), log1p sum_{u in N(s)} d_out(u),
 * log1p sum d_in(u), log1p of the 1-hop frontier size #{edges (s,u): (1-alpha)/d_out(s)
 * > r_rule d_out(u)}, log1p of the out-edges of that frontier (the 2-hop frontier),
 * log(r_rule m), log(m/n), then zeros.
 */
int fora_source_features(fora_graph *g, const fora_params *params, const int32_t *sources,
                         int32_t nsrc, float *out);

/* fora_ssppr_batch with r_max chosen per source by the model (features, forward pass
 * and r_max on the device); stats[i].rmax reports the value used. */
int fora_ssppr_batch_learned(fora_graph *g, const fora_params *params, fora_model *model,
                             const int32_t *sources, int32_t nsrc, int32_t *out_ids,
                             double *out_vals, fora_stats *stats, void *stream);

/* ---- serving: continuous batching over resident graphs ---- */

/*
 * A request loop over resident graphs (the graph handles stay owned by the caller and
 * must outlive the server).  Each graph gets lanes_per_graph lanes; a lane owns a
 * workspace for `slots` queries, a CUDA stream and a host thread.  Admission is by HBM
 * footprint: the budget (memory_budget_bytes, 0 = 80% of the free device memory) is
 * split evenly over the lanes and a lane holds as many queries as its share fits at
 * fora_workspace_bytes per query slot (residue, reserve, walk tallies, frontiers), at most
 * max_batch.  Requests queue per graph; a free lane admits the oldest queued requests
 * that share everything but k (up to its slots; after waiting up to batch_window_ms for
 * more when fewer are queued), runs them as one batched query with the largest k, and
 * returns each request its own top-k.  With admit_during_push, requests that arrive while
 * a batch is in its push rounds join it between two rounds, as long as it has free slots
 * and they share its parameters (k at most the batch's k).  Lanes run concurrently, so
 * requests that arrive while others are on the GPU also start as soon as a lane frees up
 * and overlap with them.
 * A request's result equals the same query run alone (same Philox counters), up to the
 * FP64 rounding order of the push.
 */
typedef struct {
  uint64_t memory_budget_bytes;
  int32_t lanes_per_graph;
  int32_t max_batch;
  double batch_window_ms;
  int32_t admit_during_push; /* 1: a running batch takes compatible arrivals into its free
                                slots between two push rounds (its rounds then run from a
                                host loop); 0: arrivals wait for a free lane */
  int32_t pad;
} fora_server_config;

typedef struct {
  double submit_ms, start_ms, end_ms; /* since the server was created */
  uint32_t batch_size;                /* queries in the batch that served the request */
  int32_t lane;
  uint32_t joined;                    /* 1: admitted into a running batch between two of its
                                         push rounds (admit_during_push) */
  uint32_t pad;
  fora_stats stats;
} fora_request_info;

typedef struct fora_server fora_server;

int fora_server_create(fora_graph *const *graphs, int32_t ngraphs, const fora_server_config *cfg,
                       fora_server **out);
/* Stops the lanes (queued requests are dropped) and releases their workspaces. */
void fora_server_destroy(fora_server *s);
/* Graph index and query slots of a lane (lanes are numbered graph-major). */
int fora_server_lane_capacity(const fora_server *s, int32_t lane, int32_t *graph, int32_t *slots);
/* Queue one query (params->k <= min(n, FORA_MAX_K); flags FORA_OUT_DEVICE/ASYNC ignored). */
int fora_server_submit(fora_server *s, int32_t graph, int32_t source, const fora_params *params,
                       uint64_t *ticket);
/* Wait up to timeout_ms for a request (FORA_ERR_TIMEOUT if it has not finished); on
 * success copies its top-k to HOST out_ids / out_vals [k] and its info, and forgets the
 * ticket.  Any output may be NULL. */
int fora_server_wait(fora_server *s, uint64_t ticket, double timeout_ms, int32_t *out_ids,
                     double *out_vals, fora_request_info *info);
/* Requests completed, batches run, the most lanes that were busy at once, and requests
 * that joined a batch during its push rounds.  Any output may be NULL. */
int fora_server_stats(fora_server *s, uint64_t *completed, uint64_t *batches,
                      int32_t *max_concurrent, uint64_t *joined);

/* ---- inspection entry points (parity testing) ---- */

/* Device arrays of a batch, [nsrc][n] row-major; any may be NULL. */
typedef struct {
  double *reserve;   /* pi_o after the push (input with FORA_DBG_GIVEN_PUSH) */
  double *residue;   /* r after the push (input with FORA_DBG_GIVEN_PUSH) */
  uint32_t *count;   /* walks ending at each node */
  uint64_t *acc;     /* fixed-point walk weight ending at each node (2^-63 units) */
  double *estimate;  /* pi_hat */
  const fora_balance *balance; /* NULL, or the balanced push of Alg. 3 with these costs
                                  (host struct; params->rmax is then not used) */
} fora_debug_io;

#define FORA_DBG_GIVEN_PUSH 0x1u /* skip the push; take reserve/residue from dbg (device) */

/*
 * fora_ssppr_batch with access to the intermediate arrays: with
 * FORA_DBG_GIVEN_PUSH the walk phase and top-k run on the caller's reserve
 * and residue (e.g. the oracle's); the other arrays are filled on return.
 */
int fora_ssppr_batch_debug(fora_graph *g, const fora_params *params, const int32_t *sources,
                           int32_t nsrc, int32_t *out_ids, double *out_vals, fora_stats *stats,
                           const fora_debug_io *dbg, uint32_t dbg_flags, void *stream);

/*
 * Top-k select on the device: for each of nrows rows of est ([nrows][n]
 * device doubles, all >= 0), the k largest entries with ties to the smaller
 * index, written to out_ids / out_vals ([nrows][k], device).  Uses scratch
 * memory that the call allocates (stream-ordered) and frees.
 */
int fora_topk(const double *est, int64_t n, int32_t nrows, uint32_t k, int32_t *out_ids,
              double *out_vals, void *stream);

/*
 * fora_topk without any allocation, for callers that cannot call cudaMalloc or
 * cudaFree: a free synchronises the whole device and so stalls the other streams of
 * a latency-bound serving loop, and a process that runs under a device-memory budget
 * fixed at start-up must not grow it per call.  The paper has no counterpart: this is
 * a memory-management variant of the same select.
 * Same arguments and results as fora_topk (est, out_ids and out_vals are device
 * pointers the caller owns), with at most 9 rows per call: the scratch lives in one
 * 1 MiB device array of the library, which every GPU that loads the library holds
 * until the process exits.  Larger nrows -> FORA_ERR_BAD_ARG.  The first call on a
 * device (with that device current) looks up the array's device address and keeps it
 * for the life of the process; make that first call before any stream capture.  The
 * kept address belongs to the device's primary context: do not call this entry point
 * again on a device after cudaDeviceReset (or anything else that destroys that context)
 * in the same process.  All calls share the one array: calls that overlap on the GPU
 * (on different streams or host threads) race and must be ordered by the caller.  Each
 * call synchronises `stream` before it returns.
 */
int fora_topk_noalloc(const double *est, int64_t n, int32_t nrows, uint32_t k, int32_t *out_ids,
                      double *out_vals, void *stream);

/* Evaluate the device Philox4x32-10 on count (counter[4], key[2]) rows of
 * ctr_key (host, [count][6]); writes out (host, [count][4]). */
int fora_philox_debug(const uint32_t *ctr_key, uint32_t *out, int32_t count);

/* The push's frontier test (Alg. 1: push from v while r(v) > r_max * d_out(v)) as the
 * device evaluates it, on count host triples: out[i] = 1 iff r[i] > RN64(rmax[i] * d[i]),
 * for r[i] >= 0, rmax[i] > 0 finite and d[i] >= 1.  The device decides most cases in
 * FP32 and the rest in FP64; this exposes that test for checking against plain FP64.
 * All pointers are host memory; returns FORA_ERR_BAD_ARG for count < 0 or null pointers. */
int fora_threshold_debug(const double *r, const double *rmax, const uint32_t *d, uint8_t *out,
                         int32_t count);

/*
 * Launch-shape parameters of a graph's queries (results do not depend on them, only
 * speed):  "spread_width" (1..4096, default 1): the push visits the frontier of a round
 * (grouped by source) through this many interleaved segments, so the warps in flight cover about that
 * many sources at once (wider spreads reductions on shared hub targets over more
 * addresses; narrower keeps the residue arrays in flight smaller).  "spread_hot" (0 or 1,
 * default 1): in the heavy rounds of the push a block first sums, in shared memory, its
 * pushes to the graph's hot nodes (the up to 128 nodes of highest in-degree, each >= 64)
 * over a stretch of up to 32 frontier groups of one source, then adds each sum to the
 * residue with one atomic; 0 adds every push with its own atomic (results differ only by
 * the order of FP64 additions).  The tuning read-back also answers "hot_nodes", the
 * number of hot nodes of the graph (0: spread_hot has no effect).  "walk_blocks" (3, 4
 * or 5, default 4): resident walk blocks per SM, traded against registers per thread.
 * "push_host_loop" (0 or 1, default 0): 1 launches the push rounds from a host loop with
 * one device-to-host read per round, instead of the CUDA graph whose conditional while-node
 * runs them on the device; the kernels are the same (a profiler that cannot look inside
 * conditional graph nodes sees each of them).  "pipeline" (1..4, default 1): a batched
 * query of B >= 64 sources runs as that many parts (at least 32 sources each), each on
 * its own workspace, stream and host thread, part k's push starting when part k-1's push
 * has finished, so one part's walk phase runs beside the next part's push; the call's
 * stream waits for all parts, and each part's stats carry that part's phase times.
 * Results do not depend on it.  "max_push_rounds" (1..100000, default 100000): the cap
 * on the push rounds of Alg. 1 (the loop is bounded so that it cannot run away); a query
 * whose push needs more rounds stops there and returns FORA_ERR_PUSH_NOT_CONVERGED.
 * Unknown keys and out-of-range values return FORA_ERR_BAD_ARG.
 */
int fora_graph_tune(fora_graph *g, const char *key, int64_t value);

/* The current value of a fora_graph_tune key (as set, or as the autotuner chose it).
 * Returns FORA_ERR_BAD_ARG for an unknown key or a null pointer. */
int fora_graph_tuning(fora_graph *g, const char *key, int64_t *value);

/*
 * Autotuner over the launch shapes of fora_graph_tune: runs the batched query on the
 * given sources (HOST array, a representative batch) once to warm up, then with
 * spread_width 1, 2, 4, 8, 16 keeping the fastest push phase, then (when the graph
 * has hot nodes) with "spread_hot" 0 and 1 at that width keeping the faster push, then
 * with walk_blocks 3, 4, 5 ("walk_blocks": resident 256-thread walk blocks per SM, i.e.
 * the register budget of the walk kernel) keeping the fastest walk phase (all with
 * "pipeline" 1), then, for nsrc >= 64, "pipeline" 1 or 2 by the whole batch's time (the faster of two
 * runs each).  The choices stay set on the graph; spread_width and walk_blocks are
 * returned (either pointer may be NULL), all of them through fora_graph_tuning.
 * Results of queries do not depend on them.
 */
int fora_graph_autotune(fora_graph *g, const fora_params *params, const int32_t *sources,
                        int32_t nsrc, int32_t *spread_width, int32_t *walk_blocks, void *stream);

/*
 * FORA+ walk index (Section 3.3).  After the push every residue satisfies
 * r(v) <= r_max * d_out(v), so a query needs at most
 *   omega_max(v) = ceil(RN64(RN64(r_max * d_out(v)) * C))   (Eq. index-rwnum)
 * walks from v.  fora_index_build pre-computes omega_max(v) walks from every node of g
 * for the resolved parameters of params (r_max by the rule of Section 3.2 unless
 * params->rmax > 0; C = omega / r_sum of Alg. 2), walk j from v reading the Philox stream
 * with counter (c, j, v, 2^32 - 1) and key params->seed, and keeps their end nodes on the
 * device (8 bytes per node + 4 bytes per walk), replacing any earlier index.  Queries with
 * FORA_USE_INDEX then take the first omega_v stored ends of v.  With FORA_ZERO_HOP in
 * params the stored walks are zero-hop walks (a forced first move, Section 4.1) and
 * omega_max(v) = ceil(RN64(RN64((1 - alpha) RN64(r_max * d_out(v))) * C)), an index about
 * alpha smaller, served to FORA_ZERO_HOP queries.  Not safe while queries on g run.
 * Errors: FORA_ERR_BAD_ARG (an r_max so small that a node gets no walk),
 * FORA_ERR_WALK_OVERFLOW (2^32 walks or more), FORA_ERR_OOM, FORA_ERR_CUDA.
 */
int fora_index_build(fora_graph *g, const fora_params *params, void *stream);

/* The index's r_max, C and number of stored walks (all 0 without an index). */
int fora_index_info(const fora_graph *g, double *rmax, double *walk_scale, int64_t *entries);

/* Copy the index to HOST arrays: off [n + 1] (exclusive prefix of omega_max), dest
 * [entries] (dest[off[v] + j] = end of walk j from v).  FORA_ERR_BAD_ARG without an index. */
int fora_index_export(const fora_graph *g, int64_t *off, uint32_t *dest);

/* Free the index (no-op without one). */
int fora_index_destroy(fora_graph *g);

/*
 * Device bytes a batched query of nsrc sources allocates on a graph given as HOST
 * row_ptr[n + 1] (the workspace: residue, reserve and walk tallies per source and node,
 * the frontier queues of Alg. 1, hub-chunk lists, the residual lists of Alg. 2, top-k
 * scratch and per-source state).  The same sizes decide a serving lane's slot count.
 * Host arithmetic only (no device needed).  FORA_ERR_BAD_ARG for n < 1, nsrc outside
 * [1, 65535] or a decreasing row_ptr.
 */
int fora_workspace_bytes(int64_t n, const int64_t *row_ptr, int32_t nsrc, uint64_t *bytes);

/*
 * Fault injection for tests: the nth device allocation the library makes from now on
 * (counting only its own allocations of graphs, workspaces and walk indexes, from any
 * thread) fails as if the device were out of memory, so the call making it returns
 * FORA_ERR_OOM; the allocations before and after it are real.  nth = 0 switches the
 * injection off.  The paper has no counterpart.  FORA_ERR_BAD_ARG for nth < 0.
 */
int fora_debug_fail_alloc(int64_t nth);

/*
 * 1 if this library was built with FORA_DEBUG: the hot kernels then check their device
 * indexes (nodes, edges, queue and hub-item slots, residual entries, walk-end tallies)
 * against the buffer sizes, skip an access that would fall outside and report it as
 * FORA_ERR_BOUNDS instead of touching memory; 0 for the normal build.  The paper has no
 * counterpart.
 */
int fora_debug_checks(void);

/* Message of the calling thread's last failure ("" if none): the error channel of the
 * conventions above (no exception crosses the ABI); the string stays valid until the
 * thread's next failing call. */
const char *fora_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FORA_H_ */
