// Forward Push (Alg. 1) as synchronous frontier rounds over a batch of sources.
//
// F_t holds, per source, the nodes v with r(v) > r_max * d(v) at the start of round t,
// each with the increment inc_v = (1 - alpha) a_v / d(v) of its taken residue a_v.
// Source s keeps its part of F_t in its own region of the queue (q[par][s * n + j]), so
// the frontier is grouped by source without a global sort.  Round t:
//   k_push_spread   r(u) += inc_v for every out-edge (v, u) of F_t: FP64 reductions
//                   that return nothing, so a warp never waits on an atomic.
//                   (k_push_spread_hot, the default on graphs with hot nodes, first
//                   sums a block's pushes to the few nodes of highest in-degree in
//                   shared memory; see there.)
//   k_push_take     F_{t+1} = {u : r(u) > r_max * d(u)} over the sources that pushed in
//                   round t (every other r is unchanged and below its threshold), in one
//                   streaming pass over their residues; each crossing node is appended
//                   to its source's region and taken at once:
//                   a_u = r(u); reserve(u) += alpha a_u; r(u) = 0;
//                   inc_u = (1 - alpha) a_u / d(u)   (the first half of round t+1),
//                   computed as RN(RN((1 - alpha) a_u) * RN(1 / d(u))) with the
//                   graph's reciprocal degrees (within an ulp or so of the quotient;
//                   this GPU's FP64 division costs about ten FP64 instructions).
//   k_push_advance  one block: per-source prefix of the new frontier's groups and hub
//                   items, the list of sources still pushing, the loop condition.
// The take of round t+1 happens after every add of round t (kernel boundary), so
// residue arriving at a frontier node during a round waits for the next round.
//
// Spread load balance: a warp takes 32 frontier entries with d <= kHubChunk, scans their
// degrees and walks their concatenated edge lists 128 edges per iteration (coalesced
// col reads); nodes with more out-edges are split into kHubChunk-edge hub items, one
// warp each.  Work is handed out in source order, so the warps in flight work on a few
// sources at a time and the residue arrays they add into stay in L2.
#include "fora_engine.cuh"

namespace fora {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kTakeThreads = 256;
constexpr int kSpreadThreads = 256;
constexpr uint32_t kTileNodes = kTakeTile;  // nodes of one source a warp scans per take tile

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T t = __shfl_up_sync(kFull, x, off);
    if ((int)lane_id() >= off) x += t;
  }
  return x;
}

// Block-wide exclusive scan of two counters; returns the block totals too.
__device__ __forceinline__ void block_scan2(unsigned long long a, unsigned long long b,
                                            unsigned long long* ae, unsigned long long* be,
                                            unsigned long long* at, unsigned long long* bt) {
  __shared__ unsigned long long sa[32], sb[32];
  __shared__ unsigned long long ta, tb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long ai = warp_incl_scan(a), bi = warp_incl_scan(b);
  if (lane == 31) { sa[wid] = ai; sb[wid] = bi; }
  __syncthreads();
  if (wid == 0) {
    const unsigned long long x = lane < nw ? sa[lane] : 0, y = lane < nw ? sb[lane] : 0;
    const unsigned long long xi = warp_incl_scan(x), yi = warp_incl_scan(y);
    if (lane < nw) { sa[lane] = xi - x; sb[lane] = yi - y; }
    if (lane == 31) { ta = xi; tb = yi; }
  }
  __syncthreads();
  *ae = sa[wid] + ai - a;
  *be = sb[wid] + bi - b;
  *at = ta;
  *bt = tb;
  __syncthreads();
}

__device__ __forceinline__ uint32_t hub_chunks_of(uint32_t d) {
  return d > kHubChunk ? (d + kHubChunk - 1) / kHubChunk : 0u;
}

// r > RN(rm * d), the frontier test, with FP64 arithmetic only near the threshold (this
// GPU issues about two FP64 operations per clock per SM, so the test itself would bound
// the scan).  rf is r truncated to 23 mantissa bits through its bit pattern (rf <= r <
// rf (1 + 2^-23) when r's exponent is in FP32's normal range, rf = 0 when r < 2^-126),
// tf = RN32(rmf * RN32(d)) with rmf = RN32(rm) is within 2^-22 of V = rm * d, and
// T = RN64(V) is within 2^-53 of V.  So rf below tf (1 - 2^-19) implies r < V (1 - 2^-20)
// < T, and rf above tf (1 + 2^-19) implies r > V (1 + 2^-20) > T.  Returns 0 (below),
// 1 (above) or 2 (undecided: in between, or rmf outside [2^-100, 2^60], which `fast`
// excludes, or r >= 2^128); the FP64 test decides the undecided ones.
__device__ __forceinline__ uint32_t threshold_fast(double r, float rmf, bool fast, uint32_t d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
  const uint32_t hi = (uint32_t)(bits >> 32);
  const uint32_t ex = hi >> 20;  // r >= 0: no sign bit
  if (!fast || ex > 1150u) return 2u;
  const float tf = rmf * __uint2float_rn(d);
  const float rf = ex < 897u ? 0.0f
                             : __uint_as_float(((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) |
                                               ((uint32_t)bits >> 29));
  if (rf < tf * (1.0f - 0x1p-19f)) return 0u;
  if (rf > tf * (1.0f + 0x1p-19f)) return 1u;
  return 2u;
}

// The FP64 test, kept out of line so that it is not evaluated for every node.
__device__ __noinline__ bool threshold_exact(double r, double rm, uint32_t d) {
  return r > __dmul_rn(rm, (double)d);
}

__device__ __forceinline__ bool above_threshold(double r, double rm, float rmf, bool fast,
                                                uint32_t d) {
  const uint32_t f = threshold_fast(r, rmf, fast, d);
  return f == 2u ? threshold_exact(r, rm, d) : f == 1u;
}

// The source whose range [pre[s], pre[s + 1]) holds x, for a non-decreasing prefix with
// x < pre[nsrc]: the largest s with pre[s] <= x (empty sources have pre[s] = pre[s + 1]).
__device__ __forceinline__ int slot_of(const unsigned long long* pre, int nsrc,
                                       unsigned long long x) {
  int lo = 0, hi = nsrc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_push_seed(GraphDev g, BatchDev b) {
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < b.nsrc;
       slot += gridDim.x * blockDim.x) {
    // Alg. 1 starts from r(s) = 1.  The first pass of the loop body has an empty
    // frontier (nothing to spread); its take scans every source and finds F_0.
    const uint32_t src = (uint32_t)b.sources[slot];
    b.r[(unsigned long long)slot * (unsigned long long)g.n + src] = 1.0;
    b.alist[slot] = (uint32_t)slot;
    // only r(s) is non-zero: the first take scans the source's tile alone
    b.light[slot] = 1;
    b.tile_dirty[(unsigned long long)slot * b.tiles + src / kTileNodes] = 1;
    if (b.balance) {
      // the cost rule before any push: FC = 0 against the walk cost of r_sum = 1
      const bool stop = 0.0 >= __dmul_rn(__dmul_rn(1.0, b.bal_scale), b.cost_walk);
      b.stopped[slot] = stop ? 1u : 0u;
      // Alg. 3 starts from threshold 1 and halves it while no node is above it: before the
      // first push only r(s) = 1 is non-zero, so theta halves until 1 > theta d(s)
      double theta = 1.0;
      const double ds = (double)(g.row[src + 1] - g.row[src]);
      if (!stop)
        while (!(1.0 > __dmul_rn(theta, ds))) theta = __dmul_rn(0.5, theta);
      b.theta[slot] = theta;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PushState* ps = b.ps;
    ps->cur = 1;
    ps->round = 0;
    ps->go = 1;
    ps->nact = (uint32_t)b.nsrc;
    ps->ngroups = 0;
    ps->nhub = 0;
  }
}

// 0, 1, ..., 32 as FP64 (the run lengths of spread_slice).
__constant__ double kMultiple[33] = {0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10,
                                     11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21,
                                     22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32};

// Runs of one 32-edge slice whose lanes hold consecutive CSR entries (lane order = entry
// order; inactive lanes only at the end).  Rows are sorted, so the copies of a multi-edge
// (v, u) are adjacent: a run of lanes with the same target from the same frontier node
// (`owner`) becomes one add of k * inc by its first lane (k copies counted with
// multiplicity, as Alg. 1 pushes along each of them; one rounding instead of k, which only
// reorders the FP64 sum like the atomics do).  True for the first lane of a run, with
// add = k * inc; every lane of the warp calls it.
__device__ __forceinline__ bool run_lead(uint32_t u, uint32_t owner, double inc, bool act,
                                         double& add) {
  const uint32_t lane = lane_id();
  const uint32_t pu = __shfl_up_sync(kFull, u, 1);
  const uint32_t po = __shfl_up_sync(kFull, owner, 1);
  const bool cont = act && lane > 0 && pu == u && po == owner;  // continues lane - 1's run
  const uint32_t brk = __ballot_sync(kFull, !cont);              // run starts and idle lanes
  const bool lead = act && !cont;
  uint32_t k = 1;
  if (lead) {
    const uint32_t above = brk & ~((2u << lane) - 1u);
    k = (above ? (uint32_t)__ffs(above) - 1u : 32u) - lane;
  }
  // FP64 arithmetic only in slices that hold a run (this GPU's FP64 rate is low, and most
  // slices have none); kMultiple[k] = k avoids an integer-to-FP64 conversion
  add = inc;
  if (__any_sync(kFull, k > 1u)) {
    if (k > 1u) add = __dmul_rn(inc, kMultiple[k]);
  }
  return lead;
}

// r[base + u] += inc for the active lanes of one slice, one reduction per run.
__device__ __forceinline__ void spread_slice(double* r, unsigned long long base, uint32_t u,
                                             uint32_t owner, double inc, bool act,
                                             uint32_t* err, unsigned long long n) {
  double add;
  if (run_lead(u, owner, inc, act, add) && FORA_IN_RANGE(err, u, n)) atomicAdd(&r[base + u], add);
}

// Work is handed out dynamically (kGrab groups or hub items per atomic), so the warps
// in flight always hold the next unprocessed stretch of the frontier, whatever the cost
// of each group.
constexpr unsigned long long kGrab = 4;

#ifndef FORA_SPREAD_MIN_BLOCKS
#define FORA_SPREAD_MIN_BLOCKS 6
#endif
__global__ void __launch_bounds__(kSpreadThreads, FORA_SPREAD_MIN_BLOCKS) k_push_spread(GraphDev g, BatchDev b) {
  const int cur = b.ps->cur;
  const unsigned long long ngroups = b.ps->ngroups;
  const unsigned long long nh = b.ps->nhub;
  const unsigned long long* q = b.q[cur];
  const uint32_t* cnt = b.slot_cnt + (size_t)cur * b.cnt_stride;
  const uint32_t lane = lane_id();
  const unsigned long long n = (unsigned long long)g.n;

  // groups of 32 frontier entries of one source (nodes with d <= kHubChunk), visited
  // through b.spread_width interleaved segments of the frontier
  const unsigned long long width = (unsigned long long)b.spread_width;
  const unsigned long long gseg = (ngroups + width - 1) / width;
  const unsigned long long gtotal = gseg * width;
  int cs = 0;                           // source of the cached range
  unsigned long long clo = 1, chi = 0;  // its groups [clo, chi) (empty: nothing cached)
  uint32_t ccnt = 0;
  bool clight = false;                  // the cached source's round is light: mark tiles
  for (;;) {
    unsigned long long v0 = 0;
    if (lane == 0) v0 = atomicAdd(&b.work[0], kGrab);
    v0 = __shfl_sync(kFull, v0, 0);
    if (v0 >= gtotal) break;
    const unsigned long long v1 = min(v0 + kGrab, gtotal);
    for (unsigned long long vg = v0; vg < v1; ++vg) {
      const unsigned long long grp = (vg % width) * gseg + vg / width;
      if (grp >= ngroups) continue;
      if (grp < clo || grp >= chi) {  // warp-uniform
        cs = slot_of(b.gpre, b.nsrc, grp);
        clo = b.gpre[cs];
        chi = b.gpre[cs + 1];
        ccnt = cnt[cs];
        clight = b.light[cs] != 0;
      }
      const uint32_t i = (uint32_t)(grp - clo) * 32u + lane;
      const unsigned long long base_gi = (unsigned long long)cs * n;
      uint32_t c = 0, rb = 0;
      double inc = 0.0;
      if (i < ccnt) {
        const uint32_t v = (uint32_t)q[base_gi + i];
        rb = g.row[v];
        const uint32_t d = g.row[v + 1] - rb;
        if (d <= kHubChunk) {
          c = d;
          inc = b.fa[base_gi + i];
        }
      }
      const uint32_t incl = warp_incl_scan(c);
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      const uint32_t excl = incl - c;
      for (uint32_t base = 0; base < total; base += 128) {
        uint32_t u[4], own[4];
        double ik[4];
        bool act[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t e = base + 32 * k + lane;
          int lo = 0, hi = 31;  // owner: the first lane whose inclusive prefix exceeds e
#pragma unroll
          for (int s2 = 0; s2 < 5; ++s2) {
            const int mid = (lo + hi) >> 1;
            if (__shfl_sync(kFull, incl, mid) > e) hi = mid; else lo = mid + 1;
          }
          const uint32_t ek = __shfl_sync(kFull, excl, lo);
          const uint32_t rbk = __shfl_sync(kFull, rb, lo);
          ik[k] = __shfl_sync(kFull, inc, lo);
          own[k] = (uint32_t)lo;
          act[k] = e < total;
          u[k] = act[k] ? (uint32_t)g.col[rbk + (e - ek)] : 0u;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          spread_slice(b.r, base_gi, u[k], own[k], ik[k], act[k], b.err, n);
        if (clight) {  // warp-uniform
          uint8_t* dirty = b.tile_dirty + (unsigned long long)cs * b.tiles;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (act[k] && u[k] < n) dirty[u[k] / kTileNodes] = 1;
        }
      }
    }
  }

  // hub items: kHubChunk edges of one frontier node each, same segment order
  const unsigned long long hseg = (nh + width - 1) / width;
  const unsigned long long htotal = hseg * width;
  clo = 1;
  chi = 0;
  for (;;) {
    unsigned long long v0 = 0;
    if (lane == 0) v0 = atomicAdd(&b.work[16], kGrab);
    v0 = __shfl_sync(kFull, v0, 0);
    if (v0 >= htotal) break;
    const unsigned long long v1 = min(v0 + kGrab, htotal);
    for (unsigned long long vh = v0; vh < v1; ++vh) {
      const unsigned long long h = (vh % width) * hseg + vh / width;
      if (h >= nh) continue;
      if (h < clo || h >= chi) {  // warp-uniform
        cs = slot_of(b.hpre, b.nsrc, h);
        clo = b.hpre[cs];
        chi = b.hpre[cs + 1];
        clight = b.light[cs] != 0;
      }
      const unsigned long long item =
          b.hub[cur][(unsigned long long)cs * b.hub_stride + (h - clo)];
      const unsigned long long fi = item >> kHubChunkBits;
      const uint32_t c = (uint32_t)(item & ((1ull << kHubChunkBits) - 1));
      const uint32_t v = (uint32_t)q[fi];
      const unsigned long long gbase = (unsigned long long)cs * n;
      const uint32_t rb = g.row[v], re = g.row[v + 1];
      const double inc = b.fa[fi];
      const uint32_t beg = rb + c * kHubChunk;
      const uint32_t end = min(beg + kHubChunk, re);
      uint32_t u[kHubChunk / 32];
#pragma unroll
      for (int k = 0; k < (int)(kHubChunk / 32); ++k) {
        const uint32_t p = beg + 32 * k + lane;
        u[k] = p < end ? (uint32_t)g.col[p] : 0xFFFFFFFFu;
      }
#pragma unroll
      for (int k = 0; k < (int)(kHubChunk / 32); ++k)
        spread_slice(b.r, gbase, u[k], 0u, inc, u[k] != 0xFFFFFFFFu, b.err, n);
      if (clight) {  // warp-uniform
        uint8_t* dirty = b.tile_dirty + (unsigned long long)cs * b.tiles;
#pragma unroll
        for (int k = 0; k < (int)(kHubChunk / 32); ++k)
          if (u[k] < n) dirty[u[k] / kTileNodes] = 1;
      }
    }
  }
}

// The spread with hot targets summed per block (GraphDev::scol set, BatchDev::spread_hot).
// In the R-MAT graphs a few thousand nodes of high in-degree receive a large share of all
// edge pushes, and every push is an FP64 reduction at L2, the spread's bound.  Here a
// block takes kHotRange consecutive groups (or hub items) of one interleaved segment of
// the frontier at a time.  Where the range holds at least kHotStretch items of one source
// in a heavy round (the source's round is not light), the block processes that stretch
// together: its adds to hot nodes go to a shared-memory array, and after the stretch one
// reduction per touched hot node carries each sum to r.  The rest of the range (light
// rounds, whose spread also marks the tiles it touches, and short stretches) is spread
// first, warp by warp, with one reduction per push as in k_push_spread.  Summing in
// shared memory first only regroups the FP64 sum, as the order of the atomics does.
// Range and stretch measured on the 2^20 R-MAT graph (2048 hot nodes, 5 blocks per SM):
// ranges of 16, 24, 32, 64, 128 items gave 103.4, 101.2, 100.5, 110.7, 141.3 ms of push
// with the rule's r_max (fewer, larger ranges leave blocks idle at the end of a round);
// a minimum stretch of 4, 8 or 16 items made no difference.
#ifndef FORA_HOT_RANGE
#define FORA_HOT_RANGE 32
#endif
constexpr unsigned long long kHotRange = FORA_HOT_RANGE;
#ifndef FORA_HOT_STRETCH
#define FORA_HOT_STRETCH 8
#endif
constexpr unsigned long long kHotStretch = FORA_HOT_STRETCH;

// Node id of a target code of GraphDev::scol.
__device__ __forceinline__ uint32_t hot_decode(const GraphDev& g, uint32_t code) {
  return (code & kHotBit) ? g.hot_node[code & ~kHotBit] : code;
}

__device__ __forceinline__ void hot_slice(const GraphDev& g, double* r, unsigned long long base,
                                          double* hacc, bool agg, uint32_t code, uint32_t owner,
                                          double inc, bool act, uint32_t* err,
                                          unsigned long long n) {
  double add;
  if (!run_lead(code, owner, inc, act, add)) return;
  if (code & kHotBit) {
    const uint32_t h = code & ~kHotBit;
    if (!FORA_IN_RANGE(err, h, (uint32_t)g.nhot)) return;
    if (agg) atomicAdd(&hacc[h], add);
    else atomicAdd(&r[base + g.hot_node[h]], add);
  } else if (FORA_IN_RANGE(err, code, n)) {
    atomicAdd(&r[base + code], add);
  }
}

// Light rounds: the take tile of this lane's push target is marked (when act).
__device__ __forceinline__ void hot_mark(const GraphDev& g, const BatchDev& b, int cs,
                                         uint32_t code, bool act) {
  const unsigned long long n = (unsigned long long)g.n;
  if (!act) return;
  const uint32_t x = hot_decode(g, code);
  if (x < n) b.tile_dirty[(unsigned long long)cs * b.tiles + x / kTileNodes] = 1;
}

// Group grp of source cs (its groups start at clo, its frontier has ccnt entries): the
// out-edges of 32 frontier entries with d <= kHubChunk, 128 edges per iteration.
__device__ __forceinline__ void hot_group(const GraphDev& g, const BatchDev& b,
                                          const unsigned long long* q, int cs,
                                          unsigned long long clo, uint32_t ccnt,
                                          unsigned long long grp, bool light, bool agg,
                                          double* hacc) {
  const uint32_t lane = lane_id();
  const unsigned long long n = (unsigned long long)g.n;
  const unsigned long long base_gi = (unsigned long long)cs * n;
  const uint32_t i = (uint32_t)(grp - clo) * 32u + lane;
  uint32_t c = 0, rb = 0;
  double inc = 0.0;
  if (i < ccnt) {
    const uint32_t v = (uint32_t)q[base_gi + i];
    rb = g.row[v];
    const uint32_t d = g.row[v + 1] - rb;
    if (d <= kHubChunk) {
      c = d;
      inc = b.fa[base_gi + i];
    }
  }
  const uint32_t incl = warp_incl_scan(c);
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t excl = incl - c;
  for (uint32_t base = 0; base < total; base += 128) {
    uint32_t u[4], own[4];
    double ik[4];
    bool act[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t e = base + 32 * k + lane;
      int lo = 0, hi = 31;  // owner: the first lane whose inclusive prefix exceeds e
#pragma unroll
      for (int s2 = 0; s2 < 5; ++s2) {
        const int mid = (lo + hi) >> 1;
        if (__shfl_sync(kFull, incl, mid) > e) hi = mid; else lo = mid + 1;
      }
      const uint32_t ek = __shfl_sync(kFull, excl, lo);
      const uint32_t rbk = __shfl_sync(kFull, rb, lo);
      ik[k] = __shfl_sync(kFull, inc, lo);
      own[k] = (uint32_t)lo;
      act[k] = e < total;
      u[k] = act[k] ? g.scol[rbk + (e - ek)] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      hot_slice(g, b.r, base_gi, hacc, agg, u[k], own[k], ik[k], act[k], b.err, n);
    if (light) {  // warp-uniform
#pragma unroll
      for (int k = 0; k < 4; ++k) hot_mark(g, b, cs, u[k], act[k]);
    }
  }
}

// Hub item h of source cs (its items start at clo): kHubChunk out-edges of one node.
__device__ __forceinline__ void hot_hub(const GraphDev& g, const BatchDev& b,
                                        const unsigned long long* q, int cur, int cs,
                                        unsigned long long clo, unsigned long long h, bool light,
                                        bool agg, double* hacc) {
  const uint32_t lane = lane_id();
  const unsigned long long n = (unsigned long long)g.n;
  const unsigned long long item = b.hub[cur][(unsigned long long)cs * b.hub_stride + (h - clo)];
  const unsigned long long fi = item >> kHubChunkBits;
  const uint32_t c = (uint32_t)(item & ((1ull << kHubChunkBits) - 1));
  const uint32_t v = (uint32_t)q[fi];
  const uint32_t rb = g.row[v], re = g.row[v + 1];
  const double inc = b.fa[fi];
  const uint32_t beg = rb + c * kHubChunk;
  const uint32_t end = min(beg + kHubChunk, re);
  uint32_t u[kHubChunk / 32];
  bool act[kHubChunk / 32];
#pragma unroll
  for (int k = 0; k < (int)(kHubChunk / 32); ++k) {
    const uint32_t p = beg + 32 * k + lane;
    act[k] = p < end;
    u[k] = act[k] ? g.scol[p] : 0u;
  }
#pragma unroll
  for (int k = 0; k < (int)(kHubChunk / 32); ++k)
    hot_slice(g, b.r, (unsigned long long)cs * n, hacc, agg, u[k], 0u, inc, act[k], b.err, n);
  if (light) {  // warp-uniform
#pragma unroll
    for (int k = 0; k < (int)(kHubChunk / 32); ++k) hot_mark(g, b, cs, u[k], act[k]);
  }
}

// Item x of a phase (0: groups, 1: hub items) of source cs.
__device__ __forceinline__ void hot_item(const GraphDev& g, const BatchDev& b, int phase,
                                         const unsigned long long* q, int cur,
                                         const uint32_t* cnt, int cs, unsigned long long clo,
                                         unsigned long long x, bool light, bool agg,
                                         double* hacc) {
  if (phase == 0)
    hot_group(g, b, q, cs, clo, cnt[cs], x, light, agg, hacc);
  else
    hot_hub(g, b, q, cur, cs, clo, x, light, agg, hacc);
}

// The items of source cs in the range [lo, hi) are summed in shared memory when the
// source's round is heavy and they are at least kHotStretch.
__device__ __forceinline__ bool hot_summed(const BatchDev& b, const unsigned long long* pre,
                                           int cs, unsigned long long lo, unsigned long long hi) {
  const unsigned long long s0 = max(lo, pre[cs]), s1 = min(hi, pre[cs + 1]);
  return b.light[cs] == 0 && s1 - s0 >= kHotStretch;
}

// 5 resident blocks (48 registers): 6 (40 registers, a few spilled) and 4 were slower by
// 2-4% and 3-10%.
#ifndef FORA_SPREAD_HOT_MIN_BLOCKS
#define FORA_SPREAD_HOT_MIN_BLOCKS 5
#endif
__global__ void __launch_bounds__(kSpreadThreads, FORA_SPREAD_HOT_MIN_BLOCKS)
    k_push_spread_hot(GraphDev g, BatchDev b) {
  __shared__ double hacc[kHotSlots];
  __shared__ unsigned long long s_range[2];  // one per phase: no thread reads a stale one
  __shared__ uint32_t s_next;
  const int cur = b.ps->cur;
  const unsigned long long* q = b.q[cur];
  const uint32_t* cnt = b.slot_cnt + (size_t)cur * b.cnt_stride;
  const unsigned long long width = (unsigned long long)b.spread_width;
  const uint32_t lane = lane_id();
  const unsigned long long base_n = (unsigned long long)g.n;
  for (int h = threadIdx.x; h < g.nhot; h += blockDim.x) hacc[h] = 0.0;

  // phase 0: groups, phase 1: hub items; segment k of a phase's items is
  // [k * seg, min((k + 1) * seg, total)), taken kHotRange items at a time, the ranges of
  // the segments interleaved
  for (int phase = 0; phase < 2; ++phase) {
    const unsigned long long total = phase == 0 ? b.ps->ngroups : b.ps->nhub;
    const unsigned long long* pre = phase == 0 ? b.gpre : b.hpre;
    unsigned long long* work = b.work + (phase == 0 ? 0 : 16);
    const unsigned long long seg = (total + width - 1) / width;
    const unsigned long long rseg = (seg + kHotRange - 1) / kHotRange;
    const unsigned long long rtotal = rseg * width;
    for (;;) {
      if (threadIdx.x == 0) {
        s_range[phase] = atomicAdd(work, 1ull);
        s_next = 0;
      }
      __syncthreads();
      const unsigned long long vr = s_range[phase];
      if (vr >= rtotal) break;  // block-uniform
      const unsigned long long sbeg = (vr % width) * seg;
      const unsigned long long lo = sbeg + (vr / width) * kHotRange;
      const unsigned long long hi = min(lo + kHotRange, min(sbeg + seg, total));
      // the items not summed, warp by warp with one reduction per push
      int cs = 0;
      unsigned long long clo = 1, chi = 0;
      bool skip = false, light = false;
      for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&s_next, 1u);
        k = __shfl_sync(kFull, k, 0);
        const unsigned long long x = lo + k;
        if (x >= hi) break;  // warp-uniform
        if (x < clo || x >= chi) {  // warp-uniform
          cs = slot_of(pre, b.nsrc, x);
          clo = pre[cs];
          chi = pre[cs + 1];
          skip = hot_summed(b, pre, cs, lo, hi);
          light = b.light[cs] != 0;
        }
        if (!skip) hot_item(g, b, phase, q, cur, cnt, cs, clo, x, light, false, hacc);
      }
      // the summed stretches, one source at a time with the whole block
      for (unsigned long long x = lo; x < hi;) {  // block-uniform
        const int s = slot_of(pre, b.nsrc, x);
        const unsigned long long s1 = min(hi, pre[s + 1]);
        if (hot_summed(b, pre, s, lo, hi)) {
          __syncthreads();  // s_next free, hacc zero
          if (threadIdx.x == 0) s_next = 0;
          __syncthreads();
          for (;;) {
            uint32_t k = 0;
            if (lane == 0) k = atomicAdd(&s_next, 1u);
            k = __shfl_sync(kFull, k, 0);
            if (x + k >= s1) break;  // warp-uniform
            hot_item(g, b, phase, q, cur, cnt, s, pre[s], x + k, false, true, hacc);
          }
          __syncthreads();  // every add of the stretch is in hacc
          const unsigned long long base = (unsigned long long)s * base_n;
          for (int h = threadIdx.x; h < g.nhot; h += blockDim.x) {
            const double a = hacc[h];
            if (a != 0.0) {  // every add is positive: zero means untouched
              atomicAdd(&b.r[base + g.hot_node[h]], a);
              hacc[h] = 0.0;
            }
          }
        }
        x = s1;
      }
      __syncthreads();  // s_range, s_next and hacc free for the next range
    }
  }
}

// Detection and take of the next frontier in one pass.  Warp w scans tiles w, w + W, ...
// of kTileNodes nodes of one pushing source; for 8 words of 32 nodes at a time the
// residues and both row offsets are loaded before any is used, the crossing nodes of
// the 8 words are counted, one atomic per counter reserves their places in the source's
// queue region, and the crossing nodes are taken.
// Resident blocks per SM the take and the spread are compiled for (measured on the 2^20
// graph, 256 sources: take 3 -> 4 blocks 120.4 -> 118.5 ms of push; spread 7 or 8 blocks
// instead of 6 made it slower, 128-130 ms: more scattered reductions in flight contend at L2).
#ifndef FORA_TAKE_MIN_BLOCKS
#define FORA_TAKE_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(kTakeThreads, FORA_TAKE_MIN_BLOCKS) k_push_take(GraphDev g, BatchDev b) {
  const PushState* ps = b.ps;
  const int nx = ps->cur ^ 1;
  const unsigned long long n = (unsigned long long)g.n;
  const unsigned long long tps = (n + kTileNodes - 1) / kTileNodes;
  const unsigned long long ntiles = (unsigned long long)ps->nact * tps;
  uint32_t* cnt_nx = b.slot_cnt + (size_t)nx * b.cnt_stride;
  uint32_t* hcnt_nx = b.slot_cnt + (size_t)(2 + nx) * b.cnt_stride;
  unsigned long long* qn = b.q[nx];
  unsigned long long* hn = b.hub[nx];
  const double alpha = b.alpha, beta = __dadd_rn(1.0, -b.alpha);
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const unsigned long long wpb = blockDim.x >> 5;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * wpb;
  __shared__ uint32_t stage_u[kTakeThreads / 32][256], stage_d[kTakeThreads / 32][256];
  __shared__ double stage_a[kTakeThreads / 32][256];
  uint32_t* st_u = stage_u[threadIdx.x >> 5];
  uint32_t* st_d = stage_d[threadIdx.x >> 5];
  double* st_a = stage_a[threadIdx.x >> 5];
  for (unsigned long long t = blockIdx.x * wpb + (threadIdx.x >> 5); t < ntiles; t += nwarps) {
    const uint32_t s = b.alist[t / tps];
    if (b.balance && b.stopped[s]) continue;  // warp-uniform: stopped before its first push
    if (b.light[s]) {  // warp-uniform: only the tiles this round's spread added to
      uint8_t* flag = b.tile_dirty + (unsigned long long)s * b.tiles + t % tps;
      if (*flag == 0) continue;
      __syncwarp();
      if (lane == 0) *flag = 0;
    }
    const uint32_t tb = (uint32_t)((t % tps) * kTileNodes);
    const double rm = b.rmax[s];
    const float rmf = __double2float_rn(rm);
    const bool fast = rmf >= 0x1p-100f && rmf <= 0x1p60f;
    const unsigned long long g0 = (unsigned long long)s * n;
    uint32_t t_cnt = 0;
    unsigned long long t_d = 0;
    double t_moved = 0.0;  // this lane's alpha a of the tile (balanced push only)
#pragma unroll 1
    for (uint32_t k0 = 0; k0 < kTileNodes / 32; k0 += 8) {
      // 256 consecutive nodes: residues and row offsets (nodes past n read row[n], so
      // their degree is 0) loaded before any is used; the row offset that ends the last
      // node of a word is the next lane's, and for lane 31 the next word's first
      const uint32_t ub = tb + k0 * 32;
      double rv[8];
      uint32_t d[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t u = ub + kk * 32 + lane;
        rv[kk] = u < n ? b.r[g0 + u] : 0.0;
        d[kk] = g.row[min((unsigned long long)u, n)];
      }
      const uint32_t tail = g.row[min((unsigned long long)(ub + 256), n)];
      uint32_t m[8], any = 0, mine = 0, my_h = 0, my_d = 0;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t first_next = kk < 7 ? __shfl_sync(kFull, d[kk + 1], 0) : tail;
        const uint32_t down = __shfl_down_sync(kFull, d[kk], 1);
        d[kk] = (lane < 31 ? down : first_next) - d[kk];
      }
      uint32_t above = 0, undecided = 0;  // bit kk: word kk of this lane
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t f = threshold_fast(rv[kk], rmf, fast, d[kk]);
        above |= (f == 1u ? 1u : 0u) << kk;
        undecided |= (f == 2u ? 1u : 0u) << kk;
      }
      if (__any_sync(kFull, undecided != 0)) {  // rare: a residue within 2^-19 of its threshold
        for (int kk = 0; kk < 8; ++kk)
          if (((undecided >> kk) & 1u) && threshold_exact(rv[kk], rm, d[kk])) above |= 1u << kk;
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const bool cross = (above >> kk) & 1u;
        m[kk] = __ballot_sync(kFull, cross);
        any |= m[kk];
        mine += __popc(m[kk]);
        if (cross) {
          my_h += hub_chunks_of(d[kk]);
          my_d += d[kk];
        }
      }
      if (any == 0) continue;  // warp-uniform
      // distinct nodes of one source: their degrees sum to at most m < 2^32
      const uint32_t hsum = __reduce_add_sync(kFull, my_h);
      t_d += __reduce_add_sync(kFull, my_d);
      t_cnt += mine;
      uint32_t qb = 0, hb = 0;
      if (lane == 0) {
        qb = atomicAdd(&cnt_nx[s], mine);
        if (hsum) hb = atomicAdd(&hcnt_nx[s], hsum);
      }
      qb = __shfl_sync(kFull, qb, 0);
      hb = __shfl_sync(kFull, hb, 0);
      // the batch's crossing nodes, packed in (word, lane) order into this warp's stage,
      // so the take's FP64 arithmetic runs on 32 crossing nodes per instruction
      {
        uint32_t before = 0;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          if ((m[kk] >> lane) & 1u) {
            const uint32_t e = before + __popc(m[kk] & lt_mask);
            st_u[e] = ub + kk * 32 + lane;
            st_d[e] = d[kk];
            st_a[e] = rv[kk];
          }
          before += __popc(m[kk]);
        }
      }
      __syncwarp();
      uint32_t hp = hb;
      for (uint32_t e0 = 0; e0 < mine; e0 += 32) {
        const uint32_t e = e0 + lane;
        const bool live = e < mine;
        uint32_t u = 0, dk = 1;
        double a = 0.0, rs = 0.0, inv = 0.0;
        if (live) {
          u = st_u[e];
          dk = st_d[e];
          a = st_a[e];
          rs = b.res[g0 + u];
          inv = g.invd[u];
        }
        const uint32_t nch = live ? hub_chunks_of(dk) : 0u;
        const uint32_t nch_incl = hsum ? warp_incl_scan(nch) : 0u;  // lower entries first
        if (live && FORA_IN_RANGE(b.err, qb + e, n) &&
            FORA_IN_RANGE(b.err, hp + nch_incl, b.hub_stride + 1)) {
          const unsigned long long gi = g0 + u;
          // the take: reserve += alpha a, r = 0, spread increment
          b.r[gi] = 0.0;
          const double moved = __dmul_rn(alpha, a);
          b.res[gi] = __dadd_rn(rs, moved);
          if (b.balance) t_moved = __dadd_rn(t_moved, moved);
          const unsigned long long qi = g0 + qb + e;
          qn[qi] = ((unsigned long long)s << 32) | u;
          b.fa[qi] = __dmul_rn(__dmul_rn(beta, a), inv);  // (1 - alpha) a / d
          const unsigned long long hbase =
              (unsigned long long)s * b.hub_stride + hp + (nch_incl - nch);
          for (uint32_t c = 0; c < nch; ++c) hn[hbase + c] = (qi << kHubChunkBits) | c;
        }
        if (hsum) hp += __shfl_sync(kFull, nch_incl, 31);
      }
      __syncwarp();
    }
    if (b.balance && t_cnt) {  // warp-uniform
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t_moved = __dadd_rn(t_moved, __shfl_down_sync(kFull, t_moved, o));
    }
    if (lane == 0 && t_cnt) {
      atomicAdd(&b.stats[s].pushes, (unsigned long long)t_cnt);
      atomicAdd(&b.stats[s].edge_pushes, t_d);
      if (b.balance) atomicAdd(&b.stats[s].moved, t_moved);
    }
  }
}

// End of a round (one block): the new frontier's per-source group and hub-item prefixes,
// the list of sources that still push, zeroed counters for the round after, and the
// loop condition (at most b.max_rounds push rounds).
__global__ void __launch_bounds__(1024) k_push_advance(BatchDev b,
                                                       cudaGraphConditionalHandle loop,
                                                       int in_graph) {
  PushState* ps = b.ps;
  const int cur = ps->cur, nx = cur ^ 1;
  const int nsrc = b.nsrc;
  const size_t cs = (size_t)b.cnt_stride;
  const uint32_t* cnt_nx = b.slot_cnt + (size_t)nx * cs;
  const uint32_t* hcnt_nx = b.slot_cnt + (size_t)(2 + nx) * cs;
  uint32_t* cnt_cur = b.slot_cnt + (size_t)cur * cs;
  uint32_t* hcnt_cur = b.slot_cnt + (size_t)(2 + cur) * cs;
  __shared__ unsigned long long carry_g, carry_h, carry_a;
  if (threadIdx.x == 0) { carry_g = 0; carry_h = 0; carry_a = 0; }
  __syncthreads();
  for (int base = 0; base < nsrc; base += blockDim.x) {
    const int s = base + (int)threadIdx.x;
    const uint32_t c = s < nsrc ? cnt_nx[s] : 0u;
    const uint32_t h = s < nsrc ? hcnt_nx[s] : 0u;
    // does the source's next take run: it found a frontier, or (balanced push) the cost
    // rule lets it go on, with the threshold halved when no node was above it
    bool take = c > 0;
    if (s < nsrc && b.balance) {
      if (b.stopped[s]) {
        take = false;
      } else {
        const SlotStats& st = b.stats[s];
        const double fc = __dadd_rn(__dmul_rn(b.cost_edge, (double)st.edge_pushes),
                                    __dmul_rn(b.cost_push, (double)st.pushes));
        const double wc = __dmul_rn(__dmul_rn(__dadd_rn(1.0, -st.moved), b.bal_scale), b.cost_walk);
        if (fc >= wc) {
          b.stopped[s] = 1u;  // the frontier just taken is still spread
          take = false;
        } else {
          if (c == 0) b.theta[s] = __dmul_rn(0.5, b.theta[s]);
          take = true;
        }
      }
    }
    if (s < nsrc && c > 0) b.stats[s].rounds += 1u;  // a push round of this source
    if (s < nsrc) {
      // the frontier just taken is spread next; a light one lets the next take scan only
      // the tiles it touches (a halved threshold needs a full scan)
      const unsigned long long ep = b.stats[s].edge_pushes;
      const unsigned long long round_edges = ep - b.last_edges[s];
      b.last_edges[s] = ep;
      const bool halved = b.balance && take && c == 0;
      b.light[s] = (take && !halved && round_edges < b.light_edges) ? 1 : 0;
    }
    unsigned long long ge, he, gt, ht, ae, ze, at, zt;
    block_scan2((c + 31u) / 32u, h, &ge, &he, &gt, &ht);
    block_scan2(take ? 1u : 0u, 0u, &ae, &ze, &at, &zt);
    if (s < nsrc) {
      b.gpre[s] = carry_g + ge;
      b.hpre[s] = carry_h + he;
      if (take) b.alist[carry_a + ae] = (uint32_t)s;
      cnt_cur[s] = 0;  // counters of the frontier just spread: they serve the round after
      hcnt_cur[s] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) { carry_g += gt; carry_h += ht; carry_a += at; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.gpre[nsrc] = carry_g;
    b.hpre[nsrc] = carry_h;
    ps->ngroups = carry_g;
    ps->nhub = carry_h;
    ps->nact = (uint32_t)carry_a;
    ps->cur = nx;
    ps->round += 1;
    b.work[0] = 0;  // dynamic work counters of the next spread
    b.work[16] = 0;
    // ps->round passes have run; the last one took the frontier of push round ps->round
    // (the first pass only finds F_0), so going on is allowed while that is <= the cap.
    // Another pass is needed while a source takes again or a taken frontier waits for its
    // spread (a source the cost rule just stopped).
    const bool more = carry_a > 0 || carry_g > 0 || carry_h > 0;
    const bool go = more && ps->round <= b.max_rounds;
    if (more && !go) atomicOr(b.err, kErrPushNotConverged);
    ps->go = go ? 1u : 0u;
    if (in_graph) cudaGraphSetConditional(loop, go ? 1u : 0u);
  }
}

// Sources joining a batch between two push rounds (serving): slots [first, first + k)
// (their sources, r_max and zeroed state already in place) get r(s) = 1 and enter the next
// take, and the frontier prefixes are extended over them (empty frontiers).  One block.
// The push of a source depends only on its own residues, so a source that joins later runs
// the same rounds as it would from the start.
__global__ void k_push_join(GraphDev g, BatchDev b, int first, int k) {
  PushState* ps = b.ps;
  const unsigned long long gtot = b.gpre[first], htot = b.hpre[first];
  const uint32_t nact = ps->nact;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const int slot = first + i;
    const uint32_t src = (uint32_t)b.sources[slot];
    b.r[(unsigned long long)slot * (unsigned long long)g.n + src] = 1.0;
    b.alist[nact + i] = (uint32_t)slot;
    b.light[slot] = 1;
    b.tile_dirty[(unsigned long long)slot * b.tiles + src / kTileNodes] = 1;
    b.gpre[slot + 1] = gtot;
    b.hpre[slot + 1] = htot;
  }
  __syncthreads();
  if (threadIdx.x == 0) ps->nact = nact + (uint32_t)k;
}

// The frontier test of k_push_take on given (r, r_max, d) triples.
__global__ void k_threshold_table(const double* r, const double* rm, const uint32_t* d,
                                  uint8_t* out, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float rmf = __double2float_rn(rm[i]);
  const bool fast = rmf >= 0x1p-100f && rmf <= 0x1p60f;
  out[i] = above_threshold(r[i], rm[i], rmf, fast, d[i]) ? 1 : 0;
}

}  // namespace

cudaError_t launch_threshold_table(const double* r, const double* rm, const uint32_t* d,
                                   uint8_t* out, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_threshold_table<<<(count + 255) / 256, 256, 0, st>>>(r, rm, d, out, count);
  return cudaGetLastError();
}

cudaError_t launch_push_join(const GraphDev& g, const BatchDev& b, int first, int k,
                             cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_push_join<<<1, 256, 0, st>>>(g, b, first, k);
  return cudaGetLastError();
}

cudaError_t launch_push_seed(const GraphDev& g, const BatchDev& b, cudaStream_t st) {
  const int threads = 256;
  k_push_seed<<<(b.nsrc + threads - 1) / threads, threads, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_push_body(const GraphDev& g, const BatchDev& b, int num_sms,
                             cudaGraphConditionalHandle loop, bool in_graph, cudaStream_t st) {
  // one wave of resident blocks for the spread (with the dynamic work counter the warps
  // in flight cover one contiguous window of the frontier) and for the take
  const bool hot = b.spread_hot && g.scol && g.nhot > 0;
  const void* spread = hot ? (const void*)k_push_spread_hot : (const void*)k_push_spread;
  const int spread_per_sm = resident_blocks(spread, kSpreadThreads);
  const int take_per_sm = resident_blocks((const void*)k_push_take, kTakeThreads);
  if (spread_per_sm == 0 || take_per_sm == 0) return cudaErrorInvalidConfiguration;
  if (hot)
    k_push_spread_hot<<<num_sms * spread_per_sm, kSpreadThreads, 0, st>>>(g, b);
  else
    k_push_spread<<<num_sms * spread_per_sm, kSpreadThreads, 0, st>>>(g, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_take<<<num_sms * take_per_sm, kTakeThreads, 0, st>>>(g, b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_advance<<<1, 1024, 0, st>>>(b, loop, in_graph ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace fora
