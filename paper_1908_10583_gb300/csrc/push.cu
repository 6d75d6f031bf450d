// Forward Push (Alg. 1) as synchronous frontier rounds over a batch of sources.
//
// Round t over the frontier F_t (pairs (slot, v) with r(v) > r_max * d(v)):
//   phase A  (k_push_take):    a_v = r(v); reserve(v) += alpha * a_v; r(v) = 0;
//                              inc_v = (1 - alpha) * a_v / d(v)
//   phase B  (k_push_spread):  r(u) += inc_v for every out-edge (v, u), FP64 atomics;
//                              the add that lifts r(u) above r_max * d(u) appends u to F_{t+1}
// Phase A of a round finishes before its phase B starts (two launches), so residue
// that reaches a node of F_t during round t stays in r for round t+1.  At the start
// of phase B every r(u) <= r_max * d(u) (all larger ones were just taken), and r(u)
// only grows during phase B, so exactly one add crosses the threshold per node.
//
// Phase B load balance: a warp takes 32 frontier entries, scans their degrees and
// walks their concatenated edge lists 32 edges at a time (coalesced col reads; the
// owner of an edge is found by a 5-step binary search over the lane prefix sums).
// Nodes with more than kHubChunk out-edges are instead split into kHubChunk-edge
// chunks ("hub items"), one warp per chunk.
#include "fora_engine.cuh"

namespace fora {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void append_frontier(const GraphDev& g, const BatchDev& b, int nxt,
                                                bool crossed, uint32_t slot, uint32_t u,
                                                uint32_t du) {
  const uint32_t bal = __ballot_sync(kFull, crossed);
  if (bal == 0) return;
  unsigned long long base = 0;
  if (lane_id() == 0) base = atomicAdd(&b.counters[nxt * 2], (unsigned long long)__popc(bal));
  base = __shfl_sync(kFull, base, 0);
  if (crossed) {
    const unsigned long long idx = base + __popc(bal & ((1u << lane_id()) - 1u));
    b.q[nxt][idx] = ((unsigned long long)slot << 32) | u;
    if (du > kHubChunk) {
      const uint32_t nch = (du + kHubChunk - 1) / kHubChunk;
      const unsigned long long h = atomicAdd(&b.counters[nxt * 2 + 1], (unsigned long long)nch);
      for (uint32_t c = 0; c < nch; ++c) b.hub[nxt][h + c] = (idx << kHubChunkBits) | c;
    }
  }
}

// r(u) += inc for one edge; returns through append_frontier (warp-collective: every
// lane of the warp must call it, with act = false for lanes without an edge).
__device__ __forceinline__ void relax(const GraphDev& g, const BatchDev& b, int nxt, bool act,
                                      uint32_t slot, uint32_t u, double inc) {
  bool crossed = false;
  uint32_t du = 0;
  if (act) {
    const unsigned long long gi = (unsigned long long)slot * (unsigned long long)g.n + u;
    const double old = atomicAdd(&b.r[gi], inc);
    const double now = __dadd_rn(old, inc);  // the value the atomic stored
    du = g.row[u + 1] - g.row[u];
    const double thr = __dmul_rn(b.rmax[slot], (double)du);
    crossed = (old <= thr) && (now > thr);
  }
  append_frontier(g, b, nxt, crossed, slot, u, du);
}

__global__ void k_push_init(GraphDev g, BatchDev b) {
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < b.nsrc;
       slot += gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)b.sources[slot];
    const unsigned long long gi = (unsigned long long)slot * (unsigned long long)g.n + s;
    b.r[gi] = 1.0;  // Alg. 1, line 1
    const uint32_t d = g.row[s + 1] - g.row[s];
    if (1.0 > __dmul_rn(b.rmax[slot], (double)d)) {
      const unsigned long long idx = atomicAdd(&b.counters[0], 1ull);
      b.q[0][idx] = ((unsigned long long)slot << 32) | s;
      if (d > kHubChunk) {
        const uint32_t nch = (d + kHubChunk - 1) / kHubChunk;
        const unsigned long long h = atomicAdd(&b.counters[1], (unsigned long long)nch);
        for (uint32_t c = 0; c < nch; ++c) b.hub[0][h + c] = (idx << kHubChunkBits) | c;
      }
    }
  }
}

// Phase A: take the residue of every frontier node.
__global__ void k_push_take(GraphDev g, BatchDev b, int cur, uint32_t round) {
  const unsigned long long nf = b.counters[cur * 2];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += stride) {
    const unsigned long long e = b.q[cur][i];
    const uint32_t slot = (uint32_t)(e >> 32), v = (uint32_t)e;
    const unsigned long long gi = (unsigned long long)slot * (unsigned long long)g.n + v;
    const double a = b.r[gi];
    b.r[gi] = 0.0;
    b.res[gi] = __dadd_rn(b.res[gi], __dmul_rn(b.alpha, a));
    const uint32_t d = g.row[v + 1] - g.row[v];
    b.fa[i] = __ddiv_rn(__dmul_rn(__dadd_rn(1.0, -b.alpha), a), (double)d);
    // per-source counters, aggregated over the lanes that share a source
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, slot);
    const unsigned nd = __reduce_add_sync(peers, d);
    if ((int)lane_id() == __ffs(peers) - 1) {
      atomicAdd(&b.stats[slot].pushes, (unsigned long long)__popc(peers));
      atomicAdd(&b.stats[slot].edge_pushes, (unsigned long long)nd);
      atomicMax(&b.stats[slot].rounds, round);
    }
  }
}

// Phase B: spread the taken residue along the out-edges.
__global__ void k_push_spread(GraphDev g, BatchDev b, int cur) {
  const int nxt = cur ^ 1;
  const unsigned long long nf = b.counters[cur * 2];
  const unsigned long long nh = b.counters[cur * 2 + 1];
  const uint32_t lane = lane_id();
  const unsigned long long warp =
      ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;

  // groups of 32 frontier entries (nodes with d <= kHubChunk)
  const unsigned long long ngroups = (nf + 31) / 32;
  for (unsigned long long grp = warp; grp < ngroups; grp += nwarps) {
    const unsigned long long i = grp * 32 + lane;
    uint32_t cnt = 0, rb = 0, slot = 0;
    double inc = 0.0;
    if (i < nf) {
      const unsigned long long e = b.q[cur][i];
      slot = (uint32_t)(e >> 32);
      const uint32_t v = (uint32_t)e;
      rb = g.row[v];
      const uint32_t d = g.row[v + 1] - rb;
      if (d <= kHubChunk) {
        cnt = d;
        inc = b.fa[i];
      }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, off);
      if ((int)lane >= off) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - cnt;
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t e = base + lane;
      // owner: the first lane whose inclusive prefix exceeds e
      int lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi) >> 1;
        const uint32_t im = __shfl_sync(kFull, incl, mid);
        if (im > e) hi = mid; else lo = mid + 1;
      }
      const uint32_t ek = __shfl_sync(kFull, excl, lo);
      const uint32_t rbk = __shfl_sync(kFull, rb, lo);
      const uint32_t sk = __shfl_sync(kFull, slot, lo);
      const double ik = __shfl_sync(kFull, inc, lo);
      const bool act = e < total;
      const uint32_t u = act ? (uint32_t)g.col[rbk + (e - ek)] : 0u;
      relax(g, b, nxt, act, sk, u, ik);
    }
  }

  // hub chunks
  for (unsigned long long h = warp; h < nh; h += nwarps) {
    const unsigned long long item = b.hub[cur][h];
    const unsigned long long fi = item >> kHubChunkBits;
    const uint32_t c = (uint32_t)(item & ((1ull << kHubChunkBits) - 1));
    const unsigned long long e = b.q[cur][fi];
    const uint32_t slot = (uint32_t)(e >> 32), v = (uint32_t)e;
    const uint32_t rb = g.row[v], re = g.row[v + 1];
    const double inc = b.fa[fi];
    const uint32_t beg = rb + c * kHubChunk;
    const uint32_t end = min(beg + kHubChunk, re);
    for (uint32_t p0 = beg; p0 < end; p0 += 32) {
      const uint32_t p = p0 + lane;
      const bool act = p < end;
      const uint32_t u = act ? (uint32_t)g.col[p] : 0u;
      relax(g, b, nxt, act, slot, u, inc);
    }
  }
}

}  // namespace

cudaError_t launch_push_init(const GraphDev& g, const BatchDev& b, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (b.nsrc + threads - 1) / threads;
  k_push_init<<<blocks, threads, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_push_round(const GraphDev& g, const BatchDev& b, int cur, uint64_t nf,
                              uint64_t nh, uint32_t round, int num_sms, cudaStream_t st) {
  const int threads = 256;
  const uint64_t max_blocks = (uint64_t)num_sms * 16;
  uint64_t blocks_a = (nf + threads - 1) / threads;
  if (blocks_a > max_blocks) blocks_a = max_blocks;
  if (blocks_a == 0) blocks_a = 1;
  k_push_take<<<(unsigned)blocks_a, threads, 0, st>>>(g, b, cur, round);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nxt = cur ^ 1;
  e = cudaMemsetAsync(b.counters + nxt * 2, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const uint64_t warps = (nf + 31) / 32 + nh;
  uint64_t blocks_b = (warps * 32 + threads - 1) / threads;
  if (blocks_b > max_blocks) blocks_b = max_blocks;
  if (blocks_b == 0) blocks_b = 1;
  k_push_spread<<<(unsigned)blocks_b, threads, 0, st>>>(g, b, cur);
  return cudaGetLastError();
}

}  // namespace fora
