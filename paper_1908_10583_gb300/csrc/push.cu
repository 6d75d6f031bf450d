// Forward Push (Alg. 1) as synchronous frontier rounds over a batch of sources.
//
// F_t holds the pairs (slot, v) with r(v) > r_max * d(v), sorted by (slot, v), and for
// each entry the increment inc_v = (1 - alpha) a_v / d(v) of its taken residue a_v.
// Round t:
//   k_push_spread   r(u) += inc_v for every out-edge (v, u) of F_t: FP64 reductions
//                   that return nothing, so a warp never waits on an atomic.
//   k_push_detect   F_{t+1} = {u : r(u) > r_max * d(u)} over the sources that pushed in
//                   round t (every other r is unchanged and below its threshold): one
//                   pass marks the crossing nodes in a bit mask and counts them per block,
//   k_push_scan     one block turns the per-block counts into output offsets,
//   k_push_emit     a second pass writes F_{t+1} in (slot, v) order and takes each new
//                   node's residue: a_u = r(u); reserve(u) += alpha a_u; r(u) = 0;
//                   inc_u = (1 - alpha) a_u / d(u)   (the first half of round t+1).
// The take of round t+1 happens after every add of round t (kernel boundary), so
// residue arriving at a frontier node during a round waits for the next round.
//
// Spread load balance: a warp takes 32 frontier entries with d <= kHubChunk, scans their
// degrees and walks their concatenated edge lists 128 edges per iteration (coalesced
// col reads); nodes with more out-edges are split into kHubChunk-edge hub items, one
// warp each.  Sorted frontiers keep the warps in flight on a few sources at a time, so
// the residue arrays they add into stay in L2.
#include "fora_engine.cuh"

namespace fora {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kDetectThreads = 256;
constexpr int kSpreadThreads = 256;

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

// Words of the crossing mask: one bit per (slot, node), each slot padded to whole words.
__device__ __forceinline__ unsigned long long words_per_slot(int64_t n) {
  return ((unsigned long long)n + 31) / 32;
}

__global__ void k_push_seed(GraphDev g, BatchDev b) {
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < b.nsrc;
       slot += gridDim.x * blockDim.x) {
    b.r[(unsigned long long)slot * (unsigned long long)g.n + (uint32_t)b.sources[slot]] = 1.0;
    // Alg. 1, line 1: r(s) = 1.  The detection that builds F_0 runs with parity 1:
    // it scans the sources flagged in active[1] and writes F_0 into q[0].
    b.active[b.nsrc + slot] = 1;
  }
}

__global__ void __launch_bounds__(kSpreadThreads) k_push_spread(GraphDev g, BatchDev b, int cur) {
  const unsigned long long nf = b.counters[cur * 2];
  const unsigned long long nh = b.counters[cur * 2 + 1];
  const unsigned long long* q = b.q[cur];
  const uint32_t lane = lane_id();
  const unsigned long long warp =
      ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long n = (unsigned long long)g.n;

  // groups of 32 frontier entries (nodes with d <= kHubChunk)
  const unsigned long long ngroups = (nf + 31) / 32;
  for (unsigned long long grp = warp; grp < ngroups; grp += nwarps) {
    const unsigned long long i = grp * 32 + lane;
    uint32_t cnt = 0, rb = 0;
    unsigned long long base_gi = 0;  // slot * n
    double inc = 0.0;
    if (i < nf) {
      const unsigned long long e = q[i];
      const uint32_t v = (uint32_t)e;
      base_gi = (e >> 32) * n;
      rb = g.row[v];
      const uint32_t d = g.row[v + 1] - rb;
      if (d <= kHubChunk) {
        cnt = d;
        inc = b.fa[i];
      }
    }
    const uint32_t incl = warp_incl_scan(cnt);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - cnt;
    for (uint32_t base = 0; base < total; base += 128) {
      uint32_t u[4];
      unsigned long long gb[4];
      double ik[4];
      bool act[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t e = base + 32 * k + lane;
        int lo = 0, hi = 31;  // owner: the first lane whose inclusive prefix exceeds e
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const int mid = (lo + hi) >> 1;
          if (__shfl_sync(kFull, incl, mid) > e) hi = mid; else lo = mid + 1;
        }
        const uint32_t ek = __shfl_sync(kFull, excl, lo);
        const uint32_t rbk = __shfl_sync(kFull, rb, lo);
        gb[k] = __shfl_sync(kFull, base_gi, lo);
        ik[k] = __shfl_sync(kFull, inc, lo);
        act[k] = e < total;
        u[k] = act[k] ? (uint32_t)g.col[rbk + (e - ek)] : 0u;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (act[k]) atomicAdd(&b.r[gb[k] + u[k]], ik[k]);
    }
  }

  // hub items: kHubChunk edges of one frontier node each
  for (unsigned long long h = warp; h < nh; h += nwarps) {
    const unsigned long long item = b.hub[cur][h];
    const unsigned long long fi = item >> kHubChunkBits;
    const uint32_t c = (uint32_t)(item & ((1ull << kHubChunkBits) - 1));
    const unsigned long long e = q[fi];
    const uint32_t v = (uint32_t)e;
    const unsigned long long gbase = (e >> 32) * n;
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
      if (u[k] != 0xFFFFFFFFu) atomicAdd(&b.r[gbase + u[k]], inc);
  }
}

// Element range (in mask words) of block `blk`.
__device__ __forceinline__ void word_range(unsigned long long total, int blk, int nblk,
                                           unsigned long long* beg, unsigned long long* end) {
  *beg = total * (unsigned long long)blk / (unsigned long long)nblk;
  *end = total * (unsigned long long)(blk + 1) / (unsigned long long)nblk;
}

// Pass 1: crossing mask and per-block counts (nodes, hub items) over the active slots.
// A warp takes 32 mask words (1024 nodes of one slot row, padded per slot) at a time;
// for word k the 32 lanes read 32 consecutive residues and the ballot of their tests
// is the mask word.
__global__ void __launch_bounds__(kDetectThreads) k_push_detect(GraphDev g, BatchDev b, int par) {
  const unsigned long long wps = words_per_slot(g.n);
  const unsigned long long total = (unsigned long long)b.nsrc * wps;
  unsigned long long wbeg, wend;
  word_range(total, blockIdx.x, gridDim.x, &wbeg, &wend);
  const uint32_t* act = b.active + (size_t)par * b.nsrc;
  if (blockIdx.x == 0) {  // flags of the next frontier: set by the emit pass
    uint32_t* nxt = b.active + (size_t)(par ^ 1) * b.nsrc;
    for (int s = threadIdx.x; s < b.nsrc; s += blockDim.x) nxt[s] = 0;
  }
  const uint32_t lane = lane_id();
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long nodes = 0, hubs = 0;
  for (unsigned long long gw = wbeg + 32ull * wid; gw < wend; gw += 32ull * nw) {
    uint32_t my_mask = 0;
    unsigned long long slot = gw / wps;
    unsigned long long slot_first = slot * wps;
    for (int k = 0; k < 32; ++k) {
      const unsigned long long w = gw + k;
      if (w >= wend) break;  // warp-uniform
      if (w >= slot_first + wps) { ++slot; slot_first += wps; }
      bool cross = false;
      if (act[slot]) {
        const uint32_t u = (uint32_t)((w - slot_first) * 32) + lane;
        if (u < (uint32_t)g.n) {
          const double ru = b.r[slot * (unsigned long long)g.n + u];
          if (ru > 0.0) {
            const uint32_t d = g.row[u + 1] - g.row[u];
            if (ru > __dmul_rn(b.rmax[slot], (double)d)) {
              cross = true;
              ++nodes;
              hubs += hub_chunks_of(d);
            }
          }
        }
      }
      const uint32_t m = __ballot_sync(kFull, cross);
      if ((int)lane == k) my_mask = m;
    }
    if (gw + lane < wend) b.mask[gw + lane] = my_mask;
  }
  unsigned long long ne, he, nt, ht;
  block_scan2(nodes, hubs, &ne, &he, &nt, &ht);
  if (threadIdx.x == 0) {
    b.blk_cnt[blockIdx.x] = nt;
    b.blk_walks[blockIdx.x] = ht;
  }
}

// One block: exclusive scan of the per-block counts; totals into the next counters.
__global__ void __launch_bounds__(1024) k_push_scan(BatchDev b, int nxt) {
  __shared__ unsigned long long carry_n, carry_h;
  if (threadIdx.x == 0) { carry_n = 0; carry_h = 0; }
  __syncthreads();
  for (int base = 0; base < b.residual_grid; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const unsigned long long c = i < b.residual_grid ? b.blk_cnt[i] : 0;
    const unsigned long long h = i < b.residual_grid ? b.blk_walks[i] : 0;
    unsigned long long ce, he, ct, ht;
    block_scan2(c, h, &ce, &he, &ct, &ht);
    if (i < b.residual_grid) {
      b.blk_cnt[i] = carry_n + ce;
      b.blk_walks[i] = carry_h + he;
    }
    __syncthreads();
    if (threadIdx.x == 0) { carry_n += ct; carry_h += ht; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.counters[nxt * 2] = carry_n;
    b.counters[nxt * 2 + 1] = carry_h;
  }
}

// Pass 2: write F_{t+1} in order and take the residue of its nodes.
__global__ void __launch_bounds__(kDetectThreads) k_push_emit(GraphDev g, BatchDev b, int par,
                                                              uint32_t round) {
  const int nxt = par ^ 1;
  const unsigned long long wps = words_per_slot(g.n);
  const unsigned long long total = (unsigned long long)b.nsrc * wps;
  unsigned long long wbeg, wend;
  word_range(total, blockIdx.x, gridDim.x, &wbeg, &wend);
  unsigned long long pos = b.blk_cnt[blockIdx.x];
  unsigned long long hpos = b.blk_walks[blockIdx.x];
  uint32_t* act_next = b.active + (size_t)nxt * b.nsrc;
  const double alpha = b.alpha, beta = __dadd_rn(1.0, -b.alpha);
  for (unsigned long long tile = wbeg; tile < wend; tile += kDetectThreads) {
    const unsigned long long w = tile + threadIdx.x;
    uint32_t mask = 0, nodes = 0, hubs = 0;
    unsigned long long slot = 0;
    if (w < wend) {
      mask = b.mask[w];
      if (mask) {
        slot = w / wps;
        const uint32_t u0 = (uint32_t)((w - slot * wps) * 32);
        nodes = __popc(mask);
        for (uint32_t m = mask; m; m &= m - 1) {
          const uint32_t u = u0 + __ffs(m) - 1;
          hubs += hub_chunks_of(g.row[u + 1] - g.row[u]);
        }
      }
    }
    unsigned long long ne, he, nt, ht;
    block_scan2(nodes, hubs, &ne, &he, &nt, &ht);
    if (mask) {
      const uint32_t u0 = (uint32_t)((w - slot * wps) * 32);
      unsigned long long idx = pos + ne, hidx = hpos + he;
      uint32_t dsum = 0;
      for (uint32_t m = mask; m; m &= m - 1) {
        const uint32_t u = u0 + __ffs(m) - 1;
        const unsigned long long gi = slot * (unsigned long long)g.n + u;
        const uint32_t d = g.row[u + 1] - g.row[u];
        // the take of round `round`: reserve += alpha a, r = 0, spread increment
        const double a = b.r[gi];
        b.r[gi] = 0.0;
        b.res[gi] = __dadd_rn(b.res[gi], __dmul_rn(alpha, a));
        b.q[nxt][idx] = (slot << 32) | u;
        b.fa[idx] = __ddiv_rn(__dmul_rn(beta, a), (double)d);
        const uint32_t nch = hub_chunks_of(d);
        for (uint32_t c = 0; c < nch; ++c) b.hub[nxt][hidx + c] = (idx << kHubChunkBits) | c;
        hidx += nch;
        ++idx;
        dsum += d;
      }
      act_next[slot] = 1;
      atomicAdd(&b.stats[slot].pushes, (unsigned long long)nodes);
      atomicAdd(&b.stats[slot].edge_pushes, (unsigned long long)dsum);
      atomicMax(&b.stats[slot].rounds, round);
    }
    pos += nt;
    hpos += ht;
  }
}

}  // namespace

cudaError_t launch_push_detect(const GraphDev& g, const BatchDev& b, int par, uint32_t round,
                               cudaStream_t st) {
  k_push_detect<<<b.residual_grid, kDetectThreads, 0, st>>>(g, b, par);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_scan<<<1, 1024, 0, st>>>(b, par ^ 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_emit<<<b.residual_grid, kDetectThreads, 0, st>>>(g, b, par, round);
  return cudaGetLastError();
}

cudaError_t launch_push_init(const GraphDev& g, const BatchDev& b, cudaStream_t st) {
  const int threads = 256;
  k_push_seed<<<(b.nsrc + threads - 1) / threads, threads, 0, st>>>(g, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // F_0 = {s} if 1 > r_max d(s): the detection pass over r = e_s, taken as round 1
  return launch_push_detect(g, b, /*par=*/1, /*round=*/1, st);
}

cudaError_t launch_push_round(const GraphDev& g, const BatchDev& b, int cur, uint64_t nf,
                              uint64_t nh, uint32_t round, int num_sms, cudaStream_t st) {
  const uint64_t max_blocks = (uint64_t)num_sms * 16;
  const uint64_t warps = (nf + 31) / 32 + nh;
  uint64_t blocks = (warps * 32 + kSpreadThreads - 1) / kSpreadThreads;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks == 0) blocks = 1;
  k_push_spread<<<(unsigned)blocks, kSpreadThreads, 0, st>>>(g, b, cur);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // detection scans the sources that pushed in this round (flags of parity cur) and
  // writes F_{round+1} into q[cur ^ 1], taking its residue as round round + 1
  return launch_push_detect(g, b, cur, round + 1, st);
}

}  // namespace fora
