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
    // Alg. 1: r(s) = 1.  The first pass of the loop body has an empty frontier
    // of parity 1 (nothing to spread); its detection scans the sources flagged in
    // active[1] and writes F_0 into q[0].
    b.active[b.nsrc + slot] = 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.ps->cur = 1;
    b.ps->round = 0;
  }
}

// Work is handed out dynamically (kGrab groups or hub items per atomic), so the warps
// in flight always hold the next unprocessed stretch of the sorted frontier, whatever
// the cost of each group.
constexpr unsigned long long kGrab = 4;

__global__ void __launch_bounds__(kSpreadThreads) k_push_spread(GraphDev g, BatchDev b) {
  const int cur = b.ps->cur;
  const unsigned long long nf = b.counters[cur * 2];
  const unsigned long long nh = b.counters[cur * 2 + 1];
  const unsigned long long* q = b.q[cur];
  const uint32_t lane = lane_id();
  const unsigned long long n = (unsigned long long)g.n;

  // groups of 32 frontier entries (nodes with d <= kHubChunk), visited through
  // b.spread_width interleaved segments of the sorted frontier
  const unsigned long long ngroups = (nf + 31) / 32;
  const unsigned long long width = (unsigned long long)b.spread_width;
  const unsigned long long gseg = (ngroups + width - 1) / width;
  const unsigned long long gtotal = gseg * width;
  for (;;) {
    unsigned long long v0 = 0;
    if (lane == 0) v0 = atomicAdd(&b.work[0], kGrab);
    v0 = __shfl_sync(kFull, v0, 0);
    if (v0 >= gtotal) break;
    const unsigned long long v1 = min(v0 + kGrab, gtotal);
    for (unsigned long long vg = v0; vg < v1; ++vg) {
      const unsigned long long grp = (vg % width) * gseg + vg / width;
      if (grp >= ngroups) continue;
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
          for (int s2 = 0; s2 < 5; ++s2) {
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
  }

  // hub items: kHubChunk edges of one frontier node each, same segment order
  const unsigned long long hseg = (nh + width - 1) / width;
  const unsigned long long htotal = hseg * width;
  for (;;) {
    unsigned long long v0 = 0;
    if (lane == 0) v0 = atomicAdd(&b.work[16], kGrab);
    v0 = __shfl_sync(kFull, v0, 0);
    if (v0 >= htotal) break;
    const unsigned long long v1 = min(v0 + kGrab, htotal);
    for (unsigned long long vh = v0; vh < v1; ++vh) {
      const unsigned long long h = (vh % width) * hseg + vh / width;
      if (h >= nh) continue;
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
}

// Element range (in mask words) of block `blk`.
__device__ __forceinline__ void word_range(unsigned long long total, int blk, int nblk,
                                           unsigned long long* beg, unsigned long long* end) {
  *beg = total * (unsigned long long)blk / (unsigned long long)nblk;
  *end = total * (unsigned long long)(blk + 1) / (unsigned long long)nblk;
}

// Pass 1: crossing mask, per-word hub-item counts and per-block counts (nodes, hub
// items) over the active slots.  A warp takes 32 mask words (1024 nodes, slot rows
// padded to whole words) at a time; for word k the 32 lanes test 32 consecutive nodes
// and the ballot of their tests is the mask word.  Eight words' residues are loaded
// before any is used.
__global__ void __launch_bounds__(kDetectThreads) k_push_detect(GraphDev g, BatchDev b) {
  const int par = b.ps->cur;
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
  const unsigned long long n = (unsigned long long)g.n;
  unsigned long long nodes = 0, hubs = 0;
  for (unsigned long long gw = wbeg + 32ull * wid; gw < wend; gw += 32ull * nw) {
    unsigned long long slot = gw / wps;
    // words of sources that did not push are neither scanned nor written
    if (!act[slot] && gw + 32 <= (slot + 1) * wps) continue;
    uint32_t my_mask = 0, my_hubs = 0;
    for (int k0 = 0; k0 < 32; k0 += 8) {
      double rv[8];
      uint32_t uu[8];
      unsigned long long ss[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const unsigned long long w = gw + k0 + kk;
        while (w >= (slot + 1) * wps) ++slot;
        ss[kk] = slot;
        uu[kk] = (uint32_t)((w - slot * wps) * 32) + lane;
        const bool ok = w < wend && slot < (unsigned long long)b.nsrc && act[slot] && uu[kk] < n;
        rv[kk] = ok ? b.r[slot * n + uu[kk]] : 0.0;
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        bool cross = false;
        uint32_t h = 0;
        if (rv[kk] > 0.0) {
          const uint32_t d = g.row[uu[kk] + 1] - g.row[uu[kk]];
          if (rv[kk] > __dmul_rn(b.rmax[ss[kk]], (double)d)) {
            cross = true;
            h = hub_chunks_of(d);
          }
        }
        const uint32_t m = __ballot_sync(kFull, cross);
        const uint32_t hw = __reduce_add_sync(kFull, h);
        if ((int)lane == k0 + kk) { my_mask = m; my_hubs = hw; }
        nodes += cross ? 1 : 0;
        hubs += h;
      }
    }
    const unsigned long long w = gw + lane;
    if (w < wend && act[w / wps]) {
      b.mask[w] = my_mask;
      b.hubw[w] = my_hubs;
    }
  }
  unsigned long long ne, he, nt, ht;
  block_scan2(nodes, hubs, &ne, &he, &nt, &ht);
  if (threadIdx.x == 0) {
    b.blk_cnt[blockIdx.x] = nt;
    b.blk_walks[blockIdx.x] = ht;
  }
}

// One block: exclusive scan of the per-block counts; totals into the next counters.
__global__ void __launch_bounds__(1024) k_push_scan(BatchDev b) {
  const int nxt = b.ps->cur ^ 1;
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
    b.work[0] = 0;   // dynamic work counters of the next spread
    b.work[16] = 0;
  }
}

// Pass 2: write F_{t+1} in order and take the residue of its nodes.  The block walks its
// word range in tiles of 32 words per warp; within a word the lanes are the 32 bits, so
// the residue, reserve and degree reads and the frontier writes are coalesced.
__global__ void __launch_bounds__(kDetectThreads) k_push_emit(GraphDev g, BatchDev b) {
  const int par = b.ps->cur;
  const uint32_t round = b.ps->round + 1;  // the take done here belongs to the next round
  const int nxt = par ^ 1;
  const unsigned long long wps = words_per_slot(g.n);
  const unsigned long long total = (unsigned long long)b.nsrc * wps;
  unsigned long long wbeg, wend;
  word_range(total, blockIdx.x, gridDim.x, &wbeg, &wend);
  const uint32_t* act = b.active + (size_t)par * b.nsrc;
  uint32_t* act_next = b.active + (size_t)nxt * b.nsrc;
  const double alpha = b.alpha, beta = __dadd_rn(1.0, -b.alpha);
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long n = (unsigned long long)g.n;
  unsigned long long pos = b.blk_cnt[blockIdx.x];
  unsigned long long hpos = b.blk_walks[blockIdx.x];
  for (unsigned long long tile = wbeg; tile < wend; tile += 32ull * nw) {
    const unsigned long long gw = tile + 32ull * wid;  // this warp's 32 words
    const unsigned long long w = gw + lane;
    uint32_t my_mask = 0, hubs = 0;
    if (w < wend && act[w / wps]) {
      my_mask = b.mask[w];
      if (my_mask) hubs = b.hubw[w];
    }
    const uint32_t nodes = __popc(my_mask);
    unsigned long long slot;
    unsigned long long ne, he, nt, ht;
    const unsigned long long wn = __reduce_add_sync(kFull, nodes);
    const unsigned long long wh = __reduce_add_sync(kFull, hubs);
    block_scan2(lane == 0 ? wn : 0, lane == 0 ? wh : 0, &ne, &he, &nt, &ht);
    unsigned long long p = pos + __shfl_sync(kFull, ne, 0);
    unsigned long long hp = hpos + __shfl_sync(kFull, he, 0);
    slot = gw / wps;
    uint32_t dsum = 0, cnt_slot = 0;
    for (int k0 = 0; k0 < 32; k0 += 4) {
      uint32_t m[4], u[4], d[4];
      unsigned long long sl[4];
      double a[4], rs[4];
      uint32_t any = 0;
      unsigned long long s_it = slot;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // issue every load of four words first
        m[kk] = __shfl_sync(kFull, my_mask, k0 + kk);
        any |= m[kk];
        const unsigned long long wk = gw + k0 + kk;
        while (wk >= (s_it + 1) * wps) ++s_it;
        sl[kk] = s_it;
        u[kk] = (uint32_t)((wk - s_it * wps) * 32) + lane;
        const bool bit = (m[kk] >> lane) & 1u;
        d[kk] = 0; a[kk] = 0.0; rs[kk] = 0.0;
        if (bit) {
          const unsigned long long gi = s_it * n + u[kk];
          d[kk] = g.row[u[kk] + 1] - g.row[u[kk]];
          a[kk] = b.r[gi];
          rs[kk] = b.res[gi];
        }
      }
      if (any == 0) continue;  // warp-uniform
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (m[kk] == 0) continue;
        if (sl[kk] != slot) {  // flush the counters of the previous source
          if (lane == 0 && cnt_slot) {
            atomicAdd(&b.stats[slot].pushes, (unsigned long long)cnt_slot);
            atomicAdd(&b.stats[slot].edge_pushes, (unsigned long long)dsum);
            atomicMax(&b.stats[slot].rounds, round);
            act_next[slot] = 1;
          }
          dsum = 0; cnt_slot = 0;
          slot = sl[kk];
        }
        const bool bit = (m[kk] >> lane) & 1u;
        const uint32_t nch = hub_chunks_of(d[kk]);
        const uint32_t nch_incl = warp_incl_scan(nch);  // hub items of the lower lanes first
        if (bit) {
          const unsigned long long gi = slot * n + u[kk];
          // the take of round `round`: reserve += alpha a, r = 0, spread increment
          b.r[gi] = 0.0;
          b.res[gi] = __dadd_rn(rs[kk], __dmul_rn(alpha, a[kk]));
          const unsigned long long idx = p + __popc(m[kk] & lt_mask);
          b.q[nxt][idx] = (slot << 32) | u[kk];
          b.fa[idx] = __ddiv_rn(__dmul_rn(beta, a[kk]), (double)d[kk]);
          const unsigned long long hb = hp + (nch_incl - nch);
          for (uint32_t c = 0; c < nch; ++c) b.hub[nxt][hb + c] = (idx << kHubChunkBits) | c;
        }
        p += __popc(m[kk]);
        hp += __shfl_sync(kFull, nch_incl, 31);
        dsum += __reduce_add_sync(kFull, d[kk]);
        cnt_slot += __popc(m[kk]);
      }
    }
    if (lane == 0 && cnt_slot) {
      atomicAdd(&b.stats[slot].pushes, (unsigned long long)cnt_slot);
      atomicAdd(&b.stats[slot].edge_pushes, (unsigned long long)dsum);
      atomicMax(&b.stats[slot].rounds, round);
      act_next[slot] = 1;
    }
    pos += nt;
    hpos += ht;
  }
}

// End of a round: switch to the new frontier and keep looping while it is non-empty
// (at most kMaxPushRounds rounds).
__global__ void k_push_advance(BatchDev b, cudaGraphConditionalHandle loop) {
  PushState* ps = b.ps;
  ps->cur ^= 1;
  ps->round += 1;
  const bool more = b.counters[ps->cur * 2] > 0;
  const bool go = more && ps->round < kMaxPushRounds;
  if (more && !go) atomicOr(b.err, kErrPushNotConverged);
  cudaGraphSetConditional(loop, go ? 1u : 0u);
}

}  // namespace

cudaError_t launch_push_seed(const GraphDev& g, const BatchDev& b, cudaStream_t st) {
  const int threads = 256;
  k_push_seed<<<(b.nsrc + threads - 1) / threads, threads, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_push_body(const GraphDev& g, const BatchDev& b, int num_sms,
                             cudaGraphConditionalHandle loop, cudaStream_t st) {
  // one wave of resident blocks: with the dynamic work counter the warps in flight
  // cover one contiguous window of the sorted frontier
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_spread,
                                                                  kSpreadThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  k_push_spread<<<num_sms * per_sm, kSpreadThreads, 0, st>>>(g, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_detect<<<b.residual_grid, kDetectThreads, 0, st>>>(g, b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_scan<<<1, 1024, 0, st>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_emit<<<b.residual_grid, kDetectThreads, 0, st>>>(g, b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_push_advance<<<1, 1, 0, st>>>(b, loop);
  return cudaGetLastError();
}

}  // namespace fora
