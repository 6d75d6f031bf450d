// Walk phase of Alg. 2 over a batch of sources.
//
//   k_residual_count / k_residual_scan / k_residual_emit:
//     R = {(slot, v) : r(v) > 0} in ascending (slot, v); omega_v = ceil(r(v) * C) with
//     C = omega / r_sum (Alg. 2); exclusive offsets of omega_v over R (one flat
//     walk index space for all sources) and the fixed-point weight
//     W_v = rint(r(v)/omega_v * 2^63) of every walk from v (Alg. 2: a_v r_sum/omega).
//   k_walks:
//     walk g in [0, W) belongs to the entry i with offset[i] <= g < offset[i+1] and is
//     walk j = g - offset[i] of node v; it reads its own Philox4x32-10 stream with
//     counter (c, j, v, s) and stops with probability alpha at every node
//     (Section 2.1); count[end] += 1 and acc[end] += W_v.
#include "fora_engine.cuh"

namespace fora {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kResidualThreads = 256;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Philox4x32-10 with its ten round keys given (BatchDev::round_key, kernel parameters, so
// the key schedule costs no instruction per round).
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint2* rk) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk[i].x, lo1, hi0 ^ c.w ^ rk[i].y, lo0);
  }
  return c;
}

// omega_v = ceil(RN64(r * C)); W_v = rint((r / omega_v) * 2^63)
__device__ __noinline__ unsigned long long walks_exact(double r, double C) {
  return (unsigned long long)ceil(__dmul_rn(r, C));
}
__device__ __forceinline__ unsigned long long weight_of(double r, double omega) {
  return __double2ull_rn(__dmul_rn(__ddiv_rn(r, omega), 0x1p63));
}

constexpr uint32_t kOmegaUndecided = 0xFFFFFFFFu;

// omega_v for r > 0 without FP64 arithmetic where FP32 decides it (this GPU issues about
// two FP64 operations per clock per SM).  rf = r truncated to 23 mantissa bits (rf <= r
// < rf (1 + 2^-23)) and cf = RN32(C) give P = RN32(rf * cf) within 2^-22 of V = r * C,
// and T = RN64(V) is within 2^-53 of V; so T lies strictly inside (P (1 - 2^-20),
// P (1 + 2^-20)), and when that band holds no integer, ceil(T) = floor(band) + 1.
// Returns kOmegaUndecided otherwise (an integer in the band, P >= 2^22, r outside FP32's
// normal range, or C outside [1, 2^100], which `fast` excludes).
__device__ __forceinline__ uint32_t walks_fast(double r, float cf, bool fast) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
  const uint32_t hi = (uint32_t)(bits >> 32);
  const uint32_t ex = hi >> 20;  // r > 0: no sign bit
  if (!fast || ex < 897u || ex > 1150u) return kOmegaUndecided;
  const float rf =
      __uint_as_float(((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | ((uint32_t)bits >> 29));
  const float pr = rf * cf;
  if (!(pr < 0x1p22f)) return kOmegaUndecided;
  const float lo = pr * (1.0f - 0x1p-20f), up = pr * (1.0f + 0x1p-20f);
  const float fl = floorf(lo);
  if (floorf(up) != fl || fl == lo) return kOmegaUndecided;
  return (uint32_t)fl + 1u;
}

// omega_v of this lane's residue (0 when r = 0); every lane of the warp must call it.
__device__ __forceinline__ unsigned long long walks_of(double r, double C, float cf, bool fast) {
  const bool live = __double_as_longlong(r) != 0;  // residues are >= 0, never -0
  const uint32_t f = live ? walks_fast(r, cf, fast) : 0u;
  unsigned long long w = f;
  const bool undecided = f == kOmegaUndecided;
  if (__any_sync(kFull, undecided)) {  // rare: r * C within 2^-20 of an integer
    if (undecided) w = walks_exact(r, C);
  }
  return w;
}

// The residue the walks sample: r, or (1 - alpha) r with zero-hop pruning (Section 4.1).
__device__ __forceinline__ double sampled(const BatchDev& b, double r) {
  return b.zero_hop ? __dmul_rn(__dadd_rn(1.0, -b.alpha), r) : r;
}

// Contiguous element range of block `blk` out of `nblk` over [0, total).
__device__ __forceinline__ void block_range(unsigned long long total, int blk, int nblk,
                                            unsigned long long* beg, unsigned long long* end) {
  *beg = total * (unsigned long long)blk / (unsigned long long)nblk;
  *end = total * (unsigned long long)(blk + 1) / (unsigned long long)nblk;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T t = __shfl_up_sync(kFull, x, off);
    if ((int)(threadIdx.x & 31) >= off) x += t;
  }
  return x;
}

// Block-wide exclusive scan of (count, walks) pairs; also returns the block totals.
// Every thread of the block must call it.
__device__ __forceinline__ void block_excl_scan2(unsigned long long c, unsigned long long w,
                                                 unsigned long long* ce, unsigned long long* we,
                                                 unsigned long long* ct, unsigned long long* wt) {
  __shared__ unsigned long long sc[32], sw[32];
  __shared__ unsigned long long tc, tw;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long ci = warp_incl_scan(c), wi = warp_incl_scan(w);
  if (lane == 31) { sc[wid] = ci; sw[wid] = wi; }
  __syncthreads();
  if (wid == 0) {
    const unsigned long long a = lane < nw ? sc[lane] : 0, bb = lane < nw ? sw[lane] : 0;
    const unsigned long long ai = warp_incl_scan(a), bi = warp_incl_scan(bb);
    if (lane < nw) { sc[lane] = ai - a; sw[lane] = bi - bb; }
    if (lane == 31) { tc = ai; tw = bi; }
  }
  __syncthreads();
  *ce = sc[wid] + ci - c;
  *we = sw[wid] + wi - w;
  *ct = tc;
  *wt = tw;
  __syncthreads();
}

__global__ void __launch_bounds__(kResidualThreads) k_residual_count(GraphDev g, BatchDev b) {
  const unsigned long long total = (unsigned long long)b.nsrc * (unsigned long long)g.n;
  unsigned long long beg, end;
  block_range(total, blockIdx.x, gridDim.x, &beg, &end);
  unsigned long long cnt = 0, walks = 0;
  // per-source sums, flushed whenever this thread's elements move to another source
  unsigned long long i = beg + threadIdx.x;
  uint32_t slot = (uint32_t)(i / (unsigned long long)g.n);
  unsigned long long slot_end = (unsigned long long)(slot + 1) * (unsigned long long)g.n;
  unsigned long long s_cnt = 0, s_walks = 0;
  double s_sum = 0.0;
  const float cf = __double2float_rn(b.walk_scale);
  const bool fast = cf >= 1.0f && cf <= 0x1p100f;
  for (unsigned long long base = beg; base < end; base += kResidualThreads, i += kResidualThreads) {
    const bool valid = i < end;
    while (valid && i >= slot_end) {
      if (s_cnt) {
        atomicAdd(&b.stats[slot].residual_nodes, s_cnt);
        atomicAdd(&b.stats[slot].walks, s_walks);
        atomicAdd(&b.stats[slot].rsum, s_sum);
      }
      s_cnt = 0; s_walks = 0; s_sum = 0.0;
      ++slot;
      slot_end += (unsigned long long)g.n;
    }
    const double r = valid ? b.r[i] : 0.0;
    // an entry of R needs at least one walk (omega_v = 0 only if r * C underflows)
    const unsigned long long w = walks_of(sampled(b, r), b.walk_scale, cf, fast);
    if (__double_as_longlong(r) != 0) {
      if (w > 0) { ++cnt; walks += w; }
      ++s_cnt; s_walks += w; s_sum += r;
    }
  }
  if (s_cnt && slot < (uint32_t)b.nsrc) {
    atomicAdd(&b.stats[slot].residual_nodes, s_cnt);
    atomicAdd(&b.stats[slot].walks, s_walks);
    atomicAdd(&b.stats[slot].rsum, s_sum);
  }
  unsigned long long ce, we, ct, wt;
  block_excl_scan2(cnt, walks, &ce, &we, &ct, &wt);
  if (threadIdx.x == 0) {
    b.blk_cnt[blockIdx.x] = ct;
    b.blk_walks[blockIdx.x] = wt;
  }
}

// One block: exclusive scan of the per-block totals; totals; per-source walk limit.
__global__ void __launch_bounds__(1024) k_residual_scan(BatchDev b) {
  __shared__ unsigned long long carry_c, carry_w;
  if (threadIdx.x == 0) { carry_c = 0; carry_w = 0; }
  __syncthreads();
  for (int base = 0; base < b.residual_grid; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const unsigned long long c = i < b.residual_grid ? b.blk_cnt[i] : 0;
    const unsigned long long w = i < b.residual_grid ? b.blk_walks[i] : 0;
    unsigned long long ce, we, ct, wt;
    block_excl_scan2(c, w, &ce, &we, &ct, &wt);
    if (i < b.residual_grid) {
      b.blk_cnt[i] = carry_c + ce;
      b.blk_walks[i] = carry_w + we;
    }
    __syncthreads();
    if (threadIdx.x == 0) { carry_c += ct; carry_w += wt; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.totals[0] = carry_c;
    b.totals[1] = carry_w;
    b.wr_offset[carry_c] = carry_w;
  }
  for (int s = threadIdx.x; s < b.nsrc; s += blockDim.x)
    if (b.stats[s].walks > 0xFFFFFFFFull) atomicOr(b.err, kErrWalkOverflow);
}

__global__ void __launch_bounds__(kResidualThreads) k_residual_emit(GraphDev g, BatchDev b) {
  const unsigned long long total = (unsigned long long)b.nsrc * (unsigned long long)g.n;
  unsigned long long beg, end;
  block_range(total, blockIdx.x, gridDim.x, &beg, &end);
  unsigned long long pos = b.blk_cnt[blockIdx.x];
  unsigned long long woff = b.blk_walks[blockIdx.x];
  const float cf = __double2float_rn(b.walk_scale);
  const bool fast = cf >= 1.0f && cf <= 0x1p100f;
  for (unsigned long long tile = beg; tile < end; tile += kResidualThreads) {
    const unsigned long long i = tile + threadIdx.x;
    const double r = i < end ? sampled(b, b.r[i]) : 0.0;
    const unsigned long long omega = walks_of(r, b.walk_scale, cf, fast);
    const bool live = omega >= 1;
    unsigned long long ce, we, ct, wt;
    block_excl_scan2(live ? 1ull : 0ull, omega, &ce, &we, &ct, &wt);
    if (live && FORA_IN_RANGE(b.err, pos + ce, total)) {
      const unsigned long long slot = i / (unsigned long long)g.n;
      const unsigned long long v = i - slot * (unsigned long long)g.n;
      b.wr_entry[pos + ce] = (slot << 32) | v;
      b.wr_offset[pos + ce] = woff + we;
      // the residue for now; k_residual_weight turns it into the walk weight
      b.wr_weight[pos + ce] = (unsigned long long)__double_as_longlong(r);
    }
    pos += ct;
    woff += wt;
  }
}

// W_v of every entry of R, densely over the list (omega_v = offset[i + 1] - offset[i]),
// so the FP64 division runs on 32 entries per instruction.
__global__ void __launch_bounds__(kResidualThreads) k_residual_weight(BatchDev b) {
  const unsigned long long nR = b.totals[0];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nR;
       i += stride) {
    const double r = __longlong_as_double((long long)b.wr_weight[i]);
    const double omega = (double)(b.wr_offset[i + 1] - b.wr_offset[i]);
    b.wr_weight[i] = weight_of(r, omega);
  }
}

constexpr int kWalkThreads = 256;
constexpr int kWalkWarps = kWalkThreads / 32;
constexpr int kWalksPerLane = 32;
constexpr int kChunk = 32 * kWalksPerLane;  // walks per warp chunk
constexpr uint32_t kMaxSteps = 16384u;

// Largest i in [0, nR) with off[i] <= g (off non-decreasing, off[0] = 0 <= g);
// warp-cooperative 32-ary search, every lane gets the answer.
__device__ __forceinline__ unsigned long long warp_find_entry(const unsigned long long* off,
                                                              unsigned long long nR,
                                                              unsigned long long g) {
  const unsigned lane = threadIdx.x & 31;
  unsigned long long lo = 0, hi = nR;
  while (hi - lo > 32) {
    const unsigned long long step = (hi - lo + 31) / 32;
    const unsigned long long p = lo + lane * step;
    const unsigned bal = __ballot_sync(kFull, p < hi && off[p] <= g);
    lo += (unsigned long long)(31 - __clz(bal)) * step;
    hi = min(lo + step, hi);
  }
  const unsigned long long p = lo + lane;
  const unsigned bal = __ballot_sync(kFull, p < hi && off[p] <= g);
  return lo + (unsigned long long)(31 - __clz(bal));
}

// Map walk cbeg + i (i < cnt) to its residual entry idx0 + smap[i], 32 walks at a time
// (the entries' walk offsets are read coalesced, a 5-step search per walk in registers).
__device__ __forceinline__ void map_chunk(const unsigned long long* off, unsigned long long nR,
                                          unsigned long long cbeg, uint32_t cnt,
                                          unsigned long long idx0, uint16_t* smap) {
  const uint32_t lane = threadIdx.x & 31;
  unsigned long long idxw = idx0;
  for (uint32_t rb = 0; rb < cnt; rb += 32) {
    const unsigned long long gw = cbeg + rb + lane;
    const unsigned long long o = idxw + lane < nR ? off[idxw + lane] : ~0ull;
    int lo = 0, hi = 31;  // largest j with off[idxw + j] <= gw
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const int mid = (lo + hi + 1) >> 1;
      if (__shfl_sync(kFull, o, mid) <= gw) lo = mid; else hi = mid - 1;
    }
    const unsigned long long mine = idxw + (unsigned long long)lo;
    smap[rb + lane] = (uint16_t)(mine - idx0);
    idxw = __shfl_sync(kFull, mine, 31);
  }
  __syncwarp();
}

// Target e of the walk copy of the adjacency (bit-packed when colbits > 0).
__device__ __forceinline__ uint32_t walk_target(const GraphDev& g, uint32_t e) {
  return g.colbits ? packed_target(g.colp, g.colbits, e) : (uint32_t)g.col[e];
}

constexpr uint32_t kCapped = 0xFFFFFFFFu;

// The rest of a walk whose neighbour draw at x (row offset rb, degree d) came out with
// low word below d on its first try, m0 (Lemire's method then rejects the try when the low
// word is below 2^32 mod d, probability below d / 2^32): the try is accepted or retried,
// then the walk goes on with the words taken one at a time from word `pos` of the block
// `blk` (the next block to generate is `cb`), stop tests and moves in stream order.
// Returns the end node, or kCapped when the walk reaches the step cap (or, never in
// practice, 64 rejected tries in a row).
__device__ __forceinline__ uint32_t walk_rest(const GraphDev& g, uint4 blk, int pos, uint32_t cb,
                                              uint32_t j, uint32_t v, uint32_t s, uint2 key,
                                              uint32_t t_alpha, uint32_t x, uint32_t rb,
                                              uint32_t d, unsigned long long m0,
                                              uint32_t* steps) {
  auto next = [&]() -> uint32_t {
    if (pos == 4) {
      blk = philox4x32_10(make_uint4(cb, j, v, s), key);
      ++cb;
      pos = 0;
    }
    const uint32_t w = pos == 0 ? blk.x : pos == 1 ? blk.y : pos == 2 ? blk.z : blk.w;
    ++pos;
    return w;
  };
  unsigned long long m = m0;
  bool first = true;  // the move at x has its first try in m0
  for (;;) {
    if (!first) {
      if (next() < t_alpha) return x;
      if (*steps >= kMaxSteps) return kCapped;
      const uint2 r = g.rd[x];
      rb = r.x;
      d = r.y;
      m = (unsigned long long)next() * d;
    }
    first = false;
    uint32_t low = (uint32_t)m;
    if (low < d) {
      const uint32_t reject_below = (0u - d) % d;
      int tries = 0;
      while (low < reject_below) {
        if (++tries > 64) return kCapped;
        m = (unsigned long long)next() * d;
        low = (uint32_t)m;
      }
    }
    x = walk_target(g, rb + (uint32_t)(m >> 32));
    ++*steps;
  }
}

// One move of a walk at x with the word u, on the fast path: false when the low word of
// the product is below d (a try Lemire's method may reject; walk_rest decides it, with
// rb, d and m left for it), else x becomes the chosen out-neighbour.
__device__ __forceinline__ bool fast_move(const GraphDev& g, uint32_t u, uint32_t& x,
                                          uint32_t& rb, uint32_t& d, unsigned long long& m,
                                          uint32_t* err, bool& bad) {
  if (!FORA_IN_RANGE(err, x, g.n)) { bad = true; return false; }
  const uint2 r = g.rd[x];
  rb = r.x;
  d = r.y;
  m = (unsigned long long)u * d;
  if ((uint32_t)m < d) return false;
  const uint32_t e = rb + (uint32_t)(m >> 32);
  if (!FORA_IN_RANGE(err, e, g.m)) { bad = true; return false; }
  x = walk_target(g, e);
  return true;
}

// The first kStartCache residual entries of a warp's chunk, staged in shared memory when
// the chunk starts (one coalesced load per lane), so that a lane starting a walk of one of
// them reads its data there instead of making two dependent global loads.
constexpr int kStartCache = 32;
struct StartCache {
  unsigned long long off[kStartCache];
  unsigned long long wgt[kStartCache];
  uint32_t v[kStartCache];
  uint32_t s[kStartCache];
  uint32_t slot[kStartCache];
};

__device__ __forceinline__ void fill_start_cache(const BatchDev& b, unsigned long long idx0,
                                                 unsigned long long nR, StartCache& sc) {
  const uint32_t lane = threadIdx.x & 31;
  const unsigned long long idx = idx0 + lane;
  if (idx < nR) {
    const unsigned long long entry = b.wr_entry[idx];
    const uint32_t slot = (uint32_t)(entry >> 32);
    sc.off[lane] = b.wr_offset[idx];
    sc.wgt[lane] = b.wr_weight[idx];
    sc.v[lane] = (uint32_t)entry;
    sc.slot[lane] = slot;
    sc.s[lane] = (uint32_t)b.sources[slot];
  }
  __syncwarp();
}

// Per-walk state of the walk kernels.
struct Walk {
  uint32_t x, v, j, s, slot, steps, cb, i;
  unsigned long long wgt;
  bool have;
};

// Start walk w.i of the chunk (residual entry idx0 + smap[w.i]).
__device__ __forceinline__ void start_walk(const BatchDev& b, const unsigned long long* off,
                                           unsigned long long cbeg, unsigned long long idx0,
                                           const uint16_t* smap, const StartCache& sc, Walk& w) {
  const uint32_t e = smap[w.i];
  if (e < (uint32_t)kStartCache) {
    w.slot = sc.slot[e];
    w.v = sc.v[e];
    w.s = sc.s[e];
    w.wgt = sc.wgt[e];
    w.j = (uint32_t)(cbeg + w.i - sc.off[e]);
  } else {
    unsigned long long idx = idx0 + e;
    if (!FORA_IN_RANGE(b.err, idx, b.totals[0])) idx = idx0;
    const unsigned long long entry = b.wr_entry[idx];
    w.slot = (uint32_t)(entry >> 32);
    w.v = (uint32_t)entry;
    w.j = (uint32_t)(cbeg + w.i - off[idx]);
    w.s = (uint32_t)b.sources[w.slot];
    w.wgt = b.wr_weight[idx];
  }
  w.x = w.v;
  w.steps = 0;
  w.cb = 0;
}

// One iteration of a walk on its Philox block o (block index w.cb - 1): plain walks take
// the words as stop test, move, stop test, move; zero-hop walks as move, stop test, move,
// stop test (the first move of a zero-hop walk has no stop test).  A rejected neighbour try
// (probability below d / 2^32) moves the walk off this block alignment: walk_rest then
// finishes it word by word.  Returns true when the walk stopped (at w.x); sets w.have =
// false and capped when it ran into the step cap.
template <bool kZeroHop>
__device__ __forceinline__ bool walk_block(const GraphDev& g, uint4 o, uint2 key, uint32_t t_alpha,
                                           Walk& w, bool& capped, uint32_t* err) {
  bool stop = false;
  uint32_t rb = 0, d = 0;
  unsigned long long m = 0;
  int rejected = -1;  // word index of a try that walk_rest has to decide
  bool bad = false;   // a failed index check (FORA_DEBUG builds): the walk is dropped
  const uint32_t u0 = kZeroHop ? 0u : o.x, mv0 = kZeroHop ? o.x : o.y;
  const uint32_t t1 = kZeroHop ? o.y : o.z, mv1 = kZeroHop ? o.z : o.w;
  if (!kZeroHop) stop = u0 < t_alpha;
  if (!stop) {
    if (w.steps >= kMaxSteps) { capped = true; w.have = false; return false; }
    if (fast_move(g, mv0, w.x, rb, d, m, err, bad)) {
      ++w.steps;
      stop = t1 < t_alpha;
      if (!stop) {
        if (w.steps >= kMaxSteps) { capped = true; w.have = false; return false; }
        if (fast_move(g, mv1, w.x, rb, d, m, err, bad)) {
          ++w.steps;
          if (kZeroHop) stop = o.w < t_alpha;
        } else {
          rejected = kZeroHop ? 2 : 3;
        }
      }
    } else {
      rejected = kZeroHop ? 0 : 1;
    }
  }
  if (bad) { w.have = false; return false; }
  if (rejected >= 0) {  // rare: decide the try and finish the walk word by word
    const uint32_t end = walk_rest(g, o, rejected + 1, w.cb, w.j, w.v, w.s, key, t_alpha, w.x,
                                   rb, d, m, &w.steps);
    if (end == kCapped) { capped = true; w.have = false; return false; }
    w.x = end;
    stop = true;
  }
  return stop;
}

// The end of this lane's walk w: tally it (or store it in a walk index) and count its
// moves for its source.
__device__ __forceinline__ void finish_walk(const BatchDev& b, unsigned long long n,
                                            unsigned long long cbeg, const Walk& w,
                                            unsigned long long& steps_here, uint32_t& cur_slot) {
  // the walk stops at x (Section 2.1): count it and add its weight (Alg. 2), or record
  // its end in a walk index (Section 3.3)
  if (b.walk_dest) {
    b.walk_dest[cbeg + w.i] = w.x;
  } else if (FORA_IN_RANGE(b.err, w.x, n) && FORA_IN_RANGE(b.err, w.slot, b.nsrc)) {
    Tally* t = b.tally + (unsigned long long)w.slot * n + w.x;
    if (b.want_count) atomicAdd(&t->cnt, 1u);
    atomicAdd(&t->acc, w.wgt);
  }
  if (w.slot != cur_slot) {
    if (steps_here) atomicAdd(&b.stats[cur_slot].walk_steps, steps_here);
    steps_here = 0;
    cur_slot = w.slot;
  }
  steps_here += w.steps;
}

// The walk kernel.  The flat walk range is cut into chunks of kChunk walks and chunk c goes
// to warp c mod (number of warps), so the walks in flight at any time are a narrow window
// of the source-major walk space and their end tallies stay in L2.  Per chunk the warp maps
// every walk to its residual entry (map_chunk) and stages the chunk's first entries
// (fill_start_cache); each lane runs one walk and takes the chunk's next unstarted walk
// when its walk ends (walk lengths are geometric: with a fixed share of walks per lane a
// warp would wait for its longest share).  One loop iteration consumes exactly one Philox
// block of a lane's walk (walk_block), so every lane with a walk evaluates its Philox block
// in the same iteration and the ten rounds, most of a walk's arithmetic, run on full warps;
// a walk that stops inside a block leaves the block's remaining words unused, as its stream
// definition does.
template <int kMinBlocks, bool kZeroHop>
__global__ void __launch_bounds__(kWalkThreads, kMinBlocks) k_walks(GraphDev g, BatchDev b) {
  __shared__ uint16_t smap[kWalkWarps][kChunk];
  __shared__ StartCache scache[kWalkWarps];
  if (*b.err) return;
  const unsigned long long W = b.totals[1];
  const unsigned long long nR = b.totals[0];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long nchunks = (W + kChunk - 1) / kChunk;
  const unsigned long long* off = b.wr_offset;
  const unsigned long long n = (unsigned long long)g.n;
  const uint2 key = make_uint2((uint32_t)b.seed, (uint32_t)(b.seed >> 32));
  const uint32_t t_alpha = b.alpha_threshold;
  StartCache& sc = scache[wid];
  unsigned long long steps_here = 0;  // moves of this lane's walks of source `cur_slot`
  uint32_t cur_slot = 0xFFFFFFFFu;
  bool capped = false;

  for (unsigned long long c = warp; c < nchunks; c += nwarps) {
    const unsigned long long cbeg = c * kChunk;
    const uint32_t cnt = (uint32_t)min((unsigned long long)kChunk, W - cbeg);
    const unsigned long long idx0 = warp_find_entry(off, nR, cbeg);
    map_chunk(off, nR, cbeg, cnt, idx0, smap[wid]);
    fill_start_cache(b, idx0, nR, sc);

    uint32_t next_walk = 32;  // warp-uniform: the chunk's next unstarted walk
    Walk w;
    w.i = lane;
    w.have = w.i < cnt;
    if (w.have) start_walk(b, off, cbeg, idx0, smap[wid], sc, w);
    for (;;) {
      bool stop = false;
      if (w.have) {
        const uint4 o = philox_rk(make_uint4(w.cb, w.j, w.v, w.s), b.round_key);
        ++w.cb;
        stop = walk_block<kZeroHop>(g, o, key, t_alpha, w, capped, b.err);
      }
      const bool ended = w.have && stop;
      const uint32_t ends = __ballot_sync(kFull, ended);
      if (ended) {
        finish_walk(b, n, cbeg, w, steps_here, cur_slot);
        w.i = next_walk + (uint32_t)__popc(ends & lt_mask);
        w.have = w.i < cnt;
        if (w.have) start_walk(b, off, cbeg, idx0, smap[wid], sc, w);
      }
      next_walk += (uint32_t)__popc(ends);
      if (!__any_sync(kFull, w.have)) break;
    }
    __syncwarp();
  }
  if (capped) atomicOr(b.err, kErrWalkCap);
  if (steps_here) atomicAdd(&b.stats[cur_slot].walk_steps, steps_here);
}

// FORA+ (Section 3.3): the residue whose walk count is the index's omega_max(v).
__global__ void k_index_residue(GraphDev g, double* r, double rmax) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long v = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       v < (unsigned long long)g.n; v += stride)
    r[v] = __dmul_rn(rmax, (double)(g.row[v + 1] - g.row[v]));
}

// The walk phase served from a walk index: walk j of residual entry (slot, v) ends at
// idx_dest[idx_off[v] + j] (the j-th stored walk from v) instead of being simulated.
// Walks map to entries as in k_walks (chunks of kChunk, a shared-memory map per warp).
// A walk past v's stored walks (a residue above the index's r_max) sets kErrIndexRange
// and is skipped.
__global__ void __launch_bounds__(kWalkThreads) k_walks_indexed(GraphDev g, BatchDev b,
                                                                const unsigned long long* idx_off,
                                                                const uint32_t* idx_dest) {
  __shared__ uint16_t smap[kWalkWarps][kChunk];
  if (*b.err) return;
  const unsigned long long W = b.totals[1];
  const unsigned long long nR = b.totals[0];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long nchunks = (W + kChunk - 1) / kChunk;
  const unsigned long long* off = b.wr_offset;
  bool out_of_range = false;
  for (unsigned long long c = warp; c < nchunks; c += nwarps) {
    const unsigned long long cbeg = c * kChunk;
    const uint32_t cnt = (uint32_t)min((unsigned long long)kChunk, W - cbeg);
    const unsigned long long idx0 = warp_find_entry(off, nR, cbeg);
    unsigned long long idxw = idx0;
    for (uint32_t rb = 0; rb < cnt; rb += 32) {
      const unsigned long long gw = cbeg + rb + lane;
      const unsigned long long o = idxw + lane < nR ? off[idxw + lane] : ~0ull;
      int lo = 0, hi = 31;  // largest j with off[idxw + j] <= gw
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        const int mid = (lo + hi + 1) >> 1;
        if (__shfl_sync(kFull, o, mid) <= gw) lo = mid; else hi = mid - 1;
      }
      const unsigned long long mine = idxw + (unsigned long long)lo;
      smap[wid][rb + lane] = (uint16_t)(mine - idx0);
      idxw = __shfl_sync(kFull, mine, 31);
    }
    __syncwarp();
    for (uint32_t i = lane; i < cnt; i += 32) {
      const unsigned long long idx = idx0 + smap[wid][i];
      const unsigned long long entry = b.wr_entry[idx];
      const uint32_t slot = (uint32_t)(entry >> 32), v = (uint32_t)entry;
      const unsigned long long j = cbeg + i - off[idx];
      const unsigned long long pos = idx_off[v] + j;
      if (pos >= idx_off[v + 1]) {
        out_of_range = true;
        continue;
      }
      Tally* t = b.tally + (unsigned long long)slot * (unsigned long long)g.n + idx_dest[pos];
      if (b.want_count) atomicAdd(&t->cnt, 1u);
      atomicAdd(&t->acc, b.wr_weight[idx]);
    }
    __syncwarp();
  }
  if (out_of_range) atomicOr(b.err, kErrIndexRange);
}

__global__ void k_unpack_tally(const Tally* __restrict__ t, uint32_t* cnt,
                               unsigned long long* acc, unsigned long long count) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += stride) {
    const Tally v = t[i];
    if (cnt) cnt[i] = v.cnt;
    if (acc) acc[i] = v.acc;
  }
}

__global__ void k_philox_table(const uint32_t* ck, uint32_t* out, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 o = philox4x32_10(make_uint4(ck[6 * i], ck[6 * i + 1], ck[6 * i + 2], ck[6 * i + 3]),
                                make_uint2(ck[6 * i + 4], ck[6 * i + 5]));
  out[4 * i] = o.x; out[4 * i + 1] = o.y; out[4 * i + 2] = o.z; out[4 * i + 3] = o.w;
}

}  // namespace

cudaError_t launch_residuals(const GraphDev& g, const BatchDev& b, cudaStream_t st) {
  k_residual_count<<<b.residual_grid, kResidualThreads, 0, st>>>(g, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual_scan<<<1, 1024, 0, st>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual_emit<<<b.residual_grid, kResidualThreads, 0, st>>>(g, b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual_weight<<<b.residual_grid, kResidualThreads, 0, st>>>(b);
  return cudaGetLastError();
}

// Walk kernel instances for 3, 4 or 5 resident blocks of 256 threads per SM (the register
// budget the compiler gets); b.walk_blocks picks one (launch shape only).
template <int kMinBlocks, bool kZeroHop>
cudaError_t launch_walks_t(const GraphDev& g, const BatchDev& b, int num_sms, cudaStream_t st) {
  const int per_sm = resident_blocks((const void*)k_walks<kMinBlocks, kZeroHop>, kWalkThreads);
  if (per_sm == 0) return cudaErrorInvalidConfiguration;
  k_walks<kMinBlocks, kZeroHop><<<num_sms * per_sm, kWalkThreads, 0, st>>>(g, b);
  return cudaGetLastError();
}

template <bool kZeroHop>
cudaError_t launch_walks_zh(const GraphDev& g, const BatchDev& b, int num_sms, cudaStream_t st) {
  switch (b.walk_blocks) {
    case 3: return launch_walks_t<3, kZeroHop>(g, b, num_sms, st);
    case 5: return launch_walks_t<5, kZeroHop>(g, b, num_sms, st);
    default: return launch_walks_t<4, kZeroHop>(g, b, num_sms, st);
  }
}

cudaError_t launch_walks(const GraphDev& g, const BatchDev& b, int num_sms, cudaStream_t st) {
  return b.zero_hop ? launch_walks_zh<true>(g, b, num_sms, st)
                    : launch_walks_zh<false>(g, b, num_sms, st);
}

cudaError_t launch_index_residue(const GraphDev& g, double* r, double rmax, cudaStream_t st) {
  k_index_residue<<<1024, 256, 0, st>>>(g, r, rmax);
  return cudaGetLastError();
}

cudaError_t launch_walks_indexed(const GraphDev& g, const BatchDev& b, int num_sms,
                                 const unsigned long long* idx_off, const uint32_t* idx_dest,
                                 cudaStream_t st) {
  const int per_sm = resident_blocks((const void*)k_walks_indexed, kWalkThreads);
  if (per_sm == 0) return cudaErrorInvalidConfiguration;
  k_walks_indexed<<<num_sms * per_sm, kWalkThreads, 0, st>>>(g, b, idx_off, idx_dest);
  return cudaGetLastError();
}

cudaError_t launch_unpack_tally(const Tally* t, uint32_t* cnt, unsigned long long* acc,
                                uint64_t count, int num_sms, cudaStream_t st) {
  uint64_t blocks = (count + 255) / 256;
  if (blocks > (uint64_t)num_sms * 32) blocks = (uint64_t)num_sms * 32;
  if (blocks == 0) return cudaSuccess;
  k_unpack_tally<<<(unsigned)blocks, 256, 0, st>>>(t, cnt, acc, count);
  return cudaGetLastError();
}

cudaError_t launch_philox_table(const uint32_t* ctr_key, uint32_t* out, int count,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_philox_table<<<(count + 127) / 128, 128, 0, st>>>(ctr_key, out, count);
  return cudaGetLastError();
}

}  // namespace fora
