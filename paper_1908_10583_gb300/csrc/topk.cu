// Estimate and top-k select (the query returns the k nodes with the largest
// estimated PPR, Section 2.1; ties go to the smaller id).
//
// Every element t of a row gets the 96-bit key  Z = bits(pi_hat(t)) : ~t.  pi_hat >= 0,
// so its IEEE bits order like its value, and ~t orders equal values by ascending id;
// keys are unique, so the k largest keys are exactly the answer.  Radix select over
// the key in 12-bit digits, most significant first:
//   level L:  k_topk_hist   histogram of digit L of the keys whose leading 12L bits equal
//                           the row's prefix (skipped once the row is done)
//             k_topk_select pick the digit whose bucket holds the kk-th largest key,
//                           extend the prefix, and mark the row done once every key above
//                           the bucket plus the bucket itself fits the final sort
//   then      k_topk_collect  every key >= the prefix bucket goes to the candidate list
//             k_topk_sort     bitonic sort of <= kSortCap candidates in shared memory.
// All levels are launched without host synchronisation; finished rows return at once.
#include "fora_engine.cuh"

namespace fora {

namespace {

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 key_of(double e, uint32_t t) {
  return ((u128)(unsigned long long)__double_as_longlong(e) << 32) | (u128)(~t);
}

__device__ __forceinline__ u128 prefix_of(const TopkSlot& s) {
  return ((u128)s.pa << 32) | (u128)s.pb;
}

__global__ void k_estimate(const double* __restrict__ res, const Tally* __restrict__ tally,
                           double* est, const double* r, double alpha, int zero_hop,
                           unsigned long long count) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += stride) {
    // pi_hat = reserve (+ alpha r with zero-hop pruning) + acc * 2^-63 (exact scaling)
    const double base = zero_hop ? __dadd_rn(res[i], __dmul_rn(alpha, r[i])) : res[i];
    est[i] = __dadd_rn(base, __dmul_rn(__ull2double_rn(tally[i].acc), 0x1p-63));
  }
}

__global__ void k_topk_init(TopkSlot* slots, uint32_t* hist, int nrows, uint32_t k) {
  const int row = blockIdx.x;
  if (row >= nrows) return;
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[(size_t)row * kBins + i] = 0;
  if (threadIdx.x == 0) {
    TopkSlot s;
    s.pa = 0; s.pb = 0; s.plen = 0; s.kk = k; s.done = (k == 0); s.ncand = 0; s.pad = 0;
    slots[row] = s;
  }
}

// Element range of block bx (of bpr blocks per row) over a row of n.
__device__ __forceinline__ void row_range(int64_t n, int bx, int bpr, int64_t* beg, int64_t* end) {
  *beg = n * (int64_t)bx / bpr;
  *end = n * (int64_t)(bx + 1) / bpr;
}

__global__ void __launch_bounds__(256) k_topk_hist(const double* __restrict__ est, int64_t n,
                                                   const TopkSlot* __restrict__ slots,
                                                   uint32_t* __restrict__ hist, int level) {
  const int row = blockIdx.y;
  const TopkSlot s = slots[row];
  if (s.done) return;
  __shared__ uint32_t sh[kBins];
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int shift_digit = 96 - kDigitBits * (level + 1);
  const u128 p = prefix_of(s) >> (96 - s.plen);  // s.plen = 12 * level
  int64_t beg, end;
  row_range(n, blockIdx.x, gridDim.x, &beg, &end);
  const double* e = est + (size_t)row * (size_t)n;
  const uint32_t lane = threadIdx.x & 31;
  // keys crowd into few bins (every zero estimate, and the few binades the others span, share
  // the leading digits), so the lanes of a warp that fall into the same bin add their count
  // once (their lowest lane), instead of serialising on one shared-memory counter
  for (int64_t base = beg; base < end; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    bool in = false;
    uint32_t bin = 0;
    if (t < end) {
      const u128 z = key_of(e[t], (uint32_t)t);
      in = (z >> (96 - s.plen)) == p;
      bin = (uint32_t)(z >> shift_digit) & (kBins - 1);
    }
    const unsigned members = __ballot_sync(0xFFFFFFFFu, in);
    if (in) {
      const unsigned grp = __match_any_sync(members, bin);
      if ((grp & ((1u << lane) - 1u)) == 0) atomicAdd(&sh[bin], (uint32_t)__popc(grp));
    }
  }
  __syncthreads();
  uint32_t* h = hist + (size_t)row * kBins;
  for (int i = threadIdx.x; i < kBins; i += blockDim.x)
    if (sh[i]) atomicAdd(&h[i], sh[i]);
}

// One block of 1024 threads per row; thread t owns bins 4095-4t .. 4092-4t (descending).
__global__ void __launch_bounds__(1024) k_topk_select(TopkSlot* slots, uint32_t* hist, uint32_t k,
                                                      int level) {
  const int row = blockIdx.x;
  TopkSlot s = slots[row];
  if (s.done) return;
  uint32_t* h = hist + (size_t)row * kBins;
  const int t = threadIdx.x;
  uint32_t c[4];
  uint32_t local = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    c[q] = h[kBins - 1 - (4 * t + q)];
    local += c[q];
  }
  // exclusive scan of `local` over the block (descending bin order)
  __shared__ uint32_t wsum[32];
  const int lane = t & 31, wid = t >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const uint32_t a = wsum[lane];
    uint32_t ai = a;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, ai, off);
      if (lane >= off) ai += v;
    }
    wsum[lane] = ai - a;
  }
  __syncthreads();
  uint32_t above = wsum[wid] + incl - local;  // keys in bins above this thread's bins
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (above < s.kk && s.kk <= above + c[q]) {
      const uint32_t digit = (uint32_t)(kBins - 1 - (4 * t + q));
      const int pos = 96 - kDigitBits * (level + 1);  // bit position of the digit
      const u128 p = prefix_of(s) | ((u128)digit << pos);
      s.pa = (unsigned long long)(p >> 32);
      s.pb = (uint32_t)p;
      s.plen += kDigitBits;
      s.kk -= above;
      const uint32_t sure = k - s.kk;  // keys strictly above the bucket
      s.done = (sure + c[q] <= kSortCap) || (s.plen >= 96);
      slots[row] = s;
    }
    above += c[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) h[kBins - 1 - (4 * t + q)] = 0;  // clean for the next level
}

__global__ void __launch_bounds__(256) k_topk_collect(const double* __restrict__ est, int64_t n,
                                                      TopkSlot* slots,
                                                      unsigned long long* __restrict__ cand_key,
                                                      uint32_t* __restrict__ cand_id) {
  const int row = blockIdx.y;
  const TopkSlot s = slots[row];
  if (s.plen == 0) return;  // k == 0
  const u128 p = prefix_of(s) >> (96 - s.plen);
  int64_t beg, end;
  row_range(n, blockIdx.x, gridDim.x, &beg, &end);
  const double* e = est + (size_t)row * (size_t)n;
  const unsigned lane = threadIdx.x & 31;
  for (int64_t base = beg; base < end; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    bool take = false;
    double v = 0.0;
    if (t < end) {
      v = e[t];
      take = (key_of(v, (uint32_t)t) >> (96 - s.plen)) >= p;
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
    if (bal) {
      uint32_t pos = 0;
      if (lane == 0) pos = atomicAdd(&slots[row].ncand, (uint32_t)__popc(bal));
      pos = __shfl_sync(0xFFFFFFFFu, pos, 0) + __popc(bal & ((1u << lane) - 1u));
      if (take && pos < kSortCap) {
        cand_key[(size_t)row * kSortCap + pos] = (unsigned long long)__double_as_longlong(v);
        cand_id[(size_t)row * kSortCap + pos] = (uint32_t)t;
      }
    }
  }
}

// Bitonic sort (descending by key) of one row's candidates; writes the first k.
__global__ void __launch_bounds__(1024) k_topk_sort(const TopkSlot* slots,
                                                    const unsigned long long* cand_key,
                                                    const uint32_t* cand_id, uint32_t k,
                                                    int32_t* out_ids, double* out_vals) {
  extern __shared__ unsigned char smem[];
  unsigned long long* ka = (unsigned long long*)smem;
  uint32_t* kb = (uint32_t*)(ka + kSortCap);
  const int row = blockIdx.x;
  const uint32_t nc = min(slots[row].ncand, kSortCap);
  uint32_t size = 1;
  while (size < nc) size <<= 1;
  for (uint32_t i = threadIdx.x; i < size; i += blockDim.x) {
    if (i < nc) {
      ka[i] = cand_key[(size_t)row * kSortCap + i];
      kb[i] = ~cand_id[(size_t)row * kSortCap + i];
    } else {
      ka[i] = 0;  // below every real key (a real key has ~id > 0)
      kb[i] = 0;
    }
  }
  __syncthreads();
  for (uint32_t len = 2; len <= size; len <<= 1) {
    for (uint32_t j = len >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < size; i += blockDim.x) {
        const uint32_t pr = i ^ j;
        if (pr > i) {
          const bool desc = (i & len) == 0;
          const u128 zi = ((u128)ka[i] << 32) | kb[i];
          const u128 zp = ((u128)ka[pr] << 32) | kb[pr];
          if (desc ? (zi < zp) : (zi > zp)) {
            const unsigned long long ta = ka[i]; ka[i] = ka[pr]; ka[pr] = ta;
            const uint32_t tb = kb[i]; kb[i] = kb[pr]; kb[pr] = tb;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
    out_ids[(size_t)row * k + i] = (int32_t)(~kb[i]);
    out_vals[(size_t)row * k + i] = __longlong_as_double((long long)ka[i]);
  }
}

}  // namespace

size_t topk_scratch_bytes(int nrows) {
  const size_t r = (size_t)nrows;
  return r * kBins * sizeof(uint32_t) + r * sizeof(TopkSlot) +
         r * kSortCap * (sizeof(unsigned long long) + sizeof(uint32_t)) + 256;
}

TopkScratch topk_scratch_carve(void* base, int nrows) {
  const size_t r = (size_t)nrows;
  TopkScratch s;
  unsigned char* p = (unsigned char*)base;
  s.cand_key = (unsigned long long*)p;  p += r * kSortCap * sizeof(unsigned long long);
  s.slots = (TopkSlot*)p;               p += r * sizeof(TopkSlot);
  s.hist = (uint32_t*)p;                p += r * kBins * sizeof(uint32_t);
  s.cand_id = (uint32_t*)p;
  return s;
}

cudaError_t launch_estimate(const double* res, const Tally* tally, double* est, const double* r,
                            double alpha, int zero_hop, uint64_t count, int num_sms,
                            cudaStream_t st) {
  uint64_t blocks = (count + 255) / 256;
  if (blocks > (uint64_t)num_sms * 32) blocks = (uint64_t)num_sms * 32;
  if (blocks == 0) return cudaSuccess;
  k_estimate<<<(unsigned)blocks, 256, 0, st>>>(res, tally, est, r, alpha, zero_hop, count);
  return cudaGetLastError();
}

cudaError_t launch_topk(const double* est, int64_t n, int nrows, uint32_t k, int32_t* out_ids,
                        double* out_vals, const TopkScratch& s, int num_sms, cudaStream_t st) {
  if (nrows <= 0 || k == 0) return cudaSuccess;
  k_topk_init<<<nrows, 256, 0, st>>>(s.slots, s.hist, nrows, k);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // enough blocks per row to cover the GPU, each with at least 4096 elements
  int64_t bpr = ((int64_t)num_sms * 8 + nrows - 1) / nrows;
  const int64_t max_bpr = (n + 4095) / 4096;
  if (bpr > max_bpr) bpr = max_bpr;
  if (bpr < 1) bpr = 1;
  if (bpr > 65535) bpr = 65535;
  const dim3 grid((unsigned)bpr, (unsigned)nrows);
  for (int level = 0; level < kLevels; ++level) {
    k_topk_hist<<<grid, 256, 0, st>>>(est, n, s.slots, s.hist, level);
    k_topk_select<<<nrows, 1024, 0, st>>>(s.slots, s.hist, k, level);
  }
  k_topk_collect<<<grid, 256, 0, st>>>(est, n, s.slots, s.cand_key, s.cand_id);
  const size_t smem = kSortCap * (sizeof(unsigned long long) + sizeof(uint32_t));
  e = cudaFuncSetAttribute(k_topk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_topk_sort<<<nrows, 1024, smem, st>>>(s.slots, s.cand_key, s.cand_id, k, out_ids, out_vals);
  return cudaGetLastError();
}

}  // namespace fora
