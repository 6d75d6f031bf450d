// fora_topk_noalloc: the top-k select of fora_topk with its scratch memory in a
// fixed device array instead of memory the call allocates.
//
// Some callers cannot call cudaMalloc / cudaFree: the free synchronises the whole
// device, which stalls every other stream of a latency-bound serving loop, and
// processes that run under a device-memory budget fixed at start-up must not grow it
// per call.  This entry point allocates nothing: its scratch (histograms, per-row
// select state, candidate lists) lives in g_topk_scratch below, which every GPU that
// loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "fora.h"
#include "fora_engine.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;  // 1 MiB: room for 9 rows
constexpr int kMaxDevices = 64;

// Device-side scratch of the select.  In host code this name is only a host-side
// stand-in: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_topk_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int fora_topk_noalloc(const double* est, int64_t n, int32_t nrows, uint32_t k,
                                 int32_t* out_ids, double* out_vals, void* stream) {
  if (!est || n < 1 || n > 0x7FFFFFFF || nrows < 1)
    return fora::report_error(FORA_ERR_BAD_ARG, "fora_topk_noalloc: bad arguments");
  if (k > FORA_MAX_K || (int64_t)k > n)
    return fora::report_error(FORA_ERR_BAD_ARG, "fora_topk_noalloc: k out of range");
  if (fora::topk_scratch_bytes(nrows) > kNoAllocScratchBytes)
    return fora::report_error(FORA_ERR_BAD_ARG,
                              "fora_topk_noalloc: at most 9 rows fit its 1 MiB scratch array");
  if (k == 0) return FORA_OK;
  if (!out_ids || !out_vals)
    return fora::report_error(FORA_ERR_BAD_ARG, "fora_topk_noalloc: null output");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fora::report_error(FORA_ERR_CUDA, "fora_topk_noalloc: no usable current device");
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fora::report_error(FORA_ERR_CUDA, "fora_topk_noalloc: cannot query the SM count");
  void* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the array's device address
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_topk_scratch);
      if (e != cudaSuccess || !p)
        return fora::report_error(FORA_ERR_CUDA, "fora_topk_noalloc: cudaGetSymbolAddress: %s",
                                  cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  // The select's first kernel zeroes the histograms and resets the per-row state, so
  // what an earlier call left in the array does not matter.
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = fora::launch_topk(est, n, nrows, k, out_ids, out_vals,
                                    fora::topk_scratch_carve(scratch, nrows), sms, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fora::report_error(FORA_ERR_CUDA, "fora_topk_noalloc: %s", cudaGetErrorString(e));
  return FORA_OK;
}
