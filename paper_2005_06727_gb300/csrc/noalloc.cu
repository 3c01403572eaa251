// A query entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: an application whose memory manager
// already reserved the whole GPU (a framework's caching allocator that hands
// out every byte itself), or a serving thread that must never hit the driver
// allocator because cudaMalloc can synchronise the device and stall the other
// streams.  wmd_query_device_noalloc serves them: instead of a caller-provided
// workspace it uses one fixed scratch array compiled into this library.
//
// The array lives in device global memory; every GPU that loads the library
// holds its kWmdScratchBytes until the process exits.  Host code may not use
// the array's name as a device address (on the host it is only a stand-in
// symbol), so the device address is looked up with cudaGetSymbolAddress once
// per device, with that device current.  The lookup happens in
// wmd_corpus_load (noalloc_reserve), which allocates anyway: with lazy module
// loading the driver reserves the array at that lookup, so it must not be the
// no-allocation call that triggers it.
#include <mutex>

#include "wmd_internal.h"

namespace {

// 16 MiB: enough for K of a 30-word query against ~130,000 active vocabulary
// words in float32 (the paper-shaped corpus has 53,151).
constexpr size_t kWmdScratchBytes = size_t(16) << 20;

__device__ __align__(256) unsigned char g_wmd_scratch[kWmdScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

namespace wmd {

cudaError_t noalloc_reserve(int device) {
  if (device < 0 || device >= kMaxDevices) return cudaSuccess;  // the entry point refuses such devices
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[device]) return cudaSuccess;
  int prev = -1;
  cudaGetDevice(&prev);
  void* ptr = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr, g_wmd_scratch);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e == cudaSuccess) g_scratch_ptr[device] = ptr;
  return e;
}

}  // namespace wmd

extern "C" wmd_status wmd_query_device_noalloc(wmd_corpus* corpus, const int32_t* d_q_ids,
                                               const float* d_q_w, int32_t v_r, float lambda,
                                               int32_t max_iter, wmd_precision prec,
                                               double* d_out, void* stream) {
  if (!corpus) return wmd::set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (corpus->device < 0 || corpus->device >= kMaxDevices)
    return wmd::set_error(WMD_ERR_UNSUPPORTED, "device ordinal too large for the scratch table");
  const size_t need = wmd_workspace_bytes(corpus, v_r, prec);
  if (need == 0) return wmd::set_error(WMD_ERR_INVALID_ARG, "v_r or precision out of range");
  if (need > kWmdScratchBytes)
    return wmd::set_error(WMD_ERR_UNSUPPORTED,
                          "this query needs " + std::to_string(need) +
                              " bytes of scratch; the built-in scratch array holds " +
                              std::to_string(kWmdScratchBytes) +
                              " (use wmd_query_device with a larger workspace)");

  // the address was recorded when the corpus was loaded on this device
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    scratch = g_scratch_ptr[corpus->device];
  }
  if (!scratch) return wmd::set_error(WMD_ERR_CUDA, "scratch array not reserved on this device");
  // The kernels overwrite every byte of the scratch they read (r, lambda, K,
  // and the error slots, one per cdist CTA), so nothing has to be cleared
  // between calls.
  return wmd_query_device(corpus, d_q_ids, d_q_w, v_r, lambda, max_iter, prec, scratch,
                          kWmdScratchBytes, d_out, stream);
}
