// FP32 FMA throughput of the device, measured: the denominator of the fused
// loop's roofline.  The loop is bound by FP32 issue (one FMA per K element in
// each of the SDDMM and the SpMM), so its roof is the rate at which the SMs
// retire FP32 fused multiply-adds, scalar (FFMA) or packed in pairs (FFMA2).
#include "wmd_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;   // independent float2 accumulators per thread
constexpr int kUnroll = 16;  // bodies per loop trip

// Every thread runs kChains independent chains a = a * m + c on float2 pairs,
// either as one packed FFMA2 per pair or as two scalar FFMAs.  m < 1 keeps
// the values bounded; the final test is never true for these inputs but the
// compiler cannot know that, so every chain stays live.
template <bool PACKED>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(float2 m, float2 c, int trips,
                                                            float* sink) {
  float2 a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if constexpr (PACKED) {
          a[i] = __ffma2_rn(a[i], m, c);
        } else {
          a[i].x = fmaf(a[i].x, m.x, c.x);
          a[i].y = fmaf(a[i].y, m.y, c.y);
        }
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (s == -1.f) sink[blockIdx.x] = s;
}

template <bool PACKED>
cudaError_t time_fma(int grid, int trips, cudaStream_t st, float* sink, float* ms) {
  const float2 m = make_float2(0.999f, 0.998f), c = make_float2(1e-3f, 2e-3f);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.f;
  // one untimed launch, then the fastest of three
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
    err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) {
      fma_rate_kernel<PACKED><<<grid, kThreads, 0, st>>>(m, c, trips, sink);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    if (err == cudaSuccess && rep > 0 && (best == 0.f || t < best)) best = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *ms = best;
  return err;
}

}  // namespace

extern "C" wmd_status wmd_measure_fp32_peak(int32_t device, int32_t packed, double* tflops) {
  if (!tflops) return wmd::set_error(WMD_ERR_INVALID_ARG, "tflops is null");
  int n_dev = 0;
  WMD_CUDA_TRY(cudaGetDeviceCount(&n_dev));
  if (device < 0 || device >= n_dev)
    return wmd::set_error(WMD_ERR_INVALID_ARG, "device out of range");
  int prev = 0;
  WMD_CUDA_TRY(cudaGetDevice(&prev));
  WMD_CUDA_TRY(cudaSetDevice(device));
  wmd::NvtxRange nvtx("wmd_measure_fp32_peak");
  int sms = 0, per_sm = 0;
  cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err == cudaSuccess)
    err = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel<true>,
                                                                 kThreads, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel<false>,
                                                                 kThreads, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int trips = 4096;  // about a millisecond at the expected rates
  float* sink = nullptr;
  cudaStream_t st = nullptr;
  if (err == cudaSuccess) err = cudaMalloc(&sink, sizeof(float) * grid);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  float ms = 0.f;
  if (err == cudaSuccess)
    err = packed ? time_fma<true>(grid, trips, st, sink, &ms) : time_fma<false>(grid, trips, st, sink, &ms);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  if (err != cudaSuccess) return wmd::cuda_error(err, "wmd_measure_fp32_peak");
  if (!(ms > 0.f)) return wmd::set_error(WMD_ERR_CUDA, "wmd_measure_fp32_peak: no timing");
  // flops: 2 per FMA, 2 FMAs per float2 pair
  const double flops = 4.0 * grid * kThreads * double(trips) * kUnroll * kChains;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return WMD_OK;
}
