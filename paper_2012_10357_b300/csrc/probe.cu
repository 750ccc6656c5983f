// FP32 FMA throughput probe: the measured denominator beside the derived
// FP32 peak (SMs x 128 lanes x 2 FLOP x clock) of the trace kernel's roofline.
#include <cuda_runtime.h>

#include "../../include/proceduray.h"
#include "internal.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (hides the FMA latency)
constexpr int kThreads = 256;

__device__ float g_probe_sink;

// Every thread runs kChains dependent chains a <- a * x + y for iters rounds.
// x and y keep the values bounded (fixed point y / (1 - x)); the store is
// conditional on a value the chains never reach, so nothing is optimised away.
__global__ void __launch_bounds__(kThreads) k_fma_probe(uint32_t iters, float x, float y) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.f) g_probe_sink = s;
}

}  // namespace

pr_status pr_fma_peak_probe(uint32_t iters, float* tflops_out, float* ms_out, void* stream) {
  if (!tflops_out || iters == 0 || iters > (1u << 24)) {
    pr_internal_set_error("null output or iters outside 1..2^24");
    return PR_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe, kThreads, 0);
  if (e != cudaSuccess) {
    pr_internal_set_error(std::string("fma probe set-up: ") + cudaGetErrorString(e));
    return PR_ERR_CUDA;
  }
  const unsigned int ctas = (unsigned int)(sms * (per_sm > 0 ? per_sm : 1));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fma_probe<<<ctas, kThreads, 0, st>>>(iters, 0.999f, 0.001f);   // warm-up
    e = cudaEventRecord(ev[0], st);
  }
  if (e == cudaSuccess) {
    k_fma_probe<<<ctas, kThreads, 0, st>>>(iters, 0.999f, 0.001f);
    e = cudaEventRecord(ev[1], st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  if (e == cudaSuccess) e = cudaGetLastError();
  for (cudaEvent_t v : ev)
    if (v) cudaEventDestroy(v);
  if (e != cudaSuccess) {
    pr_internal_set_error(std::string("fma probe: ") + cudaGetErrorString(e));
    return PR_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * (double)ctas * kThreads;
  *tflops_out = ms > 0.f ? (float)(flops / (ms * 1e-3) / 1e12) : 0.f;
  if (ms_out) *ms_out = ms;
  return PR_OK;
}
