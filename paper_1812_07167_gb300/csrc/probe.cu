// hps_fp64_rate: the FP64 fused multiply-add rate of the current device,
// measured (a diagnostic beside the solver; the paper has no counterpart).
// Every complex128 kernel of the solver that stays on the FMA pipes is bound
// by this rate, so it is the denominator of their roofline fractions.
#include <cuda_runtime.h>

#include "hps.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains a thread (hides the FMA latency)

__device__ double g_fp64_sink;

__global__ void __launch_bounds__(256) fp64_rate_kernel(int iters) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = 1e-3 * (threadIdx.x + c);
  const double m = 0.9999999, d = 1e-7;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = fma(a[c], m, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += a[c];
  if (s == -1.0) g_fp64_sink = s;  // never true (every chain stays positive): keeps them alive
}

}  // namespace

extern "C" int hps_fp64_rate(double *tflops, void *stream) {
  if (!tflops) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return HPS_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return HPS_ECUDA;
  }
  int rc = HPS_OK;
  float best = 1e30f;
  fp64_rate_kernel<<<blocks, threads, 0, st>>>(iters);  // warm-up (clocks, module load)
  for (int rep = 0; rep < 3 && rc == HPS_OK; rep++) {
    cudaEventRecord(e0, st);
    fp64_rate_kernel<<<blocks, threads, 0, st>>>(iters);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = HPS_ECUDA;
    else if (ms < best)
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HPS_OK) return rc;
  const double flop = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return HPS_OK;
}
