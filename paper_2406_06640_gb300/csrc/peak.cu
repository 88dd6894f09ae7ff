// Measured FP32 FMA throughput of the device: the denominator of the roofline of the ALU-bound
// kernels (the fused per-position kernel, the staged passes, the CGLS solver), next to the nominal
// figure of SMs x 128 FP32 lanes x 2 FLOP x clock. The paper has no counterpart; this is a
// measurement utility.
//
// Every thread runs kChains independent FMA chains (enough to cover the pipe latency) for `iters`
// rounds; the chains' sum is stored so nothing is optimised away. Grid: 4 CTAs of 256 threads per SM.
#include <cuda_runtime.h>

#include "ptycho.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_ffma_peak(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" ptycho_status ptycho_measure_fp32_peak(double* tflops, double* ms, void* cuda_stream) {
  if (!tflops || !ms) return PTYCHO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return PTYCHO_ECUDA;
  const int blocks = 4 * sms, threads = 256, iters = 4096;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ptycho_status st = PTYCHO_ECUDA;
  float best = 0.f;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return PTYCHO_ENOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  for (int rep = 0; rep < 6; ++rep) {  // the first run warms the clocks up; best of the rest
    cudaEventRecord(e0, s);
    k_ffma_peak<<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && (best == 0.f || t < best)) best = t;
  }
  if (cudaGetLastError() != cudaSuccess || best <= 0.f) goto done;
  *ms = best;
  *tflops = 2.0 * kChains * kUnroll * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  st = PTYCHO_OK;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
