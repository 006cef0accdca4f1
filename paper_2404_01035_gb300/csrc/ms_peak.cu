// FP32 arithmetic peak of the device, measured (the ALU roof of the step's
// roofline).  Every thread runs 8 independent chains of fused multiply-adds,
// scalar (fma.rn.f32) or paired (fma.rn.f32x2, two lanes of arithmetic per
// instruction), long enough that launch overhead is negligible; the grid
// fills every SM with 64 warps.  Flops = 2 per FMA.  The results feed a
// store that never happens (a value the chains cannot reach), so the
// compiler keeps every FMA.
#include <cuda_runtime.h>

#include "ms_device.cuh"
#include "ms_rt.h"

using namespace msgb;

namespace {

constexpr int kIters = 4096;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_fma_scalar(float m, float c, float* sink) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3f * (threadIdx.x + k);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0f) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma_paired(float m, float c, float* sink) {
  F2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = f2(1e-3f * (threadIdx.x + k), 2e-3f * (threadIdx.x + k));
  const F2 m2 = f2s(m), c2 = f2s(c);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma2(a[k], m2, c2);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += f2lo(a[k]) + f2hi(a[k]);
  if (s == -1.0f) sink[0] = s;
}

}  // namespace

extern "C" ms_status ms_peak_fp32(void* stream, int paired, double* tflops) {
  if (!tflops) return fail(nullptr, MS_ERR_ARG, "tflops is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
  float* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaMallocAsync(&sink, sizeof(float), st);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int blocks = sms * kBlocksPerSm;
  // a chain keeps its value inside (0, 1): a <- 0.5 a + 0.25
  const float m = 0.5f, c = 0.25f;
  double best = 0.0;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a, st);
    if (paired)
      k_fma_paired<<<blocks, kThreads, 0, st>>>(m, c, sink);
    else
      k_fma_scalar<<<blocks, kThreads, 0, st>>>(m, c, sink);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess || rep == 0) continue;   // the first launch warms up
    const double fmas = (double)blocks * kThreads * kIters * 8 * (paired ? 2 : 1);
    const double tf = 2.0 * fmas / (ms * 1e-3) / 1e12;
    if (tf > best) best = tf;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFreeAsync(sink, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "FMA peak kernels");
  *tflops = best;
  return MS_OK;
}
