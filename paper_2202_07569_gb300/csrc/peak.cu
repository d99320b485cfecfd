// peak.cu -- measured integer-pipe throughput of the device, the
// denominator of the answer kernels' roofline.
//
// The answer path is bound by integer instruction issue (modular
// multiplications on the 32-bit integer pipes), not by HBM, so its roofline
// needs the device's integer-op rate.  Each probe kernel runs CH
// independent dependency chains per thread on every SM (four resident
// 512-thread blocks per SM, 2048 threads) so that latency is hidden and
// only the pipe's throughput limits it; the chains feed each other
// through a double buffer, which keeps the compiler from folding the
// repeated affine steps.  Timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cwpir.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 512;

enum Op { IMAD32 = 0, MULHI32 = 1, MULLO64 = 2, MULHI64 = 3, IADD32 = 4 };

template <int OP>
__device__ __forceinline__ uint64_t step(uint64_t x, uint64_t y, uint64_t a) {
  if (OP == IMAD32) return (uint32_t)x * (uint32_t)a + (uint32_t)y;
  if (OP == MULHI32) return __umulhi((uint32_t)x, (uint32_t)a) ^ (uint32_t)y;
  if (OP == MULLO64) return x * a ^ y;
  if (OP == MULHI64) return __umul64hi(x, a) ^ y;
  return (uint32_t)x + (uint32_t)y + (uint32_t)a;  // IADD3
}

// iters * kUnroll * kChains operations per thread
template <int OP>
__global__ void __launch_bounds__(kThreads) k_int_probe(uint32_t iters, uint64_t a,
                                                         uint64_t *sink) {
  uint64_t x[kChains], y[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i)
    x[i] = (uint64_t)(threadIdx.x + 977u * blockIdx.x) * 0x9E3779B97F4A7C15ull + i;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; u += 2) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) y[i] = step<OP>(x[i], x[(i + 1) % kChains], a);
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = step<OP>(y[i], y[(i + 3) % kChains], a);
    }
  }
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= x[i];
  if (s == 0x5DEECE66Dull) sink[threadIdx.x] = s;  // keeps the chains live
}

template <int OP>
cudaError_t time_probe(int sms, uint32_t iters, uint64_t *sink, double *ops_per_s) {
  const dim3 grid(4 * sms), block(kThreads);
  const uint64_t a = 0x2545F4914F6CDD1Dull;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_int_probe<OP><<<grid, block>>>(iters, a, sink);  // warm-up
    cudaEventRecord(e0);
    k_int_probe<OP><<<grid, block>>>(iters, a, sink);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
      *ops_per_s = (double)grid.x * kThreads * iters * kUnroll * kChains / (ms * 1e-3);
    cudaEventDestroy(e1);
  }
  cudaEventDestroy(e0);
  return e;
}

}  // namespace

extern "C" int cwpir_measure_int_peaks(int device, cwpir_int_peaks *out) {
  if (!out) return CWPIR_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return CWPIR_EINVAL;
  int sms = 0, clk = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      sms <= 0)
    return CWPIR_ECUDA;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
  uint64_t *sink = nullptr;
  if (cudaMalloc(&sink, kThreads * sizeof(uint64_t)) != cudaSuccess) return CWPIR_ENOMEM;
  out->sms = sms;
  out->max_sm_mhz = clk / 1000.0;
  // iteration counts: each timed launch runs a few tens of milliseconds
  cudaError_t e = time_probe<IMAD32>(sms, 4096, sink, &out->imad32_per_s);
  if (e == cudaSuccess) e = time_probe<MULHI32>(sms, 4096, sink, &out->mulhi32_per_s);
  if (e == cudaSuccess) e = time_probe<MULLO64>(sms, 1024, sink, &out->mullo64_per_s);
  if (e == cudaSuccess) e = time_probe<MULHI64>(sms, 1024, sink, &out->mulhi64_per_s);
  if (e == cudaSuccess) e = time_probe<IADD32>(sms, 4096, sink, &out->iadd32_per_s);
  cudaFree(sink);
  return e == cudaSuccess ? CWPIR_OK : CWPIR_ECUDA;
}
