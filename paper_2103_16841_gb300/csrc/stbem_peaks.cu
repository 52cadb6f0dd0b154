// Measured FMA throughput of the device (diagnostics; no counterpart in the
// paper). The light-cone quadrature is bound by the FP32 and FP64 pipes, not
// by the tensor cores or HBM, so its roofline needs these two rates, measured
// on the device at its present clocks rather than taken from a data sheet.
//
// Each thread runs independent register-resident FMA chains (no memory
// traffic inside the timed loop); every SM is filled to its occupancy limit.
// FP32 is timed both with scalar FMAs and with the paired FMA (two lanes of a
// float2 per instruction); the larger rate is reported.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "stbem_internal.h"

namespace {

constexpr int kChains = 8;    // independent accumulators per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop iteration

// written only when a chain hits an impossible value: keeps the chains live
__device__ double g_fma_sink;

__global__ void __launch_bounds__(256) k_fma_f32(int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * (threadIdx.x + c);
  const float m = 0.9999999f, k = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5f) g_fma_sink = s;
}

__global__ void __launch_bounds__(256) k_fma_f32x2(int iters, float seed) {
  float2 a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + 1e-3f * (threadIdx.x + c), seed - 1e-3f * c);
  const float2 m = make_float2(0.9999999f, 0.9999999f), k = make_float2(1e-7f, 1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
  if (s == 1234.5f) g_fma_sink = s;
}

__global__ void __launch_bounds__(256) k_fma_f64(int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 0.9999999999, k = 1e-10;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5) g_fma_sink = s;
}

// Grows the iteration count until one launch takes >= 50 ms, then times three
// launches of that size; returns the best rate in TFLOP/s (2 flops per FMA lane).
template <typename S>
bem_status time_kernel(void (*kern)(int, S), S seed, int lanes, cudaStream_t s, double* tflops) {
  using namespace stbem;
  int per_sm = 0, dev = 0, sms = 0;
  STBEM_CUDA(cudaGetDevice(&dev));
  STBEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  STBEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
  const int blocks = sms * std::max(per_sm, 1);
  cudaEvent_t e0, e1;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  bem_status st = BEM_OK;
  double best = 0.0;
  long long iters = 64;
  int timed = 0;
  for (int round = 0; round < 40 && timed < 3; ++round) {
    cudaEventRecord(e0, s);
    kern<<<blocks, 256, 0, s>>>((int)iters, seed);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      set_error("FMA probe launch failed");
      st = BEM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < 50.f && timed == 0) {
      iters = std::min<long long>((long long)(iters * std::max(2.0, 60.0 / std::max(ms, 0.01f))), 1 << 28);
      continue;
    }
    ++timed;
    const double flops = 2.0 * lanes * (double)blocks * 256.0 * (double)iters * kUnroll * kChains;
    best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return st;
}

}  // namespace

extern "C" bem_status bem_alu_peaks(bem_context* ctx, double* fp32_tflops, double* fp64_tflops) {
  using namespace stbem;
  if (!ctx || !fp32_tflops || !fp64_tflops) {
    set_error("bem_alu_peaks: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  STBEM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  double a = 0, b = 0, c = 0;
  bem_status st = time_kernel<float>(k_fma_f32, 1.0f, 1, s, &a);
  if (st == BEM_OK) st = time_kernel<float>(k_fma_f32x2, 1.0f, 2, s, &b);
  if (st == BEM_OK) st = time_kernel<double>(k_fma_f64, 1.0, 1, s, &c);
  if (st != BEM_OK) return st;
  *fp32_tflops = std::max(a, b);
  *fp64_tflops = c;
  return BEM_OK;
}
