// gl_peaks.cu -- throughput probes of the FP32 FMA, FP64 FMA and MUFU pipes
// (libglpeaks.so, include/gl_peaks.h).  Each thread runs CH independent chains
// of one instruction; the chains are summed at the end and the sum is written
// only if it equals an impossible value, so the compiler keeps every operation
// while the kernel writes nothing in practice.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gl_peaks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

template <int CH>
__global__ void __launch_bounds__(kThreads) ffma_kernel(float* sink, int iters, float a, float b) {
  float x[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) x[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += x[i];
  if (s == -1234.5f) sink[0] = s;
}

template <int CH>
__global__ void __launch_bounds__(kThreads) dfma_kernel(float* sink, int iters, double a, double b) {
  double x[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) x[i] = 1.0 + 1e-3 * (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += x[i];
  if (s == -1234.5) sink[0] = (float)s;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// x -> rsqrt(x) has the fixed point 1 and stays in [0.5, 2] from a start there
template <int CH>
__global__ void __launch_bounds__(kThreads) mufu_kernel(float* sink, int iters) {
  float x[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) x[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = rsqrt_approx(x[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += x[i];
  if (s == -1234.5f) sink[0] = s;
}

constexpr int kChF = 8, kChD = 4, kChM = 8;

}  // namespace

extern "C" int glp_measure(int device, int kind, int repeats, double* flops_per_s,
                           double* best_ms, double* ops) {
  if (!flops_per_s || !best_ms || !ops || repeats < 1 || repeats > 100) return -1;
  if (kind != GLP_FFMA && kind != GLP_DFMA && kind != GLP_MUFU) return -1;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -3;
  const int grid = sms * kCtasPerSm;
  const double threads = (double)grid * kThreads;
  // iterations sized for launches of about 5-20 ms at B300 rates
  int iters = 0;
  double per_iter = 0.0, flops_per_op = 0.0;
  if (kind == GLP_FFMA) {
    iters = 160000;
    per_iter = kChF;
    flops_per_op = 2.0;
  } else if (kind == GLP_DFMA) {
    iters = 2500;
    per_iter = kChD;
    flops_per_op = 2.0;
  } else {
    iters = 20000;
    per_iter = kChM;
    flops_per_op = 1.0;
  }
  float* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  float best = 1e30f;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess || cudaStreamCreate(&st) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = -3;
  } else {
    for (int r = 0; r <= repeats && rc == 0; ++r) {   // launch 0 is untimed
      cudaEventRecord(e0, st);
      if (kind == GLP_FFMA)
        ffma_kernel<kChF><<<grid, kThreads, 0, st>>>(sink, iters, 0.9999f, 1e-4f);
      else if (kind == GLP_DFMA)
        dfma_kernel<kChD><<<grid, kThreads, 0, st>>>(sink, iters, 0.9999, 1e-4);
      else
        mufu_kernel<kChM><<<grid, kThreads, 0, st>>>(sink, iters);
      cudaEventRecord(e1, st);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = -3;
        break;
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = -3;
      if (r > 0 && ms < best) best = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  *ops = threads * (double)iters * per_iter;
  *best_ms = best;
  *flops_per_s = *ops * flops_per_op / (best * 1e-3);
  return 0;
}
