// Arithmetic-unit peak probes of the device, for the roofline denominators
// that MEASURED_PEAKS-style copy and bf16 GEMM figures do not cover: FP32
// FFMA, FP64 DFMA on the CUDA cores, and FP64 DMMA (mma.sync m8n8k4).  Each
// probe runs independent dependency chains in every thread of 4 CTAs per SM
// for about the requested time and reports flops / elapsed time measured with
// CUDA events; the caller samples the SM clock around it.
#include "../../include/find.h"

#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3f + c;
  const float m = 0.999999f, b = 1e-7f;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.f) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_dfma(double* out, int iters) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3 + c;
  const double m = 0.999999, b = 1e-7;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.0) out[0] = s;
}

// one m8n8k4 FP64 MMA per warp per chain step: 8 x 8 x 4 FMAs = 512 flops
__global__ void __launch_bounds__(256) k_dmma(double* out, int iters) {
  double acc[4][2];
  const double av = 1e-3 * (threadIdx.x & 31), bv = 0.5;
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 0.0;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
          : "+d"(acc[c][0]), "+d"(acc[c][1])
          : "d"(av), "d"(bv));
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  if (s == 12345.0) out[0] = s;
}

}  // namespace

extern "C" int find_peak_probe(int kind, double seconds, int device, double* tflops) {
  if (!tflops || kind < 0 || kind > 2 || !(seconds > 0.0)) return FIND_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return FIND_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  void* buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) return FIND_ENOMEM;
  const int blocks = 4 * sms, threads = 256;
  // flops per thread per iteration
  const double fpt = kind == 0 ? 2.0 * kChains : kind == 1 ? 2.0 * kChains : 4 * 512.0 / 32.0;
  auto run = [&](int iters) {
    if (kind == 0) k_ffma<<<blocks, threads>>>(static_cast<float*>(buf), iters);
    else if (kind == 1) k_dfma<<<blocks, threads>>>(static_cast<double*>(buf), iters);
    else k_dmma<<<blocks, threads>>>(static_cast<double*>(buf), iters);
  };
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int iters = 1024;
  float ms = 0.f;
  run(iters);  // warm-up
  for (int rep = 0; rep < 20; ++rep) {
    cudaEventRecord(a);
    run(iters);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    if (ms >= 1e3 * seconds) break;
    const double scale = ms > 0.f ? (1e3 * seconds) / ms : 16.0;
    const double next = iters * (scale > 16.0 ? 16.0 : (scale < 1.5 ? 1.5 : scale));
    if (next > 1.5e9) break;
    iters = (int)next;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return FIND_ECUDA;
  *tflops = (double)blocks * threads * iters * fpt / (ms * 1e-3) / 1e12;
  return FIND_OK;
}
