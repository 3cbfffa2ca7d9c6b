// Measurement utility (not an operation of the paper): throughput of the
// arithmetic units the front kernels can use -- FP64 fused multiply-add,
// FP64 warp-level MMA (mma.sync m8n8k4 .f64), FP32 fused multiply-add --
// and the latency of a dependent FP64 FMA chain, each timed with CUDA events
// on every SM of the current device.
#include <cuda_runtime.h>

#include <cstdint>

#include "chd_internal.h"

namespace {

constexpr int kThreads = 256;

// eight independent FMA chains per thread
template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, int iters, T s) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = static_cast<T>(threadIdx.x) * static_cast<T>(1e-3) + static_cast<T>(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], s, static_cast<T>(1e-9));
  }
  T r = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// eight independent accumulators of mma.sync m8n8k4 (FP64): 2 * 8 * 8 * 4
// flops per instruction and warp
__global__ void __launch_bounds__(kThreads) k_dmma_chains(double* out, int iters) {
  const double a = threadIdx.x * 1e-3, b = 1.0 + threadIdx.x * 1e-4;
  double c[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
  }
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r += c[i][0] + c[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// one thread, one dependent FP64 FMA chain
__global__ void k_dfma_latency(double* out, int iters, double s) {
  double a = 1.0 + threadIdx.x;
  for (int it = 0; it < iters; ++it) a = fma(a, s, 1e-9);
  out[threadIdx.x] = a;
}

template <class Launch>
cudaError_t time_ms(cudaStream_t st, Launch&& launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  launch(true);  // warm-up (short)
  cudaEventRecord(e0, st);
  launch(false);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace

extern "C" chd_status chd_probe_units(void* stream, double out[4]) {
  if (!out) return CHD_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CHD_ERR_CUDA;
  const int blocks = sms * 8;
  void* buf = nullptr;
  if (cudaMallocAsync(&buf, static_cast<size_t>(blocks) * kThreads * 8, st) != cudaSuccess) return CHD_ERR_OOM;
  double* d = static_cast<double*>(buf);
  float ms = 0.f;
  cudaError_t e = cudaSuccess;
  const int it64 = 4000, it32 = 40000, itmma = 2000, itlat = 200000;
  e = time_ms(st, [&](bool w) { k_fma_chains<double><<<blocks, kThreads, 0, st>>>(d, w ? 10 : it64, 0.999); }, &ms);
  if (e == cudaSuccess) out[0] = 2.0 * 8 * it64 * static_cast<double>(blocks) * kThreads / (ms * 1e-3) / 1e12;
  if (e == cudaSuccess)
    e = time_ms(st, [&](bool w) { k_dmma_chains<<<blocks, kThreads, 0, st>>>(d, w ? 10 : itmma); }, &ms);
  if (e == cudaSuccess)
    out[1] = 2.0 * 8 * 8 * 4 * 8 * itmma * static_cast<double>(blocks) * (kThreads / 32) / (ms * 1e-3) / 1e12;
  if (e == cudaSuccess)
    e = time_ms(st, [&](bool w) {
      k_fma_chains<float><<<blocks, kThreads, 0, st>>>(reinterpret_cast<float*>(d), w ? 10 : it32, 0.999f);
    }, &ms);
  if (e == cudaSuccess) out[2] = 2.0 * 8 * it32 * static_cast<double>(blocks) * kThreads / (ms * 1e-3) / 1e12;
  if (e == cudaSuccess) e = time_ms(st, [&](bool w) { k_dfma_latency<<<1, 1, 0, st>>>(d, w ? 10 : itlat, 0.999); }, &ms);
  if (e == cudaSuccess) out[3] = ms * 1e6 / itlat;
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  return e == cudaSuccess ? CHD_OK : CHD_ERR_CUDA;
}
