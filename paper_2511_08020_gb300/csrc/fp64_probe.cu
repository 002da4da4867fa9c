// FP64 throughput probes for the benchmark's roofline denominators (not part
// of libdg.so): a DFMA-chain loop, an mma.sync f64 m8n8k4 loop, and both at
// once in one launch.  Built into _lib/libfp64probe.so; bench.py loads it.
#include <cuda_runtime.h>

namespace {

// FP64 throughput probes.
__global__ void dfma_probe_kernel(double* out, int iters, double s) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], s, 1e-7);
  }
  double t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void dmma_probe_kernel(double* out, int iters) {
  double a = 1e-3 * (threadIdx.x & 7), b = 1e-3 * (threadIdx.x >> 3);
  double c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c0[k]), "+d"(c1[k])
                   : "d"(a), "d"(b));
  }
  double t = 0;
  for (int k = 0; k < 4; ++k) t += c0[k] + c1[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// Half the warps of a block run DFMA chains, the other half mma.sync f64:
// shows whether the two share one FP64 throughput limit.
__global__ void fp64_mixed_probe_kernel(double* out, int it_f, int it_m) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double t = 0;
  if (warp < nw / 2) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < it_f; ++i) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], 1.0000001, 1e-7);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) t += a[k];
  } else {
    double a = 1e-3 * (threadIdx.x & 7), b = 1e-3 * ((threadIdx.x >> 3) & 3);
    double c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
    for (int i = 0; i < it_m; ++i) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(c0[k]), "+d"(c1[k])
                     : "d"(a), "d"(b));
    }
    for (int k = 0; k < 4; ++k) t += c0[k] + c1[k];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

static cudaError_t probe_peak(double* dfma_tflops, double* dmma_tflops) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 4, threads = 128;
  double* out = nullptr;
  e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  const int it1 = 4000, it2 = 1000;
  dfma_probe_kernel<<<blocks, threads>>>(out, 10, 1.0000001);
  cudaEventRecord(e0);
  dfma_probe_kernel<<<blocks, threads>>>(out, it1, 1.0000001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *dfma_tflops = 2.0 * 8 * it1 * (double)blocks * threads / (ms * 1e-3) / 1e12;
  dmma_probe_kernel<<<blocks, threads>>>(out, 10);
  cudaEventRecord(e0);
  dmma_probe_kernel<<<blocks, threads>>>(out, it2);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *dmma_tflops = 2.0 * 8 * 8 * 4 * 4 * it2 * (double)blocks * (threads / 32) / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  cudaFree(out);
  return e;
}

static cudaError_t probe_mixed(double* total_tflops) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 4, threads = 256, itf = 4000, itm = 4000;
  double* out = nullptr;
  e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_mixed_probe_kernel<<<blocks, threads>>>(out, 10, 10);
  cudaEventRecord(e0);
  fp64_mixed_probe_kernel<<<blocks, threads>>>(out, itf, itm);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double fl = 2.0 * 8 * itf * (double)blocks * (threads / 2) + 2.0 * 8 * 8 * 4 * 4 * itm * (double)blocks * (threads / 64);
  *total_tflops = fl / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  cudaFree(out);
  return e;
}

extern "C" {

// Measured FP64 throughput of the current device (DFMA chains and mma.sync f64
// m8n8k4), TFLOP/s, from a ~50 ms probe launch each.  Synchronises.  Returns
// the cudaError_t of the probe (0 on success).
int fp64_probe_peak(double* dfma_tflops, double* dmma_tflops) {
  if (!dfma_tflops || !dmma_tflops) return (int)cudaErrorInvalidValue;
  return (int)probe_peak(dfma_tflops, dmma_tflops);
}

// Combined FP64 throughput (TFLOP/s) when half of every block's warps run DFMA
// chains and the other half mma.sync f64 at the same time: equal to the
// single-path rates if the two share one FP64 throughput limit.  Synchronises.
int fp64_probe_mixed(double* total_tflops) {
  if (!total_tflops) return (int)cudaErrorInvalidValue;
  return (int)probe_mixed(total_tflops);
}

}  // extern "C"
