// Arithmetic-throughput probe: FP64 and FP32 fused multiply-add rates of the
// current device, measured with independent FMA chains (8 per thread) over a
// grid of 16 blocks per SM.  Gives the ALU roofline of the FP64 kernels.
#include <cuda_runtime.h>

#include "../../include/gpsoc.h"

namespace {

template <class T>
__global__ void fma_chains(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

template <class T>
double rate(int sms, int iters, cudaStream_t st) {
  const int blocks = sms * 16, threads = 256;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, threads, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0, st);
  for (int r = 0; r < 3; ++r) fma_chains<T><<<blocks, threads, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double flops = 3.0 * 2.0 * 8.0 * (double)iters * blocks * threads;
  return ms > 0 ? flops / (ms * 1e-3) / 1e12 : -1.0;
}

}  // namespace

extern "C" gpsoc_status gpsoc_probe_peaks(double* fp64_tflops, double* fp32_tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GPSOC_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GPSOC_ECUDA;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return GPSOC_ECUDA;
  if (fp64_tflops) *fp64_tflops = rate<double>(sms, 1024, st);
  if (fp32_tflops) *fp32_tflops = rate<float>(sms, 16384, st);
  cudaStreamDestroy(st);
  return cudaGetLastError() == cudaSuccess ? GPSOC_OK : GPSOC_ECUDA;
}
