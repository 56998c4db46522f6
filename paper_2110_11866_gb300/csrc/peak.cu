// morlet_measure_fp64_rate: the GPU's FP64 fused multiply-add rate, measured, as the denominator of
// the FP64 path's roofline (that path is bound by the FP64 pipe, not by memory, on this GPU).
#include "../../include/morlet_sft.h"

#include <cuda_runtime.h>

namespace {

constexpr int FP64_CHAINS = 8;  // independent FMA chains per thread (enough to cover the pipe latency)

// Every thread runs FP64_CHAINS independent chains a <- a * b + c for `iters` steps (2 flops each)
// and writes one sum, so the compiler keeps every FMA.
__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, long long iters, double b, double c) {
  double a[FP64_CHAINS];
#pragma unroll
  for (int k = 0; k < FP64_CHAINS; ++k) a[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < FP64_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < FP64_CHAINS; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int st_of(cudaError_t e) {
  if (e == cudaSuccess) return MORLET_OK;
  if (e == cudaErrorMemoryAllocation) return MORLET_ERR_NOMEM;
  return MORLET_ERR_CUDA;
}

}  // namespace

extern "C" int morlet_measure_fp64_rate(double* flops, void* stream) {
  if (!flops) return MORLET_ERR_ARG;
  *flops = 0.0;
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp64_fma_kernel, 256, 0);
  if (e != cudaSuccess) return st_of(e);
  const int grid = (occ > 0 ? occ : 1) * sms;
  cudaStream_t st = (cudaStream_t)stream;
  double* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  const long long iters = 1 << 14;
  e = cudaMalloc(&d_out, sizeof(double) * (size_t)grid * 256);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {  // warm-up, then the timed launch
    fp64_fma_kernel<<<grid, 256, 0, st>>>(d_out, iters / 8, 0.999999, 1e-7);
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    fp64_fma_kernel<<<grid, 256, 0, st>>>(d_out, iters, 0.999999, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess && ms > 0.f)
    *flops = 2.0 * FP64_CHAINS * (double)iters * (double)grid * 256.0 / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_out);
  return st_of(e);
}
