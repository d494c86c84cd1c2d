// Measured CUDA-core throughput of the current device: the denominators of
// the roofline fractions of the tracing kernels, which are bound by the FP64
// (or FP32) fused multiply-add pipes, not by tensor cores or HBM.
//
// Every thread runs NCHAIN independent multiply-add chains x <- x b + c, so
// that the pipe, not the latency of one chain, limits the rate; the grid fills
// every SM with the resident blocks that fit.  One warm-up launch, then one
// launch timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"
#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int NCHAIN = 8;
constexpr int PEAK_BLOCK = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_BLOCK) fma_chains(int64_t iters, T b, T c, T* sink) {
  T x[NCHAIN];
#pragma unroll
  for (int j = 0; j < NCHAIN; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < NCHAIN; ++j) x[j] = fma(x[j], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < NCHAIN; ++j) s += x[j];
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <class T>
cudaError_t time_chains(int64_t iters, int grid, T* sink, cudaStream_t stream, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  // b < 1 and c > 0: x stays finite and away from denormals
  fma_chains<T><<<grid, PEAK_BLOCK, 0, stream>>>(iters / 8 + 1, (T)0.999, (T)1e-3, sink);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
  if (e == cudaSuccess) {
    fma_chains<T><<<grid, PEAK_BLOCK, 0, stream>>>(iters, (T)0.999, (T)1e-3, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace rtk

extern "C" rt_status rt_measure_alu_peak(int64_t iters64, int64_t iters32, double* out4,
                                         void* stream) {
  using namespace rtk;
  if (!out4) {
    set_last_error("out4 is NULL");
    return RT_EINVAL;
  }
  if (iters64 < 1 || iters32 < 1 || iters64 > ((int64_t)1 << 40) || iters32 > ((int64_t)1 << 40)) {
    set_last_error("iteration counts must be in [1, 2^40]");
    return RT_EINVAL;
  }
  int dev = 0, nsm = 0, occ64 = 0, occ32 = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, fma_chains<double>, PEAK_BLOCK, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, fma_chains<float>, PEAK_BLOCK, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(cudaGetErrorString(e));
    return RT_ECUDA;
  }
  const int g64 = nsm * (occ64 > 0 ? occ64 : 1), g32 = nsm * (occ32 > 0 ? occ32 : 1);
  const int gmax = g64 > g32 ? g64 : g32;
  void* sink = nullptr;
  e = cudaMalloc(&sink, (size_t)gmax * PEAK_BLOCK * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error("cannot allocate the result buffer of the peak measurement");
    return RT_ENOMEM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  float ms64 = 0.0f, ms32 = 0.0f;
  e = time_chains<double>(iters64, g64, (double*)sink, s, &ms64);
  if (e == cudaSuccess) e = time_chains<float>(iters32, g32, (float*)sink, s, &ms32);
  cudaFree(sink);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(cudaGetErrorString(e));
    return RT_ECUDA;
  }
  const double fma_per_thread64 = 4.0 * NCHAIN * (double)iters64;
  const double fma_per_thread32 = 4.0 * NCHAIN * (double)iters32;
  out4[0] = 2.0 * fma_per_thread64 * g64 * PEAK_BLOCK / (ms64 * 1e-3);
  out4[1] = 2.0 * fma_per_thread32 * g32 * PEAK_BLOCK / (ms32 * 1e-3);
  out4[2] = ms64;
  out4[3] = ms32;
  return RT_OK;
}
