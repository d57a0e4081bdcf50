// peaks.cu -- the device's FMA throughput in FP64 and FP32, measured by a kernel of
// independent FMA chains.  It gives the ALU roofline of the stage kernels its denominator
// (the FP64 and FP32 rates of a GB300 are not published per GPU); it has no counterpart in
// the paper.
#include <cuda_runtime.h>

#include "hweno.h"

namespace {

constexpr int kILP = 8;        // independent chains per thread
constexpr int kThreads = 256;  // threads per block
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T* out, int iters, T a, T b) {
  T x[kILP];
#pragma unroll
  for (int k = 0; k < kILP; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kILP; ++k) x[k] = fma(x[k], a, b);
  }
  T s = x[0];
#pragma unroll
  for (int k = 1; k < kILP; ++k) s += x[k];
  // a store the compiler cannot prove dead keeps every chain; it is never taken for these
  // inputs (the chains stay near b / (1 - a) = 1)
  if (s == (T)-1) out[blockIdx.x] = s;
}

template <typename T>
int measure(int device, int iters, double* flop_per_s) {
  int nsm = 0;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return HWENO_ERR_CUDA;
  const int blocks = nsm * kBlocksPerSM;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return HWENO_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int rc = HWENO_OK;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0);
    fma_chain_kernel<T><<<blocks, kThreads>>>(out, iters, (T)0.999999, (T)1e-6);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = HWENO_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != HWENO_OK) return rc;
  const double fmas = (double)blocks * kThreads * kILP * (double)iters;
  *flop_per_s = 2.0 * fmas / (best * 1e-3);
  return HWENO_OK;
}

}  // namespace

extern "C" int hweno_fma_peak(int device, int fp64, double* flop_per_s) {
  if (!flop_per_s) return HWENO_ERR_ARG;
  // about 10 ms per launch on a GB300 in either precision
  return fp64 ? measure<double>(device, 2048, flop_per_s)
              : measure<float>(device, 131072, flop_per_s);
}
