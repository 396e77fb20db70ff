// Measured FP64 FMA rate of the current GPU: the ceiling that the FP64-ALU-bound
// kernels of this library (the FP64 substitutions, the stencil, the diagonal
// tile factorizations) are compared against.  Every thread runs eight
// independent FMA chains in registers, so the FP64 pipe, not latency, sets the
// time; the grid covers every SM several times.
#include "sfcdd_internal.cuh"

namespace sfcdd {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_dfma_rate(double* __restrict__ out, int iters,
                                                             double a, double b) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
  out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace
}  // namespace sfcdd

using namespace sfcdd;

extern "C" int sfcdd_measure_fp64_rate(int reps, double* tflops, double* ms_per_launch,
                                       void* stream) {
  if (!tflops || reps < 1) return SFCDD_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  SFCDD_CUDA_OK(cudaGetDevice(&dev));
  SFCDD_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 4;
  const int iters = 4096;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* out = nullptr;
  SFCDD_CUDA_OK(cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * sizeof(double)));
  cudaEvent_t e0, e1;
  SFCDD_CUDA_OK(cudaEventCreate(&e0));
  SFCDD_CUDA_OK(cudaEventCreate(&e1));
  const double a = 0.999999, b = 1e-7;
  k_dfma_rate<<<blocks, PROBE_THREADS, 0, s>>>(out, iters, a, b);  // warm-up
  SFCDD_CUDA_OK(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) k_dfma_rate<<<blocks, PROBE_THREADS, 0, s>>>(out, iters, a, b);
  SFCDD_CUDA_OK(cudaEventRecord(e1, s));
  SFCDD_CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0.f;
  SFCDD_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  SFCDD_CUDA_OK(cudaGetLastError());
  const double fmas = (double)blocks * PROBE_THREADS * iters * PROBE_CHAINS * reps;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  if (ms_per_launch) *ms_per_launch = ms / reps;
  return SFCDD_OK;
}
