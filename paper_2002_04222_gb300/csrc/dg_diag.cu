// Diagnostics outside the method: a measured FP64 FMA throughput, the
// denominator of the residual kernels' roofline (they are bound by the FP64
// pipe, and the GPU's FP64 rate is not a published constant of this part).
#include <cuda_runtime.h>
#include "dg_internal.h"

namespace dg {

static __device__ double g_peak_sink;

// Eight independent FMA chains per thread (enough to cover the FP64 pipe's
// latency at full occupancy), ITERS steps each; a = a * b + c with b < 1
// keeps every value finite and normal.
template <int ITERS>
__global__ void __launch_bounds__(256) fp64_fma_kernel(double b, double c) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0) g_peak_sink = s;   // never true; keeps the chains alive
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_peak_fp64(int reps, double* tflops, void* stream) {
  if (reps < 1 || !tflops) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  constexpr int ITERS = 4096;
  int dev = 0, sms = 0, per_sm = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_kernel<ITERS>, 256, 0));
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  fp64_fma_kernel<ITERS><<<grid, 256, 0, s>>>(0.999999, 1e-6);  // warm-up
  DG_LAUNCHED(1);
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) fp64_fma_kernel<ITERS><<<grid, 256, 0, s>>>(0.999999, 1e-6);
  cudaEventRecord(e1, s);
  DG_LAUNCHED(reps);
  DG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * ITERS * (double)grid * 256.0 * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return DG_OK;
}
