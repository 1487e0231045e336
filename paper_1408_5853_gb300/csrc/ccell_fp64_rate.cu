// Measured FP64 FMA rate of the current GPU: the denominator of the FP64-pipe
// roofline of the time-step kernels, which are bound by FP64 issue rather
// than by memory (the scheme needs tens of FP64 operations per node-update).
//
// Every thread runs kChains independent dependent chains of DFMA, so each
// SM sub-partition always has independent FP64 work to issue; the grid holds
// four blocks of 256 threads per SM.  The chains' results are reduced into one
// value per thread and stored, so no FMA can be removed as dead code.
#include <cuda_runtime.h>

#include "ccell_internal.h"

namespace ccell {

constexpr int kChains = 8;
constexpr int kRateThreads = 256;
constexpr int kRateBlocksPerSm = 4;

__global__ void __launch_bounds__(kRateThreads) fp64_rate_kernel(int iters, double* out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (double)(tid + k);
  const double a = 0.999999, b = 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[tid] = s;
}

}  // namespace ccell

extern "C" int cc_measure_fp64_rate(double* scratch_dev, int64_t scratch_len, int32_t iters,
                                    double* fma_per_s, double* seconds, void* stream) {
  using namespace ccell;
  if (!fma_per_s || iters < 1) return CC_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CC_ECUDA;
  const int blocks = sms * kRateBlocksPerSm;
  const long long threads = (long long)blocks * kRateThreads;
  if (!scratch_dev || scratch_len < threads) return CC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CC_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CC_ECUDA;
  }
  fp64_rate_kernel<<<blocks, kRateThreads, 0, st>>>(iters / 8 + 1, scratch_dev);  // warm-up
  cudaEventRecord(e0, st);
  fp64_rate_kernel<<<blocks, kRateThreads, 0, st>>>(iters, scratch_dev);
  cudaEventRecord(e1, st);
  count_launch();
  count_launch();
  float ms = 0.0f;
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return CC_ECUDA;
  *fma_per_s = (double)threads * kChains * (double)iters / (1e-3 * (double)ms);
  if (seconds) *seconds = 1e-3 * (double)ms;
  return CC_OK;
}
