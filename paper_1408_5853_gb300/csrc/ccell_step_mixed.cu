// Mixed-precision time step, one launch per step (the task and the precision
// design are in ccell_mixed_task.cuh).
#include <cuda_runtime.h>

#include "ccell_mixed_task.cuh"

namespace ccell {

template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(256) step_mixed_kernel(const StepArgs a) {
  const int lane = threadIdx.x & 31;
  const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < a.n_tasks; w += n_warps)
    step_mixed_task<ENERGY, TRACE>(a, a.tasks[w], lane);
}

template <bool ENERGY, bool TRACE>
static void launch_mixed_variant(const StepArgs& a, cudaStream_t st) {
  static int resident[3] = {0, 0, 0};
  const int t = a.threads > 0 ? a.threads : 128, si = shape_index_m(t);
  if (resident[si] == 0) resident[si] = resident_blocks_m(step_mixed_kernel<ENERGY, TRACE>, t);
  const int need = (a.n_tasks * 32 + t - 1) / t;
  step_mixed_kernel<ENERGY, TRACE><<<need < resident[si] ? need : resident[si], t, 0, st>>>(a);
}

int launch_step_mixed(const StepArgs& a, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  if (E && T) launch_mixed_variant<true, true>(a, st);
  else if (E) launch_mixed_variant<true, false>(a, st);
  else if (T) launch_mixed_variant<false, true>(a, st);
  else launch_mixed_variant<false, false>(a, st);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The low parts of the first state buffer start at zero for every call.
int launch_mixed_init(const DevInst*, int, const Task*, int, float* lo, long long n_total,
                      void* stream) {
  return cudaMemsetAsync(lo, 0, sizeof(float) * n_total, (cudaStream_t)stream) == cudaSuccess
             ? 0 : -1;
}

}  // namespace ccell
