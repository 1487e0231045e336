// Mixed-precision time step, one launch per step (the task and the precision
// design are in ccell_mixed_task.cuh).
#include <cuda_runtime.h>

#include "ccell_mixed_task.cuh"

namespace ccell {

template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(CC_MIX_MAX_THREADS, CC_MIX_MIN_BLOCKS) step_mixed_kernel(const StepArgs a) {
  extern __shared__ float smf[];
  EAcc acc;
  eacc_init(acc);
  mixed_tiles<ENERGY, TRACE, true>(a, smf, acc);
  eacc_flush<ENERGY, TRACE>(a, acc);
}

template <bool ENERGY, bool TRACE>
static KernelCache& mixed_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE>
static int mixed_variant_resident(int threads, int smem) {
  return cached_resident(mixed_cache<ENERGY, TRACE>(), step_mixed_kernel<ENERGY, TRACE>, threads,
                         smem, kMaxTileSmem);
}

int mixed_resident_blocks(int threads, int smem) {
  int r = mixed_variant_resident<true, true>(threads, smem);
  r = min(r, mixed_variant_resident<true, false>(threads, smem));
  r = min(r, mixed_variant_resident<false, true>(threads, smem));
  return min(r, mixed_variant_resident<false, false>(threads, smem));
}

template <bool ENERGY, bool TRACE>
static int launch_mixed_variant(const StepArgs& a, cudaStream_t st) {
  const int t = a.threads > 0 ? a.threads : 128;
  const int resident = mixed_variant_resident<ENERGY, TRACE>(t, a.smem_bytes);
  if (resident < 0) return -1;
  const int blocks = a.cta_start ? a.n_cta : (a.n_tiles < resident ? a.n_tiles : resident);
  step_mixed_kernel<ENERGY, TRACE><<<blocks, t, a.smem_bytes, st>>>(a);
  return 0;
}

int launch_step_mixed(const StepArgs& a, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_mixed_variant<true, true>(a, st);
  else if (E) r = launch_mixed_variant<true, false>(a, st);
  else if (T) r = launch_mixed_variant<false, true>(a, st);
  else r = launch_mixed_variant<false, false>(a, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The low parts of the first state buffer start at zero for every call.
int launch_mixed_init(float* lo, long long n_total, void* stream) {
  return cudaMemsetAsync(lo, 0, sizeof(float) * n_total, (cudaStream_t)stream) == cudaSuccess
             ? 0 : -1;
}

}  // namespace ccell
