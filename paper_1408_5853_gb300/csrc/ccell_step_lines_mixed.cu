// Mixed-precision time step with warp-owned lines, one launch per step (the
// task is in ccell_lines_mixed.cuh; the warp structure as in
// ccell_step_lines.cu).
#include <cuda_runtime.h>

#include "ccell_lines_mixed.cuh"

#ifndef CC_LINES_MAX_THREADS
#define CC_LINES_MAX_THREADS 256
#endif
#ifndef CC_LINES_MIN_BLOCKS
#define CC_LINES_MIN_BLOCKS 1
#endif

namespace ccell {

template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(CC_LINES_MAX_THREADS, CC_LINES_MIN_BLOCKS)
    step_mixed_lines_kernel(const StepArgs a) {
  extern __shared__ double sm[];
  double* wsm = sm + (size_t)(threadIdx.x >> 5) * a.warp_doubles;
  EAcc acc;
  eacc_init(acc);
  mixed_warp_tasks<ENERGY, TRACE>(a, wsm, acc);
  eacc_flush<ENERGY, TRACE>(a, acc);
}

template <bool ENERGY, bool TRACE>
static KernelCache& mixed_lines_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE>
static int mixed_lines_variant_resident(int threads, int smem) {
  return cached_resident(mixed_lines_cache<ENERGY, TRACE>(),
                         step_mixed_lines_kernel<ENERGY, TRACE>, threads, smem, kMaxTileSmem);
}

int mixed_lines_resident_blocks(int threads, int smem) {
  int r = mixed_lines_variant_resident<true, true>(threads, smem);
  r = min(r, mixed_lines_variant_resident<true, false>(threads, smem));
  r = min(r, mixed_lines_variant_resident<false, true>(threads, smem));
  return min(r, mixed_lines_variant_resident<false, false>(threads, smem));
}

template <bool ENERGY, bool TRACE>
static int launch_mixed_lines_variant(const StepArgs& a, cudaStream_t st) {
  if (mixed_lines_variant_resident<ENERGY, TRACE>(a.threads, a.smem_bytes) < 0) return -1;
  step_mixed_lines_kernel<ENERGY, TRACE><<<a.n_cta, a.threads, a.smem_bytes, st>>>(a);
  return 0;
}

int launch_step_mixed_lines(const StepArgs& a, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_mixed_lines_variant<true, true>(a, st);
  else if (E) r = launch_mixed_lines_variant<true, false>(a, st);
  else if (T) r = launch_mixed_lines_variant<false, true>(a, st);
  else r = launch_mixed_lines_variant<false, false>(a, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
