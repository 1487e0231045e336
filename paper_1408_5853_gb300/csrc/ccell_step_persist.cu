// FP64 time step, all steps of a call in one cooperative launch (see
// ccell_step.cu for the scheme and ccell_fp64_task.cuh for one CTA tile).
#include <cuda_runtime.h>

#include "ccell_fp64_task.cuh"

namespace ccell {

// All n steps in one cooperative launch, a bounded grid barrier between steps.
template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(CC_FP64_MAX_THREADS, CC_FP64_MIN_BLOCKS) steps_fp64_persistent_kernel(const StepArgs a,
                                                                     long long n) {
  extern __shared__ double sm[];
  StepArgs s = a;
  for (long long q = 0; q < n; ++q) {
    s.step = a.step + q;
    s.Tin = (q & 1) ? a.Tout : a.Tin;
    s.Tout = (q & 1) ? const_cast<void*>(a.Tin) : a.Tout;
    EAcc acc;
    eacc_init(acc);
    fp64_tiles<ENERGY, TRACE, false>(s, sm, acc);
    eacc_flush<ENERGY, TRACE>(s, acc);
    if (!grid_barrier(a.bar, a.bar_extra, a.spin_limit, a.err)) return;
  }
}

template <bool ENERGY, bool TRACE>
static KernelCache& fp64_persistent_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE>
static int fp64_persistent_variant_resident(int threads, int smem) {
  return cached_resident(fp64_persistent_cache<ENERGY, TRACE>(), steps_fp64_persistent_kernel<ENERGY, TRACE>,
                         threads, smem, kMaxTileSmem);
}

template <bool ENERGY, bool TRACE>
static int launch_fp64_persistent_variant(const StepArgs& a, long long n, cudaStream_t st) {
  auto kern = steps_fp64_persistent_kernel<ENERGY, TRACE>;
  const int t = a.threads > 0 ? a.threads : 128;
  const int resident = fp64_persistent_variant_resident<ENERGY, TRACE>(t, a.smem_bytes);
  if (resident < 0) return -1;
  if (a.cta_start && resident < a.n_cta) return -3;
  const int blocks = a.cta_start ? a.n_cta : (a.n_tiles < resident ? a.n_tiles : resident);
  StepArgs copy = a;
  void* args[] = {&copy, &n};
  const cudaError_t e =
      cudaLaunchCooperativeKernel((const void*)kern, blocks, t, args, a.smem_bytes, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return -3;
  }
  return e == cudaSuccess ? 0 : -1;
}

int fp64_persistent_resident_blocks(int threads, int smem) {
  int r = fp64_persistent_variant_resident<true, true>(threads, smem);
  r = min(r, fp64_persistent_variant_resident<true, false>(threads, smem));
  r = min(r, fp64_persistent_variant_resident<false, true>(threads, smem));
  return min(r, fp64_persistent_variant_resident<false, false>(threads, smem));
}

int launch_steps_fp64_persistent(const StepArgs& a, long long n, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_fp64_persistent_variant<true, true>(a, n, st);
  else if (E) r = launch_fp64_persistent_variant<true, false>(a, n, st);
  else if (T) r = launch_fp64_persistent_variant<false, true>(a, n, st);
  else r = launch_fp64_persistent_variant<false, false>(a, n, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
