// Mixed-precision time step, all steps of a call in one cooperative launch.
#include <cuda_runtime.h>

#include "ccell_mixed_task.cuh"

namespace ccell {

template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(CC_MIX_MAX_THREADS, CC_MIX_MIN_BLOCKS) steps_mixed_persistent_kernel(const StepArgs a,
                                                                      long long n) {
  extern __shared__ float smf[];
  StepArgs s = a;
  for (long long q = 0; q < n; ++q) {
    s.step = a.step + q;
    s.Tin = (q & 1) ? a.Tout : a.Tin;
    s.Tout = (q & 1) ? const_cast<void*>(a.Tin) : a.Tout;
    s.lo_in = (q & 1) ? a.lo_out : a.lo_in;
    s.lo_out = (q & 1) ? const_cast<float*>(a.lo_in) : a.lo_out;
    EAcc acc;
    eacc_init(acc);
    mixed_tiles<ENERGY, TRACE, false>(s, smf, acc);
    eacc_flush<ENERGY, TRACE>(s, acc);
    if (!grid_barrier(a.bar, a.bar_extra, a.spin_limit, a.err)) return;
  }
}

template <bool ENERGY, bool TRACE>
static KernelCache& mixed_persistent_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE>
static int mixed_persistent_variant_resident(int threads, int smem) {
  return cached_resident(mixed_persistent_cache<ENERGY, TRACE>(), steps_mixed_persistent_kernel<ENERGY, TRACE>,
                         threads, smem, kMaxTileSmem);
}

template <bool ENERGY, bool TRACE>
static int launch_mixed_persistent_variant(const StepArgs& a, long long n, cudaStream_t st) {
  auto kern = steps_mixed_persistent_kernel<ENERGY, TRACE>;
  const int t = a.threads > 0 ? a.threads : 128;
  const int resident = mixed_persistent_variant_resident<ENERGY, TRACE>(t, a.smem_bytes);
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

int mixed_persistent_resident_blocks(int threads, int smem) {
  int r = mixed_persistent_variant_resident<true, true>(threads, smem);
  r = min(r, mixed_persistent_variant_resident<true, false>(threads, smem));
  r = min(r, mixed_persistent_variant_resident<false, true>(threads, smem));
  return min(r, mixed_persistent_variant_resident<false, false>(threads, smem));
}

int launch_steps_mixed_persistent(const StepArgs& a, long long n, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_mixed_persistent_variant<true, true>(a, n, st);
  else if (E) r = launch_mixed_persistent_variant<true, false>(a, n, st);
  else if (T) r = launch_mixed_persistent_variant<false, true>(a, n, st);
  else r = launch_mixed_persistent_variant<false, false>(a, n, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
