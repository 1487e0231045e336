// FP64 time step, all steps of a call in one cooperative launch with the
// field resident in shared memory (launch mode 3).
//
// Block b owns the consecutive lines J0 .. J1-1 of its CTA tiles and keeps
// them in shared memory for the whole call, between a south halo row J0-1
// and a north halo row J1.  Per step it runs its tiles in order with the tile
// code of the other launches (ccell_fp64_task.cuh), reading and writing the
// resident rows in place: the axial flux south of a tile's first line is
// handed over from the previous tile, so a tile reads a line above it before
// any store to it, and its own lines before its own stores.  Between steps
// only the boundary rows move: each block publishes its first and last lines
// of the new field to global memory and raises its step counter; its
// neighbours wait for the counter (bounded wait, as the grid barrier of the
// persistent launch) and copy those rows into their halo rows.  Rows 0 and M
// (the axial boundary rows of the scheme) are the halo rows of the first and
// last block, updated by their own stores.
#include <cuda_runtime.h>

#include "ccell_fp64_task.cuh"

namespace ccell {

// Wait until the step counters of the neighbouring blocks reach `s`
// (bounded; on timeout the error word records bit 1 and false is returned).
__device__ __forceinline__ bool wait_neighbours(const StepArgs& a, unsigned s) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    const int b = blockIdx.x;
    for (int side = -1; side <= 1 && ok; side += 2) {
      const int nb = b + side;
      if (nb < 0 || nb >= (int)gridDim.x) continue;
      volatile unsigned* f = a.nbr_flags + nb;
      long long spins = 0;
      while (*f < s) {
        if (++spins > a.spin_limit) {
          atomicOr(a.err, 2u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(CC_FP64_MAX_THREADS, 1)
    steps_fp64_resident_kernel(const StepArgs a, long long n) {
  extern __shared__ double sm[];
  const int b = blockIdx.x, B = gridDim.x;
  const int t0 = a.cta_start[b], t1 = a.cta_start[b + 1];
  const TileTask first = a.tiles[t0], last = a.tiles[t1 - 1];
  const DevInst& I = a.insts[first.inst];
  const int nr = I.nr, nrp = smem_row_stride(nr);
  const int J0 = first.j0, J1 = last.j0 + last.nl, R = J1 - J0 + 2;  // rows with the halos
  double* f = sm + a.res_offset;
  const SmemField fld{f, J0, nrp};
  double* T = const_cast<double*>(static_cast<const double*>(a.Tin)) + I.t_off;
  for (int e = threadIdx.x; e < R * nr; e += blockDim.x) {
    const int r = e / nr, i = e - r * nr;
    f[r * nrp + smem_col(i)] = T[(long long)(J0 - 1 + r) * nr + i];
  }
  __syncthreads();
  for (long long q = 0; q < n; ++q) {
    if (q > 0) {  // halo rows of T^q from the neighbours (published with parity q & 1)
      if (!wait_neighbours(a, (unsigned)q + a.bar_extra)) return;  // bar_extra: test hook
      const int par = (int)(q & 1);
      for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        if (b > 0)
          f[smem_col(i)] = __ldcg(a.xb + (((size_t)(b - 1) * 2 + par) * 2 + 1) * nr + i);
        if (b < B - 1)
          f[(size_t)(R - 1) * nrp + smem_col(i)] =
              __ldcg(a.xb + (((size_t)(b + 1) * 2 + par) * 2) * nr + i);
      }
      __syncthreads();
    }
    StepArgs st = a;
    st.step = a.step + q;
    EAcc acc;
    eacc_init(acc);
    int par = 0;
    for (int t = t0; t < t1; ++t) {  // consecutive tiles: fluxes carried from the second on
      step_fp64_tile<ENERGY, TRACE, false>(st, a.tiles[t], sm, acc, t > t0, par, fld);
      par ^= 1;
    }
    eacc_flush<ENERGY, TRACE>(st, acc);
    // publish the first and last lines of T^{q+1}, then raise the counter
    const int par1 = (int)((q + 1) & 1);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      __stcg(a.xb + (((size_t)b * 2 + par1) * 2) * nr + i, f[(size_t)nrp + smem_col(i)]);
      __stcg(a.xb + (((size_t)b * 2 + par1) * 2 + 1) * nr + i,
             f[(size_t)(R - 2) * nrp + smem_col(i)]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(a.nbr_flags + b, (unsigned)(q + 1));
  }
  // the block's lines (and the axial boundary rows of the first and last
  // block) back to the caller's field
  const int r0 = (b == 0) ? 0 : 1, r1 = (b == B - 1) ? R : R - 1;
  for (int e = threadIdx.x; e < (r1 - r0) * nr; e += blockDim.x) {
    const int r = r0 + e / nr, i = e - (r - r0) * nr;
    T[(long long)(J0 - 1 + r) * nr + i] = f[r * nrp + smem_col(i)];
  }
}

template <bool ENERGY, bool TRACE>
static KernelCache& resident_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE>
static int resident_variant_blocks(int threads, int smem) {
  return cached_resident(resident_cache<ENERGY, TRACE>(), steps_fp64_resident_kernel<ENERGY, TRACE>,
                         threads, smem, kMaxTileSmem);
}

int fp64_resident_kernel_blocks(int threads, int smem) {
  int r = resident_variant_blocks<true, true>(threads, smem);
  r = min(r, resident_variant_blocks<true, false>(threads, smem));
  r = min(r, resident_variant_blocks<false, true>(threads, smem));
  return min(r, resident_variant_blocks<false, false>(threads, smem));
}

template <bool ENERGY, bool TRACE>
static int launch_resident_variant(const StepArgs& a, long long n, cudaStream_t st) {
  const int resident = resident_variant_blocks<ENERGY, TRACE>(a.threads, a.smem_bytes);
  if (resident < 0) return -1;
  if (resident < a.n_cta) return -3;
  StepArgs copy = a;
  void* args[] = {&copy, &n};
  const cudaError_t e = cudaLaunchCooperativeKernel(
      (const void*)steps_fp64_resident_kernel<ENERGY, TRACE>, a.n_cta, a.threads, args,
      a.smem_bytes, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return -3;
  }
  return e == cudaSuccess ? 0 : -1;
}

int launch_steps_fp64_resident(const StepArgs& a, long long n, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_resident_variant<true, true>(a, n, st);
  else if (E) r = launch_resident_variant<true, false>(a, n, st);
  else if (T) r = launch_resident_variant<false, true>(a, n, st);
  else r = launch_resident_variant<false, false>(a, n, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
