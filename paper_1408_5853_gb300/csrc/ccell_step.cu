// Time-step kernels of the explicit-implicit scheme (Section 3 of Ayriyan et
// al., arXiv:1408.5853) for sm_103a.
//
// One launch per time step.  A block works on CTA tiles of consecutive axial
// lines of one instance (ccell_fp64_task.cuh): properties and the rows of
// Eq. (ABC), the interface rows of Eq. (cc_first_1) and the closures of
// Eq. (first_oder_bc) are assembled in shared memory with the lanes over
// columns; each line is then solved over G lanes (segment elimination, the
// forward sweep of Eq. (front_sweep) restricted to a segment; cyclic
// reduction of the G separator rows with warp shuffles; back substitution,
// Eq. (back_sweep)).  For G = 1 this is exactly the Thomas algorithm of the
// paper with alpha_0 = 1, beta_0 = 0 and That_N = beta_{N-1}/(1 - alpha_{N-1}).
// The blocks of a launch take equal shares of all nodes as ranges of tiles.
// This file also holds the waveform table kernel and the launch counter.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "ccell_fp64_task.cuh"

namespace ccell {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long kernel_launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// waveform table: s[n][k] = s(t_n) of instance k, t_n = t0 + n tau_k
// (Eq. (period) rectangle, or tanh-smoothed edges).  The phase arithmetic uses
// explicitly rounded operations so window edges fall exactly as in plain
// IEEE evaluation.
// ---------------------------------------------------------------------------
__global__ void waveform_kernel(const DevInst* __restrict__ insts, int n_inst,
                                long long n_steps, double t0, double* __restrict__ s_tab,
                                double* __restrict__ ds_tab) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_steps * n_inst) return;
  const long long n = idx / n_inst;
  const int k = (int)(idx - n * n_inst);
  const DevInst& I = insts[k];
  const double tn = __dadd_rn(t0, __dmul_rn((double)n, I.tau));
  const double u = __dsub_rn(tn, I.t_start);
  double s = 0.0, ds = 0.0;
  if (I.src_layer >= 0) {
    if (I.waveform == 2) {  // nu(t) p^2(t), transient turn-on of Section 3.1
      if (u >= 0.0) {
        const double kk = floor(__ddiv_rn(u, I.t_period));
        const double phi = __dsub_rn(u, __dmul_rn(kk, I.t_period));
        if (phi < I.t_on)
          s = (phi < I.edge_w) ? 1.0 - exp(-phi / (7.0 * (I.edge_w / 100.0))) : 1.0;
      }
    } else if (I.waveform == 0) {
      if (u >= 0.0) {
        const double kk = floor(__ddiv_rn(u, I.t_period));
        const double phi = __dsub_rn(u, __dmul_rn(kk, I.t_period));
        s = (phi < I.t_on) ? 1.0 : 0.0;
      }
    } else {
      double kk = floor(__dadd_rn(__ddiv_rn(__dsub_rn(u, __dmul_rn(0.5, I.t_on)), I.t_period), 0.5));
      if (kk < 0.0) kk = 0.0;
      const double phi = __dsub_rn(u, __dmul_rn(kk, I.t_period));
      const double th = tanh((phi - I.t_on) / I.edge_w);
      s = 0.5 * (tanh(phi / I.edge_w) - th);
      ds = 0.5 * (1.0 - th * th) / I.edge_w;  // d s / d t_on
    }
  }
  s_tab[idx] = s;
  if (ds_tab) ds_tab[idx] = ds;
}

int launch_waveform(const DevInst* insts, int n_inst, long long n_steps, double t0,
                    double* s_tab, void* stream, double* ds_tab) {
  const long long n = n_steps * n_inst;
  if (n <= 0) return 0;
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  waveform_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(insts, n_inst, n_steps,
                                                                          t0, s_tab, ds_tab);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Each block takes its range of tiles (consecutive lines of an instance, so
// the axial face fluxes of a tile's last line are handed to the next tile) or,
// without ranges, strides over the tiles.
template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(CC_FP64_MAX_THREADS, CC_FP64_MIN_BLOCKS) step_fp64_kernel(const StepArgs a) {
  extern __shared__ double sm[];
  EAcc acc;
  eacc_init(acc);
  fp64_tiles<ENERGY, TRACE, true>(a, sm, acc);
  eacc_flush<ENERGY, TRACE>(a, acc);
}

// Per-device opt-in to the largest dynamic shared memory and occupancy cache
// of each variant.
template <bool ENERGY, bool TRACE>
static KernelCache& fp64_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE>
static int fp64_variant_resident(int threads, int smem) {
  return cached_resident(fp64_cache<ENERGY, TRACE>(), step_fp64_kernel<ENERGY, TRACE>, threads,
                         smem, kMaxTileSmem);
}

int fp64_resident_blocks(int threads, int smem) {
  int r = fp64_variant_resident<true, true>(threads, smem);
  r = min(r, fp64_variant_resident<true, false>(threads, smem));
  r = min(r, fp64_variant_resident<false, true>(threads, smem));
  return min(r, fp64_variant_resident<false, false>(threads, smem));
}

template <bool ENERGY, bool TRACE>
static int launch_fp64_variant(const StepArgs& a, cudaStream_t st) {
  const int t = a.threads > 0 ? a.threads : 128;
  const int resident = fp64_variant_resident<ENERGY, TRACE>(t, a.smem_bytes);
  if (resident < 0) return -1;
  const int blocks = a.cta_start ? a.n_cta : (a.n_tiles < resident ? a.n_tiles : resident);
  step_fp64_kernel<ENERGY, TRACE><<<blocks, t, a.smem_bytes, st>>>(a);
  return 0;
}

int launch_step_fp64(const StepArgs& a, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_fp64_variant<true, true>(a, st);
  else if (E) r = launch_fp64_variant<true, false>(a, st);
  else if (T) r = launch_fp64_variant<false, true>(a, st);
  else r = launch_fp64_variant<false, false>(a, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
