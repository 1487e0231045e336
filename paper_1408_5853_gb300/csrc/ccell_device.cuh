// Device helpers shared by the FP64 and mixed-precision step kernels.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "ccell_internal.h"

namespace ccell {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// material functions (FP64)
// ---------------------------------------------------------------------------
// 1/d to about 1 ulp: hardware approximation of the reciprocal of the high
// word, then one cubic Newton step (e = 1 - d r, r (1 + e + e^2)).
__device__ __forceinline__ double frcp(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  const double e = fma(-d, r, 1.0);
  return fma(fma(e, e, e), r, r);
}

// 1/d to about 46 bits (one quadratic Newton step), for line systems whose
// coefficients carry FP32 accuracy only (the mixed-precision step).
__device__ __forceinline__ double frcp46(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  return fma(r, fma(-d, r, 1.0), r);
}

// Reciprocal of a line solve: full FP64 (FULL) or frcp46.
template <bool FULL>
__device__ __forceinline__ double lrcp(double d) {
  if constexpr (FULL) return frcp(d);
  else return frcp46(d);
}

// lam0 (x / t_ref)^b with the exact pow, for arguments outside the table (kept
// out of line: it is rare, and inlining it at every face evaluation would
// multiply the code and register footprint of the step kernels).
static __device__ __noinline__ double lam_pow_exact(const DevMaterial& M, double y, bool face) {
  return M.lam0s * pow((face ? 0.5 * y : y) * M.inv_tref, M.lam_b);
}

// Power law lam0 (x / t_ref)^b from the material's table: y = m 2^e with
// m in [1, 2); the scale row e holds lam0 (k t_ref)^-b 2^(e b) (k = 2 for a
// face, where y = T_a + T_b, k = 1 for a node, where y = T), and m^b is a
// degree-kPowDeg polynomial in m - c_q on mantissa interval q.  Arguments outside
// the table (or non-finite, or <= 0) take the exact pow path.
__device__ __forceinline__ double lam_pow(const DevMaterial& M, double y, bool face) {
  const long long bits = __double_as_longlong(y);
  const int e = (int)(bits >> 52) - 1023 - kPowEmin;
  if (M.ptab != nullptr && (unsigned)e < (unsigned)kPowNE) {
    const unsigned q = (unsigned)(bits >> (52 - kPowBits)) & (kPowQ - 1);
    const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double c = __longlong_as_double(0x3FF0000000000000LL | ((long long)q << (52 - kPowBits)) |
                                          (1LL << (51 - kPowBits)));
    const double* P = M.ptab + 2 * kPowNE + q * (kPowDeg + 1);
    const double u = m - c;
    double r = __ldg(P + kPowDeg);
#pragma unroll
    for (int k = kPowDeg - 1; k >= 0; --k) r = fma(r, u, __ldg(P + k));
    return r * __ldg(M.ptab + (face ? 0 : kPowNE) + e);
  }
  return lam_pow_exact(M, y, face);
}

__device__ __forceinline__ double lam_eval(const DevMaterial& M, double T) {
  if (M.lam_model == 1) return lam_pow(M, T, false);
  if (M.lam_model == 0) return M.lam0s;
  const double* b = M.lam_poly;
  return fma(fma(fma(fma(b[4], T, b[3]), T, b[2]), T, b[1]), T, b[0]);
}

__device__ __forceinline__ double lam_face(const DevMaterial& M, int rule, double Ta,
                                           double Tb) {
  if (rule == 0) {
    if (M.lam_model == 1) return lam_pow(M, Ta + Tb, true);
    return lam_eval(M, 0.5 * (Ta + Tb));
  }
  return 0.5 * (lam_eval(M, Ta) + lam_eval(M, Tb));
}

__device__ __forceinline__ double cap_eval(const DevMaterial& M, double T) {
  if (M.cap_model == 1) {
    const double x = T * M.inv_tref, y = T * M.inv_theta;
    return M.c0s * (x * x * x) * frcp(fma(y * y, y, 1.0));
  }
  if (M.cap_model == 0) return M.c0s;
  const double* a = M.cap_poly;
  return fma(fma(fma(a[3], T, a[2]), T, a[1]), T, a[0]);
}

__device__ __forceinline__ bool not_finite(double x) {
  const unsigned hi = (unsigned)(__double_as_longlong(x) >> 32);
  return (hi & 0x7ff00000u) == 0x7ff00000u;
}

// Phase 2 of a line solve.  Lane l of a group of G lanes holds the separator
// row of its segment (row e_l: a x_{e-1} + b x_e + c x_{e+1} = d) plus, from
// its downward elimination, the normalised last interior row
// (x_{e-1} + pc x_e + pa x_{e_{l-1}} = pd) and the expression of its first
// interior row in the two neighbouring separators (Dacc + P x_e - Aacc x_{e_{l-1}}).
// Substituting the neighbours' rows gives a tridiagonal system in the G
// separators, solved by parallel cyclic reduction over warp shuffles.
// Returns x at this lane's separator.
template <bool FULL = true>
__device__ __forceinline__ double solve_separators(double ae, double be, double ce, double de,
                                                   double pa, double pc, double pd, double Dacc,
                                                   double Aacc, double P, int G, int l) {
  const double D2n = __shfl_down_sync(kFull, Dacc, 1, G);
  const double A2n = __shfl_down_sync(kFull, Aacc, 1, G);
  const double C2n = -__shfl_down_sync(kFull, P, 1, G);
  double at = -ae * pa;
  double bt = fma(-ae, pc, be) - ce * A2n;
  double ct = -ce * C2n;
  double dt = fma(-ae, pd, de) - ce * D2n;
  for (int d = 1; d < G; d <<= 1) {
    const double ib = lrcp<FULL>(bt);
    const double am = __shfl_up_sync(kFull, at, d, G);
    const double cm = __shfl_up_sync(kFull, ct, d, G);
    const double dm = __shfl_up_sync(kFull, dt, d, G);
    const double ibm = __shfl_up_sync(kFull, ib, d, G);
    const double apv = __shfl_down_sync(kFull, at, d, G);
    const double cpv = __shfl_down_sync(kFull, ct, d, G);
    const double dpv = __shfl_down_sync(kFull, dt, d, G);
    const double ibp = __shfl_down_sync(kFull, ib, d, G);
    const double al = (l >= d) ? -at * ibm : 0.0;
    const double ga = (l + d < G) ? -ct * ibp : 0.0;
    const double nb = fma(ga, apv, fma(al, cm, bt));
    const double nd = fma(ga, dpv, fma(al, dm, dt));
    at = al * am;
    ct = ga * cpv;
    bt = nb;
    dt = nd;
  }
  return dt * lrcp<FULL>(bt);
}

// Energy and trace partial sums of one thread, carried over the tiles of a
// launch and flushed (warp sums, one atomic per warp and term) when the
// instance changes, at the end of a step and at the end of the launch.
struct EAcc {
  double e[5];  // dE, Q, Phi_D, Phi_I, Phi_N
  double tr;    // trapezoid-weighted z-sum of That(r_max, z)
  int inst;     // instance the sums belong to (-1: none yet)
};

__device__ __forceinline__ void eacc_init(EAcc& c) {
#pragma unroll
  for (int k = 0; k < 5; ++k) c.e[k] = 0.0;
  c.tr = 0.0;
  c.inst = -1;
}

// Called by every thread of the block (c.inst is block-uniform).
template <bool ENERGY, bool TRACE>
__device__ __forceinline__ void eacc_flush(const StepArgs& a, EAcc& c) {
  if constexpr (!(ENERGY || TRACE)) return;
  if (c.inst < 0) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (ENERGY) {
#pragma unroll
      for (int k = 0; k < 5; ++k) c.e[k] += __shfl_xor_sync(kFull, c.e[k], o);
    }
    if (TRACE) c.tr += __shfl_xor_sync(kFull, c.tr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ENERGY) {
      double* e = a.energy + (long long)c.inst * 5;
#pragma unroll
      for (int k = 0; k < 5; ++k) atomicAdd(e + k, c.e[k]);
    }
    if (TRACE) atomicAdd(a.trace + ((long long)c.inst * a.n_steps + a.step) * 2 + 1, c.tr);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) c.e[k] = 0.0;
  c.tr = 0.0;
}

// A group of consecutive warps of the block that runs one phase of a tile:
// the whole block (barrier 0, __syncthreads) or, in the pipelined launch, the
// producer or the consumer warps (a named barrier of the group's threads).
struct WarpGroup {
  int warp0, nwarps, bar;
  __device__ __forceinline__ int warp() const { return (int)(threadIdx.x >> 5) - warp0; }
  __device__ __forceinline__ int tid() const { return (int)threadIdx.x - 32 * warp0; }
  __device__ __forceinline__ int size() const { return 32 * nwarps; }
  __device__ __forceinline__ void sync() const {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * nwarps) : "memory");
  }
};

__device__ __forceinline__ WarpGroup whole_block() {
  return WarpGroup{0, (int)(blockDim.x >> 5), 0};
}

// Named barrier `id` over n threads: wait for it, or arrive without waiting
// (the arriving thread's earlier shared-memory writes are fenced first).
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  __threadfence_block();
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Phases 1-3 of a CTA tile: the tridiagonal systems of its nl lines, rows
// (a, b, c | d) in SA .. SD (line q in the padded row q of nrp doubles), solved
// in place.  Each line is split over G lanes (lane l holds rows
// [l nr/G, (l+1) nr/G)); every lane eliminates its segment downwards (the
// forward sweep of Eq. (front_sweep) restricted to the segment, keeping the
// coupling to the previous segment's last row; c', a', d' overwrite c, a, d),
// the G separator rows are solved by cyclic reduction with shuffles, and back
// substitution (Eq. (back_sweep)) leaves the solution of every row in SB.
// FULL: reciprocals to FP64 accuracy; otherwise to 46 bits for rows of FP32
// accuracy that are scaled to a unit diagonal (b is not read).
// For G = 1 this is the Thomas algorithm of the paper with alpha_0 = 1,
// beta_0 = 0 and x_N = beta_{N-1} / (1 - alpha_{N-1}).
// warp: index of this warp among the warps that solve (default: in the block).
template <bool FULL>
__device__ __forceinline__ void solve_tile_lines(double* __restrict__ SA, double* __restrict__ SB,
                                                 double* __restrict__ SC, double* __restrict__ SD,
                                                 int nl, int nr, int G, int warp = -1) {
  const int nrp = smem_row_stride(nr);
  const int lg = __ffs(G) - 1;
  const int lane = threadIdx.x & 31;
  if (warp < 0) warp = threadIdx.x >> 5;
  const int grp = lane >> lg, l = lane & (G - 1);
  const int q_req = warp * (32 >> lg) + grp;
  const bool active = q_req < nl;
  const int q = active ? q_req : nl - 1;  // idle lane groups solve a valid line, store nothing
  const int i_lo = (l * nr) >> lg;
  const int i_hi = ((l + 1) * nr) >> lg;
  const int cnt = i_hi - i_lo;  // 2 .. kRowsPerLane
  double* A = SA + (size_t)q * nrp;
  double* B = SB + (size_t)q * nrp;
  double* C = SC + (size_t)q * nrp;
  double* D = SD + (size_t)q * nrp;
  double pc = 0.0, pa = 0.0, pd = 0.0;    // c', a', d' of the previous interior row
  double Dacc = 0.0, Aacc = 0.0, P = 1.0; // first interior row = Dacc + P x_next - Aacc L
  double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;  // separator row
#pragma unroll
  for (int k = 0; k < kRowsPerLane; ++k) {
    if (k < cnt) {
      const int c = smem_col(i_lo + k);
      const double ra = A[c], rb = FULL ? B[c] : 1.0, rc = C[c], rd = D[c];
      if (k < cnt - 1) {
        const double den = (k == 0) ? rb : fma(-ra, pc, rb);
        const double r = lrcp<FULL>(den);
        const double c1 = rc * r;
        const double a1 = (k == 0) ? ra * r : -ra * pa * r;
        const double d1 = (k == 0) ? rd * r : fma(-ra, pd, rd) * r;
        if (active) {
          C[c] = c1;
          A[c] = a1;
          D[c] = d1;
        }
        Dacc = fma(P, d1, Dacc);
        Aacc = fma(P, a1, Aacc);
        P = -P * c1;
        pc = c1;
        pa = a1;
        pd = d1;
      } else {
        ae = ra; be = rb; ce = rc; de = rd;
      }
    }
  }
  const double xs = solve_separators<FULL>(ae, be, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);
  const double L = __shfl_up_sync(kFull, xs, 1, G);
  if (active) {
    double xn = xs;
    B[smem_col(i_hi - 1)] = xs;
#pragma unroll
    for (int k = kRowsPerLane - 2; k >= 0; --k) {
      if (k <= cnt - 2) {
        const int c = smem_col(i_lo + k);
        const double x = fma(-C[c], xn, fma(-A[c], L, D[c]));
        B[c] = x;
        xn = x;
      }
    }
  }
}

// Grid-wide barrier of a cooperative (co-resident) launch with a bounded wait.
// bar[0] counts arrivals, bar[1] is the generation.  Every thread fences its
// writes before thread 0 arrives; the last arrival resets the count and bumps
// the generation; the others poll the generation at most spin_limit times,
// then record a timeout (bit 1 of the error word) and report failure, so a
// failed barrier ends the kernel instead of hanging the GPU.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned extra, long long spin_limit,
                                             unsigned* err) {
  __shared__ int ok_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    int ok = 1;
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x + extra - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > spin_limit) {
          atomicOr(err, 2u);
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

// Per-device launch facts of one kernel.  cudaFuncSetAttribute acts on the
// device that is current when it is called, and the resident-block count
// depends on the device, so the dynamic shared-memory opt-in and the
// occupancy figures (per block size: 64, 128, 256 threads) are kept per
// device; a mutex makes the cache safe for concurrent host threads.
struct KernelCache {
  static constexpr int kDevices = 64;
  std::mutex mu;
  bool opted[kDevices] = {};
  int resident[kDevices][3] = {};
  int smem[kDevices][3];
  KernelCache() {
    for (auto& d : smem) d[0] = d[1] = d[2] = -1;
  }
};

static inline int shape_slot(int threads) { return threads <= 64 ? 0 : (threads <= 128 ? 1 : 2); }

// Resident blocks (SMs x blocks per SM) of `kernel` on the current device for
// a block size and dynamic shared memory, opting the kernel in to the largest
// dynamic shared memory on first use on that device.  Returns -1 if the
// current device cannot be read or lies outside the cache.
template <class K>
int cached_resident(KernelCache& c, K kernel, int threads, int smem_bytes, int smem_max) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= KernelCache::kDevices) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lock(c.mu);
  if (!c.opted[dev]) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) !=
        cudaSuccess)
      cudaGetLastError();  // the launch then reports a tile that does not fit
    c.opted[dev] = true;
  }
  const int si = shape_slot(threads);
  if (c.smem[dev][si] != smem_bytes) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem_bytes);
    c.resident[dev][si] = sms * (per_sm > 0 ? per_sm : 1);
    c.smem[dev][si] = smem_bytes;
  }
  return c.resident[dev][si];
}

}  // namespace ccell
