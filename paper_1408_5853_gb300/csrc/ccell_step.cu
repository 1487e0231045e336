// Time-step kernels of the explicit-implicit scheme (Section 3 of Ayriyan et
// al., arXiv:1408.5853) for sm_103a.
//
// One warp task covers 32/G consecutive axial lines j of one instance; each
// line is owned by G lanes, lane l holding a contiguous segment of rows
// i in [l*nr/G, (l+1)*nr/G).  Per time step and line:
//   1. every lane assembles its rows of the tridiagonal system of Eq. (ABC)
//      (regular nodes), the interface rows of Eq. (cc_first_1) and the
//      closures of Eq. (first_oder_bc), evaluating lambda(T) and c(T) in
//      registers (Eqs. (Lambda_i), (Lambda_j), (source));
//   2. it eliminates the segment's interior rows downwards (the forward
//      sweep of Eq. (front_sweep) restricted to the segment, keeping the
//      coupling to the previous segment's last row), and accumulates the
//      expression of its first interior row in terms of the two segment
//      separators;
//   3. the G separator rows form a tridiagonal system solved by parallel
//      cyclic reduction with warp shuffles;
//   4. back substitution (Eq. (back_sweep)) inside each segment.
// For G = 1 this is exactly the Thomas algorithm of the paper with
// alpha_0 = 1, beta_0 = 0 and That_N = beta_{N-1}/(1 - alpha_{N-1}).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "ccell_internal.h"

namespace ccell {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long kernel_launch_count() { return g_launches.load(std::memory_order_relaxed); }

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

// Power law lam0 (x / t_ref)^b from the material's table: y = m 2^e with
// m in [1, 2); the scale row e holds lam0 (k t_ref)^-b 2^(e b) (k = 2 for a
// face, where y = T_a + T_b, k = 1 for a node, where y = T), and m^b is a
// degree-5 polynomial in m - c_q on mantissa interval q.  Arguments outside
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
    double r = fma(__ldg(P + 5), u, __ldg(P + 4));
    r = fma(r, u, __ldg(P + 3));
    r = fma(r, u, __ldg(P + 2));
    r = fma(r, u, __ldg(P + 1));
    r = fma(r, u, __ldg(P + 0));
    return r * __ldg(M.ptab + (face ? 0 : kPowNE) + e);
  }
  return M.lam0s * pow((face ? 0.5 * y : y) * M.inv_tref, M.lam_b);
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

// ---------------------------------------------------------------------------
// waveform table: s[n][k] = s(t_n) of instance k, t_n = t0 + n tau_k
// (Eq. (period) rectangle, or tanh-smoothed edges).  The phase arithmetic uses
// explicitly rounded operations so window edges fall exactly as in plain
// IEEE evaluation.
// ---------------------------------------------------------------------------
__global__ void waveform_kernel(const DevInst* __restrict__ insts, int n_inst,
                                long long n_steps, double t0, double* __restrict__ s_tab) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n_steps * n_inst) return;
  const long long n = idx / n_inst;
  const int k = (int)(idx - n * n_inst);
  const DevInst& I = insts[k];
  const double tn = __dadd_rn(t0, __dmul_rn((double)n, I.tau));
  const double u = __dsub_rn(tn, I.t_start);
  double s = 0.0;
  if (I.src_layer >= 0) {
    if (I.waveform == 0) {
      if (u >= 0.0) {
        const double kk = floor(__ddiv_rn(u, I.t_period));
        const double phi = __dsub_rn(u, __dmul_rn(kk, I.t_period));
        s = (phi < I.t_on) ? 1.0 : 0.0;
      }
    } else {
      double kk = floor(__dadd_rn(__ddiv_rn(__dsub_rn(u, __dmul_rn(0.5, I.t_on)), I.t_period), 0.5));
      if (kk < 0.0) kk = 0.0;
      const double phi = __dsub_rn(u, __dmul_rn(kk, I.t_period));
      s = 0.5 * (tanh(phi / I.edge_w) - tanh((phi - I.t_on) / I.edge_w));
    }
  }
  s_tab[idx] = s;
}

int launch_waveform(const DevInst* insts, int n_inst, long long n_steps, double t0,
                    double* s_tab, void* stream) {
  const long long n = n_steps * n_inst;
  if (n <= 0) return 0;
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  waveform_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(insts, n_inst, n_steps,
                                                                          t0, s_tab);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// FP64 step
// ---------------------------------------------------------------------------
template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(128) step_fp64_kernel(const StepArgs a) {
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (wid >= a.n_tasks) return;  // uniform per warp
  const int lane = threadIdx.x & 31;
  const Task tk = a.tasks[wid];
  const DevInst& I = a.insts[tk.inst];
  const int G = I.G;
  const int lg = __ffs(G) - 1;
  const int grp = lane >> lg, l = lane & (G - 1);
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j_req = tk.j0 + grp;
  const bool active = j_req <= M - 1;
  const int j = active ? j_req : M - 1;  // idle lane groups recompute a valid line
  const int i_lo = (l * nr) >> lg;
  const int i_hi = ((l + 1) * nr) >> lg;
  const int cnt = i_hi - i_lo;  // 2 .. kRowsPerLane

  const double* Tin = static_cast<const double*>(a.Tin) + I.t_off;
  double* Tout = static_cast<double*>(a.Tout) + I.t_off;
  const double* Tj = Tin + (long long)j * nr;
  const double* Ts = Tj - nr;
  const double* Tn = Tj + nr;
  const ZGeo zg = I.zg[j];
  const double s = a.s_tab[a.step * a.n_inst + tk.inst];
  const double tau = I.tau, inv_tau = I.inv_tau;
  const int frule = I.face_rule;

  double cp[kRowsPerLane], ap[kRowsPerLane], dp[kRowsPerLane], mm[kRowsPerLane];
  double pc = 0.0, pa = 0.0, pd = 0.0;   // c', a', d' of the previous interior row
  double Dacc = 0.0, Aacc = 0.0, P = 1.0; // first interior row = Dacc + P x_next - Aacc L
  double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;  // separator row
  double le_prev = 0.0;
  bool have_le = false;
  double eQ = 0.0, eD = 0.0, eN = 0.0;

  double Tm1 = (i_lo > 0) ? Tj[i_lo - 1] : 0.0;
  double T0 = Tj[i_lo];

  // ---- 1. assemble rows and eliminate the segment downwards
#pragma unroll
  for (int k = 0; k < kRowsPerLane; ++k) {
    if (k < cnt) {
      const int i = i_lo + k;
      const RowGeo g = I.rg[i];
      const double Tp1 = (i < N) ? Tj[i + 1] : 0.0;
      double ra, rb, rc, rd, m = 0.0;
      if (g.cls == RC_REGULAR) {
        const DevMaterial& Mt = I.mat[g.seg];
        const double tS = Ts[i], tN = Tn[i];
        const double lw = have_le ? le_prev : lam_face(Mt, frule, Tm1, T0);
        const double le = lam_face(Mt, frule, T0, Tp1);
        const double ls = lam_face(Mt, frule, tS, T0);
        const double ln = lam_face(Mt, frule, T0, tN);
        const double rhoc = Mt.rho * cap_eval(Mt, T0);
        // Eq. (Lambda_j), explicit in T
        const double Lj = ln * (tN - T0) * zg.gzn - ls * (T0 - tS) * zg.gzs;
        double X = 0.0;  // Eq. (source)
        if (g.seg == I.src_layer && s != 0.0) {
          X = I.q0 * s;
          if (I.g_model == 1) X *= I.g_ref / sqrt(T0);
        }
        // Eq. (ABC)
        const double A = -g.gA * lw, C = -g.gC * le;
        const double rct = rhoc * inv_tau;
        ra = A;
        rc = C;
        rb = rct - A - C;
        rd = fma(rct, T0, Lj + X);
        le_prev = le;
        have_le = true;
        if (ENERGY) {
          const double V = g.V2 * zg.etabar;
          m = V * rhoc;
          eQ = fma(tau * V, X, eQ);
          if (j == 1) {
            const double f = tau * g.V2 * ls * (tS - T0) / zg.eta_s;
            if (I.bc_z0 == CC_DIRICHLET) eD += f; else eN += f;
          }
          if (j == M - 1) {
            const double f = tau * g.V2 * ln * (tN - T0) / zg.eta_n;
            if (I.bc_zmax == CC_DIRICHLET) eD += f; else eN += f;
          }
        }
      } else if (g.cls == RC_IFACE) {
        // Eq. (cc_first_1)/(cc_first_3) as the row (a, b, c | 0)
        double lm, lp;
        if (I.interface_rule == 0) {
          lm = lam_eval(I.mat[g.segw], T0);
          lp = lam_eval(I.mat[g.seg], T0);
        } else {
          lm = g.rw * lam_face(I.mat[g.segw], frule, Tm1, T0);
          lp = g.re * lam_face(I.mat[g.seg], frule, T0, Tp1);
        }
        ra = -lm * g.he;
        rc = -lp * g.hw;
        rb = fma(lm, g.he, lp * g.hw);
        rd = 0.0;
        have_le = false;
      } else if (g.cls == RC_AXIS) {  // That_0 = That_1
        ra = 0.0; rb = 1.0; rc = -1.0; rd = 0.0;
        have_le = false;
      } else {  // r = r_max
        if (I.bc_rmax == CC_DIRICHLET) { ra = 0.0; rb = 1.0; rc = 0.0; rd = I.t_d; }
        else { ra = -1.0; rb = 1.0; rc = 0.0; rd = 0.0; }
        have_le = false;
      }
      mm[k] = m;
      if (k < cnt - 1) {
        const double den = (k == 0) ? rb : fma(-ra, pc, rb);
        const double r = frcp(den);
        const double c1 = rc * r;
        const double a1 = (k == 0) ? ra * r : -ra * pa * r;
        const double d1 = (k == 0) ? rd * r : fma(-ra, pd, rd) * r;
        cp[k] = c1;
        ap[k] = a1;
        dp[k] = d1;
        Dacc = fma(P, d1, Dacc);
        Aacc = fma(P, a1, Aacc);
        P = -P * c1;
        pc = c1;
        pa = a1;
        pd = d1;
      } else {
        ae = ra; be = rb; ce = rc; de = rd;
      }
      Tm1 = T0;
      T0 = Tp1;
    }
  }

  // ---- 2. separator system: row e_l couples the separators of lanes l-1, l, l+1
  const double D2n = __shfl_down_sync(kFull, Dacc, 1, G);
  const double A2n = __shfl_down_sync(kFull, Aacc, 1, G);
  const double C2n = -__shfl_down_sync(kFull, P, 1, G);
  double at = -ae * pa;
  double bt = fma(-ae, pc, be) - ce * A2n;
  double ct = -ce * C2n;
  double dt = fma(-ae, pd, de) - ce * D2n;
  for (int d = 1; d < G; d <<= 1) {  // parallel cyclic reduction
    const double ib = frcp(bt);
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
  const double xs = dt * frcp(bt);  // this lane's separator (last row)

  // ---- 3. back substitution inside the segment
  const double L = __shfl_up_sync(kFull, xs, 1, G);
  {
    double xn = xs;
#pragma unroll
    for (int k = kRowsPerLane - 2; k >= 0; --k) {
      if (k <= cnt - 2) {
        const double x = fma(-cp[k], xn, fma(-ap[k], L, dp[k]));
        dp[k] = x;
        xn = x;
      }
    }
#pragma unroll
    for (int k = 0; k < kRowsPerLane; ++k)
      if (k == cnt - 1) dp[k] = xs;  // dp[k] = x_k for every row of the segment
  }
  const double xfirst = dp[0];
  const double xnext = __shfl_down_sync(kFull, xfirst, 1, G);  // first row of lane l+1

  // ---- 4. stores, boundary rows, energy and trace epilogue
  double eE = 0.0, eI = 0.0;
  bool bad = false;
  if (active) {
    double* Oj = Tout + (long long)j * nr;
    const bool row0 = (j == 1), rowM = (j == M - 1);
    double* O0 = Tout;
    double* OM = Tout + (long long)M * nr;
#pragma unroll
    for (int k = 0; k < kRowsPerLane; ++k) {
      if (k < cnt) {
        const int i = i_lo + k;
        const double x = dp[k];
        bad |= not_finite(x);
        Oj[i] = x;
        if (row0) O0[i] = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : x;
        if (rowM) OM[i] = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : x;
        if (ENERGY) {
          eE = fma(mm[k], x - Tj[i], eE);
          const int cls = I.rg[i].cls;
          if (cls == RC_IFACE || cls == RC_OUTER) {
            const double xw = (k == 0) ? L : dp[k > 0 ? k - 1 : 0];
            const double Tw = Tj[i - 1], Ti = Tj[i];
            const RowGeo gw = I.rg[i - 1];
            const double ke = tau * gw.V2 * zg.etabar * gw.gC *
                              lam_face(I.mat[gw.seg], frule, Tw, Ti);
            const double fw = ke * (x - xw);  // into node i-1 (regular)
            if (cls == RC_OUTER) {
              if (I.bc_rmax == CC_DIRICHLET) eD += fw; else eN += fw;
            } else {
              const double xe = (k == cnt - 1) ? xnext : dp[k < kRowsPerLane - 1 ? k + 1 : k];  // x_{i+1}
              const RowGeo ge = I.rg[i + 1];
              const double kw = tau * ge.V2 * zg.etabar * ge.gA *
                                lam_face(I.mat[ge.seg], frule, Ti, Tj[i + 1]);
              eI += fw + kw * (x - xe);  // into node i+1 (regular)
            }
          }
        }
      }
    }
  }
  if (bad) atomicOr(a.err, 1u);

  if (ENERGY || TRACE) {
    double tr = 0.0;
    if (TRACE && active && l == G - 1) {  // this lane owns That(r_max, z_j)
      tr = zg.wnorm * xs;
      double* trs = a.trace + ((long long)tk.inst * a.n_steps + a.step) * 2;
      if (j == 1) {
        const double x0 = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : xs;
        tr = fma(I.zg[0].wnorm, x0, tr);
        trs[0] = x0;
      }
      if (j == M - 1) {
        const double xM = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : xs;
        tr = fma(I.zg[M].wnorm, xM, tr);
      }
    }
    if (!active) { eE = eQ = eD = eI = eN = 0.0; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (ENERGY) {
        eE += __shfl_xor_sync(kFull, eE, o);
        eQ += __shfl_xor_sync(kFull, eQ, o);
        eD += __shfl_xor_sync(kFull, eD, o);
        eI += __shfl_xor_sync(kFull, eI, o);
        eN += __shfl_xor_sync(kFull, eN, o);
      }
      if (TRACE) tr += __shfl_xor_sync(kFull, tr, o);
    }
    if (lane == 0) {
      if (ENERGY) {
        double* e = a.energy + (long long)tk.inst * 5;
        atomicAdd(e + 0, eE);
        atomicAdd(e + 1, eQ);
        atomicAdd(e + 2, eD);
        atomicAdd(e + 3, eI);
        atomicAdd(e + 4, eN);
      }
      if (TRACE) atomicAdd(a.trace + ((long long)tk.inst * a.n_steps + a.step) * 2 + 1, tr);
    }
  }
}

int launch_step_fp64(const StepArgs& a, void* stream) {
  const int threads = 128;
  const int blocks = (a.n_tasks * 32 + threads - 1) / threads;
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  if (E && T) step_fp64_kernel<true, true><<<blocks, threads, 0, st>>>(a);
  else if (E) step_fp64_kernel<true, false><<<blocks, threads, 0, st>>>(a);
  else if (T) step_fp64_kernel<false, true><<<blocks, threads, 0, st>>>(a);
  else step_fp64_kernel<false, false><<<blocks, threads, 0, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_step_mixed(const StepArgs&, void*) { return -2; }
int launch_mixed_init(const DevInst*, int, const Task*, int, float*, long long, void*) {
  return -2;
}

}  // namespace ccell
