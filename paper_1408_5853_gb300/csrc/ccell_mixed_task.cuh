// Mixed-precision time-step task (same scheme as ccell_step.cu, Section 3 of the
// paper): conductivities, heat capacities, the explicit axial operator and
// the row coefficients run in FP32; the tridiagonal elimination, the
// separator solve, the update and the energy sums run in FP64.
//
// State.  The caller's field is FP32.  Inside one call the temperature is the
// FP32 pair hi + lo (the low parts live in context scratch and start at zero):
// per-step increments near the heater are ~1e-5 K against an FP32 spacing of
// ~3e-6 K at 20-45 K, so rounding the state to one FP32 per step would drift
// by up to ~1e-2 K over 1e4 steps; the pair keeps ~48 bits.
//
// Delta form.  The unknown of the line system is dT = That - T: rows
// A dT_{i-1} + B dT_i + C dT_{i+1} = R with R = Lambda_i[T] + Lambda_j[T] + X,
// which is Eq. (scheme_eq) minus the same equation at That = T.  R is small,
// so its FP32 rounding is relative to the increment, not to T.  Temperature
// differences are taken on the pair, (hi_a - hi_b) + (lo_a - lo_b).
#pragma once
#include "ccell_device.cuh"

namespace ccell {

// ---------------------------------------------------------------------------
// FP32 material functions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lam32(const DevMaterial& M, float T) {
  if (M.lam_model == 1) return M.lam0s_f * __powf(T * M.inv_tref_f, M.lam_b_f);
  if (M.lam_model == 0) return M.lam0s_f;
  const float* b = M.lam_poly_f;
  return fmaf(fmaf(fmaf(fmaf(b[4], T, b[3]), T, b[2]), T, b[1]), T, b[0]);
}

__device__ __forceinline__ float lam_face32(const DevMaterial& M, int rule, float Ta, float Tb) {
  if (rule == 0) return lam32(M, 0.5f * (Ta + Tb));
  return 0.5f * (lam32(M, Ta) + lam32(M, Tb));
}

__device__ __forceinline__ float cap32(const DevMaterial& M, float T) {
  if (M.cap_model == 1) {
    const float x = T * M.inv_tref_f, y = T * M.inv_theta_f;
    return M.c0s_f * (x * x * x) * __frcp_rn(fmaf(y * y, y, 1.0f));
  }
  if (M.cap_model == 0) return M.c0s_f;
  const float* a = M.cap_poly_f;
  return fmaf(fmaf(fmaf(a[3], T, a[2]), T, a[1]), T, a[0]);
}

// ---------------------------------------------------------------------------
// one warp task
// ---------------------------------------------------------------------------
template <bool ENERGY, bool TRACE>
__device__ __forceinline__ void step_mixed_task(const StepArgs& a, const Task tk, const int lane) {
  const DevInst& I = a.insts[tk.inst];
  const int G = I.G;
  const int lg = __ffs(G) - 1;
  const int grp = lane >> lg, l = lane & (G - 1);
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j_req = tk.j0 + grp;
  const bool active = j_req <= M - 1;
  const int j = active ? j_req : M - 1;
  const int i_lo = (l * nr) >> lg;
  const int i_hi = ((l + 1) * nr) >> lg;
  const int cnt = i_hi - i_lo;

  const float* Hin = static_cast<const float*>(a.Tin) + I.t_off;
  const float* Lin = a.lo_in + I.t_off;
  float* Hout = static_cast<float*>(a.Tout) + I.t_off;
  float* Lout = a.lo_out + I.t_off;
  const long long rj = (long long)j * nr;
  const float* Hj = Hin + rj;
  const float* Lj_ = Lin + rj;
  const ZGeo zg = I.zg[j];
  const float s = (float)a.s_tab[a.step * a.n_inst + tk.inst];
  const int frule = I.face_rule;
  const float inv_tau = I.inv_tau_f, tau = I.tau_f;

  double cp[kRowsPerLane], ap[kRowsPerLane], dp[kRowsPerLane];
  float mm[kRowsPerLane];
  double pc = 0.0, pa = 0.0, pd = 0.0;
  double Dacc = 0.0, Aacc = 0.0, P = 1.0;
  double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;
  float le_prev = 0.0f;
  bool have_le = false;
  double eQ = 0.0, eD = 0.0, eN = 0.0;

  float hm1 = (i_lo > 0) ? __ldcg(Hj + (i_lo - 1)) : 0.0f, lm1 = (i_lo > 0) ? __ldcg(Lj_ + (i_lo - 1)) : 0.0f;
  float h0 = __ldcg(Hj + (i_lo)), l0 = __ldcg(Lj_ + (i_lo));

  // ---- 1. FP32 rows in delta form, FP64 downward elimination
#pragma unroll
  for (int k = 0; k < kRowsPerLane; ++k) {
    if (k < cnt) {
      const int i = i_lo + k;
      const RowGeo& g = I.rg[i];
      const int cls = g.cls;
      const float hp1 = (i < N) ? __ldcg(Hj + (i + 1)) : 0.0f, lp1 = (i < N) ? __ldcg(Lj_ + (i + 1)) : 0.0f;
      const float dW = (hm1 - h0) + (lm1 - l0);  // T_{i-1} - T_i
      const float dE = (hp1 - h0) + (lp1 - l0);  // T_{i+1} - T_i
      float fa, fb, fc, fd, m = 0.0f;
      if (cls == RC_REGULAR) {
        const DevMaterial& Mt = I.mat[g.seg];
        const float hs = __ldcg(Hj + (i - nr)), ls_ = __ldcg(Lj_ + (i - nr)), hn = __ldcg(Hj + (i + nr)), ln_ = __ldcg(Lj_ + (i + nr));
        const float dS = (hs - h0) + (ls_ - l0), dN = (hn - h0) + (ln_ - l0);
        const float lw = have_le ? le_prev : lam_face32(Mt, frule, hm1, h0);
        const float le = lam_face32(Mt, frule, h0, hp1);
        const float ls = lam_face32(Mt, frule, hs, h0);
        const float ln = lam_face32(Mt, frule, h0, hn);
        const float rhoc = Mt.rho_f * cap32(Mt, h0);
        const float Ljv = fmaf(ln * zg.gzn_f, dN, ls * zg.gzs_f * dS);  // Eq. (Lambda_j)
        float X = 0.0f;
        if (g.seg == I.src_layer && s != 0.0f) {
          X = I.q0_f * s;
          if (I.g_model == 1) X *= I.g_ref_f * rsqrtf(h0);
        }
        const float A = -g.gA_f * lw, C = -g.gC_f * le;
        fa = A;
        fc = C;
        fb = fmaf(rhoc, inv_tau, -A - C);
        fd = fmaf(-A, dW, fmaf(-C, dE, Ljv + X));
        le_prev = le;
        have_le = true;
        if (ENERGY) {
          const float V = g.V2_f * zg.etabar_f;
          m = V * rhoc;
          eQ += (double)(tau * V * X);
          if (j == 1) {
            const double f = (double)(tau * g.V2_f * ls * dS / (float)zg.eta_s);
            if (I.bc_z0 == CC_DIRICHLET) eD += f; else eN += f;
          }
          if (j == M - 1) {
            const double f = (double)(tau * g.V2_f * ln * dN / (float)zg.eta_n);
            if (I.bc_zmax == CC_DIRICHLET) eD += f; else eN += f;
          }
        }
      } else if (cls == RC_IFACE) {
        float lmv, lpv;
        if (I.interface_rule == 0) {
          lmv = lam32(I.mat[g.segw], h0);
          lpv = lam32(I.mat[g.seg], h0);
        } else {
          lmv = g.rw_f * lam_face32(I.mat[g.segw], frule, hm1, h0);
          lpv = g.re_f * lam_face32(I.mat[g.seg], frule, h0, hp1);
        }
        fa = -lmv * g.he_f;
        fc = -lpv * g.hw_f;
        fb = fmaf(lmv, g.he_f, lpv * g.hw_f);
        fd = -fmaf(fa, dW, fc * dE);
        have_le = false;
      } else if (cls == RC_AXIS) {  // dT_0 - dT_1 = T_1 - T_0
        fa = 0.0f; fb = 1.0f; fc = -1.0f; fd = dE;
        have_le = false;
      } else {
        if (I.bc_rmax == CC_DIRICHLET) {
          fa = 0.0f; fb = 1.0f; fc = 0.0f; fd = (I.td_hi - h0) + (I.td_lo - l0);
        } else {
          fa = -1.0f; fb = 1.0f; fc = 0.0f; fd = dW;  // dT_N - dT_{N-1} = T_{N-1} - T_N
        }
        have_le = false;
      }
      mm[k] = m;
      const double ra = fa, rb = fb, rc = fc, rd = fd;  // exact widening
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
      hm1 = h0; lm1 = l0;
      h0 = hp1; l0 = lp1;
    }
  }

  // ---- 2. separators, 3. back substitution (FP64)
  const double xs = solve_separators(ae, be, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);
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
      if (k == cnt - 1) dp[k] = xs;
  }
  const double xnext = __shfl_down_sync(kFull, dp[0], 1, G);

  // ---- 4. pair update, boundary rows, energy, trace
  double eE = 0.0, eI = 0.0, surf = 0.0;
  bool bad = false;
  if (active) {
    const bool row0 = (j == 1), rowM = (j == M - 1);
#pragma unroll
    for (int k = 0; k < kRowsPerLane; ++k) {
      if (k < cnt) {
        const int i = i_lo + k;
        const double x = dp[k];
        bad |= not_finite(x);
        const float hi = __ldcg(Hj + (i)), lo = __ldcg(Lj_ + (i));
        const float v = lo + __double2float_rn(x);
        const float h1 = hi + v;
        const float l1 = v - (h1 - hi);  // exact: h1 + l1 = hi + v
        Hout[rj + i] = h1;
        Lout[rj + i] = l1;
        if (row0) {
          Hout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.td_hi : h1;
          Lout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.td_lo : l1;
        }
        if (rowM) {
          Hout[(long long)M * nr + i] = (I.bc_zmax == CC_DIRICHLET) ? I.td_hi : h1;
          Lout[(long long)M * nr + i] = (I.bc_zmax == CC_DIRICHLET) ? I.td_lo : l1;
        }
        if (TRACE && i == N) surf = ((double)hi + (double)lo) + x;
        if (ENERGY) {
          eE = fma((double)mm[k], x, eE);
          const int cls = I.rg[i].cls;
          if (cls == RC_IFACE || cls == RC_OUTER) {
            // heat through the edges between this node and its regular
            // neighbours, at the new temperatures: k (dT_old + d(dT))
            const double xw = (k == 0) ? L : dp[k > 0 ? k - 1 : 0];
            const float hw = __ldcg(Hj + (i - 1)), lw_ = __ldcg(Lj_ + (i - 1));
            const float dT = (hi - hw) + (lo - lw_);
            const RowGeo& gw = I.rg[i - 1];
            const float kw = tau * gw.V2_f * zg.etabar_f * gw.gC_f *
                             lam_face32(I.mat[gw.seg], frule, hw, hi);
            const double fw = (double)kw * ((double)dT + (x - xw));
            if (cls == RC_OUTER) {
              if (I.bc_rmax == CC_DIRICHLET) eD += fw; else eN += fw;
            } else {
              const double xe = (k == cnt - 1) ? xnext : dp[k < kRowsPerLane - 1 ? k + 1 : k];
              const float he = __ldcg(Hj + (i + 1)), le_ = __ldcg(Lj_ + (i + 1));
              const float dTe = (hi - he) + (lo - le_);
              const RowGeo& ge = I.rg[i + 1];
              const float ke = tau * ge.V2_f * zg.etabar_f * ge.gA_f *
                               lam_face32(I.mat[ge.seg], frule, hi, he);
              eI += fw + (double)ke * ((double)dTe + (x - xe));
            }
          }
        }
      }
    }
  }
  if (bad) atomicOr(a.err, 1u);

  if (ENERGY || TRACE) {
    double tr = 0.0;
    if (TRACE && active && l == G - 1) {
      tr = zg.wnorm * surf;
      double* trs = a.trace + ((long long)tk.inst * a.n_steps + a.step) * 2;
      if (j == 1) {
        const double x0 = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : surf;
        tr = fma(I.zg[0].wnorm, x0, tr);
        trs[0] = x0;
      }
      if (j == M - 1) {
        const double xM = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : surf;
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

template <class K>
static int resident_blocks_m(K kernel, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  return sms * (per_sm > 0 ? per_sm : 1);
}

static inline int shape_index_m(int threads) { return threads <= 64 ? 0 : (threads <= 128 ? 1 : 2); }

}  // namespace ccell
