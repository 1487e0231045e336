// Mixed-precision time step with warp-owned lines (launch mode 2): the warp
// structure of ccell_lines.cuh with the precision split of
// ccell_mixed_task.cuh -- FP32 state pair hi + lo, FP32 conductivities, heat
// capacities, explicit axial operator and rows in delta form (unknown
// dT = That - T, Section 3 of the paper minus the same equation at That = T),
// each row scaled to a unit diagonal in FP32 and widened exactly; the
// tridiagonal elimination, separator solve, back substitution and the energy
// sums in FP64.
// FP32 <-> FP64 conversions use the integer forms of ccell_mixed_task.cuh.
#pragma once
#include "ccell_mixed_task.cuh"

namespace ccell {

template <bool ENERGY, bool TRACE>
__device__ __forceinline__ void mixed_warp_task(const StepArgs& a, const TileTask tk,
                                                double* __restrict__ wsm, EAcc& acc) {
  if (tk.inst != acc.inst) {  // warp-uniform
    eacc_flush<ENERGY, TRACE>(a, acc);
    acc.inst = tk.inst;
  }
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int G = I.G, lg = __ffs(G) - 1, ng = 32 >> lg;
  const int lane = threadIdx.x & 31, grp = lane >> lg, l = lane & (G - 1);
  const int frule = I.face_rule, n_if = I.n_if;
  const int i_lo = (l * nr) >> lg, i_hi = ((l + 1) * nr) >> lg, cnt = i_hi - i_lo;
  const int gb = grp * nr;
  double* C1 = wsm;
  double* A1 = C1 + kWarpRowStride;
  double* D1 = A1 + kWarpRowStride;  // d', then the increment dT
  double* MM = D1 + kWarpRowStride;  // V rho c
  float* FS = reinterpret_cast<float*>(MM + kWarpRowStride);  // south face fluxes
  // [group][interface]: lambda_w*, lambda_e*, (kw, ke, dTw, dTe as FP32 in the last two doubles)
  double* sI = MM + 2 * kWarpRowStride;
  const LaneGeo& LG = *I.lg;
  const float* Hin = static_cast<const float*>(a.Tin) + I.t_off;
  const float* Lin = a.lo_in + I.t_off;
  float* Hout = static_cast<float*>(a.Tout) + I.t_off;
  float* Lout = a.lo_out + I.t_off;
  const float s = (float)a.s_tab[a.step * a.n_inst + tk.inst];
  const float inv_tau = I.inv_tau_f, tau = I.tau_f;
  const float Xs = (I.src_layer >= 0) ? I.q0_f * s : 0.0f;
  const int ja = tk.j0 + (grp * tk.nl) / ng, jb = tk.j0 + ((grp + 1) * tk.nl) / ng;
  const int iters = (tk.nl + ng - 1) / ng;
  double eQ = 0.0, eD = 0.0, eN = 0.0, eI = 0.0, eE = 0.0, tr = 0.0;
  bool bad = false;

  for (int q = 0; q < iters; ++q) {
    const bool valid = ja + q < jb;
    const int j = valid ? ja + q : (ja < jb ? jb - 1 : tk.j0);
    const long long o = (long long)j * nr;
    const ZGeo& zg = I.zg[j];

    // ---- 1. nodal conductivities of the interface rows, Eq. (cc_first_3)
    if (I.interface_rule == 0 && n_if > 0) {
      for (int it = lane; it < ng * n_if; it += 32) {
        const int gg = it / n_if;
        const int i = I.if_i[it - gg * n_if];
        const int ga = tk.j0 + (gg * tk.nl) / ng, gz = tk.j0 + ((gg + 1) * tk.nl) / ng;
        const int jj = ga + q < gz ? ga + q : (ga < gz ? gz - 1 : tk.j0);
        const RowGeo& g = I.rg[i];
        if (g.cls == RC_IFACE) {
          const float h = __ldg(Hin + (long long)jj * nr + i);
          float* K = reinterpret_cast<float*>(sI + 4 * it);
          K[0] = lam32(I.mat[g.segw], h);
          K[1] = lam32(I.mat[g.seg], h);
        }
      }
      __syncwarp();
    }

    // ---- the south fluxes of the first line of the run
    if (q == 0) {
#pragma unroll 1
      for (int k = 0; k < cnt; ++k) {
        const int i = i_lo + k;
        const float hs = __ldg(Hin + o - nr + i), ls = __ldg(Lin + o - nr + i);
        const float hc = __ldg(Hin + o + i), lc = __ldg(Lin + o + i);
        const int seg = (LG.meta[k * G + l] >> 4) & 15;
        FS[smem_col(gb + i)] = lam_face32(I.mat[seg], frule, hs, hc) * ((hc - hs) + (lc - ls));
      }
    }

    // ---- 2. FP32 rows in delta form, FP64 downward elimination; lanes over rows
    float le_last = 0.0f, dE_last = 0.0f;  // east face and T_{i+1} - T_i of the last row
    {
      const int i = i_hi - 1;
      if (i < N) {
        const float h0 = __ldg(Hin + o + i), h1 = __ldg(Hin + o + i + 1);
        le_last = lam_face32(I.mat[I.rg[i].seg], frule, h0, h1);
        dE_last = (h1 - h0) + (__ldg(Lin + o + i + 1) - __ldg(Lin + o + i));
      }
    }
    float lw = __shfl_up_sync(kFull, le_last, 1, G);
    float dW = -__shfl_up_sync(kFull, dE_last, 1, G);
    float hc = __ldg(Hin + o + i_lo), lc = __ldg(Lin + o + i_lo);
    double pc = 0.0, pa = 0.0, pd = 0.0;
    double Dacc = 0.0, Aacc = 0.0, P = 1.0;
    double ae = 0.0, ce = 0.0, de = 0.0;
    float he = 0.0f, lE = 0.0f;
    if (cnt > 1) {
      he = __ldg(Hin + o + i_lo + 1);
      lE = __ldg(Lin + o + i_lo + 1);
    }
    float hn = __ldg(Hin + o + nr + i_lo), ln = __ldg(Lin + o + nr + i_lo);
#pragma unroll 1
    for (int k = 0; k < cnt; ++k) {
      const int i = i_lo + k;
      const int c = smem_col(gb + i);
      const int e = k * G + l;
      const int meta = LG.meta[e];
      const int cls = meta & 15, seg = (meta >> 4) & 15;
      const DevMaterial& Mt = I.mat[seg];
      const bool last = k == cnt - 1;
      // the next row's T(i+1, j) and T(i, j+1), loaded one row ahead
      float he2 = 0.0f, lE2 = 0.0f, hn2 = 0.0f, ln2 = 0.0f;
      if (k + 2 < cnt) {
        he2 = __ldg(Hin + o + i + 2);
        lE2 = __ldg(Lin + o + i + 2);
      }
      if (k + 1 < cnt) {
        hn2 = __ldg(Hin + o + nr + i + 1);
        ln2 = __ldg(Lin + o + nr + i + 1);
      }
      const float dN = (hn - hc) + (ln - lc);                  // T_{j+1} - T_j
      const float dE = last ? dE_last : (he - hc) + (lE - lc);  // T_{i+1} - T_i
      const float le = last ? le_last : lam_face32(Mt, frule, hc, he);
      const float fn = lam_face32(Mt, frule, hc, hn) * dN;
      const float rhoc = Mt.rho_f * cap32(Mt, hc);
      const float fs = FS[c];
      const float Ljv = fmaf(zg.gzn_f, fn, -zg.gzs_f * fs);  // Eq. (Lambda_j)
      float X = (seg == I.src_layer) ? Xs : 0.0f;            // Eq. (source)
      if (I.g_model == 1 && X != 0.0f) X *= I.g_ref_f * rsqrtf(hc);
      float fa = -LG.gA_f[e] * lw, fc = -LG.gC_f[e] * le;    // Eq. (ABC)
      float fb = fmaf(rhoc, inv_tau, -fa - fc);
      float fd = fmaf(-fa, dW, fmaf(-fc, dE, Ljv + X));
      if (cls == RC_REGULAR) {
        if (ENERGY) {
          const float V2f = LG.V2_f[e];
          const float V = V2f * zg.etabar_f;
          MM[c] = widen_f32(V * rhoc);
          if (valid && X != 0.0f) eQ = fma(widen_f32(tau * V), widen_f32(X), eQ);
          if (valid && j == 1) {
            const double f = widen_f32(-tau * V2f * fs / (float)zg.eta_s);
            if (I.bc_z0 == CC_DIRICHLET) eD += f; else eN += f;
          }
          if (valid && j == M - 1) {
            const double f = widen_f32(tau * V2f * fn / (float)zg.eta_n);
            if (I.bc_zmax == CC_DIRICHLET) eD += f; else eN += f;
          }
        }
      } else {
        const RowGeo& g = I.rg[i];
        if (cls == RC_IFACE) {
          const float* K = reinterpret_cast<const float*>(sI + 4 * (grp * n_if + g.ifo));
          float lmv, lpv;
          if (I.interface_rule == 0) {
            lmv = K[0];
            lpv = K[1];
          } else {
            lmv = g.rw_f * lw;
            lpv = g.re_f * le;
          }
          fa = -lmv * g.he_f;
          fc = -lpv * g.hw_f;
          fb = fmaf(lmv, g.he_f, lpv * g.hw_f);
          fd = -fmaf(fa, dW, fc * dE);
        } else if (cls == RC_AXIS) {  // dT_0 - dT_1 = T_1 - T_0
          fa = 0.0f; fb = 1.0f; fc = -1.0f; fd = dE;
        } else if (I.bc_rmax == CC_DIRICHLET) {  // r = r_max
          fa = 0.0f; fb = 1.0f; fc = 0.0f; fd = (I.td_hi - hc) + (I.td_lo - lc);
        } else {  // dT_N - dT_{N-1} = T_{N-1} - T_N
          fa = -1.0f; fb = 1.0f; fc = 0.0f; fd = dW;
        }
        if (ENERGY) {
          MM[c] = 0.0;
          if (cls == RC_IFACE || cls == RC_OUTER) {
            // heat-flow coefficients to the regular neighbours and the old
            // temperature differences across those edges
            const RowGeo& gw = I.rg[i - 1];
            float* K = reinterpret_cast<float*>(sI + 4 * (grp * n_if + g.ifo));
            K[2] = tau * gw.V2_f * gw.gC_f * zg.etabar_f * lw;
            if (i < N) {
              const RowGeo& ge = I.rg[i + 1];
              K[3] = tau * ge.V2_f * ge.gA_f * zg.etabar_f * le;
            } else {
              K[3] = 0.0f;
            }
            K[4] = -dW;
            K[5] = -dE;
          }
        }
      }
      FS[c] = fn;
      // the row divided by its diagonal in FP32, then widened exactly
      const float ib = __fdividef(1.0f, fb);
      const double ra = widen_f32(fa * ib), rc = widen_f32(fc * ib), rd = widen_f32(fd * ib);
      if (!last) {
        double c1, a1, d1;
        if (k == 0) {  // unit diagonal: nothing to eliminate
          c1 = rc;
          a1 = ra;
          d1 = rd;
        } else {
          const double r = frcp46(fma(-ra, pc, 1.0));
          c1 = rc * r;
          a1 = -ra * pa * r;
          d1 = fma(-ra, pd, rd) * r;
        }
        C1[c] = c1;
        A1[c] = a1;
        D1[c] = d1;
        Dacc = fma(P, d1, Dacc);
        Aacc = fma(P, a1, Aacc);
        P = -P * c1;
        pc = c1;
        pa = a1;
        pd = d1;
      } else {
        ae = ra; ce = rc; de = rd;
      }
      lw = le;
      dW = -dE;
      hc = he;
      lc = lE;
      he = he2;
      lE = lE2;
      hn = hn2;
      ln = ln2;
    }

    // ---- 3. separators; 4. back substitution into D1 (unit diagonal)
    const double xs = solve_separators<false>(ae, 1.0, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);
    const double L = __shfl_up_sync(kFull, xs, 1, G);
    {
      double xn = xs;
      D1[smem_col(gb + i_hi - 1)] = xs;
#pragma unroll 4
      for (int k = cnt - 2; k >= 0; --k) {
        const int c = smem_col(gb + i_lo + k);
        const double x = fma(-C1[c], xn, fma(-A1[c], L, D1[c]));
        D1[c] = x;
        xn = x;
      }
    }
    __syncwarp();

    // ---- 5. pair update, boundary rows, trace, energy; lanes over columns
    for (int cc = lane; cc < ng * nr; cc += 32) {
      const int gg = cc / nr, i = cc - gg * nr;
      const int ga = tk.j0 + (gg * tk.nl) / ng, gz = tk.j0 + ((gg + 1) * tk.nl) / ng;
      if (ga + q >= gz) continue;
      const int jj = ga + q;
      const long long rj = (long long)jj * nr;
      const double xd = D1[smem_col(cc)];
      bad |= not_finite(xd);
      const float x = narrow_f64(xd);
      if (ENERGY) eE = fma(MM[smem_col(cc)], xd, eE);
      const float hi = __ldg(Hin + rj + i), lo = __ldg(Lin + rj + i);
      const float v = lo + x;
      const float h1 = hi + v;
      const float l1 = v - (h1 - hi);  // exact: h1 + l1 = hi + v
      Hout[rj + i] = h1;
      Lout[rj + i] = l1;
      if (jj == 1) {
        Hout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.td_hi : h1;
        Lout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.td_lo : l1;
      }
      if (jj == M - 1) {
        const long long rM = (long long)M * nr + i;
        Hout[rM] = (I.bc_zmax == CC_DIRICHLET) ? I.td_hi : h1;
        Lout[rM] = (I.bc_zmax == CC_DIRICHLET) ? I.td_lo : l1;
      }
      if (TRACE && i == N) {  // That(r_max, z_j)
        const double surf = (widen_f32(hi) + widen_f32(lo)) + xd;
        tr = fma(I.zg[jj].wnorm, surf, tr);
        if (jj == 1) {
          const double x0 = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : surf;
          tr = fma(I.zg[0].wnorm, x0, tr);
          a.trace[((long long)tk.inst * a.n_steps + a.step) * 2] = x0;
        }
        if (jj == M - 1) {
          const double xM = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : surf;
          tr = fma(I.zg[M].wnorm, xM, tr);
        }
      }
    }
    if (ENERGY) {
      // heat through the edges between each interface (or r_max) node and its
      // regular neighbours, at the new temperatures: k (dT_old + d(dT))
      for (int it = lane; it < ng * n_if; it += 32) {
        const int gg = it / n_if;
        const int ga = tk.j0 + (gg * tk.nl) / ng, gz = tk.j0 + ((gg + 1) * tk.nl) / ng;
        if (ga + q >= gz) continue;
        const int i = I.if_i[it - gg * n_if];
        const float* K = reinterpret_cast<const float*>(sI + 4 * it);
        const double x = D1[smem_col(gg * nr + i)];
        const double fw = widen_f32(K[2]) * (widen_f32(K[4]) + (x - D1[smem_col(gg * nr + i - 1)]));
        if (I.rg[i].cls == RC_OUTER) {
          if (I.bc_rmax == CC_DIRICHLET) eD += fw; else eN += fw;
        } else {
          eI += fw + widen_f32(K[3]) * (widen_f32(K[5]) + (x - D1[smem_col(gg * nr + i + 1)]));
        }
      }
    }
    __syncwarp();  // the next line reuses the warp's shared memory
  }
  if (bad) atomicOr(a.err, 1u);
  if (ENERGY) {
    acc.e[0] += eE;
    acc.e[1] += eQ;
    acc.e[2] += eD;
    acc.e[3] += eI;
    acc.e[4] += eN;
  }
  if (TRACE) acc.tr += tr;
}

template <bool ENERGY, bool TRACE>
__device__ __forceinline__ void mixed_warp_tasks(const StepArgs& a, double* __restrict__ wsm,
                                                 EAcc& acc) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int t0 = a.cta_start[w], t1 = a.cta_start[w + 1];
  for (int t = t0; t < t1; ++t) mixed_warp_task<ENERGY, TRACE>(a, a.tiles[t], wsm, acc);
}

}  // namespace ccell
