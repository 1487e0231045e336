// FP64 time step with warp-owned lines (launch mode 2): every warp advances
// its own run of consecutive axial lines from start to end, with no barrier
// between the warps of a block.  Per line j (Section 3 of the paper):
//   1. (paper interface rule) the nodal conductivities lambda*_m(T_i*) of the
//      interface rows, Eq. (cc_first_3), with the lanes over interface nodes;
//   2. with the lanes over rows (lane l of a group of G lanes holds the rows
//      [l nr/G, (l+1) nr/G)): every conductivity and heat capacity once --
//      the radial faces lambda_{i+1/2} (Eq. (Lambda_i); a lane's first west
//      face is its left neighbour's last east face), the axial north face
//      flux lambda_{i,j+1/2} (T_{i,j+1} - T_ij) (Eq. (Lambda_j)), kept in
//      registers as the south flux of the next line, and rho c(T) / tau -- the
//      row of Eq. (ABC) with the source of Eq. (source) (or the interface row
//      of Eq. (cc_first_1), or a closure of Eq. (first_oder_bc)), and at once
//      the downward elimination of the lane's segment (the forward sweep of
//      Eq. (front_sweep) restricted to the segment, keeping the coupling to
//      the previous segment's last row);
//   3. the G separator rows by cyclic reduction with shuffles;
//   4. back substitution, Eq. (back_sweep), into the warp's shared memory;
//   5. with the lanes over columns: coalesced stores of That, the axial
//      boundary rows, the surface trace and the energy terms.
// Lines of a warp's run are split over its 32/G lane groups; the south face
// fluxes are carried from line to line in the warp's shared memory (the first
// line of a run evaluates them once more).  The row loop is not unrolled and
// the row geometry is read in lane-major order (LaneGeo), so each load of it
// is one coalesced access per warp.
// For G = 1 the line solve is the Thomas algorithm of the paper with
// alpha_0 = 1, beta_0 = 0 and That_N = beta_{N-1}/(1 - alpha_{N-1}).
// Rectangles only (stepped outlines use the CTA-tile kernels).
#pragma once
#include "ccell_fp64_task.cuh"

namespace ccell {

template <bool ENERGY, bool TRACE>
__device__ __forceinline__ void fp64_warp_task(const StepArgs& a, const TileTask tk,
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
  const int gb = grp * nr;  // first column of this group's line in the warp rows
  double* C1 = wsm;
  double* A1 = C1 + kWarpRowStride;
  double* D1 = A1 + kWarpRowStride;  // d', then That
  double* MM = D1 + kWarpRowStride;  // V2 rho c / tau
  double* FS = MM + kWarpRowStride;  // south face fluxes, carried to the next line
  double* sI = FS + kWarpRowStride;  // [group][interface]: lambda_w*, lambda_e*, kw, ke
  const LaneGeo& LG = *I.lg;
  const double* Tin = static_cast<const double*>(a.Tin) + I.t_off;
  double* Tout = static_cast<double*>(a.Tout) + I.t_off;
  const double s = a.s_tab[a.step * a.n_inst + tk.inst];
  const double Xs = (I.src_layer >= 0) ? I.q0 * s : 0.0;
  // lines [ja, jb) of this lane group; idle groups run a valid line unstored
  const int ja = tk.j0 + (grp * tk.nl) / ng, jb = tk.j0 + ((grp + 1) * tk.nl) / ng;
  const int iters = (tk.nl + ng - 1) / ng;
  double eQ = 0.0, eD = 0.0, eN = 0.0, eI = 0.0, eE = 0.0, tr = 0.0;
  bool bad = false;

  for (int q = 0; q < iters; ++q) {
    const bool valid = ja + q < jb;
    const int j = valid ? ja + q : (ja < jb ? jb - 1 : tk.j0);
    const double* row = Tin + (long long)j * nr;
    const ZGeo& zg = I.zg[j];

    // ---- 1. nodal conductivities of the interface rows, Eq. (cc_first_3)
    if (I.interface_rule == 0 && n_if > 0) {  // warp-uniform
      for (int it = lane; it < ng * n_if; it += 32) {
        const int gg = it / n_if;
        const int i = I.if_i[it - gg * n_if];
        const int ga = tk.j0 + (gg * tk.nl) / ng, gz = tk.j0 + ((gg + 1) * tk.nl) / ng;
        const int jj = ga + q < gz ? ga + q : (ga < gz ? gz - 1 : tk.j0);
        const RowGeo& g = I.rg[i];
        if (g.cls == RC_IFACE) {
          const double T = __ldg(Tin + (long long)jj * nr + i);
          sI[4 * it] = lam_eval(I.mat[g.segw], T);
          sI[4 * it + 1] = lam_eval(I.mat[g.seg], T);
        }
      }
      __syncwarp();
    }

    // ---- the south fluxes of the first line of the run
    if (q == 0) {
#pragma unroll 1
      for (int k = 0; k < cnt; ++k) {
        const int i = i_lo + k;
        const double Ts = __ldg(row - nr + i), Tc = __ldg(row + i);
        const int seg = (LG.meta[k * G + l] >> 4) & 15;
        FS[smem_col(gb + i)] = lam_face(I.mat[seg], frule, Ts, Tc) * (Tc - Ts);
      }
    }

    // ---- 2. rows and downward elimination, lanes over rows
    double le_last = 0.0;  // east face of this lane's last row (lane l+1 needs it as west face)
    {
      const int i = i_hi - 1;
      if (i < N)
        le_last = lam_face(I.mat[I.rg[i].seg], frule, __ldg(row + i), __ldg(row + i + 1));
    }
    double lw = __shfl_up_sync(kFull, le_last, 1, G);
    double Tc = __ldg(row + i_lo);
    double pc = 0.0, pa = 0.0, pd = 0.0;     // c', a', d' of the previous row
    double Dacc = 0.0, Aacc = 0.0, P = 1.0;  // first row = Dacc + P x_sep - Aacc L
    double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;
    double Te = (cnt > 1) ? __ldg(row + i_lo + 1) : 0.0, Tn = __ldg(row + nr + i_lo);
#pragma unroll 1
    for (int k = 0; k < cnt; ++k) {
      const int i = i_lo + k;
      const int c = smem_col(gb + i);
      const int e = k * G + l;
      const int meta = LG.meta[e];
      const int cls = meta & 15, seg = (meta >> 4) & 15;
      const DevMaterial& Mt = I.mat[seg];
      const bool last = k == cnt - 1;
      // T(i+1, j) and T(i, j+1) of the next row, loaded one row ahead
      const double Te2 = (k + 2 < cnt) ? __ldg(row + i + 2) : 0.0;
      const double Tn2 = (k + 1 < cnt) ? __ldg(row + nr + i + 1) : 0.0;
      const double le = last ? le_last : lam_face(Mt, frule, Tc, Te);
      const double fn = lam_face(Mt, frule, Tc, Tn) * (Tn - Tc);
      const double rct = rct_eval(Mt, Tc);
      const double fs = FS[c];
      double X = (seg == I.src_layer) ? Xs : 0.0;  // Eq. (source)
      if (I.g_model == 1 && X != 0.0) X *= I.g_ref / sqrt(Tc);
      // Eq. (ABC) with Eq. (Lambda_j), explicit in T
      double ra = -LG.gA[e] * lw, rc = -LG.gC[e] * le;
      double rb = rct - ra - rc;
      double rd = fma(rct, Tc, fma(zg.gzn, fn, fma(-zg.gzs, fs, X)));
      double m = 0.0;
      if (cls == RC_REGULAR) {
        if (ENERGY) {
          const double V2 = LG.V2[e];
          m = V2 * rct;
          if (valid && X != 0.0) eQ = fma(zg.etabar * I.tau * V2, X, eQ);
          if (valid && j == 1) {
            const double f = -I.tau * V2 * fs / zg.eta_s;
            if (I.bc_z0 == CC_DIRICHLET) eD += f; else eN += f;
          }
          if (valid && j == M - 1) {
            const double f = I.tau * V2 * fn / zg.eta_n;
            if (I.bc_zmax == CC_DIRICHLET) eD += f; else eN += f;
          }
        }
      } else {
        const RowGeo& g = I.rg[i];
        if (cls == RC_IFACE) {  // Eq. (cc_first_1)/(cc_first_3) as the row (a, b, c | 0)
          const double* K = sI + 4 * (grp * n_if + g.ifo);
          double lmv, lpv;
          if (I.interface_rule == 0) {
            lmv = K[0];
            lpv = K[1];
          } else {
            lmv = g.rw * lw;
            lpv = g.re * le;
          }
          ra = -lmv * g.he;
          rc = -lpv * g.hw;
          rb = fma(lmv, g.he, lpv * g.hw);
          rd = 0.0;
        } else if (cls == RC_AXIS) {  // That_0 = That_1
          ra = 0.0; rb = 1.0; rc = -1.0; rd = 0.0;
        } else if (I.bc_rmax == CC_DIRICHLET) {  // r = r_max
          ra = 0.0; rb = 1.0; rc = 0.0; rd = I.t_d;
        } else {
          ra = -1.0; rb = 1.0; rc = 0.0; rd = 0.0;
        }
        if (ENERGY && (cls == RC_IFACE || cls == RC_OUTER)) {
          // heat-flow coefficients to the regular neighbours
          const RowGeo& gw = I.rg[i - 1];
          const RowGeo& ge = I.rg[i < N ? i + 1 : i];
          double* K = sI + 4 * (grp * n_if + g.ifo);
          K[2] = I.tau * gw.V2 * zg.etabar * gw.gC * lw;
          K[3] = (i < N) ? I.tau * ge.V2 * zg.etabar * ge.gA * le : 0.0;
        }
      }
      if (ENERGY) MM[c] = m;
      FS[c] = fn;
      if (!last) {
        const double den = (k == 0) ? rb : fma(-ra, pc, rb);
        const double r = frcp(den);
        const double c1 = rc * r;
        const double a1 = (k == 0) ? ra * r : -ra * pa * r;
        const double d1 = (k == 0) ? rd * r : fma(-ra, pd, rd) * r;
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
        ae = ra; be = rb; ce = rc; de = rd;
      }
      lw = le;
      Tc = Te;
      Te = Te2;
      Tn = Tn2;
    }

    // ---- 3. separators; 4. back substitution into D1
    const double xs = solve_separators<true>(ae, be, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);
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

    // ---- 5. stores, boundary rows, trace, energy; lanes over the columns of
    // all groups' lines
    {
      int qe = -1;
      double eEq = 0.0, ebt = 0.0;
      for (int cc = lane; cc < ng * nr; cc += 32) {
        const int gg = cc / nr, i = cc - gg * nr;
        const int ga = tk.j0 + (gg * tk.nl) / ng, gz = tk.j0 + ((gg + 1) * tk.nl) / ng;
        if (ga + q >= gz) continue;  // idle group: nothing to store
        const int jj = ga + q;
        const double x = D1[smem_col(cc)];
        bad |= not_finite(x);
        Tout[(long long)jj * nr + i] = x;
        if (jj == 1) Tout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : x;
        if (jj == M - 1) Tout[(long long)M * nr + i] = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : x;
        if (ENERGY) {
          if (gg != qe) {  // per-line factor etabar tau of the capacities
            eE = fma(ebt, eEq, eE);
            eEq = 0.0;
            ebt = I.zg[jj].etabar * I.tau;
            qe = gg;
          }
          eEq = fma(MM[smem_col(cc)], x - __ldg(Tin + (long long)jj * nr + i), eEq);
        }
        if (TRACE && i == N) {  // That(r_max, z_j)
          tr = fma(I.zg[jj].wnorm, x, tr);
          if (jj == 1) {
            const double x0 = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : x;
            tr = fma(I.zg[0].wnorm, x0, tr);
            a.trace[((long long)tk.inst * a.n_steps + a.step) * 2] = x0;
          }
          if (jj == M - 1) {
            const double xM = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : x;
            tr = fma(I.zg[M].wnorm, xM, tr);
          }
        }
      }
      if (ENERGY) {
        eE = fma(ebt, eEq, eE);
        // heat through the radial edges between each interface (or r_max)
        // node and its regular neighbours, at That
        for (int it = lane; it < ng * n_if; it += 32) {
          const int gg = it / n_if;
          const int ga = tk.j0 + (gg * tk.nl) / ng, gz = tk.j0 + ((gg + 1) * tk.nl) / ng;
          if (ga + q >= gz) continue;
          const int i = I.if_i[it - gg * n_if];
          const double* K = sI + 4 * it;
          const double x = D1[smem_col(gg * nr + i)];
          const double fw = K[2] * (x - D1[smem_col(gg * nr + i - 1)]);  // into node i-1
          if (I.rg[i].cls == RC_OUTER) {
            if (I.bc_rmax == CC_DIRICHLET) eD += fw; else eN += fw;
          } else {
            eI += fw + K[3] * (x - D1[smem_col(gg * nr + i + 1)]);  // and into node i+1
          }
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

// The warp tasks of warp w: [cta_start[w], cta_start[w + 1]) (w = block x
// warps per block + warp).
template <bool ENERGY, bool TRACE>
__device__ __forceinline__ void fp64_warp_tasks(const StepArgs& a, double* __restrict__ wsm,
                                                EAcc& acc) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int t0 = a.cta_start[w], t1 = a.cta_start[w + 1];
  for (int t = t0; t < t1; ++t) fp64_warp_task<ENERGY, TRACE>(a, a.tiles[t], wsm, acc);
}

}  // namespace ccell
