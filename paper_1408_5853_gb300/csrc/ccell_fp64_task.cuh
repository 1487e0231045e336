// FP64 time step of one CTA tile, shared by the per-step and the persistent
// kernels.
//
// A tile is nl consecutive axial lines j0 .. j0+nl-1 of one instance.  Per
// time step:
//   0. with the warp lanes over consecutive columns i (radial nodes) and each
//      warp marching down the lines of its columns, every conductivity and
//      heat capacity is evaluated once -- the axial face fluxes
//      lambda_{i,j+1/2} (T_{i,j+1} - T_ij) (Eq. (Lambda_j); a face is shared
//      by the two lines it separates), the radial faces lambda_{i+1/2,j}
//      (Eq. (Lambda_i); the west face comes from the neighbouring lane) and
//      rho c(T_ij) / tau -- and the rows of the tridiagonal systems are
//      assembled into shared memory: Eq. (ABC) for regular nodes with the
//      source of Eq. (source), the interface rows of Eq. (cc_first_1) and the
//      closures of Eq. (first_oder_bc);
//   1. each line is split over G lanes (lane l holds rows [l nr/G,
//      (l+1) nr/G)); every lane eliminates its segment downwards (the forward
//      sweep of Eq. (front_sweep) restricted to the segment, keeping the
//      coupling to the previous segment's last row);
//   2. the G separator rows are solved by cyclic reduction with shuffles;
//   3. back substitution (Eq. (back_sweep)) inside each segment;
//   4. with the lanes over columns again: stores, axial boundary rows,
//      surface trace and energy terms.
// For G = 1 the line solve is the Thomas algorithm of the paper with
// alpha_0 = 1, beta_0 = 0 and That_N = beta_{N-1}/(1 - alpha_{N-1}).
#pragma once
#include "ccell_device.cuh"

// Launch bounds of the FP64 step kernels (register budget per thread).
#ifndef CC_FP64_MAX_THREADS
#define CC_FP64_MAX_THREADS 256
#endif
#ifndef CC_FP64_MIN_BLOCKS
#define CC_FP64_MIN_BLOCKS 1
#endif

namespace ccell {

// rho c(T) / tau from the folded material constants.  The Debye-saturated
// form takes its reciprocal to 2^-46 (one Newton step): rho c / tau multiplies
// only the increment That - T of its row (Eq. (ABC): (rho c / tau)(That - T) =
// the fluxes + X), so the relative error it leaves in a step's increment,
// <= 2^-46, is below the FP64 rounding of the temperature itself.
__device__ __forceinline__ double rct_eval(const DevMaterial& M, double T) {
  if (M.cap_model == 1) {
    const double T3 = T * T * T;
    return M.rct_k * T3 * frcp46(fma(M.inv_theta3, T3, 1.0));
  }
  if (M.cap_model == 0) return M.rct_k;
  const double* a = M.cap_poly;
  return M.rho_tau * fma(fma(fma(a[3], T, a[2]), T, a[1]), T, a[0]);
}

// Field values of the current step: read-only within a launch.  CACHED loads
// may go through L1 (per-step launches); otherwise they are L2-only, coherent
// with the other blocks of a persistent launch.
template <bool CACHED>
__device__ __forceinline__ double ld_field(const double* p) {
  if constexpr (CACHED) return __ldg(p);
  else return __ldcg(p);
}

// The field as the tile sees it: T^n at (line j, node i) and the store of
// That.  In global memory (per-step and persistent launches: separate input
// and output buffers) ...
template <bool CACHED>
struct GlobalField {
  const double* in;
  double* out;
  int nr;
  __device__ __forceinline__ GlobalField(const StepArgs& a, const DevInst& I)
      : in(static_cast<const double*>(a.Tin) + I.t_off),
        out(static_cast<double*>(a.Tout) + I.t_off), nr(I.nr) {}
  __device__ __forceinline__ double at(int j, int i) const {
    return ld_field<CACHED>(in + (long long)j * nr + i);
  }
  __device__ __forceinline__ void put(int j, int i, double v) const {
    out[(long long)j * nr + i] = v;
  }
};

// ... or resident in shared memory (a block's lines J0 .. J1-1 between a
// south halo row J0-1 and a north halo row J1, padded rows of nrp doubles,
// updated in place: a tile reads line j only before its own stores of line j,
// and the lines above it only after they are stored by no one earlier).
struct SmemField {
  double* f;
  int J0, nrp;
  __device__ __forceinline__ double at(int j, int i) const {
    return f[(j - J0 + 1) * nrp + smem_col(i)];
  }
  __device__ __forceinline__ void put(int j, int i, double v) const {
    f[(j - J0 + 1) * nrp + smem_col(i)] = v;
  }
};

// Row buffers of one FP64 tile of nl lines (padded rows of nrp doubles): the
// four rows of every line's system, the heat capacities, and four values per
// line and interface node.
struct Fp64Tile {
  double *SA, *SB, *SC, *SD;  // a then a', b then That, c then c', d then d'
  double *SM, *sI;            // V2 rho c / tau (energy); lambda_w(T), lambda_e(T), kw, ke
};

__device__ __forceinline__ Fp64Tile fp64_tile_at(double* base, int nl, int nrp) {
  Fp64Tile B;
  B.SA = base;
  B.SB = B.SA + (size_t)nl * nrp;
  B.SC = B.SB + (size_t)nl * nrp;
  B.SD = B.SC + (size_t)nl * nrp;
  B.SM = B.SD + (size_t)nl * nrp;
  B.sI = B.SM + (size_t)nl * nrp;
  return B;
}

// Phases 0a-0b of a tile, run by the warps of g: nodal conductivities of the
// interface rows, then properties and rows with the lanes over columns into
// the tile's row buffers.  The axial fluxes south of the first line come from
// cin if carry; those north of the last line go to cout.  STP: the tile holds
// a line of a stepped outline that is narrow or borders a narrow one (other
// tiles skip the checks).
template <bool ENERGY, bool STP, class F>
__device__ __forceinline__ void fp64_produce(const StepArgs& a, const TileTask tk, const Fp64Tile& B,
                                             const double* __restrict__ cin, double* __restrict__ cout,
                                             bool carry, const WarpGroup& grp, EAcc& acc,
                                             const F& fld) {
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j0 = tk.j0, nl = tk.nl;
  const int nrp = smem_row_stride(nr);
  const int frule = I.face_rule;
  const int n_if = I.n_if;
  const int warp = grp.warp(), lane = threadIdx.x & 31, nwarps = grp.nwarps;
  double* SA = B.SA;
  double* SB = B.SB;
  double* SC = B.SC;
  double* SD = B.SD;
  double* SM = B.SM;
  double* sI = B.sI;
  const double s = a.s_tab[a.step * a.n_inst + tk.inst];

  // ---- 0a. nodal conductivities of the interface rows, Eq. (cc_first_3)
  if (I.interface_rule == 0 && n_if > 0) {  // block-uniform
    for (int it = grp.tid(); it < nl * n_if; it += grp.size()) {
      const int q = it / n_if;
      const int i = I.if_i[it - q * n_if];
      const RowGeo& g = I.rg[i];
      if (g.cls == RC_IFACE) {
        const double T = fld.at(j0 + q, i);
        sI[4 * it] = lam_eval(I.mat[g.segw], T);
        sI[4 * it + 1] = lam_eval(I.mat[g.seg], T);
      }
    }
  }
  grp.sync();  // the interface values, and the previous tile's carried fluxes

  // ---- 0b. properties and rows, lanes over columns.  Block b of a warp
  // covers columns 31b .. 31b+31; lane 0 (column 31b) only supplies the face
  // (31b, 31b+1) and the row is assembled by the previous block (for b = 0,
  // lane 0 owns the axis row).  The nb x nl (block, line) items are split
  // into equal contiguous ranges, one per warp, in block-major order; a warp
  // marches down the lines of a block carrying the south face flux.
  {
    const int nb = (N + 30) / 31;
    const int n_items = nb * nl;
    const int end = (int)((long long)(warp + 1) * n_items / nwarps);
    for (int idx = (int)((long long)warp * n_items / nwarps); idx < end;) {
      const int b = idx / nl, q0 = idx - b * nl;
      const int q1 = min(nl, q0 + (end - idx));
      idx += q1 - q0;
      const int i = 31 * b + lane;
      const int ic = i <= N ? i : N;
      const bool own = (i <= N) && (lane > 0 || b == 0);
      const RowGeo g = I.rg[ic];
      const DevMaterial& Mt = I.mat[g.seg];
      const int ie = ic < N ? ic + 1 : ic;
      const bool edge = (g.cls == RC_IFACE || g.cls == RC_OUTER);
      double gwV = 0.0, gwC = 0.0, geV = 0.0, geA = 0.0;  // regular neighbours of an edge node
      if (ENERGY && edge) {
        const RowGeo& gw = I.rg[ic - 1];
        const RowGeo& ge = I.rg[ie];
        gwV = gw.V2; gwC = gw.gC; geV = ge.V2; geA = ge.gA;
      }
      // T(i, j-1), T(i, j), T(i, j+1) and T(i+1, j) of line j = j0 + q; the
      // values of the next line are loaded one iteration ahead
      double Tc = fld.at(j0 + q0, ic);
      double Tn = fld.at(j0 + q0 + 1, ic);
      double Te = fld.at(j0 + q0, ie);
      double fs;
      if (carry && q0 == 0) {
        fs = cin[smem_col(ic)];
      } else {
        const double Ts = fld.at(j0 + q0 - 1, ic);
        const double ls = lam_face(Mt, frule, Ts, Tc);
        fs = ls * (Tc - Ts);
        if (a.adi_lamz && own && j0 + q0 == 1) a.adi_lamz[I.t_off + ic] = ls;  // face (0, 1)
      }
      for (int q = q0; q < q1; ++q) {
        const int j = j0 + q;
        double Tn_next = 0.0, Te_next = 0.0;
        if (q + 1 < q1) {
          Tn_next = fld.at(j + 2, ic);
          Te_next = fld.at(j + 1, ie);
        }
        const double ln = lam_face(Mt, frule, Tc, Tn);  // face (j, j+1)
        // no heat through a face to a node outside a stepped outline
        const double fn = (STP && j + 1 >= I.j_narrow && ic > I.i_step) ? 0.0 : ln * (Tn - Tc);
        const int cls = STP ? line_class(I, g.cls, ic, j) : g.cls;
        const double le = (ic < N) ? lam_face(Mt, frule, Tc, Te) : 0.0;  // face (i, i+1)
        const double lw = __shfl_up_sync(kFull, le, 1);                  // face (i-1, i)
        const double rct = rct_eval(Mt, Tc);                             // rho c / tau
        const ZGeo& zg = I.zg[j];
        double ra, rb, rc, rd, m = 0.0;
        if (cls == RC_REGULAR) {
          double X = 0.0;  // Eq. (source)
          if (g.seg == I.src_layer && s != 0.0) {
            X = I.q0 * s;
            if (I.g_model == 1) X *= I.g_ref / sqrt(Tc);
          }
          // Eq. (ABC) with Eq. (Lambda_j), explicit in T, from the face fluxes
          const double A = -g.gA * lw, C = -g.gC * le;
          ra = A;
          rc = C;
          rb = rct - A - C;
          if (a.adi_lj) {  // the axial half step of the ADI variant needs Lambda_j alone
            const double Lj = fma(zg.gzn, fn, -zg.gzs * fs);
            rd = fma(rct, Tc, Lj + X);
            if (own) {
              const long long o = I.t_off + (long long)j * nr + ic;
              a.adi_rct[o] = rct;
              a.adi_lj[o] = Lj;
              a.adi_lamz[o] = ln;
            }
          } else {
            rd = fma(rct, Tc, fma(zg.gzn, fn, fma(-zg.gzs, fs, X)));
          }
          if (ENERGY && own) {
            m = g.V2 * rct;  // V rho c / (etabar tau)
            if (X != 0.0) acc.e[1] = fma(zg.etabar * I.tau * g.V2, X, acc.e[1]);
            if (j == 1) {
              const double f = -I.tau * g.V2 * fs / zg.eta_s;
              if (I.bc_z0 == CC_DIRICHLET) acc.e[2] += f; else acc.e[4] += f;
            }
            if (j == M - 1) {
              const double f = I.tau * g.V2 * fn / zg.eta_n;
              if (I.bc_zmax == CC_DIRICHLET) acc.e[2] += f; else acc.e[4] += f;
            }
          }
        } else if (cls == RC_IFACE) {
          // Eq. (cc_first_1)/(cc_first_3) as the row (a, b, c | 0)
          double lmv, lpv;
          if (I.interface_rule == 0) {
            lmv = sI[4 * (q * n_if + g.ifo)];
            lpv = sI[4 * (q * n_if + g.ifo) + 1];
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
        } else if (!STP || cls == RC_OUTER) {  // r = r_max, or the outer node of a narrow line
          if (I.bc_rmax == CC_DIRICHLET) { ra = 0.0; rb = 1.0; rc = 0.0; rd = I.t_d; }
          else { ra = -1.0; rb = 1.0; rc = 0.0; rd = 0.0; }
        } else {  // outside the domain: a decoupled row, the old value is stored
          ra = 0.0; rb = 1.0; rc = 0.0; rd = 0.0;
        }
        if (ENERGY && own && edge) {
          // heat-flow coefficients to the regular neighbours (faces at T^n)
          const bool in = !STP || cls != RC_OUTSIDE;
          double* K = sI + 4 * (q * n_if + g.ifo);
          K[2] = in ? I.tau * gwV * zg.etabar * gwC * lw : 0.0;
          K[3] = in ? I.tau * geV * zg.etabar * geA * le : 0.0;
        }
        if (own && q == nl - 1) cout[smem_col(ic)] = fn;
        if (own) {
          const size_t o = (size_t)q * nrp + smem_col(ic);
          SA[o] = ra;
          SB[o] = rb;
          SC[o] = rc;
          SD[o] = rd;
          if (ENERGY) SM[o] = m;
        }
        Tc = Tn;
        Tn = Tn_next;
        Te = Te_next;
        fs = fn;
      }
    }
  }
}

// Phase 4 of a tile, run by the threads of g after the line solves: stores,
// axial boundary rows, surface trace and energy terms, with the threads over
// the nodes of the tile.
template <bool ENERGY, bool TRACE, bool STP, class F>
__device__ __forceinline__ void fp64_finish(const StepArgs& a, const TileTask tk, const Fp64Tile& B,
                                            const WarpGroup& grp, EAcc& acc, const F& fld) {
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j0 = tk.j0, nl = tk.nl;
  const int nrp = smem_row_stride(nr);
  const int n_if = I.n_if;
  const double* SB = B.SB;
  const double* SM = B.SM;
  const double* sI = B.sI;
  double eE = 0.0, eD = 0.0, eN = 0.0, eI = 0.0, tr = 0.0;
  // ---- 4. stores, boundary rows, trace and energy, lanes over columns
  {
    bool bad = false;
    // threads over the nl x nr nodes of the tile, line by line (all threads
    // stay busy when nr is below the block size)
    int q = grp.tid() / nr, i = grp.tid() - q * nr, qe = -1;
    double eEq = 0.0;
    for (; q < nl;) {
      const int j = j0 + q;
      if (ENERGY && q != qe) {  // per-line factor etabar tau of the capacities
        if (qe >= 0) eE = fma(I.zg[j0 + qe].etabar * I.tau, eEq, eE);
        eEq = 0.0;
        qe = q;
      }
      const int c = smem_col(i);
      const double x = SB[(size_t)q * nrp + c];
      bad |= not_finite(x);
      const bool outside = STP && j >= I.j_narrow && i > I.i_step;
      const double told = (ENERGY || outside) ? fld.at(j, i) : 0.0;  // before the store
      fld.put(j, i, outside ? told : x);  // nodes outside a stepped outline keep their values
      if (j == 1) fld.put(0, i, (I.bc_z0 == CC_DIRICHLET) ? I.t_d : x);
      if (j == M - 1)
        fld.put(M, i, (STP && M >= I.j_narrow && i > I.i_step) ? fld.at(M, i)
                      : (I.bc_zmax == CC_DIRICHLET) ? I.t_d : x);
      if (ENERGY) eEq = fma(SM[(size_t)q * nrp + c], x - told, eEq);
      if (TRACE && i == N) {  // That(r_max, z_j)
        tr = fma(I.zg[j].wnorm, x, tr);
        if (j == 1) {
          const double x0 = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : x;
          tr = fma(I.zg[0].wnorm, x0, tr);
          a.trace[((long long)tk.inst * a.n_steps + a.step) * 2] = x0;
        }
        if (j == M - 1) {
          const double xM = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : x;
          tr = fma(I.zg[M].wnorm, xM, tr);
        }
      }
      i += grp.size();
      while (i >= nr) {
        i -= nr;
        ++q;
      }
    }
    if (ENERGY && qe >= 0) eE = fma(I.zg[j0 + qe].etabar * I.tau, eEq, eE);
    if (bad) atomicOr(a.err, 1u);
    if (ENERGY) {
      // heat through the radial edges between each interface (or r_max) node
      // and its regular neighbours, at That
      for (int it = grp.tid(); it < nl * n_if; it += grp.size()) {
        const int q = it / n_if;
        const int i = I.if_i[it - q * n_if];
        const double* Bq = SB + (size_t)q * nrp;
        const double* K = sI + 4 * it;
        const double x = Bq[smem_col(i)];
        const double fw = K[2] * (x - Bq[smem_col(i - 1)]);  // into node i-1
        const int cls = STP ? line_class(I, I.rg[i].cls, i, j0 + q) : I.rg[i].cls;
        if (cls == RC_OUTER) {
          if (I.bc_rmax == CC_DIRICHLET) eD += fw; else eN += fw;
        } else if (!STP || cls == RC_IFACE) {
          eI += fw + K[3] * (x - Bq[smem_col(i + 1)]);  // and into node i+1
        }
      }
      acc.e[0] += eE;
      acc.e[2] += eD;
      acc.e[3] += eI;
      acc.e[4] += eN;
    }
    if (TRACE) acc.tr += tr;
  }
}

// One tile with the whole block: rows, solves, stores, separated by block
// barriers.  sm starts with two rows of axial face fluxes (row par ^ 1 holds
// those south of the tile's first line if carry; those north of its last
// line go to row par), then the tile's row buffers.
template <bool ENERGY, bool TRACE, bool STP, class F>
__device__ __forceinline__ void step_fp64_tile(const StepArgs& a, const TileTask tk,
                                               double* __restrict__ sm, EAcc& acc, bool carry,
                                               int par, const F& fld) {
  if (tk.inst != acc.inst) {  // block-uniform
    eacc_flush<ENERGY, TRACE>(a, acc);
    acc.inst = tk.inst;
  }
  const DevInst& I = a.insts[tk.inst];
  const int nrp = smem_row_stride(I.nr);
  const Fp64Tile B = fp64_tile_at(sm + 2 * (size_t)nrp, tk.nl, nrp);
  const WarpGroup all = whole_block();
  fp64_produce<ENERGY, STP>(a, tk, B, sm + (size_t)(par ^ 1) * nrp, sm + (size_t)par * nrp, carry,
                            all, acc, fld);
  __syncthreads();
  // ---- 1.-3. line solves, lanes over the rows of a line
  solve_tile_lines<true>(B.SA, B.SB, B.SC, B.SD, tk.nl, I.nr, I.G);
  __syncthreads();
  fp64_finish<ENERGY, TRACE, STP>(a, tk, B, all, acc, fld);
  __syncthreads();  // the next tile reuses the shared memory
}

// The tiles of this block: its range, or a stride over all tiles.
template <bool ENERGY, bool TRACE, bool CACHED>
__device__ __forceinline__ void fp64_tiles(const StepArgs& a, double* __restrict__ sm, EAcc& acc) {
  int t0 = blockIdx.x, t1 = a.n_tiles, dt = gridDim.x;
  if (a.cta_start) {
    t0 = a.cta_start[blockIdx.x];
    t1 = a.cta_start[blockIdx.x + 1];
    dt = 1;
  }
  int prev_inst = -1, prev_end = -1, par = 0;
  for (int t = t0; t < t1; t += dt) {
    const TileTask tk = a.tiles[t];
    const bool carry = (tk.inst == prev_inst && tk.j0 == prev_end);
    const DevInst& I = a.insts[tk.inst];
    const GlobalField<CACHED> fld(a, I);
    if (tk.j0 + tk.nl >= I.j_narrow)
      step_fp64_tile<ENERGY, TRACE, true>(a, tk, sm, acc, carry, par, fld);
    else
      step_fp64_tile<ENERGY, TRACE, false>(a, tk, sm, acc, carry, par, fld);
    prev_inst = tk.inst;
    prev_end = tk.j0 + tk.nl;
    par ^= 1;
  }
}

}  // namespace ccell
