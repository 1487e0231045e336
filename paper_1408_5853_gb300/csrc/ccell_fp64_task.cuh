// FP64 time step of one CTA tile, shared by the per-step and the persistent
// kernels.
//
// A tile is nl consecutive axial lines j0 .. j0+nl-1 of one instance; each
// warp of the CTA owns 32/G of them and each line is split over G lanes (lane
// l holds rows [l nr/G, (l+1) nr/G)).  Per time step:
//   0. the CTA stages the field rows j0-1 .. j0+nl (contiguous in global
//      memory) into shared memory, padded so lanes 16 rows apart do not share
//      a bank, and evaluates, with all threads over the columns, every
//      conductivity and heat capacity the tile needs: the axial faces
//      lambda_{i,j+1/2} (a face is shared by the two lines it separates and
//      is evaluated once), the radial faces lambda_{i+1/2,j} and
//      rho c(T_ij) / tau (Eqs. (Lambda_i), (Lambda_j));
//   1. every lane assembles its rows of the tridiagonal system of Eq. (ABC)
//      (regular nodes), the interface rows of Eq. (cc_first_1) and the
//      closures of Eq. (first_oder_bc) from those values and the source of
//      Eq. (source), and eliminates the segment's interior rows downwards
//      (the forward sweep of Eq. (front_sweep) restricted to the segment,
//      keeping the coupling to the previous segment's last row);
//   2. the G separator rows are solved by cyclic reduction with shuffles;
//   3. back substitution (Eq. (back_sweep)) inside each segment;
//   4. stores, axial boundary rows, surface trace and energy terms.
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

// rho c(T) / tau from the folded material constants
__device__ __forceinline__ double rct_eval(const DevMaterial& M, double T) {
  if (M.cap_model == 1) {
    const double T3 = T * T * T;
    return M.rct_k * T3 * frcp(fma(M.inv_theta3, T3, 1.0));
  }
  if (M.cap_model == 0) return M.rct_k;
  const double* a = M.cap_poly;
  return M.rho_tau * fma(fma(fma(a[3], T, a[2]), T, a[1]), T, a[0]);
}

// Copy the field rows j0-1 .. j0+nl of a tile into a staging buffer with
// asynchronous 8-byte copies (one commit group).  Only for per-step launches:
// the copies read through L1, which is coherent with earlier launches but not
// with other blocks of the same launch.
__device__ __forceinline__ void stage_rows_async(const StepArgs& a, const TileTask tk,
                                                 double* sT) {
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, nrp = smem_row_stride(nr);
  const double* src = static_cast<const double*>(a.Tin) + I.t_off + (long long)(tk.j0 - 1) * nr;
  for (int r = 0; r < tk.nl + 2; ++r)
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(sT + r * nrp + smem_col(i));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                   :: "r"(dst), "l"(src + (long long)r * nr + i) : "memory");
    }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// One tile.  PREFETCH: the tile's rows were staged by stage_rows_async into
// sT, and the rows of next (if next.nl > 0) are staged into sTn meanwhile;
// otherwise the rows are loaded here (L2 loads, coherent within a launch).
template <bool ENERGY, bool TRACE, bool PREFETCH>
__device__ __forceinline__ void step_fp64_tile(const StepArgs& a, const TileTask tk,
                                               double* __restrict__ sT, double* __restrict__ sTn,
                                               const TileTask next, double* __restrict__ sW,
                                               EAcc& acc) {
  if (tk.inst != acc.inst) {  // block-uniform
    eacc_flush<ENERGY, TRACE>(a, acc);
    acc.inst = tk.inst;
  }
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int G = I.G;
  const int lg = __ffs(G) - 1;
  const int lpw = 32 >> lg;
  const int j0 = tk.j0, nl = tk.nl;
  const int nrp = smem_row_stride(nr);
  const int frule = I.face_rule;
  const int n_if = I.n_if;
  double* sF = sW;                      // axial face fluxes lambda (T_{j+1} - T_j), r = 0..nl
  double* sR = sF + (size_t)(nl + 1) * nrp;  // radial faces (i, i+1) of lines j0 .. j0+nl-1
  double* sX = sR + (size_t)nl * nrp;        // rho c / tau, then V2 rho c, then That
  double* sI = sX + (size_t)nl * nrp;        // interface rows: lambda_w(T), lambda_e(T)
  double* Tout = static_cast<double*>(a.Tout) + I.t_off;

  // ---- 0. stage the rows (sT rows 0 .. nl+1 = lines j0-1 .. j0+nl)
  if constexpr (PREFETCH) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (next.nl > 0) stage_rows_async(a, next, sTn);
  } else {
    const double* src = static_cast<const double*>(a.Tin) + I.t_off + (long long)(j0 - 1) * nr;
    for (int r = 0; r < nl + 2; ++r)
      for (int i = threadIdx.x; i < nr; i += blockDim.x)
        sT[r * nrp + smem_col(i)] = __ldcg(src + (long long)r * nr + i);
    __syncthreads();
  }
  // Then every conductivity and heat capacity of the tile, with all threads
  // over the columns (independent items): the axial faces (each shared by two
  // lines, evaluated once) as fluxes, the radial faces (segment [r_i, r_{i+1}]
  // lies in layer rg[i].seg), rho c(T)/tau at the nodes, and the nodal
  // conductivities of the interface rows.
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    const DevMaterial& Mt = I.mat[I.rg[i].seg];
    const int c = smem_col(i), c1 = smem_col(i < N ? i + 1 : i);
    double Tlo = sT[c];
#pragma unroll 2
    for (int r = 0; r <= nl; ++r) {
      const double Thi = sT[(r + 1) * nrp + c];
      sF[r * nrp + c] = lam_face(Mt, frule, Tlo, Thi) * (Thi - Tlo);
      if (r < nl) {
        sR[r * nrp + c] = (i < N) ? lam_face(Mt, frule, Thi, sT[(r + 1) * nrp + c1]) : 0.0;
        sX[r * nrp + c] = rct_eval(Mt, Thi);
      }
      Tlo = Thi;
    }
  }
  if (I.interface_rule == 0) {
    for (int it = threadIdx.x; it < nl * n_if; it += blockDim.x) {
      const int q = it / n_if;
      const RowGeo& g = I.rg[I.if_i[it - q * n_if]];
      if (g.cls == RC_IFACE) {
        const double T = sT[(q + 1) * nrp + smem_col(I.if_i[it - q * n_if])];
        sI[2 * it] = lam_eval(I.mat[g.segw], T);
        sI[2 * it + 1] = lam_eval(I.mat[g.seg], T);
      }
    }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> lg, l = lane & (G - 1);
  const int q_req = warp * lpw + grp;
  const bool active = q_req < nl;
  const int q = active ? q_req : nl - 1;  // idle lane groups recompute a valid line
  const int j = j0 + q;
  const int i_lo = (l * nr) >> lg;
  const int i_hi = ((l + 1) * nr) >> lg;
  const int cnt = i_hi - i_lo;  // 2 .. kRowsPerLane
  const double* Tj = sT + (q + 1) * nrp;
  const double* Fs = sF + q * nrp;   // face (j-1, j)
  const double* Fn = Fs + nrp;       // face (j, j+1)
  const ZGeo zg = I.zg[j];
  const double s = a.s_tab[a.step * a.n_inst + tk.inst];
  const double etau = zg.etabar * I.tau;  // V tau = V2 etabar tau

  double cp[kRowsPerLane], ap[kRowsPerLane], dp[kRowsPerLane];
  const double* Rq = sR + q * nrp;  // radial faces of line j
  double* Xq = sX + q * nrp;        // rho c / tau; V2 rho c from phase 1; That from phase 4
  double pc = 0.0, pa = 0.0, pd = 0.0;    // c', a', d' of the previous interior row
  double Dacc = 0.0, Aacc = 0.0, P = 1.0; // first interior row = Dacc + P x_next - Aacc L
  double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;  // separator row
  double eQ = 0.0, eD = 0.0, eN = 0.0;    // source: sum V2 X (times etabar tau at the end)
  double lw = (i_lo > 0) ? Rq[smem_col(i_lo - 1)] : 0.0;  // face (i-1, i)

  // ---- 1. assemble rows and eliminate the segment downwards
#pragma unroll
  for (int k = 0; k < kRowsPerLane; ++k) {
    if (k < cnt) {
      const int i = i_lo + k;
      const int c = smem_col(i);
      const RowGeo g = I.rg[i];
      const double T0 = Tj[c];
      const double le = Rq[c];  // face (i, i+1)
      double ra, rb, rc, rd, m = 0.0;
      if (g.cls == RC_REGULAR) {
        const double fs = Fs[c], fn = Fn[c];  // lambda (T - T_S), lambda (T_N - T)
        const double rct = Xq[c];  // rho c / tau
        // Eq. (Lambda_j), explicit in T, from the face fluxes
        const double Lj = fma(zg.gzn, fn, -zg.gzs * fs);
        double X = 0.0;  // Eq. (source)
        if (g.seg == I.src_layer && s != 0.0) {
          X = I.q0 * s;
          if (I.g_model == 1) X *= I.g_ref / sqrt(T0);
        }
        // Eq. (ABC)
        const double A = -g.gA * lw, C = -g.gC * le;
        ra = A;
        rc = C;
        rb = rct - A - C;
        rd = fma(rct, T0, Lj + X);
        if (ENERGY) {
          m = g.V2 * rct;  // V rho c / (etabar tau)
          if (X != 0.0) eQ = fma(g.V2, X, eQ);
          if (j == 1) {
            const double f = -I.tau * g.V2 * fs / zg.eta_s;
            if (I.bc_z0 == CC_DIRICHLET) eD += f; else eN += f;
          }
          if (j == M - 1) {
            const double f = I.tau * g.V2 * fn / zg.eta_n;
            if (I.bc_zmax == CC_DIRICHLET) eD += f; else eN += f;
          }
        }
      } else if (g.cls == RC_IFACE) {
        // Eq. (cc_first_1)/(cc_first_3) as the row (a, b, c | 0)
        double lmv, lpv;
        if (I.interface_rule == 0) {
          lmv = sI[2 * (q * n_if + g.ifo)];
          lpv = sI[2 * (q * n_if + g.ifo) + 1];
        } else {
          lmv = g.rw * lw;
          lpv = g.re * le;
        }
        ra = -lmv * g.he;
        rc = -lpv * g.hw;
        rb = fma(lmv, g.he, lpv * g.hw);
        rd = 0.0;
      } else if (g.cls == RC_AXIS) {  // That_0 = That_1
        ra = 0.0; rb = 1.0; rc = -1.0; rd = 0.0;
      } else {  // r = r_max
        if (I.bc_rmax == CC_DIRICHLET) { ra = 0.0; rb = 1.0; rc = 0.0; rd = I.t_d; }
        else { ra = -1.0; rb = 1.0; rc = 0.0; rd = 0.0; }
      }
      lw = le;
      if (ENERGY && active) Xq[c] = m;
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
    }
  }

  // ---- 2. separator system (one row per lane), cyclic reduction
  const double xs = solve_separators(ae, be, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);

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
    for (int k = 0; k < kRowsPerLane; ++k)  // dp[k] = x_k for every row of the segment
      dp[k] = (k == cnt - 1) ? xs : dp[k];  // (a select: an indexed store would demote dp to local memory)
  }

  // ---- 4. stores, boundary rows, energy and trace epilogue
  double eE = 0.0;
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
          const int c = smem_col(i);
          eE = fma(Xq[c], x - Tj[c], eE);  // V2 rho c (That - T)
          Xq[c] = x;
        }
      }
    }
  }
  if (bad) atomicOr(a.err, 1u);

  if (TRACE && active && l == G - 1) {  // this lane owns That(r_max, z_j)
    double tr = zg.wnorm * xs;
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
    acc.tr += tr;
  }
  if (ENERGY && active) {
    acc.e[0] += etau * eE;
    acc.e[1] += etau * eQ;
    acc.e[2] += eD;
    acc.e[4] += eN;
  }
  if (ENERGY && I.n_if > 0) {
    // heat through the radial edges between each interface (or r_max) node
    // and its regular neighbours, at That, with the faces' conductivities at
    // T^n (Eq. (Lambda_i)); one thread per (line, interface) of the tile
    __syncthreads();  // sX complete
    for (int it = threadIdx.x; it < nl * I.n_if; it += blockDim.x) {
      const int qq = it / I.n_if;
      const int i = I.if_i[it - qq * I.n_if];
      const double* Rr = sR + qq * nrp;
      const double* Xr = sX + qq * nrp;
      const double x = Xr[smem_col(i)];
      const double etab = I.zg[j0 + qq].etabar;
      const RowGeo gw = I.rg[i - 1];
      const double kw = I.tau * gw.V2 * etab * gw.gC * Rr[smem_col(i - 1)];
      const double fw = kw * (x - Xr[smem_col(i - 1)]);  // into node i-1
      if (I.rg[i].cls == RC_OUTER) {
        if (I.bc_rmax == CC_DIRICHLET) acc.e[2] += fw; else acc.e[4] += fw;
      } else {
        const RowGeo ge = I.rg[i + 1];
        const double ke = I.tau * ge.V2 * etab * ge.gA * Rr[smem_col(i)];
        acc.e[3] += fw + ke * (x - Xr[smem_col(i + 1)]);  // and into node i+1
      }
    }
  }
  __syncthreads();  // the next tile reuses the shared memory
}

// Resident blocks per SM x SMs for a kernel, block size and shared memory.
template <class K>
static int resident_blocks(K kernel, int threads, int smem = 0) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return sms * (per_sm > 0 ? per_sm : 1);
}

static inline int shape_index(int threads) { return threads <= 64 ? 0 : (threads <= 128 ? 1 : 2); }

}  // namespace ccell
