// Reverse-time discrete adjoint of the FP64 time step (Section 3 scheme).
//
// One step maps T^n to That = T^{n+1}: on every line j = 1..M-1 the rows
// a_i That_{i-1} + b_i That_i + c_i That_{i+1} = f_i (Eq. (ABC), the interface
// rows of Eq. (cc_first_1), the closures of Eq. (first_oder_bc)), then the
// axial boundary rows.  With mu = dJ/dThat, the adjoint of a line solve is
// xi = M^{-T} mu; the derivatives of J with respect to T^n and to the
// parameters theta = (q0, t_on, lam_scale[m], cap_scale[m]) are
// sum_i xi_i d r_i / d(.), r_i = f_i - (a_i y_{i-1} + b_i y_i + c_i y_{i+1})
// at fixed y = That.
//
//  adj_tile_kernel    per CTA tile of lines: rebuild (a, b, c) at T^n with
//                     the lanes over columns, then solve the transposed
//                     systems in shared memory with the segment elimination
//                     and shuffle cyclic reduction of the forward step (mu
//                     includes the loss seed of step n and the folded axial
//                     boundary rows).  The radial face conductivity of every
//                     node, its two derivatives, rho c / tau and its
//                     derivative are evaluated here once and left for the
//                     gather (five values per node, read back from L2).
//  adj_gather_kernel  per node: dJ/dT^n from xi of the node's own row and of
//                     the four neighbouring rows that read its temperature
//                     (no atomics on the field), plus the parameter terms of
//                     its own row (shuffle sums per warp, shared sums per
//                     block, one global atomic per block and parameter).  It
//                     evaluates only the axial faces and their derivatives.
#include <cuda_runtime.h>

#include "ccell_device.cuh"

namespace ccell {

// Derivatives below take their reciprocals to 2^-46 (frcp46): they enter
// dJ/dT and the parameter terms linearly, where a relative error of 2^-46 is
// far below the rounding of the reverse sweep's sums.

// d lambda / dT at a node, given lambda(T)
__device__ __forceinline__ double dlam_node(const DevMaterial& M, double T, double lamT) {
  if (M.lam_model == 1) return M.lam_b * lamT * frcp46(T);
  if (M.lam_model == 0) return 0.0;
  const double* b = M.lam_poly;
  return fma(fma(fma(4.0 * b[4], T, 3.0 * b[3]), T, 2.0 * b[2]), T, b[1]);
}

// face conductivity and its derivatives with respect to (Ta, Tb)
__device__ __forceinline__ void lam_face_d(const DevMaterial& M, int rule, double Ta, double Tb,
                                           double& l, double& da, double& db) {
  if (rule == 0) {
    if (M.lam_model == 1) {  // lambda((Ta+Tb)/2) = K (Ta+Tb)^b: d/dTa = b lambda / (Ta+Tb)
      const double y = Ta + Tb;
      l = lam_pow(M, y, true);
      da = db = M.lam_b * l * frcp46(y);
    } else {
      const double Tm = 0.5 * (Ta + Tb);
      l = lam_eval(M, Tm);
      da = db = 0.5 * dlam_node(M, Tm, l);
    }
  } else {
    const double la = lam_eval(M, Ta), lb = lam_eval(M, Tb);
    l = 0.5 * (la + lb);
    da = 0.5 * dlam_node(M, Ta, la);
    db = 0.5 * dlam_node(M, Tb, lb);
  }
}

// rho c(T) / tau as the forward step evaluates it (rct_eval), and its
// derivative in T.  Debye-saturated form r = k T^3 / (1 + T^3/theta^3):
// dr/dT = 3 k T^2 / (1 + T^3/theta^3)^2.
__device__ __forceinline__ void rct_d(const DevMaterial& M, double T, double& r, double& dr) {
  if (M.cap_model == 1) {
    const double T2 = T * T, T3 = T2 * T;
    const double rd = frcp46(fma(M.inv_theta3, T3, 1.0));
    r = M.rct_k * T3 * rd;
    dr = 3.0 * M.rct_k * T2 * rd * rd;
  } else if (M.cap_model == 0) {
    r = M.rct_k;
    dr = 0.0;
  } else {
    const double* a = M.cap_poly;
    r = M.rho_tau * fma(fma(fma(a[3], T, a[2]), T, a[1]), T, a[0]);
    dr = M.rho_tau * fma(fma(3.0 * a[3], T, 2.0 * a[2]), T, a[1]);
  }
}

// ---------------------------------------------------------------------------
// transposed line solves, one CTA tile of nl lines at a time
// ---------------------------------------------------------------------------
// Forward row (a, b, c) of node i on a line at T^n: Eq. (ABC) for regular
// nodes, Eq. (cc_first_3) for interface nodes, the closures at the axis and
// at r_max.  lw, le: face conductivities (i-1, i) and (i, i+1); rct: rho c /
// tau of a regular node.
__device__ __forceinline__ void forward_row(const DevInst& I, const RowGeo& g, double T0,
                                            double lw, double le, double rct, double& ra,
                                            double& rb, double& rc) {
  if (g.cls == RC_REGULAR) {
    ra = -g.gA * lw;
    rc = -g.gC * le;
    rb = rct - ra - rc;
  } else if (g.cls == RC_IFACE) {
    double lm, lp;
    if (I.interface_rule == 0) {
      lm = lam_eval(I.mat[g.segw], T0);
      lp = lam_eval(I.mat[g.seg], T0);
    } else {
      lm = g.rw * lw;
      lp = g.re * le;
    }
    ra = -lm * g.he;
    rc = -lp * g.hw;
    rb = fma(lm, g.he, lp * g.hw);
  } else if (g.cls == RC_AXIS) {
    ra = 0.0; rb = 1.0; rc = -1.0;
  } else {
    ra = (I.bc_rmax == CC_DIRICHLET) ? 0.0 : -1.0;
    rb = 1.0;
    rc = 0.0;
  }
}

// The transposed system M^T xi = mu of line j has rows (c_{i-1}, b_i, a_{i+1} |
// mu_i).  Rows are assembled with the lanes over columns: block b of a warp
// covers columns 30b .. 30b+31, lanes 1..30 own columns 30b+1 .. 30b+30 (and
// lane 0 the axis for b = 0); lane 0 hands c of its column to lane 1 and lane
// 31 hands a of its column to lane 30.  Each radial face conductivity is
// evaluated once per lane (the west face comes from the left lane).  The
// systems are then solved with the segment elimination and shuffle cyclic
// reduction of the forward step, and xi is stored with the threads over the
// nodes of the tile.
__global__ void __launch_bounds__(CC_ADJ_MAX_THREADS) adj_tile_kernel(const AdjArgs a) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    const TileTask tk = a.tiles[t];
    const DevInst& I = a.insts[tk.inst];
    const int nr = I.nr, N = nr - 1, M = I.nz - 1;
    const int j0 = tk.j0, nl = tk.nl;
    const int nrp = smem_row_stride(nr);
    const int frule = I.face_rule;
    double* SA = sm;
    double* SB = SA + (size_t)nl * nrp;
    double* SC = SB + (size_t)nl * nrp;
    double* SD = SC + (size_t)nl * nrp;
    const double* X = a.x + I.t_off;
    const double* Lam = a.lam + I.t_off;
    const double sd = a.seed[(long long)tk.inst * a.n_steps + a.step];
    const double w0 = I.zg[0].wnorm, wM = I.zg[M].wnorm;
    {
      const int nb = (N + 29) / 30;
      const int n_items = nb * nl;
      const int end = (int)((long long)(warp + 1) * n_items / nwarps);
      for (int idx = (int)((long long)warp * n_items / nwarps); idx < end;) {
        const int b = idx / nl, q0 = idx - b * nl;
        const int q1 = min(nl, q0 + (end - idx));
        idx += q1 - q0;
        const int i = 30 * b + lane;
        const int ic = i <= N ? i : N;
        const bool own = (i <= N) && ((lane >= 1 && lane <= 30) || (b == 0 && lane == 0));
        const RowGeo g = I.rg[ic];
        const DevMaterial& Mt = I.mat[g.seg];
        const int ie = ic < N ? ic + 1 : ic;
        const double* row = X + (long long)(j0 + q0) * nr;
        double Tc = __ldg(row + ic), Te = __ldg(row + ie);
        for (int q = q0; q < q1; ++q) {
          const int j = j0 + q;
          double Tc_next = 0.0, Te_next = 0.0;
          if (q + 1 < q1) {
            Tc_next = __ldg(row + nr + ic);
            Te_next = __ldg(row + nr + ie);
          }
          row += nr;
          double le = 0.0, lea = 0.0, leb = 0.0;  // face (i, i+1) and its derivatives
          if (ic < N) lam_face_d(Mt, frule, Tc, Te, le, lea, leb);
          const double lw = __shfl_up_sync(kFull, le, 1);  // face (i-1, i)
          double rct = 0.0, drct = 0.0;
          if (g.cls == RC_REGULAR) rct_d(Mt, Tc, rct, drct);
          double fa, fb, fc;
          forward_row(I, g, Tc, lw, le, rct, fa, fb, fc);
          const double cw = __shfl_up_sync(kFull, fc, 1);    // c_{i-1}
          const double ae = __shfl_down_sync(kFull, fa, 1);  // a_{i+1}
          if (own) {
            const long long rj = (long long)j * nr;
            // values of this node for the gather, read back from L2
            double* st = a.st + I.t_off + rj + ic;
            st[0] = le;
            st[a.st_stride] = lea;
            st[2 * a.st_stride] = leb;
            st[3 * a.st_stride] = rct;
            st[4 * a.st_stride] = drct;
            double rd = __ldg(Lam + rj + ic);
            if (ic == N) rd = fma(sd, I.zg[j].wnorm, rd);
            if (j == 1 && I.bc_z0 == CC_NEUMANN) rd += __ldg(Lam + ic) + ((ic == N) ? sd * w0 : 0.0);
            if (j == M - 1 && I.bc_zmax == CC_NEUMANN)
              rd += __ldg(Lam + (long long)M * nr + ic) + ((ic == N) ? sd * wM : 0.0);
            const size_t o = (size_t)q * nrp + smem_col(ic);
            SA[o] = (ic > 0) ? cw : 0.0;
            SB[o] = fb;
            SC[o] = (ic < N) ? ae : 0.0;
            SD[o] = rd;
          }
          Tc = Tc_next;
          Te = Te_next;
        }
      }
    }
    __syncthreads();
    solve_tile_lines<true>(SA, SB, SC, SD, nl, nr, I.G);
    __syncthreads();
    {
      double* XI = a.xi + I.t_off;
      int q = threadIdx.x / nr, i = threadIdx.x - q * nr;
      for (; q < nl;) {
        XI[(long long)(j0 + q) * nr + i] = SB[(size_t)q * nrp + smem_col(i)];
        i += blockDim.x;
        while (i >= nr) {
          i -= nr;
          ++q;
        }
      }
    }
    __syncthreads();  // the next tile reuses the shared memory
  }
}

int launch_adj_tile(const AdjArgs& a, void* stream) {
  static KernelCache cache;
  const int resident = cached_resident(cache, adj_tile_kernel, a.threads, a.smem_bytes,
                                       kMaxTileSmem);
  if (resident < 0) return -1;
  const int blocks = a.n_tiles < resident ? a.n_tiles : resident;
  adj_tile_kernel<<<blocks, a.threads, a.smem_bytes, (cudaStream_t)stream>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// per-node gather of dJ/dT^n and of the parameter terms
// ---------------------------------------------------------------------------
constexpr int kGradMax = 2 + 2 * CC_MAX_LAYERS;

// Warp task (column block cb, line block jb): lane l holds column 31 cb + l
// (lane 0 of cb > 0 only supplies its east face to lane 1) on the lines
// gl jb .. gl jb + gl - 1 (gl = a.gather_lines).  The radial faces come from
// the tile kernel (the west face from the left lane); each axial face and its
// derivatives are evaluated once per line block: the north face per line, the
// south face carried from the previous line (one extra evaluation at the top
// of the block).
__global__ void __launch_bounds__(256) adj_gather_kernel(const AdjArgs a) {
  __shared__ double sg[kGradMax];
  const int inst = blockIdx.y;
  const DevInst& I = a.insts[inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int L = a.n_layers[inst];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kGradMax) sg[threadIdx.x] = 0.0;
  __syncthreads();
  // this column's parameter terms over its lines: q0, t_on, lam_scale[mL],
  // cap_scale[mC] (a second lam_scale term at mL2 for interface columns);
  // summed over the warp per parameter below
  double pq = 0.0, pt = 0.0, pl = 0.0, pl2 = 0.0, pc = 0.0;
  int mL = -1, mL2 = -1, mC = -1;
  const int gl = a.gather_lines;
  const int ncb = (N + 30) / 31, njb = (M + gl) / gl;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w < ncb * njb) {  // warp-uniform
    const int cb = w % ncb, jb = w / ncb;
    const int i = 31 * cb + lane;
    const int ic = i <= N ? i : N;
    const bool own = (i <= N) && (lane > 0 || cb == 0);
    const double* X = a.x + I.t_off;
    const double* Y = a.y + I.t_off;
    const double* XI = a.xi + I.t_off;
    const RowGeo g = I.rg[ic];
    const int frule = I.face_rule;
    const bool regular = (g.cls == RC_REGULAR);
    const DevMaterial& Mt = I.mat[g.seg];
    const int j_lo = gl * jb;
    const int j_hi = min(j_lo + gl - 1, M);
    double Ts = (j_lo >= 1) ? X[(long long)(j_lo - 1) * nr + ic] : 0.0;
    double T = X[(long long)j_lo * nr + ic];
    double lS = 0.0, lSa = 0.0, lSb = 0.0;  // face (j-1, j) of a regular column
    if (regular && j_lo >= 1) lam_face_d(Mt, frule, Ts, T, lS, lSa, lSb);
    for (int j = j_lo; j <= j_hi; ++j) {  // same lines for the whole warp
      const long long rj = (long long)j * nr;
      const double Tn = (j <= M - 1) ? X[rj + nr + ic] : 0.0;
      const bool line = (j >= 1 && j <= M - 1);  // own row belongs to a solved line (warp-uniform)
      // radial faces (i, i+1) of material seg[i] as the tile kernel left them
      // (zero at i = N), (i-1, i) from the left lane; needed on solved lines only
      double lE = 0.0, lEa = 0.0, lEb = 0.0;
      if (line) {
        const double* st = a.st + I.t_off + rj + ic;
        lE = st[0];
        lEa = st[a.st_stride];
        lEb = st[2 * a.st_stride];
      }
      double lW = __shfl_up_sync(kFull, lE, 1);
      double lWb = __shfl_up_sync(kFull, lEb, 1);
      if (i == 0) lW = lWb = 0.0;
      // axial face (j, j+1) of a regular column
      double lN = 0.0, lNa = 0.0, lNb = 0.0;
      if (regular && j <= M - 1) lam_face_d(Mt, frule, T, Tn, lN, lNa, lNb);
      if (own) {
        const double yi = Y[rj + ic];
        double acc = 0.0;
        // That differences to the radial neighbours on this line (zero off the line and at the
        // ends); the neighbours' rows read them with the opposite sign
        double gw = 0.0, ge = 0.0;
        if (line) {
          if (ic >= 1) gw = Y[rj + ic - 1] - yi;
          if (ic <= N - 1) ge = Y[rj + ic + 1] - yi;
        }
        // rows i-1 and i+1 of the same line
        if (line) {
          if (ic >= 1) {
            const RowGeo& gm = I.rg[ic - 1];
            const double xw = XI[rj + ic - 1];
            if (gm.cls == RC_REGULAR) acc = fma(xw * gm.gC * lWb, -gw, acc);
            else if (gm.cls == RC_IFACE && I.interface_rule == 1)
              acc = fma(xw * gm.re * lWb * gm.hw, -gw, acc);
          }
          if (ic <= N - 1) {
            const RowGeo& gp = I.rg[ic + 1];
            const double xe = XI[rj + ic + 1];
            if (gp.cls == RC_REGULAR) acc = fma(xe * gp.gA * lEa, -ge, acc);
            else if (gp.cls == RC_IFACE && I.interface_rule == 1)
              acc = fma(xe * gp.rw * lEa * gp.he, -ge, acc);
          }
        }
        if (regular) {
          const int m = g.seg;
          // rows (i, j+1) and (i, j-1) read T through their south / north faces
          if (j + 1 >= 1 && j + 1 <= M - 1)
            acc = fma(XI[rj + nr + ic] * I.zg[j + 1].gzs, fma(-lNa, Tn - T, lN), acc);
          if (j - 1 >= 1 && j - 1 <= M - 1)
            acc = fma(XI[rj - nr + ic] * I.zg[j - 1].gzn, fma(lSb, T - Ts, lS), acc);
          if (line) {
            const double xi = XI[rj + ic];
            const ZGeo& zg = I.zg[j];
            const double rct = a.st[3 * a.st_stride + I.t_off + rj + ic];
            const double drct = a.st[4 * a.st_stride + I.t_off + rj + ic];
            const double dN = Tn - T, dS = T - Ts;
            double d0 = fma(drct, T - yi, rct);
            d0 = fma(fma(lNa, dN, -lN), zg.gzn, d0);
            d0 = fma(-fma(lSb, dS, lS), zg.gzs, d0);
            d0 = fma(g.gA * lWb, gw, d0);
            d0 = fma(g.gC * lEa, ge, d0);
            const bool heat = (m == I.src_layer);
            const long long sidx = a.step * a.n_inst + inst;
            double gT = 1.0, dgT = 0.0;
            if (heat && I.g_model == 1) {
              gT = I.g_ref * rsqrt(T);
              dgT = -0.5 * gT * frcp46(T);
            }
            if (heat) d0 = fma(I.q0 * a.s_tab[sidx], dgT, d0);
            acc = fma(xi, d0, acc);
            // parameters of this row
            const double lam_part =
                fma(g.gC * lE, ge, fma(g.gA * lW, gw, fma(lN * zg.gzn, dN, -lS * zg.gzs * dS)));
            pl = fma(xi * lam_part, Mt.inv_lam_scale, pl);
            mL = m;
            pc = fma(xi * rct * (T - yi), Mt.inv_cap_scale, pc);
            mC = m;
            if (heat) {
              pq = fma(xi * a.s_tab[sidx], gT, pq);
              pt = fma(xi * I.q0 * a.ds_tab[sidx], gT, pt);
            }
          }
        } else if (g.cls == RC_IFACE && line) {
          const double xi = XI[rj + ic];
          const int mi = g.segw, mo = g.seg;
          double lm, lp, dlm, dlp;
          if (I.interface_rule == 0) {
            lm = lam_eval(I.mat[mi], T);
            lp = lam_eval(I.mat[mo], T);
            dlm = dlam_node(I.mat[mi], T, lm);
            dlp = dlam_node(I.mat[mo], T, lp);
          } else {
            lm = g.rw * lW;
            lp = g.re * lE;
            dlm = g.rw * lWb;
            dlp = g.re * lEa;
          }
          acc = fma(xi, fma(dlm * g.he, gw, dlp * g.hw * ge), acc);
          pl = fma(xi * lm * g.he * gw, I.mat[mi].inv_lam_scale, pl);
          mL = mi;
          pl2 = fma(xi * lp * g.hw * ge, I.mat[mo].inv_lam_scale, pl2);
          mL2 = mo;
        }
        a.lam_out[I.t_off + rj + ic] = acc;
      }
      Ts = T;
      T = Tn;
      lS = lN;
      lSa = lNa;
      lSb = lNb;
    }
  }
  // warp sums per parameter (the block is warp-uniform here)
  for (int p = 0; p < 2 + 2 * L; ++p) {
    double v;
    if (p == 0) v = pq;
    else if (p == 1) v = pt;
    else if (p < 2 + L) v = (mL == p - 2 ? pl : 0.0) + (mL2 == p - 2 ? pl2 : 0.0);
    else v = (mC == p - 2 - L) ? pc : 0.0;
    if (__any_sync(kFull, v != 0.0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (lane == 0) atomicAdd(&sg[p], v);
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 + 2 * L && sg[threadIdx.x] != 0.0)
    atomicAdd(a.grad + a.grad_off[inst] + threadIdx.x, sg[threadIdx.x]);
}

int launch_adj_gather(const AdjArgs& a, int max_nr, int max_nz, void* stream) {
  const int threads = 256;
  const int gl = a.gather_lines;
  const long long warps = (long long)((max_nr - 1 + 30) / 31) * ((max_nz + gl - 1) / gl);
  const dim3 grid((unsigned)((warps * 32 + threads - 1) / threads), (unsigned)a.n_inst);
  adj_gather_kernel<<<grid, threads, 0, (cudaStream_t)stream>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// loss and seeds: J = sum_n tau (Sbar_n - target_n)^2, seed_n = dJ/dSbar_n
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) adj_seed_kernel(const DevInst* __restrict__ insts,
                                                       const double* __restrict__ trace,
                                                       const double* __restrict__ target,
                                                       long long n_steps, double* seed,
                                                       double* loss) {
  __shared__ double part[256];
  const int inst = blockIdx.x;
  const double tau = insts[inst].tau;
  double acc = 0.0;
  for (long long n = threadIdx.x; n < n_steps; n += blockDim.x) {
    const long long q = (long long)inst * n_steps + n;
    const double e = trace[2 * q + 1] - target[q];
    seed[q] = 2.0 * tau * e;
    acc = fma(tau * e, e, acc);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) loss[inst] = part[0];
}

int launch_adj_seed(const DevInst* insts, int n_inst, const double* trace, const double* target,
                    long long n_steps, double* seed, double* loss, void* stream) {
  adj_seed_kernel<<<n_inst, 256, 0, (cudaStream_t)stream>>>(insts, trace, target, n_steps, seed,
                                                            loss);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
