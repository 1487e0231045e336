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
//  adj_line_kernel    per line: rebuild (a, b, c) at T^n, then solve the
//                     transposed system with the same segment elimination and
//                     shuffle cyclic reduction as the forward solve
//                     (mu includes the loss seed of step n and the folded
//                     axial boundary rows).
//  adj_gather_kernel  per node: dJ/dT^n from xi of the node's own row and of
//                     the four neighbouring rows that read its temperature
//                     (no atomics on the field), plus the parameter terms of
//                     its own row (shuffle sums per warp, shared sums per
//                     block, one global atomic per block and parameter).
#include <cuda_runtime.h>

#include "ccell_device.cuh"

namespace ccell {

// d lambda / dT at a node, given lambda(T)
__device__ __forceinline__ double dlam_node(const DevMaterial& M, double T, double lamT) {
  if (M.lam_model == 1) return M.lam_b * lamT * frcp(T);
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
      da = db = M.lam_b * l * frcp(y);
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

// c(T) and dc/dT
__device__ __forceinline__ void cap_d(const DevMaterial& M, double T, double& c, double& dc) {
  if (M.cap_model == 1) {
    const double x = T * M.inv_tref, y = T * M.inv_theta;
    const double rd = frcp(fma(y * y, y, 1.0));
    c = M.c0s * (x * x * x) * rd;
    dc = 3.0 * c * frcp(T) * rd;  // c0 x^3/(1+y^3): derivative (3c/T)/(1+y^3)
  } else if (M.cap_model == 0) {
    c = M.c0s;
    dc = 0.0;
  } else {
    const double* a = M.cap_poly;
    c = fma(fma(fma(a[3], T, a[2]), T, a[1]), T, a[0]);
    dc = fma(fma(3.0 * a[3], T, 2.0 * a[2]), T, a[1]);
  }
}

// ---------------------------------------------------------------------------
// transposed line solve
// ---------------------------------------------------------------------------
__device__ __forceinline__ void adj_line_task(const AdjArgs& a, const Task tk, const int lane) {
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
  const long long rj = (long long)j * nr;
  const double* Tj = a.x + I.t_off + rj;
  double* Sa = a.sa + I.t_off + rj;
  double* Sb = a.sb + I.t_off + rj;
  double* Sc = a.sc + I.t_off + rj;
  const int frule = I.face_rule;

  // pass 1: the rows of the forward step at T^n
  {
    double Tm1 = (i_lo > 0) ? Tj[i_lo - 1] : 0.0;
    double T0 = Tj[i_lo];
    double le_prev = 0.0;
    bool have_le = false;
#pragma unroll
    for (int k = 0; k < kRowsPerLane; ++k) {
      if (k < cnt) {
        const int i = i_lo + k;
        const RowGeo& g = I.rg[i];
        const double Tp1 = (i < N) ? Tj[i + 1] : 0.0;
        double ra, rb, rc;
        if (g.cls == RC_REGULAR) {
          const DevMaterial& Mt = I.mat[g.seg];
          const double lw = have_le ? le_prev : lam_face(Mt, frule, Tm1, T0);
          const double le = lam_face(Mt, frule, T0, Tp1);
          const double rct = Mt.rho * cap_eval(Mt, T0) * I.inv_tau;
          ra = -g.gA * lw;
          rc = -g.gC * le;
          rb = rct - ra - rc;
          le_prev = le;
          have_le = true;
        } else if (g.cls == RC_IFACE) {
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
          have_le = false;
        } else if (g.cls == RC_AXIS) {
          ra = 0.0; rb = 1.0; rc = -1.0;
          have_le = false;
        } else {
          ra = (I.bc_rmax == CC_DIRICHLET) ? 0.0 : -1.0;
          rb = 1.0;
          rc = 0.0;
          have_le = false;
        }
        if (active) {
          Sa[i] = ra;
          Sb[i] = rb;
          Sc[i] = rc;
        }
        Tm1 = T0;
        T0 = Tp1;
      }
    }
  }
  __syncwarp();

  // pass 2: M^T xi = mu, rows (c_{i-1}, b_i, a_{i+1} | mu_i)
  const double* Lam = a.lam + I.t_off;
  const double sd = a.seed[(long long)tk.inst * a.n_steps + a.step];
  const bool fold0 = (j == 1) && (I.bc_z0 == CC_NEUMANN);
  const bool foldM = (j == M - 1) && (I.bc_zmax == CC_NEUMANN);
  const double wj = I.zg[j].wnorm, w0 = I.zg[0].wnorm, wM = I.zg[M].wnorm;

  double cp[kRowsPerLane], ap[kRowsPerLane], dp[kRowsPerLane];
  double pc = 0.0, pa = 0.0, pd = 0.0;
  double Dacc = 0.0, Aacc = 0.0, P = 1.0;
  double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;
#pragma unroll
  for (int k = 0; k < kRowsPerLane; ++k) {
    if (k < cnt) {
      const int i = i_lo + k;
      const double ra = (i > 0) ? Sc[i - 1] : 0.0;
      const double rb = Sb[i];
      const double rc = (i < N) ? Sa[i + 1] : 0.0;
      double rd = Lam[rj + i];
      if (i == N) rd = fma(sd, wj, rd);
      if (fold0) rd += Lam[i] + ((i == N) ? sd * w0 : 0.0);
      if (foldM) rd += Lam[(long long)M * nr + i] + ((i == N) ? sd * wM : 0.0);
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
  const double xs = solve_separators(ae, be, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);
  const double L = __shfl_up_sync(kFull, xs, 1, G);
  double xn = xs;
#pragma unroll
  for (int k = kRowsPerLane - 2; k >= 0; --k) {
    if (k <= cnt - 2) {
      const double x = fma(-cp[k], xn, fma(-ap[k], L, dp[k]));
      dp[k] = x;
      xn = x;
    }
  }
  if (active) {
    double* XI = a.xi + I.t_off + rj;
#pragma unroll
    for (int k = 0; k < kRowsPerLane; ++k)
      if (k < cnt) XI[i_lo + k] = (k == cnt - 1) ? xs : dp[k];
  }
}

__global__ void __launch_bounds__(128) adj_line_kernel(const AdjArgs a) {
  const int lane = threadIdx.x & 31;
  const int n_warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < a.n_tasks; w += n_warps)
    adj_line_task(a, a.tasks[w], lane);
}

int launch_adj_line(const AdjArgs& a, void* stream) {
  constexpr int threads = 128;
  static int resident = 0;
  if (resident == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_line_kernel, threads, 0);
    resident = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int need = (a.n_tasks * 32 + threads - 1) / threads;
  adj_line_kernel<<<need < resident ? need : resident, threads, 0, (cudaStream_t)stream>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// per-node gather of dJ/dT^n and of the parameter terms
// ---------------------------------------------------------------------------
constexpr int kGradMax = 2 + 2 * CC_MAX_LAYERS;

__global__ void __launch_bounds__(256) adj_gather_kernel(const AdjArgs a) {
  __shared__ double sg[kGradMax];
  const int inst = blockIdx.y;
  const DevInst& I = a.insts[inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int L = a.n_layers[inst];
  if (threadIdx.x < kGradMax) sg[threadIdx.x] = 0.0;
  __syncthreads();
  // this node's parameter terms: q0, t_on, lam_scale[mL], cap_scale[mC]
  // (a second lam_scale term at mL2 for interface rows); summed over the warp
  // per parameter below, so that the block's shared sums see one add per warp
  double pq = 0.0, pt = 0.0, pl = 0.0, pl2 = 0.0, pc = 0.0;
  int mL = -1, mL2 = -1, mC = -1;
  const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node < (long long)nr * I.nz) {
    const int j = (int)(node / nr), i = (int)(node - (long long)j * nr);
    const double* X = a.x + I.t_off;
    const double* Y = a.y + I.t_off;
    const double* XI = a.xi + I.t_off;
    const long long rj = (long long)j * nr;
    const double T = X[rj + i];
    const RowGeo& g = I.rg[i];
    const int frule = I.face_rule;
    const bool line = (j >= 1 && j <= M - 1);  // own row belongs to a solved line
    const double tau_inv = I.inv_tau;
    double acc = 0.0;
    // radial faces (i-1, i) of material seg[i-1] and (i, i+1) of material seg[i]
    double lW = 0.0, lWa = 0.0, lWb = 0.0, lE = 0.0, lEa = 0.0, lEb = 0.0;
    if (i >= 1) lam_face_d(I.mat[I.rg[i - 1].seg], frule, X[rj + i - 1], T, lW, lWa, lWb);
    if (i <= N - 1) lam_face_d(I.mat[g.seg], frule, T, X[rj + i + 1], lE, lEa, lEb);
    const double yi = Y[rj + i];
    // rows i-1 and i+1 of the same line
    if (line) {
      if (i >= 1) {
        const RowGeo& gw = I.rg[i - 1];
        const double xw = XI[rj + i - 1], dy = yi - Y[rj + i - 1];
        if (gw.cls == RC_REGULAR) acc = fma(xw * gw.gC * lWb, dy, acc);
        else if (gw.cls == RC_IFACE && I.interface_rule == 1)
          acc = fma(xw * gw.re * lWb * gw.hw, dy, acc);
      }
      if (i <= N - 1) {
        const RowGeo& ge = I.rg[i + 1];
        const double xe = XI[rj + i + 1], dy = yi - Y[rj + i + 1];
        if (ge.cls == RC_REGULAR) acc = fma(xe * ge.gA * lEa, dy, acc);
        else if (ge.cls == RC_IFACE && I.interface_rule == 1)
          acc = fma(xe * ge.rw * lEa * ge.he, dy, acc);
      }
    }
    if (g.cls == RC_REGULAR) {
      const int m = g.seg;
      const DevMaterial& Mt = I.mat[m];
      // axial faces (j-1, j) and (j, j+1)
      double lS = 0.0, lSa = 0.0, lSb = 0.0, lN = 0.0, lNa = 0.0, lNb = 0.0;
      const double Ts = (j >= 1) ? X[rj - nr + i] : 0.0, Tn = (j <= M - 1) ? X[rj + nr + i] : 0.0;
      if (j >= 1) lam_face_d(Mt, frule, Ts, T, lS, lSa, lSb);
      if (j <= M - 1) lam_face_d(Mt, frule, T, Tn, lN, lNa, lNb);
      // rows (i, j+1) and (i, j-1) read T through their south / north faces
      if (j + 1 >= 1 && j + 1 <= M - 1)
        acc = fma(XI[rj + nr + i] * I.zg[j + 1].gzs, fma(-lNa, Tn - T, lN), acc);
      if (j - 1 >= 1 && j - 1 <= M - 1)
        acc = fma(XI[rj - nr + i] * I.zg[j - 1].gzn, fma(lSb, T - Ts, lS), acc);
      if (line) {
        const double xi = XI[rj + i];
        const ZGeo& zg = I.zg[j];
        double c, dc;
        cap_d(Mt, T, c, dc);
        const double rct = Mt.rho * c * tau_inv, drct = Mt.rho * dc * tau_inv;
        const double gw = Y[rj + i - 1] - yi, ge = Y[rj + i + 1] - yi;
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
          dgT = -0.5 * gT * frcp(T);
        }
        if (heat) d0 = fma(I.q0 * a.s_tab[sidx], dgT, d0);
        acc = fma(xi, d0, acc);
        // parameters of this row
        const double lam_part =
            fma(g.gC * lE, ge, fma(g.gA * lW, gw, fma(lN * zg.gzn, dN, -lS * zg.gzs * dS)));
        pl = xi * lam_part * Mt.inv_lam_scale;
        mL = m;
        pc = xi * rct * (T - yi) * Mt.inv_cap_scale;
        mC = m;
        if (heat) {
          pq = xi * a.s_tab[sidx] * gT;
          pt = xi * I.q0 * a.ds_tab[sidx] * gT;
        }
      }
    } else if (g.cls == RC_IFACE && line) {
      const double xi = XI[rj + i];
      const int mi = g.segw, mo = g.seg;
      const double gw = Y[rj + i - 1] - yi, ge = Y[rj + i + 1] - yi;
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
      pl = xi * lm * g.he * gw * I.mat[mi].inv_lam_scale;
      mL = mi;
      pl2 = xi * lp * g.hw * ge * I.mat[mo].inv_lam_scale;
      mL2 = mo;
    }
    a.lam_out[I.t_off + rj + i] = acc;
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
      if ((threadIdx.x & 31) == 0) atomicAdd(&sg[p], v);
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 + 2 * L && sg[threadIdx.x] != 0.0)
    atomicAdd(a.grad + a.grad_off[inst] + threadIdx.x, sg[threadIdx.x]);
}

int launch_adj_gather(const AdjArgs& a, long long max_nodes, void* stream) {
  const int threads = 256;
  const dim3 grid((unsigned)((max_nodes + threads - 1) / threads), (unsigned)a.n_inst);
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
