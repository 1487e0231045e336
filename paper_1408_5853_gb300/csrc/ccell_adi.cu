// ADI variant of the time step (Peaceman-Rachford), the scheme the paper
// names as the unconditionally stable alternative to its own (Section 3,
// after Eq. (stability_condition)).  Two half steps of tau/2, properties and
// source frozen at (T^n, t_n):
//   rho c (T* - T^n)/(tau/2)     = Lambda_i[T*] + Lambda_j[T^n]     + X   (radial lines)
//   rho c (T^n+1 - T*)/(tau/2)   = Lambda_i[T*] + Lambda_j[T^n+1]   + X   (axial columns)
// The first half step is the tile kernel of the paper's step at tau/2; it
// also leaves rho c/(tau/2), Lambda_j[T^n] and the axial face conductivities
// of the regular nodes.  Subtracting the two equations, the second becomes
//   rho c/(tau/2) T^n+1 - Lambda_j[T^n+1] = rho c/(tau/2) (2 T* - T^n) - Lambda_j[T^n],
// one tridiagonal system along z per column of regular nodes (this file),
// split over the threads of a block.  Then the non-regular
// columns take their radial relations with the new values (axis, r_max,
// interface rows of Eq. (cc_first_3) with lambda* at T^n), the axial
// boundary rows are set, and the surface trace is formed.
#include <cuda_runtime.h>

#include "ccell_device.cuh"

namespace ccell {

// One block per column of regular nodes.  Each thread eliminates its run of
// rows downwards (c', a', d' to global scratch, coalesced over the threads),
// the S separator rows are solved by cyclic reduction through shared memory,
// and each thread substitutes back.  The same partitioned elimination as the
// radial lines (solve_tile_lines), with the separators spread over the block.
__global__ void __launch_bounds__(kAdiLanes) adi_axial_kernel(const AdiArgs a) {
  __shared__ double sA[kAdiLanes], sB[kAdiLanes], sC[kAdiLanes], sI[kAdiLanes];
  const int s = threadIdx.x;
  for (int w = blockIdx.x; w < a.n_tasks; w += gridDim.x) {
    const AdiTask tk = a.tasks[w];
    const DevInst& I = a.insts[tk.inst];
    const int nr = I.nr, M = I.nz - 1, L = M - 1;  // rows j = 1 .. M-1
    int S = kAdiLanes;
    while (S > 1 && L < 2 * S) S >>= 1;
    const bool act = s < S;
    const int lo = 1 + (int)(((long long)s * L) / S), hi = 1 + (int)(((long long)(s + 1) * L) / S);
    const int cnt = act ? hi - lo : 0;  // >= 1
    const long long col = I.t_off + tk.i;
    const size_t plane = (size_t)a.n_tasks * a.rows_max * kAdiLanes;
    double* Cp = a.scr + ((size_t)w * a.rows_max) * kAdiLanes + s;
    double* Ap = Cp + plane;
    double* Dp = Ap + plane;
    double pc = 0.0, pa = 0.0, pd = 0.0;
    double Dacc = 0.0, Aacc = 0.0, P = 1.0;
    double ae = 0.0, be = 1.0, ce = 0.0, de = 0.0;
    double ls = act ? a.lamz[col + (long long)(lo - 1) * nr] : 0.0;  // face (j-1, j), carried
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
      const int j = lo + k;
      const long long o = col + (long long)j * nr;
      const ZGeo& zg = I.zg[j];
      const double rct = a.rct[o];
      const double ln = a.lamz[o];  // face (j, j+1)
      double ra = -zg.gzs * ls;
      double rc = -zg.gzn * ln;
      ls = ln;
      double rb = rct - ra - rc;
      double rd = fma(rct, 2.0 * a.Tx[o] - a.Tn[o], -a.lj[o]);
      if (j == 1) {  // T_0 = T_1 or T_D folded into the row
        if (I.bc_z0 == CC_DIRICHLET) rd = fma(-ra, I.t_d, rd); else rb += ra;
        ra = 0.0;
      }
      if (j == M - 1) {  // T_M = T_D or T_M-1
        if (I.bc_zmax == CC_DIRICHLET) rd = fma(-rc, I.t_d, rd); else rb += rc;
        rc = 0.0;
      }
      if (k < cnt - 1) {
        const double den = (k == 0) ? rb : fma(-ra, pc, rb);
        const double r = frcp(den);
        const double c1 = rc * r;
        const double a1 = (k == 0) ? ra * r : -ra * pa * r;
        const double d1 = (k == 0) ? rd * r : fma(-ra, pd, rd) * r;
        Cp[(size_t)k * kAdiLanes] = c1;
        Ap[(size_t)k * kAdiLanes] = a1;
        Dp[(size_t)k * kAdiLanes] = d1;
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
    // separator rows in the separators of the neighbouring segments: the
    // first interior row of segment s+1 is Dacc + P x_{s+1} - Aacc x_s
    sA[s] = Dacc;
    sB[s] = Aacc;
    sC[s] = P;
    __syncthreads();
    const int sn = (s + 1 < S) ? s + 1 : s;  // the last separator has c = 0
    double at = -ae * pa;
    double bt = fma(-ae, pc, be) - ce * sB[sn];
    double ct = ce * sC[sn];
    double dt = fma(-ae, pd, de) - ce * sA[sn];
    __syncthreads();
    // parallel cyclic reduction over the S separators
    for (int d = 1; d < S; d <<= 1) {
      const double ib = frcp(bt);
      sA[s] = at; sB[s] = ct; sC[s] = dt; sI[s] = ib;
      __syncthreads();
      double al = 0.0, ga = 0.0, am = 0.0, cm = 0.0, dm = 0.0, apv = 0.0, cpv = 0.0, dpv = 0.0;
      if (act && s >= d) {
        al = -at * sI[s - d];
        am = sA[s - d]; cm = sB[s - d]; dm = sC[s - d];
      }
      if (act && s + d < S) {
        ga = -ct * sI[s + d];
        apv = sA[s + d]; cpv = sB[s + d]; dpv = sC[s + d];
      }
      __syncthreads();
      const double nb = fma(ga, apv, fma(al, cm, bt));
      const double nd = fma(ga, dpv, fma(al, dm, dt));
      at = al * am;
      ct = ga * cpv;
      bt = nb;
      dt = nd;
    }
    const double xs = dt * frcp(bt);
    sA[s] = xs;
    __syncthreads();
    const double Lp = (s > 0) ? sA[s - 1] : 0.0;
    __syncthreads();  // the shared arrays are reused by the next column
    if (act) {
      bool bad = not_finite(xs);
      a.Tx[col + (long long)(hi - 1) * nr] = xs;
      double xn = xs;
      for (int k = cnt - 2; k >= 0; --k) {
        const double x = fma(-Cp[(size_t)k * kAdiLanes], xn,
                             fma(-Ap[(size_t)k * kAdiLanes], Lp, Dp[(size_t)k * kAdiLanes]));
        bad |= not_finite(x);
        a.Tx[col + (long long)(lo + k) * nr] = x;
        xn = x;
      }
      if (bad) atomicOr(a.err, 1u);
    }
  }
}

// Lines per block of the completion kernel.
constexpr int kFinishLines = 16;

// Blocks over (line range, instance): the non-regular columns of the lines,
// then the axial boundary rows (by the blocks owning lines 1 and M-1) and the
// trace (block partial sums, one atomic per block).
__global__ void __launch_bounds__(256) adi_finish_kernel(const AdiArgs a) {
  const int k = blockIdx.y;
  const DevInst& I = a.insts[k];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j_lo = 1 + blockIdx.x * kFinishLines;
  if (j_lo > M - 1) return;  // block-uniform
  const int j_hi = min(M - 1, j_lo + kFinishLines - 1);
  const int nj = j_hi - j_lo + 1;
  const double* Tn = a.Tn + I.t_off;
  double* X = a.Tx + I.t_off;
  bool bad = false;
  // interface nodes: lm (T_i - T_i-1)/h_i = lp (T_i+1 - T_i)/h_i+1, lambda at T^n
  const int n_if = I.n_if;
  for (int it = threadIdx.x; it < nj * n_if; it += blockDim.x) {
    const int jj = it / n_if;
    const int i = I.if_i[it - jj * n_if];
    const RowGeo& g = I.rg[i];
    if (g.cls != RC_IFACE) continue;
    const long long o = (long long)(j_lo + jj) * nr + i;
    double lm, lp;
    if (I.interface_rule == 0) {
      lm = lam_eval(I.mat[g.segw], Tn[o]);
      lp = lam_eval(I.mat[g.seg], Tn[o]);
    } else {
      lm = g.rw * lam_face(I.mat[g.segw], I.face_rule, Tn[o - 1], Tn[o]);
      lp = g.re * lam_face(I.mat[g.seg], I.face_rule, Tn[o], Tn[o + 1]);
    }
    const double x = fma(lm * g.he, X[o - 1], lp * g.hw * X[o + 1]) / fma(lm, g.he, lp * g.hw);
    bad |= not_finite(x);
    X[o] = x;
  }
  // axis and r_max columns
  for (int j = j_lo + threadIdx.x; j <= j_hi; j += blockDim.x) {
    const long long o = (long long)j * nr;
    X[o] = X[o + 1];
    X[o + N] = (I.bc_rmax == CC_DIRICHLET) ? I.t_d : X[o + N - 1];
  }
  if (bad) atomicOr(a.err, 1u);
  __syncthreads();
  // axial boundary rows, from lines 1 and M-1 (complete now)
  if (j_lo == 1)
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
      X[i] = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : X[nr + i];
  if (j_hi == M - 1)
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
      X[(long long)M * nr + i] = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : X[(long long)(M - 1) * nr + i];
  if (a.trace) {  // That(r_max, z_0) and the trapezoid-weighted mean over z
    __syncthreads();
    __shared__ double part[8];
    double s = 0.0;
    for (int j = j_lo + threadIdx.x; j <= j_hi; j += blockDim.x)
      s = fma(I.zg[j].wnorm, X[(long long)j * nr + N], s);
    if (threadIdx.x == 0) {
      if (j_lo == 1) s = fma(I.zg[0].wnorm, X[N], s);
      if (j_hi == M - 1) s = fma(I.zg[M].wnorm, X[(long long)M * nr + N], s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
      double* tr = a.trace + ((long long)k * a.n_steps + a.step) * 2;
      if (j_lo == 1) tr[0] = X[N];
      atomicAdd(tr + 1, t);
    }
  }
}

int launch_adi_axial(const AdiArgs& a, void* stream) {
  if (a.n_tasks > 0)
    adi_axial_kernel<<<a.n_tasks, kAdiLanes, 0, (cudaStream_t)stream>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_adi_finish(const AdiArgs& a, void* stream) {
  const dim3 grid((unsigned)((a.lines_max + kFinishLines - 1) / kFinishLines), (unsigned)a.n_inst);
  adi_finish_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccell
