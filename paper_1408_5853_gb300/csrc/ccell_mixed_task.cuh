// Mixed-precision time-step task (same scheme as ccell_step.cu, Section 3 of the
// paper): conductivities, heat capacities, the explicit axial operator and
// the row coefficients run in FP32; the tridiagonal elimination, the
// separator solve, the update and the energy sums run in FP64.
//
// Conversions between FP32 and FP64 issue on the FP64 pipe, the pipe that
// bounds this scheme on GB300, so the widening of the row coefficients and
// the rounding of the increment to FP32 are done with integer operations on
// the bit patterns (exact widening; round to nearest even; values below the
// FP32 normal range, |x| < 2^-126, flush to zero).
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

// (double)f for normal, zero, infinite and NaN f (subnormal f become +-0).
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned mag = b & 0x7fffffffu;
  unsigned hi = (mag >> 3) + (896u << 20);
  hi = (mag < 0x00800000u) ? 0u : hi;
  hi = (mag >= 0x7f800000u) ? (0x7ff00000u | ((mag >> 3) & 0x000fffffu)) : hi;
  const unsigned lo = (mag < 0x00800000u) ? 0u : (b << 29);
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// x rounded to the nearest FP32 (ties to even); |x| < 2^-126 gives +-0,
// overflow gives +-inf, NaN stays NaN.
__device__ __forceinline__ float narrow_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ffu);
  unsigned f = ((unsigned)(E - 896) << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  f = (E < 897) ? 0u : f;
  const bool nan = E == 2047 && ((hi & 0x000fffffu) | lo) != 0u;
  f = (E > 1150) ? (nan ? 0x7fc00000u : 0x7f800000u) : f;
  return __uint_as_float(f | (hi & 0x80000000u));
}

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
// one CTA tile of nl consecutive lines (the tile structure of the FP64 step,
// ccell_fp64_task.cuh): properties and FP32 rows with the lanes over columns,
// FP64 line solves with the lanes over the rows of a line, then the pair
// update with the lanes over columns again.
// ---------------------------------------------------------------------------
template <bool CACHED>
__device__ __forceinline__ float ld_state(const float* p) {
  if constexpr (CACHED) return __ldg(p);
  else return __ldcg(p);
}

// Row buffers of one mixed-precision tile of nl lines (padded rows of nrp):
// the four rows of every line's system (FP64), then in FP32 the capacities
// and kMixIf floats per line and interface node.
struct MixTile {
  double *SA, *SB, *SC, *SD;  // a, b (then the increment dT), c, d
  float *FM, *sI;             // V rho c (energy); lam_w, lam_e, kw, ke, dTw, dTe per interface
  // packed layout (pipelined launch): per node the FP32 row (a, c, d) and
  // V rho c; the FP64 increment later replaces (a, c) of its node
  float4* Q;
};

// Packed rows: the FP64 increment stored over (a, c) of a node, and read back.
__device__ __forceinline__ void put_packed_x(float4* Q, int c, double x) {
  *reinterpret_cast<double*>(Q + c) = x;
}
__device__ __forceinline__ double packed_x(const float4* Q, int c) {
  return *reinterpret_cast<const double*>(Q + c);
}

__device__ __forceinline__ MixTile mix_tile_packed_at(float* base, int nl, int nrp) {
  MixTile B{};
  B.Q = reinterpret_cast<float4*>(base);
  B.sI = base + 4 * (size_t)nl * nrp;
  return B;
}

__device__ __forceinline__ MixTile mix_tile_at(float* base, int nl, int nrp) {
  MixTile B;
  B.SA = reinterpret_cast<double*>(base);
  B.SB = B.SA + (size_t)nl * nrp;
  B.SC = B.SB + (size_t)nl * nrp;
  B.SD = B.SC + (size_t)nl * nrp;
  B.FM = reinterpret_cast<float*>(B.SD + (size_t)nl * nrp);
  B.sI = B.FM + (size_t)nl * nrp;
  return B;
}

// Phases 0a-0b of a tile, run by the warps of g: nodal conductivities of the
// interface rows, then FP32 properties and rows in delta form with the lanes
// over columns, widened into the tile's FP64 rows.  The axial fluxes south of
// the first line come from cin if carry, those north of the last line go to
// cout.  STP: the tile holds a line of a stepped outline that is narrow or
// borders a narrow one (other tiles skip the checks).
template <bool ENERGY, bool CACHED, bool STP, bool PACKED = false>
__device__ __forceinline__ void mixed_produce(const StepArgs& a, const TileTask tk, const MixTile& B,
                                              const float* __restrict__ cin, float* __restrict__ cout,
                                              bool carry, const WarpGroup& grp, EAcc& acc) {
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j0 = tk.j0, nl = tk.nl;
  const int nrp = smem_row_stride(nr);
  const int frule = I.face_rule;
  const int n_if = I.n_if;
  const int warp = grp.warp(), lane = threadIdx.x & 31, nwarps = grp.nwarps;
  double* SA = B.SA;
  double* SC = B.SC;
  double* SD = B.SD;
  float* FM = B.FM;
  float* sI = B.sI;
  const float* Hin = static_cast<const float*>(a.Tin) + I.t_off;
  const float* Lin = a.lo_in + I.t_off;
  const float s = (float)a.s_tab[a.step * a.n_inst + tk.inst];
  const float inv_tau = I.inv_tau_f, tau = I.tau_f;
  double eQ = 0.0, eD = 0.0, eN = 0.0;

  // ---- 0a. nodal conductivities of the interface rows, Eq. (cc_first_3)
  if (I.interface_rule == 0 && n_if > 0) {
    for (int it = grp.tid(); it < nl * n_if; it += grp.size()) {
      const int q = it / n_if;
      const int i = I.if_i[it - q * n_if];
      const RowGeo& g = I.rg[i];
      if (g.cls == RC_IFACE) {
        const float h = ld_state<CACHED>(Hin + (long long)(j0 + q) * nr + i);
        sI[kMixIf * it] = lam32(I.mat[g.segw], h);
        sI[kMixIf * it + 1] = lam32(I.mat[g.seg], h);
      }
    }
  }
  grp.sync();  // the interface values, and the previous tile's carried fluxes

  // ---- 0b. FP32 properties and rows in delta form, lanes over columns
  // (block b covers columns 31b .. 31b+31; see the FP64 tile)
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
      const RowGeo& g = I.rg[ic];
      const int cls0 = g.cls, seg = g.seg;
      const DevMaterial& Mt = I.mat[seg];
      const int ie = ic < N ? ic + 1 : ic;
      const bool edge = (cls0 == RC_IFACE || cls0 == RC_OUTER);
      float gwk = 0.0f, gek = 0.0f;  // tau V2 gC of the west, tau V2 gA of the east neighbour
      if (ENERGY && edge) {
        const RowGeo& gw = I.rg[ic - 1];
        const RowGeo& ge = I.rg[ie];
        gwk = tau * gw.V2_f * gw.gC_f;
        gek = tau * ge.V2_f * ge.gA_f;
      }
      long long o = (long long)(j0 + q0) * nr;  // line j
      float hc = ld_state<CACHED>(Hin + o + ic), lc = ld_state<CACHED>(Lin + o + ic);
      float hn = ld_state<CACHED>(Hin + o + nr + ic), ln = ld_state<CACHED>(Lin + o + nr + ic);
      float he = ld_state<CACHED>(Hin + o + ie), lE = ld_state<CACHED>(Lin + o + ie);
      float fs;  // lambda (T - T_S) on the face south of line j
      if (carry && q0 == 0) {
        fs = cin[smem_col(ic)];
      } else {
        const float hs = ld_state<CACHED>(Hin + o - nr + ic), ls = ld_state<CACHED>(Lin + o - nr + ic);
        fs = lam_face32(Mt, frule, hs, hc) * ((hc - hs) + (lc - ls));
      }
      for (int q = q0; q < q1; ++q) {
        const int j = j0 + q;
        float hn2 = 0.0f, ln2 = 0.0f, he2 = 0.0f, lE2 = 0.0f;  // next line, loaded ahead
        if (q + 1 < q1) {
          hn2 = ld_state<CACHED>(Hin + o + 2 * nr + ic);
          ln2 = ld_state<CACHED>(Lin + o + 2 * nr + ic);
          he2 = ld_state<CACHED>(Hin + o + nr + ie);
          lE2 = ld_state<CACHED>(Lin + o + nr + ie);
        }
        o += nr;
        const float dN = (hn - hc) + (ln - lc);       // T_{j+1} - T_j
        const float dE = (he - hc) + (lE - lc);       // T_{i+1} - T_i
        const float dW = -__shfl_up_sync(kFull, dE, 1);  // T_{i-1} - T_i
        // no heat through a face to a node outside a stepped outline
        const float fn = (STP && j + 1 >= I.j_narrow && ic > I.i_step)
                             ? 0.0f : lam_face32(Mt, frule, hc, hn) * dN;
        const int cls = STP ? line_class(I, cls0, ic, j) : cls0;
        const float le = (ic < N) ? lam_face32(Mt, frule, hc, he) : 0.0f;  // face (i, i+1)
        const float lw = __shfl_up_sync(kFull, le, 1);                     // face (i-1, i)
        const float rhoc = Mt.rho_f * cap32(Mt, hc);
        const ZGeo& zg = I.zg[j];
        float fa, fb, fc, fd, m = 0.0f;
        if (cls == RC_REGULAR) {
          const float Ljv = fmaf(zg.gzn_f, fn, -zg.gzs_f * fs);  // Eq. (Lambda_j)
          float X = 0.0f;
          if (seg == I.src_layer && s != 0.0f) {
            X = I.q0_f * s;
            if (I.g_model == 1) X *= I.g_ref_f * rsqrtf(hc);
          }
          const float A = -g.gA_f * lw, C = -g.gC_f * le;
          fa = A;
          fc = C;
          fb = fmaf(rhoc, inv_tau, -A - C);
          fd = fmaf(-A, dW, fmaf(-C, dE, Ljv + X));
          if (ENERGY && own) {
            const float V = g.V2_f * zg.etabar_f;
            m = V * rhoc;
            if (X != 0.0f) eQ = fma(widen_f32(tau * V), widen_f32(X), eQ);
            if (j == 1) {
              const double f = widen_f32(-tau * g.V2_f * fs / (float)zg.eta_s);
              if (I.bc_z0 == CC_DIRICHLET) eD += f; else eN += f;
            }
            if (j == M - 1) {
              const double f = widen_f32(tau * g.V2_f * fn / (float)zg.eta_n);
              if (I.bc_zmax == CC_DIRICHLET) eD += f; else eN += f;
            }
          }
        } else if (cls == RC_IFACE) {
          float lmv, lpv;
          if (I.interface_rule == 0) {
            lmv = sI[kMixIf * (q * n_if + g.ifo)];
            lpv = sI[kMixIf * (q * n_if + g.ifo) + 1];
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
        } else if (STP && cls == RC_OUTSIDE) {  // outside the domain: decoupled, dT = 0
          fa = 0.0f; fb = 1.0f; fc = 0.0f; fd = 0.0f;
        } else if (I.bc_rmax == CC_DIRICHLET) {  // r = r_max or a narrow line's outer node
          fa = 0.0f; fb = 1.0f; fc = 0.0f; fd = (I.td_hi - hc) + (I.td_lo - lc);
        } else {  // dT_N - dT_{N-1} = T_{N-1} - T_N
          fa = -1.0f; fb = 1.0f; fc = 0.0f; fd = dW;
        }
        if (ENERGY && own && edge) {
          // heat-flow coefficients to the regular neighbours and the old
          // temperature differences across those edges
          const bool in = !STP || cls != RC_OUTSIDE;
          float* K = sI + kMixIf * (q * n_if + g.ifo);
          K[2] = in ? gwk * zg.etabar_f * lw : 0.0f;
          K[3] = in ? gek * zg.etabar_f * le : 0.0f;
          K[4] = in ? -dW : 0.0f;
          K[5] = in ? -dE : 0.0f;
        }
        if (own && q == nl - 1) cout[smem_col(ic)] = fn;
        if (own) {
          const size_t w = (size_t)q * nrp + smem_col(ic);
          // the row divided by its diagonal in FP32 (the solve takes b = 1),
          // then widened exactly (packed: widened by the solve)
          const float ib = __fdividef(1.0f, fb);
          if constexpr (PACKED) {
            B.Q[w] = make_float4(fa * ib, fc * ib, fd * ib, m);
          } else {
            SA[w] = widen_f32(fa * ib);
            SC[w] = widen_f32(fc * ib);
            SD[w] = widen_f32(fd * ib);
            if (ENERGY) FM[w] = m;
          }
        }
        hc = hn; lc = ln;
        hn = hn2; ln = ln2;
        he = he2; lE = lE2;
        fs = fn;
      }
    }
  }
  if (ENERGY) {
    acc.e[1] += eQ;
    acc.e[2] += eD;
    acc.e[4] += eN;
  }
}

// Phase 4 of a tile, run by the threads of g after the line solves: pair
// update, axial boundary rows, surface trace and the energy terms, with the
// threads over the nodes of the tile.
template <bool ENERGY, bool TRACE, bool CACHED, bool STP, bool PACKED = false>
__device__ __forceinline__ void mixed_finish(const StepArgs& a, const TileTask tk, const MixTile& B,
                                             const WarpGroup& grp, EAcc& acc) {
  const DevInst& I = a.insts[tk.inst];
  const int nr = I.nr, N = nr - 1, M = I.nz - 1;
  const int j0 = tk.j0, nl = tk.nl;
  const int nrp = smem_row_stride(nr);
  const int n_if = I.n_if;
  const double* SB = B.SB;
  const float* FM = B.FM;
  const float* sI = B.sI;
  const float* Hin = static_cast<const float*>(a.Tin) + I.t_off;
  const float* Lin = a.lo_in + I.t_off;
  float* Hout = static_cast<float*>(a.Tout) + I.t_off;
  float* Lout = a.lo_out + I.t_off;
  double eE = 0.0, eD = 0.0, eN = 0.0, eI = 0.0, tr = 0.0;
  // ---- 4. pair update, boundary rows, trace, interface energy; lanes over columns
  {
    bool bad = false;
    // threads over the nl x nr nodes of the tile, line by line
    int q = grp.tid() / nr, i = grp.tid() - q * nr;
    for (; q < nl;) {
      const int j = j0 + q;
      const long long rj = (long long)j * nr;
      const int c = smem_col(i);
      const double xd = PACKED ? packed_x(B.Q, q * nrp + c) : SB[(size_t)q * nrp + c];
      bad |= not_finite(xd);
      const float x = narrow_f64(xd);
      if (ENERGY) eE = fma(widen_f32(PACKED ? B.Q[q * nrp + c].w : FM[(size_t)q * nrp + c]), xd, eE);
      const float hi = ld_state<CACHED>(Hin + rj + i), lo = ld_state<CACHED>(Lin + rj + i);
      const float v = lo + x;
      float h1 = hi + v;
      float l1 = v - (h1 - hi);  // exact: h1 + l1 = hi + v
      if (STP && j >= I.j_narrow && i > I.i_step) {  // outside a stepped outline: unchanged
        h1 = hi;
        l1 = lo;
      }
      Hout[rj + i] = h1;
      Lout[rj + i] = l1;
      if (j == 1) {
        Hout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.td_hi : h1;
        Lout[i] = (I.bc_z0 == CC_DIRICHLET) ? I.td_lo : l1;
      }
      if (j == M - 1) {
        const long long rM = (long long)M * nr + i;
        if (STP && M >= I.j_narrow && i > I.i_step) {
          Hout[rM] = ld_state<CACHED>(Hin + rM);
          Lout[rM] = ld_state<CACHED>(Lin + rM);
        } else {
          Hout[rM] = (I.bc_zmax == CC_DIRICHLET) ? I.td_hi : h1;
          Lout[rM] = (I.bc_zmax == CC_DIRICHLET) ? I.td_lo : l1;
        }
      }
      if (TRACE && i == N) {  // That(r_max, z_j)
        const double surf = (widen_f32(hi) + widen_f32(lo)) + xd;
        tr = fma(I.zg[j].wnorm, surf, tr);
        if (j == 1) {
          const double x0 = (I.bc_z0 == CC_DIRICHLET) ? I.t_d : surf;
          tr = fma(I.zg[0].wnorm, x0, tr);
          a.trace[((long long)tk.inst * a.n_steps + a.step) * 2] = x0;
        }
        if (j == M - 1) {
          const double xM = (I.bc_zmax == CC_DIRICHLET) ? I.t_d : surf;
          tr = fma(I.zg[M].wnorm, xM, tr);
        }
      }
      i += grp.size();
      while (i >= nr) {
        i -= nr;
        ++q;
      }
    }
    if (bad) atomicOr(a.err, 1u);
    if (ENERGY) {
      // heat through the edges between each interface (or r_max) node and its
      // regular neighbours, at the new temperatures: k (dT_old + d(dT))
      for (int it = grp.tid(); it < nl * n_if; it += grp.size()) {
        const int q = it / n_if;
        const int i = I.if_i[it - q * n_if];
        auto xat = [&](int ii) {
          return PACKED ? packed_x(B.Q, q * nrp + smem_col(ii)) : SB[(size_t)q * nrp + smem_col(ii)];
        };
        const float* K = sI + kMixIf * it;
        const double x = xat(i);
        const double fw = widen_f32(K[2]) * (widen_f32(K[4]) + (x - xat(i - 1)));
        const int cls = STP ? line_class(I, I.rg[i].cls, i, j0 + q) : I.rg[i].cls;
        if (cls == RC_OUTER) {
          if (I.bc_rmax == CC_DIRICHLET) eD += fw; else eN += fw;
        } else if (!STP || cls == RC_IFACE) {
          eI += fw + widen_f32(K[3]) * (widen_f32(K[5]) + (x - xat(i + 1)));
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

// Line solves of a mixed tile with packed rows (unit diagonal), run by one
// group of warps (warp: index in the group): the FP32 rows are widened on
// read, the eliminated FP64 coefficients of a lane's segment stay in its
// registers, and each solution replaces (a, c) of its node.  Same segment
// elimination, separator cyclic reduction and back substitution as
// solve_tile_lines.
__device__ __forceinline__ void solve_mixed_packed(float4* __restrict__ Q, int nl, int nr, int G,
                                                   int warp) {
  const int nrp = smem_row_stride(nr);
  const int lg = __ffs(G) - 1;
  const int lane = threadIdx.x & 31;
  const int grp = lane >> lg, l = lane & (G - 1);
  const int q_req = warp * (32 >> lg) + grp;
  const bool active = q_req < nl;
  const int q = active ? q_req : nl - 1;  // idle lane groups solve a valid line, store nothing
  const int i_lo = (l * nr) >> lg;
  const int i_hi = ((l + 1) * nr) >> lg;
  const int cnt = i_hi - i_lo;  // 2 .. kRowsPerLane
  float4* R = Q + (size_t)q * nrp;
  double cc[kRowsPerLane], aa[kRowsPerLane], dd[kRowsPerLane];
  double pc = 0.0, pa = 0.0, pd = 0.0;
  double Dacc = 0.0, Aacc = 0.0, P = 1.0;
  double ae = 0.0, ce = 0.0, de = 0.0;
#pragma unroll
  for (int k = 0; k < kRowsPerLane; ++k) {
    if (k < cnt) {
      const float4 v = R[smem_col(i_lo + k)];
      const double ra = widen_f32(v.x), rc = widen_f32(v.y), rd = widen_f32(v.z);
      if (k < cnt - 1) {
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
        cc[k] = c1;
        aa[k] = a1;
        dd[k] = d1;
        Dacc = fma(P, d1, Dacc);
        Aacc = fma(P, a1, Aacc);
        P = -P * c1;
        pc = c1;
        pa = a1;
        pd = d1;
      } else {
        ae = ra; ce = rc; de = rd;
      }
    }
  }
  const double xs = solve_separators<false>(ae, 1.0, ce, de, pa, pc, pd, Dacc, Aacc, P, G, l);
  const double L = __shfl_up_sync(kFull, xs, 1, G);
  if (active) {
    double xn = xs;
    put_packed_x(R, smem_col(i_hi - 1), xs);
#pragma unroll
    for (int k = kRowsPerLane - 2; k >= 0; --k) {
      if (k <= cnt - 2) {
        const double x = fma(-cc[k], xn, fma(-aa[k], L, dd[k]));
        put_packed_x(R, smem_col(i_lo + k), x);
        xn = x;
      }
    }
  }
}

// One tile with the whole block: rows, solves, stores, separated by block
// barriers.  sm starts with two rows of axial face fluxes (row par ^ 1 holds
// those south of the tile's first line if carry; those north of its last
// line go to row par), then the tile's row buffers.
template <bool ENERGY, bool TRACE, bool CACHED, bool STP>
__device__ __forceinline__ void step_mixed_tile(const StepArgs& a, const TileTask tk,
                                                float* __restrict__ sm, EAcc& acc, bool carry,
                                                int par) {
  if (tk.inst != acc.inst) {  // block-uniform
    eacc_flush<ENERGY, TRACE>(a, acc);
    acc.inst = tk.inst;
  }
  const DevInst& I = a.insts[tk.inst];
  const int nrp = smem_row_stride(I.nr);
  const MixTile B = mix_tile_at(sm + 2 * (size_t)nrp, tk.nl, nrp);
  const WarpGroup all = whole_block();
  mixed_produce<ENERGY, CACHED, STP>(a, tk, B, sm + (size_t)(par ^ 1) * nrp,
                                     sm + (size_t)par * nrp, carry, all, acc);
  __syncthreads();
  // ---- 1.-3. FP64 line solves, lanes over the rows of a line (unit diagonal)
  solve_tile_lines<false>(B.SA, B.SB, B.SC, B.SD, tk.nl, I.nr, I.G);
  __syncthreads();
  mixed_finish<ENERGY, TRACE, CACHED, STP>(a, tk, B, all, acc);
  __syncthreads();  // the next tile reuses the shared memory
}

// The tiles of this block: its range, or a stride over all tiles.
template <bool ENERGY, bool TRACE, bool CACHED>
__device__ __forceinline__ void mixed_tiles(const StepArgs& a, float* __restrict__ sm, EAcc& acc) {
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
    if (tk.j0 + tk.nl >= a.insts[tk.inst].j_narrow)
      step_mixed_tile<ENERGY, TRACE, CACHED, true>(a, tk, sm, acc, carry, par);
    else
      step_mixed_tile<ENERGY, TRACE, CACHED, false>(a, tk, sm, acc, carry, par);
    prev_inst = tk.inst;
    prev_end = tk.j0 + tk.nl;
    par ^= 1;
  }
}

// Launch bounds of the mixed-precision step kernels.
#ifndef CC_MIX_MAX_THREADS
#define CC_MIX_MAX_THREADS 256
#endif
#ifndef CC_MIX_MIN_BLOCKS
#define CC_MIX_MIN_BLOCKS 1
#endif

}  // namespace ccell
