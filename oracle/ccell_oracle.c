/*
 * ccell_oracle.c -- plain, slow, FP64 CPU oracle of the explicit-implicit
 * heat-conduction time step of Ayriyan et al., "Algorithm and Simulation of
 * Heat Conduction Process for Design of a Thin Multilayer Technical Device"
 * (arXiv:1408.5853).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The CUDA product path
 * never links, loads or calls it, and shares no code with it.
 *
 * What it computes (Section 3 of the paper):
 *   rho c (That - T)/tau = Lambda_i[That] + Lambda_j[T] + X          Eq. (scheme_eq)
 * radial direction r (index i) implicit, axial direction z (index j)
 * explicit; every line j = 1..M-1 is a tridiagonal system in i solved by the
 * Thomas algorithm, Eqs. (front_sweep), (ABC), (back_sweep), with the axis and
 * outer closures Eqs. (first_oder_bc), (alphabeta_ini), (T_ini_for_back_sweep)
 * and the layer-interface rows Eqs. (cc_first_1)-(cc_first_3).
 *
 * Readings of points the paper leaves open (the labels are used below):
 *   A1 face conductivity lambda_{i+1/2,j} = lambda_m((T_ij + T_i+1,j)/2)
 *      (face_rule 0); face_rule 1 = mean of the two nodal values.
 *   A2 boundary conditions per face are flags: default Neumann at r=r_max and
 *      z=0, Dirichlet T_D at z=z_max (Eq. (boundcond)), symmetry at r=0.
 *   A3 interface rows: paper Eq. (cc_first_3) with lambda* at the old
 *      interface temperature (interface_rule 0); interface_rule 1 uses the
 *      r-weighted face fluxes of the neighbouring rows (conservative).
 *      Interface nodes carry no heat capacity, no axial term, no source.
 *   A4 X and the waveform s(t) are evaluated at (T^n, t_n), t_n = t0 + n*tau;
 *      the rectangular pulse uses the half-open windows of Eq. (period).
 *   A5 the transient p^2(t) of Eq. (transient_function) with the exponent
 *      read as negative (or_waveform).
 *   A13 no FMA contraction: build with -ffp-contract=off.
 *   A19 ADI variant: Peaceman-Rachford over two half steps of tau/2
 *      (or_step_adi_n).
 *   A20 stepped outline r in [0, r_max(z)]: beyond z_step only the inner
 *      layers continue, the step face is insulated (or_outline).
 *
 * Array layout: T[j*nr + i], i = 0..nr-1 radial (contiguous), j = 0..nz-1
 * axial; a line j is one contiguous row of nr values.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LAYERS 8

/* node classes in r */
#define OR_AXIS 0      /* i = 0, closure That_0 = That_1               */
#define OR_REGULAR 1   /* interior node inside one layer               */
#define OR_IFACE 2     /* node on the border between two layers         */
#define OR_OUTER 3     /* i = N, closure Neumann or Dirichlet           */

typedef struct {
  /* geometry */
  int n_layers;
  double thickness[OR_MAX_LAYERS]; /* innermost (r = 0) first, metres    */
  int nr, nz;                      /* nodes, including boundary nodes    */
  double length;                   /* z extent, metres                   */
  int bc_rmax, bc_z0, bc_zmax;     /* 0 Neumann, 1 Dirichlet             */
  double t_dirichlet;              /* K                                  */
  int placement;                   /* 0 vertex nodes, 1 half-cell ghosts */
  int face_rule, interface_rule;
  /* materials, per layer */
  double rho[OR_MAX_LAYERS];
  int lam_model[OR_MAX_LAYERS];    /* 0 const, 1 power law, 2 polynomial */
  double lam0[OR_MAX_LAYERS], lam_b[OR_MAX_LAYERS];
  int cap_model[OR_MAX_LAYERS];    /* 0 const, 1 Debye-saturating, 2 poly */
  double c0[OR_MAX_LAYERS], theta[OR_MAX_LAYERS];
  double t_ref[OR_MAX_LAYERS];
  double lam_scale[OR_MAX_LAYERS], cap_scale[OR_MAX_LAYERS];
  double lam_poly[OR_MAX_LAYERS][5]; /* b_0..b_4, Eq. (poly_cond)       */
  double cap_poly[OR_MAX_LAYERS][4]; /* a_0..a_3, Eq. (poly_cap)        */
  /* heating source, Eqs. (source), (current), (period) */
  int src_layer;                   /* -1: no source                      */
  double q0;                       /* W/m^3 amplitude                    */
  double t_period, t_on, t_start;  /* s                                  */
  int waveform;                    /* 0 rectangle nu(t), 1 tanh edges    */
  double edge_w;                   /* s, tanh edge width                 */
  int g_model;                     /* 0: g = 1, 1: g = g_ref/sqrt(T)     */
  double g_ref;
  /* stepped outline (reading A20): 0 = rectangle; k >= 1: beyond z_step
   * only the k innermost layers continue */
  int step_layers;
  double z_step;                   /* metres                             */
} or_problem;

/* ------------------------------------------------------------------ */
/* grid: Eq. (uniform_grid), uniform inside each layer                 */
/* ------------------------------------------------------------------ */

/* Cells per layer: proportional to thickness, largest remainder, at least
 * 2 cells per layer, ties to the lower layer index. */
static int cells_per_layer(const or_problem* p, int* n) {
  int L = p->n_layers, N = p->nr - 1;
  double total = 0.0, ideal[OR_MAX_LAYERS], rem[OR_MAX_LAYERS];
  for (int m = 0; m < L; m++) total += p->thickness[m];
  int sum = 0;
  for (int m = 0; m < L; m++) {
    ideal[m] = (double)N * p->thickness[m] / total;
    n[m] = (int)floor(ideal[m]);
    rem[m] = ideal[m] - (double)n[m];
    if (n[m] < 2) n[m] = 2;
    sum += n[m];
  }
  int R = N - sum;
  int used[OR_MAX_LAYERS] = {0};
  while (R > 0) {
    int best = -1;
    for (int m = 0; m < L; m++)
      if (!used[m] && (best < 0 || rem[m] > rem[best])) best = m;
    if (best < 0) { memset(used, 0, sizeof used); continue; }
    used[best] = 1; n[best]++; R--;
  }
  while (R < 0) {
    int best = -1;
    for (int m = 0; m < L; m++)
      if (n[m] > 2 && (best < 0 || n[m] > n[best])) best = m;
    if (best < 0) return -1;
    n[best]--; R++;
  }
  return 0;
}

/* r[nr], z[nz], rclass[nr], seg[nr] (layer of segment [r_i, r_{i+1}];
 * seg[N] = last layer).  Returns 0 or -1 on an invalid problem. */
int or_grid(const or_problem* p, double* r, double* z, int* rclass, int* seg) {
  int N = p->nr - 1, M = p->nz - 1;
  if (p->n_layers < 1 || p->n_layers > OR_MAX_LAYERS || N < 2 || M < 2) return -1;
  if (p->placement == 0) {
    int n[OR_MAX_LAYERS];
    if (cells_per_layer(p, n)) return -1;
    int i = 0;
    double start = 0.0;
    for (int m = 0; m < p->n_layers; m++) {
      double h = p->thickness[m] / (double)n[m];
      for (int k = 0; k < n[m]; k++, i++) {
        r[i] = start + (double)k * h;
        seg[i] = m;
        rclass[i] = (k == 0 && m > 0) ? OR_IFACE : OR_REGULAR;
      }
      start += p->thickness[m];
    }
    r[N] = start;
    seg[N] = p->n_layers - 1;
    rclass[0] = OR_AXIS;
    rclass[N] = OR_OUTER;
  } else {
    /* half-cell ghosts: Neumann faces lie on the physical boundary; a
     * Dirichlet boundary carries a node.  Single layer only. */
    if (p->n_layers != 1) return -1;
    double R = p->thickness[0];
    double off_hi = p->bc_rmax ? 0.0 : 0.5;
    double h = R / ((double)N - 0.5 - off_hi);
    for (int i = 0; i <= N; i++) {
      r[i] = ((double)i - 0.5) * h;
      seg[i] = 0;
      rclass[i] = OR_REGULAR;
    }
    rclass[0] = OR_AXIS;
    rclass[N] = OR_OUTER;
  }
  if (p->placement == 0) {
    double eta = p->length / (double)M;
    for (int j = 0; j <= M; j++) z[j] = (double)j * eta;
  } else {
    double lo = p->bc_z0 ? 0.0 : 0.5, hi = p->bc_zmax ? 0.0 : 0.5;
    double eta = p->length / ((double)M - lo - hi);
    for (int j = 0; j <= M; j++) z[j] = ((double)j - lo) * eta;
  }
  return 0;
}

/* Stepped outline of the domain, r in [0, r_max(z)], z in [0, z_max(r)]
 * (Section 2; reading A20).  The paper's cell has its outer layers only on
 * z in [0, z_0] (the working surface r = r_max, Section 5); beyond z_0 the
 * inner layers continue alone to the thermostat end z_max.  Here: the lines
 * j with z_j > z_step (j >= j_narrow) hold only the step_layers innermost
 * layers; their outer node is the interface node i_step that starts layer
 * step_layers, and it takes the r_max closure; nodes i > i_step of those
 * lines lie outside the domain.  A rectangle gives j_narrow = nz, i_step = N.
 * Returns 0, or -1 for an outline this scheme does not take (vertex
 * placement only; line 1 must be a full-width line). */
int or_outline(const or_problem* p, const double* z, const int* rclass, int* i_step,
               int* j_narrow) {
  const int N = p->nr - 1, M = p->nz - 1;
  *i_step = N;
  *j_narrow = p->nz;
  if (p->step_layers == 0) return 0;
  if (p->step_layers < 0 || p->step_layers >= p->n_layers || p->placement != 0) return -1;
  int k = 0;
  for (int i = 1; i < N; i++)
    if (rclass[i] == OR_IFACE && ++k == p->step_layers) { *i_step = i; break; }
  if (k != p->step_layers) return -1;
  /* a node on the step face belongs to the full-width part */
  const double zs = p->z_step + 1e-9 * p->length;
  for (int j = 0; j <= M; j++)
    if (z[j] > zs) { *j_narrow = j; break; }
  if (*j_narrow < 2) return -1;
  return 0;
}

/* 1 if the outline is a rectangle (no narrow line): the ADI variant and the
 * adjoint take rectangles only */
static int rect_outline(const or_problem* p, const double* z, const int* cls) {
  int i_step, j_narrow;
  return or_outline(p, z, cls, &i_step, &j_narrow) == 0 && j_narrow == p->nz;
}

/* ------------------------------------------------------------------ */
/* material functions                                                  */
/* ------------------------------------------------------------------ */

/* lambda_m(T): power law lambda0 (T/T_ref)^b, or Eq. (poly_cond) */
static double lam_m(const or_problem* p, int m, double T) {
  double v;
  switch (p->lam_model[m]) {
    case 0: v = p->lam0[m]; break;
    case 1: v = p->lam0[m] * pow(T / p->t_ref[m], p->lam_b[m]); break;
    default: {
      const double* b = p->lam_poly[m];
      v = b[0] + b[1] * T + b[2] * T * T + b[3] * T * T * T + b[4] * T * T * T * T;
    }
  }
  return p->lam_scale[m] * v;
}

/* c_m(T): c0 (T/T_ref)^3 / (1 + (T/theta)^3), or Eq. (poly_cap) */
static double cap_m(const or_problem* p, int m, double T) {
  double v;
  switch (p->cap_model[m]) {
    case 0: v = p->c0[m]; break;
    case 1: {
      double x = T / p->t_ref[m], y = T / p->theta[m];
      v = p->c0[m] * (x * x * x) / (1.0 + y * y * y);
    } break;
    default: {
      const double* a = p->cap_poly[m];
      v = a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T;
    }
  }
  return p->cap_scale[m] * v;
}

/* face conductivity between nodes with temperatures Ta, Tb (reading A1) */
static double lam_face(const or_problem* p, int m, double Ta, double Tb) {
  if (p->face_rule == 0) return lam_m(p, m, 0.5 * (Ta + Tb));
  return 0.5 * (lam_m(p, m, Ta) + lam_m(p, m, Tb));
}

/* waveform s(t) = nu(t) p(t) of Eqs. (current), (period); p == 1.
 * waveform 1: tanh-smoothed edges of width edge_w around the nearest pulse.
 * waveform 2: nu(t) p^2(t), the transient turn-on of Eq. (transient_function)
 *   with the sign of the exponent read as negative (A5): p^2 = 1 -
 *   exp(-(t - n t_prd) / (7 tau*)) for t in [n t_prd, n t_prd + tau), else 1;
 *   tau = edge_w and tau* = tau / 100 (Section 3.1). */
double or_waveform(const or_problem* p, double t) {
  double u = t - p->t_start;
  if (p->waveform == 2) {
    if (u < 0.0) return 0.0;
    double k = floor(u / p->t_period);
    double phi = u - k * p->t_period;
    if (!(phi < p->t_on)) return 0.0;
    if (phi < p->edge_w) return 1.0 - exp(-phi / (7.0 * (p->edge_w / 100.0)));
    return 1.0;
  }
  if (p->waveform == 0) {
    if (u < 0.0) return 0.0;
    double k = floor(u / p->t_period);
    double phi = u - k * p->t_period;
    return (phi < p->t_on) ? 1.0 : 0.0;
  }
  double k = floor((u - 0.5 * p->t_on) / p->t_period + 0.5);
  if (k < 0.0) k = 0.0;
  double phi = u - k * p->t_period;
  return 0.5 * (tanh(phi / p->edge_w) - tanh((phi - p->t_on) / p->edge_w));
}

/* X_m(T, t) of Eq. (source): q0 s(t) g(T) in the heater layer only */
static double source(const or_problem* p, int m, double T, double s) {
  if (m != p->src_layer || s == 0.0) return 0.0;
  double g = (p->g_model == 1) ? p->g_ref / sqrt(T) : 1.0;
  return p->q0 * s * g;
}

/* ------------------------------------------------------------------ */
/* stability bound, Eq. (stability_condition)                          */
/* ------------------------------------------------------------------ */
double or_tau_stab(const or_problem* p, double t_lo, double t_hi, int n_samples) {
  int N = p->nr - 1, M = p->nz - 1;
  double* r = (double*)malloc(sizeof(double) * (N + 1));
  double* z = (double*)malloc(sizeof(double) * (M + 1));
  int* cls = (int*)malloc(sizeof(int) * (N + 1));
  int* seg = (int*)malloc(sizeof(int) * (N + 1));
  double out = -1.0;
  if (or_grid(p, r, z, cls, seg) == 0) {
    double eta2 = 1e300;
    for (int j = 1; j <= M; j++) {
      double e = z[j] - z[j - 1];
      if (e * e < eta2) eta2 = e * e;
    }
    double ratio = 1e300;
    for (int m = 0; m < p->n_layers; m++)
      for (int s = 0; s < n_samples; s++) {
        double T = t_lo + (t_hi - t_lo) * (double)s / (double)(n_samples > 1 ? n_samples - 1 : 1);
        double q = p->rho[m] * cap_m(p, m, T) / lam_m(p, m, T);
        if (q < ratio) ratio = q;
      }
    out = 0.5 * eta2 * ratio;
  }
  free(r); free(z); free(cls); free(seg);
  return out;
}

/* Neumaier compensated addition */
static void kadd(double* s, double* c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
  else *c += (x - t) + *s;
  *s = t;
}

/* ------------------------------------------------------------------ */
/* the tridiagonal system of one line                                  */
/* ------------------------------------------------------------------ */
/*
 * Rows (a, b, c | f) of the system for That on line j (1 <= j <= M-1) from
 * the field T at waveform value s: row i reads
 *   a_i That_{i-1} + b_i That_i + c_i That_{i+1} = f_i,   i = 0..Nj,
 * with Eq. (ABC) for regular nodes, the interface condition Eq. (cc_first_1)
 * written as a row for interface nodes, That_0 = That_1 at the axis
 * (Eq. (first_oder_bc)) and, at the outer node Nj of the line, That_Nj =
 * That_Nj-1 (Neumann) or the Dirichlet value.
 */
static void line_rows(const or_problem* p, const double* T, int j, double s, double tau,
                      const double* r, const double* z, const int* cls, const int* seg,
                      int Nj, int i_step, int j_narrow, double* a, double* b, double* c,
                      double* f) {
  const int nr = p->nr;
  const double* Tj = T + (size_t)j * nr;
  const double* Ts = T + (size_t)(j - 1) * nr;  /* line j-1 */
  const double* Tn = T + (size_t)(j + 1) * nr;  /* line j+1 */
  const double eta_s = z[j] - z[j - 1], eta_n = z[j + 1] - z[j];
  const double etabar = 0.5 * (eta_n + eta_s);
  /* lines j +- 1 narrower than this one close the axial faces of the
   * columns beyond their outer node */
  const int wide_s = (j - 1 < j_narrow), wide_n = (j + 1 < j_narrow);
  a[0] = 0.0; b[0] = 1.0; c[0] = -1.0; f[0] = 0.0;
  for (int i = 1; i <= Nj - 1; i++) {
    const double h_w = r[i] - r[i - 1], h_e = r[i + 1] - r[i];
    if (cls[i] == OR_IFACE) {
      const int mi = seg[i - 1], mo = seg[i];
      double lm, lp;                  /* lambda*_m, lambda*_m+1 */
      if (p->interface_rule == 0) {
        /* Eq. (cc_first_1): lambda*_m (T_i* - T_i*-1)/h_i* =
         * lambda*_m+1 (T_i*+1 - T_i*)/h_i*+1, lambda* at T_i*,j */
        lm = lam_m(p, mi, Tj[i]);
        lp = lam_m(p, mo, Tj[i]);
      } else {
        /* same row with the r-weighted face conductivities of the
         * neighbouring regular rows: flux continuity that conserves */
        lm = 0.5 * (r[i] + r[i - 1]) * lam_face(p, mi, Tj[i - 1], Tj[i]);
        lp = 0.5 * (r[i] + r[i + 1]) * lam_face(p, mo, Tj[i], Tj[i + 1]);
      }
      /* times h_i* h_i*+1 */
      a[i] = -lm * h_e;
      c[i] = -lp * h_w;
      b[i] = lm * h_e + lp * h_w;
      f[i] = 0.0;
      continue;
    }
    const int m = seg[i];
    const double T0 = Tj[i];
    const double hbar = 0.5 * (h_e + h_w);
    const double r_w = 0.5 * (r[i] + r[i - 1]), r_e = 0.5 * (r[i] + r[i + 1]);
    const double lw = lam_face(p, m, Tj[i - 1], T0);
    const double le = lam_face(p, m, T0, Tj[i + 1]);
    const double rc = p->rho[m] * cap_m(p, m, T0);
    /* Eq. (Lambda_j), explicit in T; no heat crosses a face to a node
     * outside the domain (Eq. (boundcond)) */
    const double fn = (wide_n || i <= i_step)
                          ? lam_face(p, m, T0, Tn[i]) * (Tn[i] - T0) / eta_n : 0.0;
    const double fs = (wide_s || i <= i_step)
                          ? lam_face(p, m, Ts[i], T0) * (T0 - Ts[i]) / eta_s : 0.0;
    const double Lj = (fn - fs) / etabar;
    const double X = source(p, m, T0, s);
    /* Eq. (ABC) */
    const double A = -r_w * lw / (r[i] * hbar * h_w);
    const double C = -r_e * le / (r[i] * hbar * h_e);
    const double B = (r_w * lw / h_w + r_e * le / h_e) / (r[i] * hbar) + rc / tau;
    const double F = rc / tau * T0 + Lj + X;
    a[i] = A;
    b[i] = B;
    c[i] = C;
    f[i] = F;
  }
  if (p->bc_rmax == 0) { a[Nj] = -1.0; b[Nj] = 1.0; c[Nj] = 0.0; f[Nj] = 0.0; }
  else { a[Nj] = 0.0; b[Nj] = 1.0; c[Nj] = 0.0; f[Nj] = p->t_dirichlet; }
}

/* Test access to line_rows: the rows of line j (1 <= j <= nz-2) for the
 * field T at time t with step tau, *n_rows = Nj + 1 (the rows the sweep of
 * or_step_n solves).  Returns 0, or -1 on an invalid problem or line. */
int or_line_rows(const or_problem* p, const double* T, int j, double t, double tau, double* a,
                 double* b, double* c, double* f, int* n_rows) {
  const int N = p->nr - 1, M = p->nz - 1;
  if (j < 1 || j > M - 1) return -1;
  double* r = (double*)malloc(sizeof(double) * (N + 1));
  double* z = (double*)malloc(sizeof(double) * (M + 1));
  int* cls = (int*)malloc(sizeof(int) * (N + 1));
  int* seg = (int*)malloc(sizeof(int) * (N + 1));
  int i_step = 0, j_narrow = 0, rc = -1;
  if (r && z && cls && seg && or_grid(p, r, z, cls, seg) == 0 &&
      or_outline(p, z, cls, &i_step, &j_narrow) == 0) {
    const int Nj = (j >= j_narrow) ? i_step : N;
    line_rows(p, T, j, or_waveform(p, t), tau, r, z, cls, seg, Nj, i_step, j_narrow, a, b, c, f);
    *n_rows = Nj + 1;
    rc = 0;
  }
  free(r); free(z); free(cls); free(seg);
  return rc;
}

/* ------------------------------------------------------------------ */
/* n time steps                                                        */
/* ------------------------------------------------------------------ */
/*
 * T       [nz*nr] in/out temperature field (K).
 * trace   [n_steps*2] or NULL: after step n, (That(r_max, z_0),
 *         trapezoid-weighted mean over z of That(r_max, z)).
 * energy  [5] or NULL, accumulated (added to): stored heat dE, injected
 *         source Q, flux through Dirichlet edges, through interface edges,
 *         through Neumann/ghost edges.  dE = Q + PhiD + PhiI + PhiN holds for
 *         the discrete scheme up to rounding.
 * Returns 0, or -1 on an invalid problem.
 */
int or_step_n(const or_problem* p, double* T, long n_steps, double t0, double tau,
              double* trace, double* energy) {
  const int N = p->nr - 1, M = p->nz - 1, nr = p->nr;
  double* r = (double*)malloc(sizeof(double) * (N + 1));
  double* z = (double*)malloc(sizeof(double) * (M + 1));
  int* cls = (int*)malloc(sizeof(int) * (N + 1));
  int* seg = (int*)malloc(sizeof(int) * (N + 1));
  double* Th = (double*)malloc(sizeof(double) * (size_t)nr * (M + 1));
  double* part = (double*)malloc(sizeof(double) * 5 * (size_t)(M + 1)); /* per line */
  int i_step = 0, j_narrow = 0;
  if (!r || !z || !cls || !seg || !Th || !part || or_grid(p, r, z, cls, seg) ||
      or_outline(p, z, cls, &i_step, &j_narrow)) {
    free(r); free(z); free(cls); free(seg); free(Th); free(part);
    return -1;
  }
  const double two_pi = 2.0 * 3.14159265358979323846;
  double esum[5] = {0, 0, 0, 0, 0}, ecmp[5] = {0, 0, 0, 0, 0};

  for (long n = 0; n < n_steps; n++) {
    const double tn = t0 + (double)n * tau;
    const double s = or_waveform(p, tn);

#pragma omp parallel
    {
      double* alpha = (double*)malloc(sizeof(double) * (N + 1));
      double* beta = (double*)malloc(sizeof(double) * (N + 1));
      double* ra = (double*)malloc(sizeof(double) * (N + 1));  /* rows of line j */
      double* rb = (double*)malloc(sizeof(double) * (N + 1));
      double* rcv = (double*)malloc(sizeof(double) * (N + 1));
      double* rf = (double*)malloc(sizeof(double) * (N + 1));
#pragma omp for schedule(static)
      for (int j = 1; j <= M - 1; j++) {
        const double* Tj = T + (size_t)j * nr;
        double* Thj = Th + (size_t)j * nr;
        /* outer node of this line (a narrower line ends at i_step) */
        const int Nj = (j >= j_narrow) ? i_step : N;
        line_rows(p, T, j, s, tau, r, z, cls, seg, Nj, i_step, j_narrow, ra, rb, rcv, rf);

        /* forward sweep, Eqs. (front_sweep), (cc_first_3) */
        alpha[0] = 1.0;                     /* Eq. (alphabeta_ini) */
        beta[0] = 0.0;
        for (int i = 1; i <= Nj - 1; i++) {
          if (cls[i] == OR_IFACE) {
            /* Eq. (cc_first_3), with lambda*_m h_i*+1 = -a and
             * lambda*_m+1 h_i* = -c of the interface row */
            const double lmh = -ra[i], lph = -rcv[i];
            const double den = lph + lmh * (1.0 - alpha[i - 1]);
            alpha[i] = lph / den;
            beta[i] = lmh * beta[i - 1] / den;
            continue;
          }
          const double den = rb[i] + ra[i] * alpha[i - 1];
          alpha[i] = -rcv[i] / den;
          beta[i] = (rf[i] - ra[i] * beta[i - 1]) / den;
        }
        /* Eq. (T_ini_for_back_sweep) or the Dirichlet value */
        Thj[Nj] = (p->bc_rmax == 0) ? beta[Nj - 1] / (1.0 - alpha[Nj - 1]) : p->t_dirichlet;
        for (int i = Nj - 1; i >= 0; i--) Thj[i] = alpha[i] * Thj[i + 1] + beta[i]; /* Eq. (back_sweep) */
        for (int i = Nj + 1; i <= N; i++) Thj[i] = Tj[i];  /* outside the domain */
      }
      free(alpha); free(beta); free(ra); free(rb); free(rcv); free(rf);
    }

    /* axial boundary rows (line 0 always has the full width) */
    const int NM = (M >= j_narrow) ? i_step : N;
    for (int i = 0; i <= N; i++) {
      Th[i] = p->bc_z0 ? p->t_dirichlet : Th[(size_t)nr + i];
      Th[(size_t)M * nr + i] = (i > NM) ? T[(size_t)M * nr + i]
                               : p->bc_zmax ? p->t_dirichlet : Th[(size_t)(M - 1) * nr + i];
    }

    /* energy terms of this step, per line then summed in line order */
    if (energy) {
#pragma omp parallel for schedule(static)
      for (int j = 1; j <= M - 1; j++) {
        const double* Tj = T + (size_t)j * nr;
        const double* Ts = T + (size_t)(j - 1) * nr;
        const double* Tn = T + (size_t)(j + 1) * nr;
        const double* Hj = Th + (size_t)j * nr;
        const double eta_s = z[j] - z[j - 1], eta_n = z[j + 1] - z[j];
        const double etabar = 0.5 * (eta_n + eta_s);
        double e[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
        const int Nj = (j >= j_narrow) ? i_step : N;
        for (int i = 1; i <= Nj - 1; i++) {
          if (cls[i] != OR_REGULAR) continue;
          const int m = seg[i];
          const double h_w = r[i] - r[i - 1], h_e = r[i + 1] - r[i];
          const double hbar = 0.5 * (h_e + h_w);
          const double r_w = 0.5 * (r[i] + r[i - 1]), r_e = 0.5 * (r[i] + r[i + 1]);
          const double V = two_pi * r[i] * hbar * etabar;
          kadd(&e[0], &c[0], V * p->rho[m] * cap_m(p, m, Tj[i]) * (Hj[i] - Tj[i]));
          kadd(&e[1], &c[1], tau * V * source(p, m, Tj[i], s));
          /* radial edges to non-regular neighbours (implicit fluxes) */
          if (cls[i - 1] != OR_REGULAR) {
            double f = tau * two_pi * etabar * r_w * lam_face(p, m, Tj[i - 1], Tj[i]) *
                       (Hj[i - 1] - Hj[i]) / h_w;
            kadd(cls[i - 1] == OR_IFACE ? &e[3] : &e[4], cls[i - 1] == OR_IFACE ? &c[3] : &c[4], f);
          }
          const int ce = (i + 1 == Nj) ? OR_OUTER : cls[i + 1];  /* outer node of the line */
          if (ce != OR_REGULAR) {
            double f = tau * two_pi * etabar * r_e * lam_face(p, m, Tj[i], Tj[i + 1]) *
                       (Hj[i + 1] - Hj[i]) / h_e;
            int k = (ce == OR_IFACE) ? 3 : (p->bc_rmax ? 2 : 4);
            kadd(&e[k], &c[k], f);
          }
          /* axial edges to the boundary rows (explicit fluxes) */
          if (j == 1) {
            double f = tau * two_pi * r[i] * hbar * lam_face(p, m, Ts[i], Tj[i]) *
                       (Ts[i] - Tj[i]) / eta_s;
            int k = p->bc_z0 ? 2 : 4;
            kadd(&e[k], &c[k], f);
          }
          if (j == M - 1 && i <= NM) {
            double f = tau * two_pi * r[i] * hbar * lam_face(p, m, Tj[i], Tn[i]) *
                       (Tn[i] - Tj[i]) / eta_n;
            int k = p->bc_zmax ? 2 : 4;
            kadd(&e[k], &c[k], f);
          }
        }
        for (int k = 0; k < 5; k++) part[5 * (size_t)j + k] = e[k] + c[k];
      }
      for (int j = 1; j <= M - 1; j++)
        for (int k = 0; k < 5; k++) kadd(&esum[k], &ecmp[k], part[5 * (size_t)j + k]);
    }

    memcpy(T, Th, sizeof(double) * (size_t)nr * (M + 1));

    if (trace) {
      /* trapezoid over the r = r_max surface, the full-width lines */
      double wsum = 0.0, acc = 0.0;
      for (int j = 0; j <= M && j < j_narrow; j++) {
        double w = 0.0;
        if (j > 0) w += 0.5 * (z[j] - z[j - 1]);
        if (j < M && j + 1 < j_narrow) w += 0.5 * (z[j + 1] - z[j]);
        wsum += w;
        acc += w * T[(size_t)j * nr + N];
      }
      trace[2 * n] = T[N];
      trace[2 * n + 1] = acc / wsum;
    }
  }
  if (energy)
    for (int k = 0; k < 5; k++) energy[k] += esum[k] + ecmp[k];
  free(r); free(z); free(cls); free(seg); free(Th); free(part);
  return 0;
}

/* ------------------------------------------------------------------ */
/* ADI variant (Peaceman-Rachford), implicit in both directions        */
/* ------------------------------------------------------------------ */
/*
 * The paper mentions the Alternating Direction Implicit method (Section 3,
 * after Eq. (stability_condition)) as the unconditionally stable alternative
 * to its scheme.  Reading taken (A19): the Peaceman-Rachford splitting of
 * Eq. (scheme_eq) over two half steps of tau/2, with the operators of
 * Eqs. (Lambda_i), (Lambda_j) and the source of Eq. (source), all material
 * properties and X frozen at (T^n, t_n) (this time level is a choice the
 * pins do not distinguish from T*: parity unpinned for it alone):
 *   half step 1:  rho c (T* - T^n)/(tau/2)      = Lambda_i[T*]      + Lambda_j[T^n]     + X
 *   half step 2:  rho c (T^n+1 - T*)/(tau/2)    = Lambda_i[T*]      + Lambda_j[T^n+1]   + X
 * Half step 1 is the paper's step with tau/2 (radial lines, interface rows
 * and closures as there).  Half step 2 is a tridiagonal system along z for
 * each column i of regular nodes (rows j = 1..M-1; T_0 = T_1 or T_D and
 * T_M = T_D or T_M-1 folded in); then the columns of non-regular nodes take
 * their radial relations with the new neighbours -- axis T_0 = T_1, r_max
 * Neumann T_N = T_N-1 or Dirichlet T_D, interface nodes the row of
 * Eq. (cc_first_3) (lambda* at T^n) -- and the axial boundary rows are set as
 * in the paper's step.  trace as in or_step_n; no energy terms.
 */
int or_step_adi_n(const or_problem* p, double* T, long n_steps, double t0, double tau,
                  double* trace) {
  const int N = p->nr - 1, M = p->nz - 1, nr = p->nr;
  const size_t nn = (size_t)nr * (M + 1);
  double* r = (double*)malloc(sizeof(double) * (N + 1));
  double* z = (double*)malloc(sizeof(double) * (M + 1));
  int* cls = (int*)malloc(sizeof(int) * (N + 1));
  int* seg = (int*)malloc(sizeof(int) * (N + 1));
  double* Ts = (double*)malloc(sizeof(double) * nn);  /* T*     */
  double* Tn = (double*)malloc(sizeof(double) * nn);  /* T^n+1  */
  if (!r || !z || !cls || !seg || !Ts || !Tn || or_grid(p, r, z, cls, seg) ||
      !rect_outline(p, z, cls)) {
    free(r); free(z); free(cls); free(seg); free(Ts); free(Tn);
    return -1;
  }
  const double h = 0.5 * tau;
  for (long n = 0; n < n_steps; n++) {
    const double tn = t0 + (double)n * tau;
    const double s = or_waveform(p, tn);
    /* half step 1: the paper's step with tau/2 */
    memcpy(Ts, T, sizeof(double) * nn);
    if (or_step_n(p, Ts, 1, tn, h, NULL, NULL)) {
      free(r); free(z); free(cls); free(seg); free(Ts); free(Tn);
      return -1;
    }
    memcpy(Tn, Ts, sizeof(double) * nn);
    /* half step 2: one tridiagonal system in j per column of regular nodes */
#pragma omp parallel
    {
      double* a = (double*)malloc(sizeof(double) * (M + 1));
      double* b = (double*)malloc(sizeof(double) * (M + 1));
      double* c = (double*)malloc(sizeof(double) * (M + 1));
      double* f = (double*)malloc(sizeof(double) * (M + 1));
#pragma omp for schedule(static)
      for (int i = 1; i <= N - 1; i++) {
        if (cls[i] != OR_REGULAR) continue;
        const int m = seg[i];
        const double h_w = r[i] - r[i - 1], h_e = r[i + 1] - r[i];
        const double hbar = 0.5 * (h_e + h_w);
        const double r_w = 0.5 * (r[i] + r[i - 1]), r_e = 0.5 * (r[i] + r[i + 1]);
        for (int j = 1; j <= M - 1; j++) {
          const double* Tj = T + (size_t)j * nr;        /* T^n, line j   */
          const double* Sj = Ts + (size_t)j * nr;       /* T*,  line j   */
          const double eta_s = z[j] - z[j - 1], eta_n = z[j + 1] - z[j];
          const double etabar = 0.5 * (eta_n + eta_s);
          const double T0 = Tj[i];
          const double rc = p->rho[m] * cap_m(p, m, T0);
          const double lw = lam_face(p, m, Tj[i - 1], T0);
          const double le = lam_face(p, m, T0, Tj[i + 1]);
          const double ls = lam_face(p, m, T[(size_t)(j - 1) * nr + i], T0);
          const double ln = lam_face(p, m, T0, T[(size_t)(j + 1) * nr + i]);
          /* Eq. (Lambda_i) applied to T*, explicit here */
          const double Li = (r_e * le * (Sj[i + 1] - Sj[i]) / h_e -
                             r_w * lw * (Sj[i] - Sj[i - 1]) / h_w) / (r[i] * hbar);
          /* Eq. (Lambda_j) applied to T^n+1: coefficients of T_j-1, T_j+1 */
          a[j] = -ls / (eta_s * etabar);
          c[j] = -ln / (eta_n * etabar);
          b[j] = rc / h - a[j] - c[j];
          f[j] = rc / h * Sj[i] + Li + source(p, m, T0, s);
        }
        /* z closures folded into the first and last rows */
        if (p->bc_z0) { f[1] -= a[1] * p->t_dirichlet; } else { b[1] += a[1]; }
        if (p->bc_zmax) { f[M - 1] -= c[M - 1] * p->t_dirichlet; } else { b[M - 1] += c[M - 1]; }
        /* Thomas algorithm in j */
        for (int j = 2; j <= M - 1; j++) {
          const double w = a[j] / b[j - 1];
          b[j] -= w * c[j - 1];
          f[j] -= w * f[j - 1];
        }
        double x = f[M - 1] / b[M - 1];
        Tn[(size_t)(M - 1) * nr + i] = x;
        for (int j = M - 2; j >= 1; j--) {
          x = (f[j] - c[j] * x) / b[j];
          Tn[(size_t)j * nr + i] = x;
        }
      }
      free(a); free(b); free(c); free(f);
    }
    /* radial relations of the non-regular columns with the new values */
    for (int j = 1; j <= M - 1; j++) {
      double* Hj = Tn + (size_t)j * nr;
      const double* Tj = T + (size_t)j * nr;
      for (int i = 1; i <= N - 1; i++) {
        if (cls[i] != OR_IFACE) continue;
        const int mi = seg[i - 1], mo = seg[i];
        const double h_w = r[i] - r[i - 1], h_e = r[i + 1] - r[i];
        double lm, lp;
        if (p->interface_rule == 0) {
          lm = lam_m(p, mi, Tj[i]);
          lp = lam_m(p, mo, Tj[i]);
        } else {
          lm = 0.5 * (r[i] + r[i - 1]) * lam_face(p, mi, Tj[i - 1], Tj[i]);
          lp = 0.5 * (r[i] + r[i + 1]) * lam_face(p, mo, Tj[i], Tj[i + 1]);
        }
        /* lm (T_i - T_i-1)/h_i = lp (T_i+1 - T_i)/h_i+1, Eq. (cc_first_1) */
        Hj[i] = (lm * h_e * Hj[i - 1] + lp * h_w * Hj[i + 1]) / (lm * h_e + lp * h_w);
      }
      Hj[0] = Hj[1];
      Hj[N] = p->bc_rmax ? p->t_dirichlet : Hj[N - 1];
    }
    /* axial boundary rows */
    for (int i = 0; i <= N; i++) {
      Tn[i] = p->bc_z0 ? p->t_dirichlet : Tn[(size_t)nr + i];
      Tn[(size_t)M * nr + i] = p->bc_zmax ? p->t_dirichlet : Tn[(size_t)(M - 1) * nr + i];
    }
    memcpy(T, Tn, sizeof(double) * nn);
    if (trace) {
      double wsum = 0.0, acc = 0.0;
      for (int j = 0; j <= M; j++) {
        double w = 0.0;
        if (j > 0) w += 0.5 * (z[j] - z[j - 1]);
        if (j < M) w += 0.5 * (z[j + 1] - z[j]);
        wsum += w;
        acc += w * T[(size_t)j * nr + N];
      }
      trace[2 * n] = T[N];
      trace[2 * n + 1] = acc / wsum;
    }
  }
  free(r); free(z); free(cls); free(seg); free(Ts); free(Tn);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* discrete adjoint of or_step_n                                       */
/* ------------------------------------------------------------------ */
/*
 * One step maps T^n to That = T^{n+1}: for every line j = 1..M-1 the rows
 * a_i That_{i-1} + b_i That_i + c_i That_{i+1} = f_i (regular rows: Eq. (ABC);
 * interface rows: Eq. (cc_first_1) written as (-lm h_{i*+1}, lm h_{i*+1} +
 * lp h_{i*}, -lp h_{i*} | 0); closures of Eq. (first_oder_bc)), then the axial
 * boundary rows.  The coefficients depend on T^n through lambda, c and X, and
 * on the parameters theta = (q0, t_on, lam_scale[m], cap_scale[m]).
 *
 * Given mu = dJ/dThat, the adjoint of a line solve is xi = M^{-T} mu, and
 * dJ/dT^n, dJ/dtheta follow from the residual r_i = f_i - (a_i y_{i-1} +
 * b_i y_i + c_i y_{i+1}) with y = That held fixed: dJ/dv = sum_i xi_i dr_i/dv.
 */

/* d lambda_m / dT */
static double dlam_m(const or_problem* p, int m, double T) {
  double v;
  switch (p->lam_model[m]) {
    case 0: v = 0.0; break;
    case 1: v = p->lam0[m] * p->lam_b[m] * pow(T / p->t_ref[m], p->lam_b[m] - 1.0) / p->t_ref[m]; break;
    default: {
      const double* b = p->lam_poly[m];
      v = b[1] + 2.0 * b[2] * T + 3.0 * b[3] * T * T + 4.0 * b[4] * T * T * T;
    }
  }
  return p->lam_scale[m] * v;
}

/* d c_m / dT */
static double dcap_m(const or_problem* p, int m, double T) {
  double v;
  switch (p->cap_model[m]) {
    case 0: v = 0.0; break;
    case 1: {
      double x = T / p->t_ref[m], y = T / p->theta[m], d = 1.0 + y * y * y;
      /* c0 x^3 / (1 + y^3): derivative 3 c0 x^2 / t_ref / (1+y^3) - c0 x^3 3 y^2 / theta / (1+y^3)^2 */
      v = p->c0[m] * (3.0 * x * x / p->t_ref[m] / d - x * x * x * 3.0 * y * y / p->theta[m] / (d * d));
    } break;
    default: {
      const double* a = p->cap_poly[m];
      v = a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T;
    }
  }
  return p->cap_scale[m] * v;
}

/* face conductivity and its derivatives with respect to the two temperatures */
static void lam_face_d(const or_problem* p, int m, double Ta, double Tb, double* l, double* da,
                       double* db) {
  if (p->face_rule == 0) {
    double Tm = 0.5 * (Ta + Tb);
    *l = lam_m(p, m, Tm);
    *da = *db = 0.5 * dlam_m(p, m, Tm);
  } else {
    *l = 0.5 * (lam_m(p, m, Ta) + lam_m(p, m, Tb));
    *da = 0.5 * dlam_m(p, m, Ta);
    *db = 0.5 * dlam_m(p, m, Tb);
  }
}

/* d s / d t_on of the waveform at time t */
static double dwave_dton(const or_problem* p, double t) {
  if (p->waveform == 0) return 0.0;
  double u = t - p->t_start;
  double k = floor((u - 0.5 * p->t_on) / p->t_period + 0.5);
  if (k < 0.0) k = 0.0;
  double phi = u - k * p->t_period;
  double th = tanh((phi - p->t_on) / p->edge_w);
  return 0.5 * (1.0 - th * th) / p->edge_w;
}

/* g(T) of the source and its derivative */
static double src_g(const or_problem* p, double T) {
  return (p->g_model == 1) ? p->g_ref / sqrt(T) : 1.0;
}
static double src_dg(const or_problem* p, double T) {
  return (p->g_model == 1) ? -0.5 * p->g_ref / (T * sqrt(T)) : 0.0;
}

/*
 * Vector-Jacobian product of one step.  x: T^n, y: T^{n+1} (as produced by
 * or_step_n from x), mu: dJ/dT^{n+1} (modified: the axial boundary rows are
 * folded into lines 1 and M-1).  Adds dJ/dT^n to xbar and dJ/dtheta to gbar
 * (2 + 2 n_layers: q0, t_on, lam_scale[], cap_scale[]).
 */
int or_step_vjp(const or_problem* p, const double* x, const double* y, double* mu, double tn,
                double tau, double* xbar, double* gbar) {
  const int N = p->nr - 1, M = p->nz - 1, nr = p->nr, L = p->n_layers;
  double* r = (double*)malloc(sizeof(double) * (N + 1));
  double* z = (double*)malloc(sizeof(double) * (M + 1));
  int* cls = (int*)malloc(sizeof(int) * (N + 1));
  int* seg = (int*)malloc(sizeof(int) * (N + 1));
  double* a = (double*)malloc(sizeof(double) * (N + 1));
  double* b = (double*)malloc(sizeof(double) * (N + 1));
  double* c = (double*)malloc(sizeof(double) * (N + 1));
  double* xi = (double*)malloc(sizeof(double) * (N + 1));
  double* cw = (double*)malloc(sizeof(double) * (N + 1));
  double* dw = (double*)malloc(sizeof(double) * (N + 1));
  if (!r || !z || !cls || !seg || !a || !b || !c || !xi || !cw || !dw || or_grid(p, r, z, cls, seg) ||
      !rect_outline(p, z, cls)) {
    free(r); free(z); free(cls); free(seg); free(a); free(b); free(c); free(xi); free(cw); free(dw);
    return -1;
  }
  const double s = or_waveform(p, tn);
  const double ds_dton = (p->src_layer >= 0) ? dwave_dton(p, tn) : 0.0;
  /* axial boundary rows: That_0 = That_1 (Neumann) or T_D; That_M likewise */
  for (int i = 0; i <= N; i++) {
    if (!p->bc_z0) mu[(size_t)nr + i] += mu[i];
    mu[i] = 0.0;
    if (!p->bc_zmax) mu[(size_t)(M - 1) * nr + i] += mu[(size_t)M * nr + i];
    mu[(size_t)M * nr + i] = 0.0;
  }
  for (int j = 1; j <= M - 1; j++) {
    const double* Tj = x + (size_t)j * nr;
    const double* Ts = x + (size_t)(j - 1) * nr;
    const double* Tn = x + (size_t)(j + 1) * nr;
    const double* yj = y + (size_t)j * nr;
    const double* mj = mu + (size_t)j * nr;
    double* xb = xbar + (size_t)j * nr;
    double* xbs = xbar + (size_t)(j - 1) * nr;
    double* xbn = xbar + (size_t)(j + 1) * nr;
    const double eta_s = z[j] - z[j - 1], eta_n = z[j + 1] - z[j];
    const double etabar = 0.5 * (eta_n + eta_s);
    /* rows of the line system */
    for (int i = 0; i <= N; i++) {
      if (i == 0) { a[i] = 0.0; b[i] = 1.0; c[i] = -1.0; continue; }
      if (i == N) {
        if (p->bc_rmax) { a[i] = 0.0; b[i] = 1.0; c[i] = 0.0; }
        else { a[i] = -1.0; b[i] = 1.0; c[i] = 0.0; }
        continue;
      }
      const double h_w = r[i] - r[i - 1], h_e = r[i + 1] - r[i];
      if (cls[i] == OR_IFACE) {
        double lm, lp;
        if (p->interface_rule == 0) {
          lm = lam_m(p, seg[i - 1], Tj[i]);
          lp = lam_m(p, seg[i], Tj[i]);
        } else {
          lm = 0.5 * (r[i] + r[i - 1]) * lam_face(p, seg[i - 1], Tj[i - 1], Tj[i]);
          lp = 0.5 * (r[i] + r[i + 1]) * lam_face(p, seg[i], Tj[i], Tj[i + 1]);
        }
        a[i] = -lm * h_e; b[i] = lm * h_e + lp * h_w; c[i] = -lp * h_w;
        continue;
      }
      const int m = seg[i];
      const double hbar = 0.5 * (h_e + h_w);
      const double r_w = 0.5 * (r[i] + r[i - 1]), r_e = 0.5 * (r[i] + r[i + 1]);
      const double lw = lam_face(p, m, Tj[i - 1], Tj[i]);
      const double le = lam_face(p, m, Tj[i], Tj[i + 1]);
      const double rc = p->rho[m] * cap_m(p, m, Tj[i]);
      a[i] = -r_w * lw / (r[i] * hbar * h_w);
      c[i] = -r_e * le / (r[i] * hbar * h_e);
      b[i] = (r_w * lw / h_w + r_e * le / h_e) / (r[i] * hbar) + rc / tau;
    }
    /* xi = M^{-T} mu_j: Thomas on the transposed rows (c_{i-1}, b_i, a_{i+1}) */
    cw[0] = a[1] / b[0];
    dw[0] = mj[0] / b[0];
    for (int i = 1; i <= N; i++) {
      const double sub = c[i - 1], sup = (i < N) ? a[i + 1] : 0.0;
      const double den = b[i] - sub * cw[i - 1];
      cw[i] = sup / den;
      dw[i] = (mj[i] - sub * dw[i - 1]) / den;
    }
    xi[N] = dw[N];
    for (int i = N - 1; i >= 0; i--) xi[i] = dw[i] - cw[i] * xi[i + 1];
    /* partial derivatives of the residuals */
    for (int i = 1; i <= N - 1; i++) {
      const double h_w = r[i] - r[i - 1], h_e = r[i + 1] - r[i];
      const double X = xi[i];
      if (X == 0.0) continue;
      if (cls[i] == OR_IFACE) {
        const int mi = seg[i - 1], mo = seg[i];
        const double gw = yj[i - 1] - yj[i], ge = yj[i + 1] - yj[i];
        if (p->interface_rule == 0) {
          /* r = lm h_e (y_{i-1} - y_i) + lp h_w (y_{i+1} - y_i) */
          xb[i] += X * (dlam_m(p, mi, Tj[i]) * h_e * gw + dlam_m(p, mo, Tj[i]) * h_w * ge);
          gbar[2 + mi] += X * lam_m(p, mi, Tj[i]) * h_e * gw / p->lam_scale[mi];
          gbar[2 + mo] += X * lam_m(p, mo, Tj[i]) * h_w * ge / p->lam_scale[mo];
        } else {
          const double rw = 0.5 * (r[i] + r[i - 1]), re = 0.5 * (r[i] + r[i + 1]);
          double l1, d1a, d1b, l2, d2a, d2b;
          lam_face_d(p, mi, Tj[i - 1], Tj[i], &l1, &d1a, &d1b);
          lam_face_d(p, mo, Tj[i], Tj[i + 1], &l2, &d2a, &d2b);
          xb[i - 1] += X * rw * d1a * h_e * gw;
          xb[i] += X * (rw * d1b * h_e * gw + re * d2a * h_w * ge);
          xb[i + 1] += X * re * d2b * h_w * ge;
          gbar[2 + mi] += X * rw * l1 * h_e * gw / p->lam_scale[mi];
          gbar[2 + mo] += X * re * l2 * h_w * ge / p->lam_scale[mo];
        }
        continue;
      }
      const int m = seg[i];
      const double hbar = 0.5 * (h_e + h_w);
      const double r_w = 0.5 * (r[i] + r[i - 1]), r_e = 0.5 * (r[i] + r[i + 1]);
      const double gA = r_w / (r[i] * hbar * h_w), gC = r_e / (r[i] * hbar * h_e);
      const double T0 = Tj[i];
      double lw, lw_a, lw_b, le, le_a, le_b, ls, ls_a, ls_b, ln, ln_a, ln_b;
      lam_face_d(p, m, Tj[i - 1], T0, &lw, &lw_a, &lw_b);
      lam_face_d(p, m, T0, Tj[i + 1], &le, &le_a, &le_b);
      lam_face_d(p, m, Ts[i], T0, &ls, &ls_a, &ls_b);
      lam_face_d(p, m, T0, Tn[i], &ln, &ln_a, &ln_b);
      const double rc = p->rho[m] * cap_m(p, m, T0);
      const double drc = p->rho[m] * dcap_m(p, m, T0);
      const double gw = yj[i - 1] - yj[i], ge = yj[i + 1] - yj[i];
      const double dN = Tn[i] - T0, dS = T0 - Ts[i];
      /* r = rc/tau (T0 - y_i) + (ln dN/eta_n - ls dS/eta_s)/etabar + X
       *     + gA lw (y_{i-1} - y_i) + gC le (y_{i+1} - y_i) */
      double d0 = drc / tau * (T0 - yj[i]) + rc / tau;
      d0 += (ln_a * dN - ln) / eta_n / etabar - (ls_b * dS + ls) / eta_s / etabar;
      d0 += gA * lw_b * gw + gC * le_a * ge;
      if (m == p->src_layer) d0 += p->q0 * s * src_dg(p, T0);
      xb[i] += X * d0;
      xb[i - 1] += X * gA * lw_a * gw;
      xb[i + 1] += X * gC * le_b * ge;
      xbn[i] += X * (ln_b * dN + ln) / eta_n / etabar;
      xbs[i] += X * (-ls_a * dS + ls) / eta_s / etabar;
      /* parameters */
      const double lam_part = (ln * dN / eta_n - ls * dS / eta_s) / etabar + gA * lw * gw + gC * le * ge;
      gbar[2 + m] += X * lam_part / p->lam_scale[m];
      gbar[2 + L + m] += X * rc / tau * (T0 - yj[i]) / p->cap_scale[m];
      if (m == p->src_layer) {
        gbar[0] += X * s * src_g(p, T0);
        gbar[1] += X * p->q0 * ds_dton * src_g(p, T0);
      }
    }
  }
  free(r); free(z); free(cls); free(seg); free(a); free(b); free(c); free(xi); free(cw); free(dw);
  return 0;
}

/*
 * Loss J = sum_n tau (Sbar_n - target_n)^2 over the n_steps steps from T0 at
 * t0 (Sbar_n: the z-mean surface temperature after step n, trace column 1 of
 * or_step_n), its gradient with respect to theta (grad[2 + 2 n_layers]) and,
 * if dT0 is not NULL, with respect to T0.  States are checkpointed every
 * ckpt steps and recomputed segment by segment in the reverse sweep.
 */
int or_adjoint(const or_problem* p, const double* T0, long n_steps, double t0, double tau,
               const double* target, int ckpt, double* loss, double* grad, double* dT0) {
  const int N = p->nr - 1, M = p->nz - 1, nr = p->nr, L = p->n_layers;
  const size_t nodes = (size_t)nr * (M + 1);
  if (ckpt < 1) ckpt = 1;
  const long n_ck = (n_steps + ckpt - 1) / ckpt;
  double* ck = (double*)malloc(sizeof(double) * nodes * (size_t)(n_ck > 0 ? n_ck : 1));
  double* seg_states = (double*)malloc(sizeof(double) * nodes * (size_t)(ckpt + 1));
  double* trace = (double*)malloc(sizeof(double) * 2 * (size_t)(n_steps > 0 ? n_steps : 1));
  double* lam = (double*)calloc(nodes, sizeof(double));
  double* lam2 = (double*)calloc(nodes, sizeof(double));
  double* w = (double*)malloc(sizeof(double) * (M + 1));
  double* r = (double*)malloc(sizeof(double) * (N + 1));
  double* z = (double*)malloc(sizeof(double) * (M + 1));
  int* cls = (int*)malloc(sizeof(int) * (N + 1));
  int* seg = (int*)malloc(sizeof(int) * (N + 1));
  int rc = -1;
  if (!ck || !seg_states || !trace || !lam || !lam2 || !w || !r || !z || !cls || !seg ||
      or_grid(p, r, z, cls, seg) || !rect_outline(p, z, cls))
    goto done;
  {
    double wsum = 0.0;
    for (int j = 0; j <= M; j++) {
      w[j] = 0.0;
      if (j > 0) w[j] += 0.5 * (z[j] - z[j - 1]);
      if (j < M) w[j] += 0.5 * (z[j + 1] - z[j]);
      wsum += w[j];
    }
    for (int j = 0; j <= M; j++) w[j] /= wsum;
  }
  /* forward sweep with checkpoints */
  memcpy(seg_states, T0, sizeof(double) * nodes);
  *loss = 0.0;
  for (long n = 0; n < n_steps; n++) {
    if (n % ckpt == 0) memcpy(ck + nodes * (size_t)(n / ckpt), seg_states, sizeof(double) * nodes);
    if (or_step_n(p, seg_states, 1, t0 + (double)n * tau, tau, trace + 2 * n, NULL)) goto done;
    const double e = trace[2 * n + 1] - target[n];
    *loss += tau * e * e;
  }
  for (int k = 0; k < 2 + 2 * L; k++) grad[k] = 0.0;
  /* reverse sweep */
  for (long k = n_ck - 1; k >= 0; k--) {
    const long n_lo = k * ckpt, n_hi = (n_lo + ckpt < n_steps) ? n_lo + ckpt : n_steps;
    memcpy(seg_states, ck + nodes * (size_t)k, sizeof(double) * nodes);
    for (long n = n_lo; n < n_hi; n++) {
      memcpy(seg_states + nodes * (size_t)(n - n_lo + 1), seg_states + nodes * (size_t)(n - n_lo),
             sizeof(double) * nodes);
      if (or_step_n(p, seg_states + nodes * (size_t)(n - n_lo + 1), 1, t0 + (double)n * tau, tau,
                    NULL, NULL))
        goto done;
    }
    for (long n = n_hi - 1; n >= n_lo; n--) {
      /* dJ/dT^{n+1} from the loss term of step n */
      const double e = trace[2 * n + 1] - target[n];
      for (int j = 0; j <= M; j++) lam[(size_t)j * nr + N] += 2.0 * tau * e * w[j];
      memset(lam2, 0, sizeof(double) * nodes);
      if (or_step_vjp(p, seg_states + nodes * (size_t)(n - n_lo), seg_states + nodes * (size_t)(n - n_lo + 1),
                      lam, t0 + (double)n * tau, tau, lam2, grad))
        goto done;
      double* t = lam; lam = lam2; lam2 = t;
    }
  }
  if (dT0) memcpy(dT0, lam, sizeof(double) * nodes);
  rc = 0;
done:
  free(ck); free(seg_states); free(trace); free(lam); free(lam2); free(w); free(r); free(z);
  free(cls); free(seg);
  return rc;
}
