// Host-side set-up shared by the entry points of the C ABI: descriptor checks,
// the grid of Eq. (uniform_grid) with a node on every layer border, the
// stepped outline of Section 2, the stability bound of Eq.
// (stability_condition), and the per-node and per-layer device tables.  No
// function here allocates: outputs go to caller-provided arrays, so the
// no-allocation entry point uses the same code as cc_step_n.
#include <cmath>
#include <cstring>

#include "ccell_host.h"

namespace ccell {

int valid_desc(const cc_geometry_desc& d) {
  if (d.n_layers < 1 || d.n_layers > CC_MAX_LAYERS) return CC_EINVAL;
  if (d.nr < 3 || d.nz < 3) return CC_EINVAL;
  if (d.nr > kMaxNr) return CC_EUNSUPPORTED;
  if (!(d.length_m > 0.0) || !std::isfinite(d.length_m)) return CC_EINVAL;
  for (int m = 0; m < d.n_layers; ++m)
    if (!(d.thickness_m[m] > 0.0) || !std::isfinite(d.thickness_m[m])) return CC_EINVAL;
  auto b01 = [](int v) { return v == 0 || v == 1; };
  if (!b01(d.bc_rmax) || !b01(d.bc_z0) || !b01(d.bc_zmax) || !b01(d.placement) ||
      !b01(d.precision) || !b01(d.face_rule) || !b01(d.interface_rule))
    return CC_EINVAL;
  if (d.placement == 1 && d.n_layers != 1) return CC_EINVAL;
  if (d.placement == 0 && d.nr - 1 < 2 * d.n_layers) return CC_EINVAL;
  if (!std::isfinite(d.t_dirichlet_K)) return CC_EINVAL;
  if (d.step_layers < 0 || d.step_layers >= d.n_layers) return CC_EINVAL;
  if (d.step_layers > 0 && (d.placement != 0 || !std::isfinite(d.z_step_m))) return CC_EINVAL;
  return CC_OK;
}

bool valid_material(const cc_material& m) {
  if (!(m.rho > 0.0) || !(m.lam_scale > 0.0) || !(m.cap_scale > 0.0)) return false;
  if (m.lam_model < 0 || m.lam_model > 2 || m.cap_model < 0 || m.cap_model > 2) return false;
  if (m.lam_model == 1 && !(m.t_ref > 0.0)) return false;
  if (m.cap_model == 1 && (!(m.t_ref > 0.0) || !(m.theta > 0.0))) return false;
  return true;
}

int valid_source(const cc_source& s, int n_layers) {
  if (s.layer < -1 || s.layer >= n_layers) return CC_EINVAL;
  if (s.layer >= 0) {
    if (!(s.t_period > 0.0) || !(s.t_on >= 0.0) || s.waveform < 0 || s.waveform > 2 ||
        s.g_model < 0 || s.g_model > 1 || !std::isfinite(s.q0))
      return CC_EINVAL;
    if (s.waveform >= 1 && !(s.edge_w > 0.0)) return CC_EINVAL;
  }
  return CC_OK;
}

void layer_cells(const cc_geometry_desc& d, int* n) {
  const int L = d.n_layers, N = d.nr - 1;
  double total = 0.0;
  for (int m = 0; m < L; ++m) total += d.thickness_m[m];
  double frac[CC_MAX_LAYERS];
  int assigned = 0;
  for (int m = 0; m < L; ++m) {
    const double share = (double)N * d.thickness_m[m] / total;
    const double fl = std::floor(share);
    n[m] = (int)fl;
    frac[m] = share - fl;
    if (n[m] < 2) n[m] = 2;
    assigned += n[m];
  }
  // layers by decreasing remainder, ties in layer order (stable insertion sort)
  int order[CC_MAX_LAYERS];
  for (int m = 0; m < L; ++m) {
    int k = m;
    while (k > 0 && frac[order[k - 1]] < frac[m]) {
      order[k] = order[k - 1];
      --k;
    }
    order[k] = m;
  }
  for (int k = 0; assigned < N; k = (k + 1) % L, ++assigned) n[order[k]]++;
  while (assigned > N) {  // minimum-count overflow: take from the largest layer
    int big = -1;
    for (int m = 0; m < L; ++m)
      if (n[m] > 2 && (big < 0 || n[m] > n[big])) big = m;
    n[big]--;
    assigned--;
  }
}

void build_grid(const cc_geometry_desc& d, double* r, double* z, int* cls, int* seg) {
  const int N = d.nr - 1, M = d.nz - 1;
  for (int i = 0; i <= N; ++i) {
    r[i] = 0.0;
    cls[i] = RC_REGULAR;
    seg[i] = 0;
  }
  for (int j = 0; j <= M; ++j) z[j] = 0.0;
  if (d.placement == 0) {
    int n[CC_MAX_LAYERS];
    layer_cells(d, n);
    int i = 0;
    double r0 = 0.0;
    for (int m = 0; m < d.n_layers; ++m) {
      const double h = d.thickness_m[m] / (double)n[m];
      for (int k = 0; k < n[m]; ++k, ++i) {
        r[i] = r0 + (double)k * h;
        seg[i] = m;
        if (k == 0 && m > 0) cls[i] = RC_IFACE;
      }
      r0 += d.thickness_m[m];
    }
    r[N] = r0;
    seg[N] = d.n_layers - 1;
    const double eta = d.length_m / (double)M;
    for (int j = 0; j <= M; ++j) z[j] = (double)j * eta;
  } else {
    // a Neumann face sits half a cell inside its outermost node
    const double hi_r = d.bc_rmax == CC_DIRICHLET ? 0.0 : 0.5;
    const double h = d.thickness_m[0] / ((double)N - 0.5 - hi_r);
    for (int i = 0; i <= N; ++i) r[i] = ((double)i - 0.5) * h;
    const double lo_z = d.bc_z0 == CC_DIRICHLET ? 0.0 : 0.5;
    const double hi_z = d.bc_zmax == CC_DIRICHLET ? 0.0 : 0.5;
    const double eta = d.length_m / ((double)M - lo_z - hi_z);
    for (int j = 0; j <= M; ++j) z[j] = ((double)j - lo_z) * eta;
  }
  cls[0] = RC_AXIS;
  cls[N] = RC_OUTER;
}

// The lines with z_j > z_step (a node on the step face counts as below it)
// keep only the step_layers innermost layers and end at the interface node
// that starts layer step_layers.  Line 1 must keep the full width.
int build_outline(const cc_geometry_desc& d, const double* z, const int* cls, int& i_step,
                  int& j_narrow) {
  const int N = d.nr - 1, M = d.nz - 1;
  i_step = N;
  j_narrow = d.nz;
  if (d.step_layers == 0) return CC_OK;
  int k = 0;
  for (int i = 1; i < N; ++i)
    if (cls[i] == RC_IFACE && ++k == d.step_layers) {
      i_step = i;
      break;
    }
  if (k != d.step_layers) return CC_EINVAL;
  const double zs = d.z_step_m + 1e-9 * d.length_m;
  for (int j = 0; j <= M; ++j)
    if (z[j] > zs) {
      j_narrow = j;
      break;
    }
  return j_narrow < 2 ? CC_EINVAL : CC_OK;
}

double lam_host(const cc_material& m, double T) {
  double v;
  if (m.lam_model == 0) v = m.lam0;
  else if (m.lam_model == 1) v = m.lam0 * std::pow(T / m.t_ref, m.lam_b);
  else {
    v = 0.0;
    for (int k = 4; k >= 0; --k) v = v * T + m.lam_poly[k];
  }
  return m.lam_scale * v;
}

double cap_host(const cc_material& m, double T) {
  double v;
  if (m.cap_model == 0) v = m.c0;
  else if (m.cap_model == 1) {
    const double x = T / m.t_ref, y = T / m.theta;
    v = m.c0 * x * x * x / (1.0 + y * y * y);
  } else {
    v = 0.0;
    for (int k = 3; k >= 0; --k) v = v * T + m.cap_poly[k];
  }
  return m.cap_scale * v;
}

double tau_stab_of(const cc_geometry_desc& d, const cc_material* mat, const double* z) {
  double eta2 = INFINITY;
  for (int j = 1; j < d.nz; ++j) {
    const double e = z[j] - z[j - 1];
    eta2 = std::fmin(eta2, e * e);
  }
  double lo = d.t_guard_lo_K, hi = d.t_guard_hi_K;
  if (!(hi > lo)) {
    lo = d.t_dirichlet_K;
    hi = 100.0;
  }
  double ratio = INFINITY;
  const int ns = 257;
  for (int m = 0; m < d.n_layers; ++m)
    for (int s = 0; s < ns; ++s) {
      const double T = lo + (hi - lo) * (double)s / (double)(ns - 1);
      const double q = mat[m].rho * cap_host(mat[m], T) / lam_host(mat[m], T);
      if (q < ratio) ratio = q;
    }
  return 0.5 * eta2 * ratio;
}

void fill_row_geo(const double* r, const int* cls, const int* seg, int nr, RowGeo* out) {
  const int N = nr - 1;
  for (int i = 0; i <= N; ++i) {
    RowGeo g{};
    g.cls = cls[i];
    g.seg = seg[i];
    g.segw = i > 0 ? seg[i - 1] : seg[0];
    if (i > 0 && i < N) {
      const double hw = r[i] - r[i - 1], he = r[i + 1] - r[i];
      const double hbar = 0.5 * (hw + he);
      const double rw = 0.5 * (r[i] + r[i - 1]), re = 0.5 * (r[i] + r[i + 1]);
      g.hw = hw;
      g.he = he;
      g.rw = rw;
      g.re = re;
      g.gA = rw / (r[i] * hbar * hw);
      g.gC = re / (r[i] * hbar * he);
      g.V2 = 2.0 * M_PI * r[i] * hbar;
    }
    g.gA_f = (float)g.gA;
    g.gC_f = (float)g.gC;
    g.hw_f = (float)g.hw;
    g.he_f = (float)g.he;
    g.rw_f = (float)g.rw;
    g.re_f = (float)g.re;
    g.V2_f = (float)g.V2;
    out[i] = g;
  }
  number_ifaces(out, nr);
}

void fill_lane_geo(const RowGeo* rg, int nr, int G, LaneGeo& out) {
  std::memset(&out, 0, sizeof out);
  int lg = 0;
  while ((1 << lg) < G) ++lg;
  for (int l = 0; l < G; ++l) {
    const int i_lo = (l * nr) >> lg, i_hi = ((l + 1) * nr) >> lg;
    for (int k = 0; k < i_hi - i_lo; ++k) {
      const RowGeo& g = rg[i_lo + k];
      const int e = k * G + l;
      out.gA[e] = g.gA;
      out.gC[e] = g.gC;
      out.V2[e] = g.V2;
      out.gA_f[e] = g.gA_f;
      out.gC_f[e] = g.gC_f;
      out.V2_f[e] = g.V2_f;
      out.meta[e] = (g.cls & 15) | ((g.seg & 15) << 4) | ((g.ifo + 1) << 8);
    }
  }
}

void fill_z_geo(const double* z, int nz, int j_narrow, ZGeo* out) {
  const int M = nz - 1;
  // trapezoid weights of the r = r_max surface (the full-width lines)
  double wsum = 0.0;
  for (int j = 0; j <= M; ++j) {
    double w = 0.0;
    if (j < j_narrow) {
      if (j > 0) w += 0.5 * (z[j] - z[j - 1]);
      if (j < M && j + 1 < j_narrow) w += 0.5 * (z[j + 1] - z[j]);
    }
    out[j] = ZGeo{};
    out[j].wnorm = w;
    wsum += w;
  }
  for (int j = 0; j <= M; ++j) {
    ZGeo& q = out[j];
    q.wnorm /= wsum;
    if (j > 0 && j < M) {
      const double es = z[j] - z[j - 1], en = z[j + 1] - z[j];
      const double eb = 0.5 * (es + en);
      q.eta_s = es;
      q.eta_n = en;
      q.etabar = eb;
      q.gzs = 1.0 / (eb * es);
      q.gzn = 1.0 / (eb * en);
    }
    q.gzs_f = (float)q.gzs;
    q.gzn_f = (float)q.gzn;
    q.etabar_f = (float)q.etabar;
  }
}

void fold_material(const cc_material& s, double tau, DevMaterial& t) {
  const double inv_tau = 1.0 / tau;
  t.rho = s.rho;
  t.lam_model = s.lam_model;
  t.cap_model = s.cap_model;
  t.lam0s = s.lam0 * s.lam_scale;
  t.inv_lam_scale = 1.0 / s.lam_scale;
  t.inv_cap_scale = 1.0 / s.cap_scale;
  t.lam_b = s.lam_b;
  t.inv_tref = 1.0 / s.t_ref;
  t.c0s = s.c0 * s.cap_scale;
  t.inv_theta = 1.0 / s.theta;
  for (int q = 0; q < 5; ++q) t.lam_poly[q] = s.lam_poly[q] * s.lam_scale;
  for (int q = 0; q < 4; ++q) t.cap_poly[q] = s.cap_poly[q] * s.cap_scale;
  const double rho_tau = s.rho * inv_tau;
  t.rho_tau = rho_tau;  // cap_poly already carries cap_scale
  t.inv_theta3 = 1.0 / (s.theta * s.theta * s.theta);
  t.rct_k = s.cap_model == 1 ? rho_tau * t.c0s / (s.t_ref * s.t_ref * s.t_ref)
                             : rho_tau * t.c0s;
  t.rho_f = (float)t.rho;
  t.lam0s_f = (float)t.lam0s;
  t.lam_b_f = (float)t.lam_b;
  t.inv_tref_f = (float)t.inv_tref;
  t.c0s_f = (float)t.c0s;
  t.inv_theta_f = (float)t.inv_theta;
  for (int q = 0; q < 5; ++q) t.lam_poly_f[q] = (float)t.lam_poly[q];
  for (int q = 0; q < 4; ++q) t.cap_poly_f[q] = (float)t.cap_poly[q];
  t.ptab = nullptr;
}

void fill_inst_scalars(const cc_geometry_desc& d, const cc_source& src, double tau, int G,
                       int j_narrow, int i_step, long long t_off, const int* cls,
                       DevInst& D) {
  std::memset(&D, 0, sizeof D);
  D.nr = d.nr;
  D.nz = d.nz;
  D.G = G;
  D.bc_rmax = d.bc_rmax;
  D.bc_z0 = d.bc_z0;
  D.bc_zmax = d.bc_zmax;
  D.face_rule = d.face_rule;
  D.interface_rule = d.interface_rule;
  D.src_layer = src.layer;
  D.waveform = src.waveform;
  D.g_model = src.g_model;
  D.j_narrow = j_narrow;
  D.i_step = i_step;
  D.t_off = t_off;
  D.t_d = d.t_dirichlet_K;
  D.tau = tau;
  D.inv_tau = 1.0 / tau;
  D.q0 = src.q0;
  D.t_period = src.t_period;
  D.t_on = src.t_on;
  D.t_start = src.t_start;
  D.edge_w = src.edge_w;
  D.g_ref = src.g_ref;
  D.tau_f = (float)D.tau;
  D.inv_tau_f = (float)D.inv_tau;
  D.q0_f = (float)D.q0;
  D.g_ref_f = (float)D.g_ref;
  D.td_hi = (float)D.t_d;
  D.td_lo = (float)(D.t_d - (double)D.td_hi);
  D.n_if = 0;  // interface and r_max nodes, ascending
  for (int i = 0; i < d.nr; ++i)
    if ((cls[i] == RC_IFACE || cls[i] == RC_OUTER) && D.n_if < CC_MAX_LAYERS) D.if_i[D.n_if++] = i;
}

int choose_lanes(int nr, int rows) {
  int G = 1;
  while (G < 32 && (nr + G - 1) / G > rows && nr >= 4 * G) G <<= 1;
  while ((nr + G - 1) / G > kRowsPerLane) G <<= 1;
  return G;
}

}  // namespace ccell
