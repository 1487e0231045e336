// cc_step_n_noalloc: the FP64 time step for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code embedded in a framework whose
// allocator owns (and may have reserved) all device memory, real-time loops
// that forbid allocation after start-up, or hosts that hand the library only
// the buffers they own.  cc_step_n allocates its context tables and scratch
// lazily on the device, so this entry point instead keeps every piece of
// scratch it needs (instance tables, work list, waveform table, error word and
// the ping-pong partner of the caller's field) in one file-scope static device
// array of a fixed size.  That array is created when the library's device code
// is loaded on a GPU and stays held by every GPU that loads the library until
// the process exits.  The call allocates nothing, on the device or the host:
// host-side tables are staged in file-scope static buffers.
//
// Device addresses: host code only sees a host-side stand-in for the static
// array's name, so the device address is fetched once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on
// the device; make that first call before any stream capture.
//
// Sharing: every call uses the same array, which keeps the contents of the
// last call.  Calls whose work overlaps on the GPU (other streams, other host
// threads) race on it; serialise them.  The error word is cleared at the start
// of every call; the rest is rewritten before it is read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "ccell_internal.h"

namespace {

using namespace ccell;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffInst = 0;
constexpr size_t kOffErr = align256(kOffInst + sizeof(DevInst));
constexpr size_t kOffRg = align256(kOffErr + sizeof(unsigned));
constexpr size_t kOffZg = align256(kOffRg + sizeof(RowGeo) * CC_NOALLOC_MAX_NR);
constexpr size_t kOffTile = align256(kOffZg + sizeof(ZGeo) * CC_NOALLOC_MAX_NZ);
constexpr size_t kOffS = align256(kOffTile + sizeof(TileTask) * CC_NOALLOC_MAX_NZ);
constexpr size_t kOffT2 = align256(kOffS + sizeof(double) * CC_NOALLOC_MAX_STEPS);
constexpr size_t kScratchBytes = align256(kOffT2 + sizeof(double) * CC_NOALLOC_MAX_NODES);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;                        // guards the host staging below
unsigned char* g_dev_ptr[kMaxDevices];  // device address of the array, per device

// host staging of the tables (no heap use)
DevInst h_inst;
RowGeo h_rg[CC_NOALLOC_MAX_NR];
ZGeo h_zg[CC_NOALLOC_MAX_NZ];
TileTask h_tile[CC_NOALLOC_MAX_NZ];
double h_r[CC_NOALLOC_MAX_NR], h_z[CC_NOALLOC_MAX_NZ];
int h_cls[CC_NOALLOC_MAX_NR], h_seg[CC_NOALLOC_MAX_NR];

// Same grid rule as cc_create_geometry (cells per layer proportional to
// thickness, largest remainder with ties to the lower layer, >= 2 per layer).
void grid(const cc_geometry_desc& d) {
  const int N = d.nr - 1, M = d.nz - 1, L = d.n_layers;
  for (int i = 0; i <= N; ++i) {
    h_cls[i] = RC_REGULAR;
    h_seg[i] = 0;
  }
  if (d.placement == 0) {
    double total = 0.0, frac[CC_MAX_LAYERS];
    int n[CC_MAX_LAYERS], used[CC_MAX_LAYERS] = {0}, assigned = 0;
    for (int m = 0; m < L; ++m) total += d.thickness_m[m];
    for (int m = 0; m < L; ++m) {
      const double share = (double)N * d.thickness_m[m] / total;
      const double fl = std::floor(share);
      n[m] = (int)fl;
      frac[m] = share - fl;
      if (n[m] < 2) n[m] = 2;
      assigned += n[m];
    }
    while (assigned < N) {
      int best = -1;
      for (int m = 0; m < L; ++m)
        if (!used[m] && (best < 0 || frac[m] > frac[best])) best = m;
      if (best < 0) {
        std::memset(used, 0, sizeof used);
        continue;
      }
      used[best] = 1;
      n[best]++;
      assigned++;
    }
    while (assigned > N) {
      int big = -1;
      for (int m = 0; m < L; ++m)
        if (n[m] > 2 && (big < 0 || n[m] > n[big])) big = m;
      n[big]--;
      assigned--;
    }
    int i = 0;
    double r0 = 0.0;
    for (int m = 0; m < L; ++m) {
      const double h = d.thickness_m[m] / (double)n[m];
      for (int k = 0; k < n[m]; ++k, ++i) {
        h_r[i] = r0 + (double)k * h;
        h_seg[i] = m;
        if (k == 0 && m > 0) h_cls[i] = RC_IFACE;
      }
      r0 += d.thickness_m[m];
    }
    h_r[N] = r0;
    h_seg[N] = L - 1;
    const double eta = d.length_m / (double)M;
    for (int j = 0; j <= M; ++j) h_z[j] = (double)j * eta;
  } else {
    const double hi_r = d.bc_rmax == CC_DIRICHLET ? 0.0 : 0.5;
    const double h = d.thickness_m[0] / ((double)N - 0.5 - hi_r);
    for (int i = 0; i <= N; ++i) h_r[i] = ((double)i - 0.5) * h;
    const double lo_z = d.bc_z0 == CC_DIRICHLET ? 0.0 : 0.5;
    const double hi_z = d.bc_zmax == CC_DIRICHLET ? 0.0 : 0.5;
    const double eta = d.length_m / ((double)M - lo_z - hi_z);
    for (int j = 0; j <= M; ++j) h_z[j] = ((double)j - lo_z) * eta;
  }
  h_cls[0] = RC_AXIS;
  h_cls[N] = RC_OUTER;
}

double lam_h(const cc_material& m, double T) {
  double v = m.lam0;
  if (m.lam_model == 1) v = m.lam0 * std::pow(T / m.t_ref, m.lam_b);
  if (m.lam_model == 2) {
    v = 0.0;
    for (int k = 4; k >= 0; --k) v = v * T + m.lam_poly[k];
  }
  return m.lam_scale * v;
}

double cap_h(const cc_material& m, double T) {
  double v = m.c0;
  if (m.cap_model == 1) {
    const double x = T / m.t_ref, y = T / m.theta;
    v = m.c0 * x * x * x / (1.0 + y * y * y);
  }
  if (m.cap_model == 2) {
    v = 0.0;
    for (int k = 3; k >= 0; --k) v = v * T + m.cap_poly[k];
  }
  return m.cap_scale * v;
}

bool ok01(int v) { return v == 0 || v == 1; }

int validate(const cc_geometry_desc& d, const cc_material* mat, const cc_source& s) {
  if (d.n_layers < 1 || d.n_layers > CC_MAX_LAYERS || d.nr < 3 || d.nz < 3) return CC_EINVAL;
  if (d.nr > CC_NOALLOC_MAX_NR || d.nz > CC_NOALLOC_MAX_NZ ||
      (long long)d.nr * d.nz > CC_NOALLOC_MAX_NODES)
    return CC_EINVAL;
  if (d.precision != CC_FP64 || !ok01(d.bc_rmax) || !ok01(d.bc_z0) || !ok01(d.bc_zmax) ||
      !ok01(d.placement) || !ok01(d.face_rule) || !ok01(d.interface_rule))
    return CC_EINVAL;
  if (d.placement == 1 && d.n_layers != 1) return CC_EINVAL;
  if (d.step_layers != 0) return CC_EUNSUPPORTED;  // rectangles only
  if (d.placement == 0 && d.nr - 1 < 2 * d.n_layers) return CC_EINVAL;
  if (!(d.length_m > 0.0) || !std::isfinite(d.t_dirichlet_K)) return CC_EINVAL;
  for (int m = 0; m < d.n_layers; ++m) {
    if (!(d.thickness_m[m] > 0.0)) return CC_EINVAL;
    const cc_material& q = mat[m];
    if (!(q.rho > 0.0) || !(q.lam_scale > 0.0) || !(q.cap_scale > 0.0) || q.lam_model < 0 ||
        q.lam_model > 2 || q.cap_model < 0 || q.cap_model > 2)
      return CC_EINVAL;
    if ((q.lam_model == 1 || q.cap_model == 1) && !(q.t_ref > 0.0)) return CC_EINVAL;
    if (q.cap_model == 1 && !(q.theta > 0.0)) return CC_EINVAL;
  }
  if (s.layer < -1 || s.layer >= d.n_layers) return CC_EINVAL;
  if (s.layer >= 0 && (!(s.t_period > 0.0) || !(s.t_on >= 0.0) || s.waveform < 0 ||
                       s.waveform > 1 || s.g_model < 0 || s.g_model > 1 ||
                       (s.waveform == 1 && !(s.edge_w > 0.0))))
    return CC_EINVAL;
  return CC_OK;
}

}  // namespace

extern "C" int cc_step_n_noalloc(const cc_geometry_desc* desc, const cc_material* materials,
                                 const cc_source* source, double* T_dev, int64_t n_steps,
                                 double t0_s, double dt_s, double* trace_dev, double* energy_dev,
                                 void* stream) {
  if (!desc || !materials || !source || !T_dev || n_steps < 0 || !std::isfinite(t0_s) ||
      !(dt_s > 0.0) || !std::isfinite(dt_s))
    return CC_EINVAL;
  if (n_steps > CC_NOALLOC_MAX_STEPS) return CC_EINVAL;
  const cc_geometry_desc& d = *desc;
  int rc = validate(d, materials, *source);
  if (rc != CC_OK) return rc;
  if (n_steps == 0) return CC_OK;

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CC_ECUDA;
  if (!g_dev_ptr[dev]) {  // once per device, with that device current
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CC_ECUDA;
    }
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* base = g_dev_ptr[dev];

  grid(d);
  const int N = d.nr - 1, M = d.nz - 1;
  // stability guard, Eq. (stability_condition)
  {
    double eta2 = INFINITY, ratio = INFINITY;
    for (int j = 1; j <= M; ++j) eta2 = std::fmin(eta2, (h_z[j] - h_z[j - 1]) * (h_z[j] - h_z[j - 1]));
    double lo = d.t_guard_lo_K, hi = d.t_guard_hi_K;
    if (!(hi > lo)) {
      lo = d.t_dirichlet_K;
      hi = 100.0;
    }
    for (int m = 0; m < d.n_layers; ++m)
      for (int s = 0; s < 257; ++s) {
        const double T = lo + (hi - lo) * (double)s / 256.0;
        ratio = std::fmin(ratio, materials[m].rho * cap_h(materials[m], T) / lam_h(materials[m], T));
      }
    const char* force = std::getenv("CC_FORCE_UNSTABLE");
    if (dt_s > 0.5 * eta2 * ratio * (1.0 + 1e-12) && !(force && force[0] == '1'))
      return CC_EUNSTABLE;
  }

  // tables
  for (int i = 0; i <= N; ++i) {
    RowGeo g{};
    g.cls = h_cls[i];
    g.seg = h_seg[i];
    g.segw = i > 0 ? h_seg[i - 1] : h_seg[0];
    if (i > 0 && i < N) {
      const double hw = h_r[i] - h_r[i - 1], he = h_r[i + 1] - h_r[i];
      const double hbar = 0.5 * (hw + he);
      const double rw = 0.5 * (h_r[i] + h_r[i - 1]), re = 0.5 * (h_r[i] + h_r[i + 1]);
      g.hw = hw;
      g.he = he;
      g.rw = rw;
      g.re = re;
      g.gA = rw / (h_r[i] * hbar * hw);
      g.gC = re / (h_r[i] * hbar * he);
      g.V2 = 2.0 * M_PI * h_r[i] * hbar;
    }
    h_rg[i] = g;
  }
  number_ifaces(h_rg, d.nr);
  double wsum = 0.0;
  for (int j = 0; j <= M; ++j) {
    double w = 0.0;
    if (j > 0) w += 0.5 * (h_z[j] - h_z[j - 1]);
    if (j < M) w += 0.5 * (h_z[j + 1] - h_z[j]);
    h_zg[j] = ZGeo{};
    h_zg[j].wnorm = w;
    wsum += w;
  }
  for (int j = 0; j <= M; ++j) {
    h_zg[j].wnorm /= wsum;
    if (j > 0 && j < M) {
      const double es = h_z[j] - h_z[j - 1], en = h_z[j + 1] - h_z[j];
      const double eb = 0.5 * (es + en);
      h_zg[j].eta_s = es;
      h_zg[j].eta_n = en;
      h_zg[j].etabar = eb;
      h_zg[j].gzs = 1.0 / (eb * es);
      h_zg[j].gzn = 1.0 / (eb * en);
    }
  }
  int G = 1;
  while (G < 32 && (d.nr + G - 1) / G > kRowsPerLane) G <<= 1;
  const int lpc = 4 * (32 / G);  // CTA tiles of the FP64 step: 4 warps, 128 threads
  int n_tiles = 0;
  for (int j0 = 1; j0 <= M - 1; j0 += lpc) h_tile[n_tiles++] = TileTask{0, j0, std::min(lpc, M - j0), 0};
  const int smem = fp64_tile_smem_bytes(std::min(lpc, M - 1), d.nr);

  std::memset(&h_inst, 0, sizeof h_inst);
  h_inst.nr = d.nr;
  h_inst.nz = d.nz;
  h_inst.G = G;
  h_inst.bc_rmax = d.bc_rmax;
  h_inst.bc_z0 = d.bc_z0;
  h_inst.bc_zmax = d.bc_zmax;
  h_inst.face_rule = d.face_rule;
  h_inst.interface_rule = d.interface_rule;
  h_inst.src_layer = source->layer;
  h_inst.waveform = source->waveform;
  h_inst.g_model = source->g_model;
  h_inst.j_narrow = d.nz;  // rectangle
  h_inst.i_step = d.nr - 1;
  h_inst.t_d = d.t_dirichlet_K;
  h_inst.tau = dt_s;
  h_inst.inv_tau = 1.0 / dt_s;
  h_inst.q0 = source->q0;
  h_inst.t_period = source->t_period;
  h_inst.t_on = source->t_on;
  h_inst.t_start = source->t_start;
  h_inst.edge_w = source->edge_w;
  h_inst.g_ref = source->g_ref;
  fill_iface_list(h_rg, d.nr, h_inst);
  h_inst.rg = reinterpret_cast<const RowGeo*>(base + kOffRg);
  h_inst.zg = reinterpret_cast<const ZGeo*>(base + kOffZg);
  for (int m = 0; m < d.n_layers; ++m) {
    const cc_material& s = materials[m];
    DevMaterial& t = h_inst.mat[m];
    t.rho = s.rho;
    t.lam_model = s.lam_model;
    t.cap_model = s.cap_model;
    t.lam0s = s.lam0 * s.lam_scale;
    t.lam_b = s.lam_b;
    t.inv_tref = 1.0 / s.t_ref;
    t.c0s = s.c0 * s.cap_scale;
    t.inv_theta = 1.0 / s.theta;
    for (int q = 0; q < 5; ++q) t.lam_poly[q] = s.lam_poly[q] * s.lam_scale;
    for (int q = 0; q < 4; ++q) t.cap_poly[q] = s.cap_poly[q] * s.cap_scale;
    const double rho_tau = s.rho / dt_s;
    t.rho_tau = rho_tau;
    t.inv_theta3 = 1.0 / (s.theta * s.theta * s.theta);
    t.rct_k = s.cap_model == 1 ? rho_tau * t.c0s / (s.t_ref * s.t_ref * s.t_ref) : rho_tau * t.c0s;
  }

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // pageable sources: each copy has consumed its host buffer when it returns
  if (cudaMemcpyAsync(base + kOffInst, &h_inst, sizeof h_inst, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + kOffRg, h_rg, sizeof(RowGeo) * d.nr, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + kOffZg, h_zg, sizeof(ZGeo) * d.nz, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + kOffTile, h_tile, sizeof(TileTask) * n_tiles, cudaMemcpyHostToDevice,
                      st) ||
      cudaMemsetAsync(base + kOffErr, 0, sizeof(unsigned), st))
    return CC_ECUDA;
  if (trace_dev && cudaMemsetAsync(trace_dev, 0, sizeof(double) * 2 * n_steps, st))
    return CC_ECUDA;

  const DevInst* dinst = reinterpret_cast<const DevInst*>(base + kOffInst);
  double* s_tab = reinterpret_cast<double*>(base + kOffS);
  double* T2 = reinterpret_cast<double*>(base + kOffT2);
  if (launch_waveform(dinst, 1, n_steps, t0_s, s_tab, stream)) return CC_ECUDA;
  StepArgs a{};
  a.insts = dinst;
  a.tiles = reinterpret_cast<const TileTask*>(base + kOffTile);
  a.n_tiles = n_tiles;
  a.smem_bytes = smem;
  a.threads = 128;
  a.n_inst = 1;
  a.s_tab = s_tab;
  a.trace = trace_dev;
  a.n_steps = n_steps;
  a.energy = energy_dev;
  a.err = reinterpret_cast<unsigned*>(base + kOffErr);
  void* bufs[2] = {T_dev, T2};
  for (long long s = 0; s < n_steps; ++s) {
    a.step = s;
    a.Tin = bufs[s & 1];
    a.Tout = bufs[(s + 1) & 1];
    if (launch_step_fp64(a, stream)) return CC_ECUDA;
  }
  const size_t bytes = sizeof(double) * (size_t)d.nr * d.nz;
  if ((n_steps & 1) && cudaMemcpyAsync(T_dev, T2, bytes, cudaMemcpyDeviceToDevice, st))
    return CC_ECUDA;
  // report a non-finite temperature before the scratch is reused
  unsigned err = 0;
  if (cudaMemcpyAsync(&err, base + kOffErr, sizeof err, cudaMemcpyDeviceToHost, st) ||
      cudaStreamSynchronize(st))
    return CC_ECUDA;
  return (err & 1u) ? CC_ENONFINITE : CC_OK;
}
