// cc_step_n_noalloc: the FP64 time step for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code embedded in a framework whose
// allocator owns (and may have reserved) all device memory, real-time loops
// that forbid allocation after start-up, or hosts that hand the library only
// the buffers they own.  cc_step_n allocates its context tables and scratch
// lazily on the device, so this entry point instead keeps every piece of
// scratch it needs (instance tables, work list, waveform table, power-law
// tables, error word and the ping-pong partner of the caller's field) in one
// file-scope static device array of a fixed size.  That array is created when
// the library's device code is loaded on a GPU and stays held by every GPU
// that loads the library until the process exits.  The call allocates nothing, on the device or the host:
// host-side tables are staged in file-scope static buffers.  The grid,
// descriptor checks, stability guard and device tables come from the same host
// code as cc_step_n (ccell_grid.cpp), so both entry points run the same
// numerics; this one uses CTA tiles of 128 threads without block ranges.
//
// Device addresses: host code only sees a host-side stand-in for the static
// array's name, so the device address is fetched once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on
// the device.  Every call copies pageable host tables and waits for its own
// work, so no call of this entry point can be captured in a CUDA graph.
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

#include "ccell_host.h"

namespace {

using namespace ccell;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffInst = 0;
constexpr size_t kOffErr = align256(kOffInst + sizeof(DevInst));
constexpr size_t kOffRg = align256(kOffErr + sizeof(unsigned));
constexpr size_t kOffZg = align256(kOffRg + sizeof(RowGeo) * CC_NOALLOC_MAX_NR);
constexpr size_t kOffTile = align256(kOffZg + sizeof(ZGeo) * CC_NOALLOC_MAX_NZ);
constexpr size_t kOffS = align256(kOffTile + sizeof(TileTask) * CC_NOALLOC_MAX_NZ);
constexpr size_t kOffTab = align256(kOffS + sizeof(double) * CC_NOALLOC_MAX_STEPS);
constexpr size_t kOffT2 = align256(kOffTab + sizeof(double) * kPowTabLen * CC_MAX_LAYERS);
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
double h_tab[kPowTabLen * CC_MAX_LAYERS];
double h_r[CC_NOALLOC_MAX_NR], h_z[CC_NOALLOC_MAX_NZ];
int h_cls[CC_NOALLOC_MAX_NR], h_seg[CC_NOALLOC_MAX_NR];

int validate(const cc_geometry_desc& d, const cc_material* mat, const cc_source& s) {
  const int v = valid_desc(d);
  if (v != CC_OK) return v;
  if (d.nr > CC_NOALLOC_MAX_NR || d.nz > CC_NOALLOC_MAX_NZ ||
      (long long)d.nr * d.nz > CC_NOALLOC_MAX_NODES)
    return CC_EINVAL;
  if (d.precision != CC_FP64) return CC_EINVAL;
  if (d.step_layers != 0) return CC_EUNSUPPORTED;  // rectangles only
  for (int m = 0; m < d.n_layers; ++m)
    if (!valid_material(mat[m])) return CC_EINVAL;
  return valid_source(s, d.n_layers);
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

  build_grid(d, h_r, h_z, h_cls, h_seg);
  const int M = d.nz - 1;
  // stability guard, Eq. (stability_condition)
  {
    const char* force = std::getenv("CC_FORCE_UNSTABLE");
    if (dt_s > tau_stab_of(d, materials, h_z) * (1.0 + 1e-12) && !(force && force[0] == '1'))
      return CC_EUNSTABLE;
  }

  // tables
  fill_row_geo(h_r, h_cls, h_seg, d.nr, h_rg);
  fill_z_geo(h_z, d.nz, d.nz, h_zg);
  const int G = choose_lanes(d.nr);
  const int lpc = 4 * (32 / G);  // CTA tiles of the FP64 step: 4 warps, 128 threads
  int n_tiles = 0;
  for (int j0 = 1; j0 <= M - 1; j0 += lpc) h_tile[n_tiles++] = TileTask{0, j0, std::min(lpc, M - j0), 0};
  const int smem = fp64_tile_smem_bytes(std::min(lpc, M - 1), d.nr);

  fill_inst_scalars(d, *source, dt_s, G, d.nz, d.nr - 1, 0, h_cls, h_inst);
  h_inst.rg = reinterpret_cast<const RowGeo*>(base + kOffRg);
  h_inst.zg = reinterpret_cast<const ZGeo*>(base + kOffZg);
  const double* dtab = reinterpret_cast<const double*>(base + kOffTab);
  for (int m = 0; m < d.n_layers; ++m) {
    const cc_material& s = materials[m];
    DevMaterial& t = h_inst.mat[m];
    fold_material(s, dt_s, t);
    if (s.lam_model == 1) {  // the power-law table of cc_step_n
      const double lam0s = s.lam0 * s.lam_scale;
      if (build_pow_table(s.lam_b, lam0s * std::pow(2.0 * s.t_ref, -s.lam_b),
                          lam0s * std::pow(s.t_ref, -s.lam_b), h_tab + (size_t)m * kPowTabLen))
        t.ptab = dtab + (size_t)m * kPowTabLen;
    }
  }

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // pageable sources: each copy has consumed its host buffer when it returns
  if (cudaMemcpyAsync(base + kOffInst, &h_inst, sizeof h_inst, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + kOffRg, h_rg, sizeof(RowGeo) * d.nr, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + kOffZg, h_zg, sizeof(ZGeo) * d.nz, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + kOffTile, h_tile, sizeof(TileTask) * n_tiles, cudaMemcpyHostToDevice,
                      st) ||
      cudaMemcpyAsync(base + kOffTab, h_tab, sizeof(double) * kPowTabLen * d.n_layers,
                      cudaMemcpyHostToDevice, st) ||
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
