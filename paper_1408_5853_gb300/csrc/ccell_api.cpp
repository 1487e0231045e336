// Host side of the C ABI declared in include/ccell.h: descriptor validation,
// the non-uniform grid of Eq. (uniform_grid), device tables, the stability
// guard of Eq. (stability_condition), and the launch sequence of cc_step_n.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ccell_host.h"

using namespace ccell;

namespace {

struct Instance {
  cc_geometry_desc d{};
  cc_material mat[CC_MAX_LAYERS]{};
  bool mat_set = false;
  cc_source src{};
  double dt = 0.0;
  std::vector<double> r, z;
  std::vector<int> cls, seg;
  int j_narrow = 0, i_step = 0;  // stepped outline (rectangle: nz, nr - 1)
  int G = 1;
  long long t_off = 0;
};

}  // namespace

struct cc_ctx {
  std::vector<Instance> inst;
  int precision = CC_FP64;
  long long total_nodes = 0;
  int failed = 0;  // sticky cc_status after a device failure
  // device state
  int device = -1;
  bool dirty = true;
  DevInst* d_inst = nullptr;
  RowGeo* d_rg = nullptr;
  ZGeo* d_zg = nullptr;
  TileTask* d_tiles = nullptr;
  int n_tiles = 0;
  size_t tiles_cap = 0;
  int smem_bytes = 0;
  int* d_cta = nullptr;       // FP64 step: first tile of each block (n_cta + 1)
  int n_cta = 0;
  size_t cta_cap = 0;
  // launch mode 2 (warp-owned lines): warp tasks and each warp's first task
  bool lines_ok = false;      // FP64 context of rectangles
  LaneGeo* d_lg = nullptr;    // lane-major rows per instance (mode 2)
  size_t lg_cap = 0;
  TileTask* d_wtasks = nullptr;
  int* d_wcta = nullptr;
  size_t wtasks_cap = 0, wcta_cap = 0;
  int lines_blocks = 0, lines_smem = 0, lines_warp_doubles = 0;
  // launch mode 3 (field resident in shared memory): per-block tiles,
  // boundary-row exchange buffer and step counters
  bool res_ok = false;
  TileTask* d_rtiles = nullptr;
  int* d_rcta = nullptr;
  size_t rtiles_cap = 0, rcta_cap = 0;
  double* d_xb = nullptr;
  size_t xb_cap = 0;
  unsigned* d_rflags = nullptr;
  size_t rflags_cap = 0;
  int res_blocks = 0, res_smem = 0, res_offset = 0;
  // launch modes 4 and 5 (pipelined tiles): tiles and blocks of the launch
  bool pipe_ok = false;
  TileTask* d_ptiles = nullptr;
  int* d_pcta = nullptr;
  size_t ptiles_cap = 0, pcta_cap = 0;
  int pipe_blocks = 0, pipe_smem = 0, pipe_buf = 0, pipe_producers = 0;
  void* d_T2 = nullptr;       // ping-pong partner of the caller's field
  float* d_lo = nullptr;      // mixed precision: low-order parts (two buffers)
  double* d_s = nullptr;      // waveform table
  double* d_ptab = nullptr;   // power-law tables [instance][layer][kPowTabLen]
  long long s_cap = 0;
  unsigned* d_err = nullptr;
  std::vector<double> uploaded_dt;
  // adjoint scratch, grown on demand
  double* d_adj = nullptr;
  size_t adj_cap = 0;
  // launch shape (modes as in cc_set_launch), threads per block, target rows
  // per lane (sets the lanes per line G); the default is set per precision
  // at creation
  int mode = 4, threads = 128, rows = kRowsPerLane;
  bool tasks_dirty = true;
  void* d_tune = nullptr;  // autotuner copy of the caller's field
  // ADI variant: column tasks and scratch, built on first use
  AdiTask* d_adi_tasks = nullptr;
  int n_adi_tasks = 0, adi_rows = 0;
  double* d_adi = nullptr;
  size_t adi_scratch = 0;
};

namespace {

double tau_stab(const Instance& in) { return tau_stab_of(in.d, in.mat, in.z.data()); }

// The grid of a valid descriptor into vectors sized here.
void grid_of(const cc_geometry_desc& d, std::vector<double>& r, std::vector<double>& z,
             std::vector<int>& cls, std::vector<int>& seg) {
  r.resize(d.nr);
  z.resize(d.nz);
  cls.resize(d.nr);
  seg.resize(d.nr);
  build_grid(d, r.data(), z.data(), cls.data(), seg.data());
}

bool force_unstable() {
  const char* v = std::getenv("CC_FORCE_UNSTABLE");
  return v && v[0] == '1';
}

void free_device(cc_ctx* c) {
  cudaFree(c->d_inst);
  cudaFree(c->d_rg);
  cudaFree(c->d_zg);
  cudaFree(c->d_tiles);
  c->d_tiles = nullptr;
  c->tiles_cap = 0;
  cudaFree(c->d_cta);
  c->d_cta = nullptr;
  c->cta_cap = 0;
  c->n_cta = 0;
  cudaFree(c->d_ptiles);
  cudaFree(c->d_pcta);
  c->d_ptiles = nullptr;
  c->d_pcta = nullptr;
  c->ptiles_cap = c->pcta_cap = 0;
  cudaFree(c->d_rtiles);
  cudaFree(c->d_rcta);
  cudaFree(c->d_xb);
  cudaFree(c->d_rflags);
  c->d_rtiles = nullptr;
  c->d_rcta = nullptr;
  c->d_xb = nullptr;
  c->d_rflags = nullptr;
  c->rtiles_cap = c->rcta_cap = c->xb_cap = c->rflags_cap = 0;
  cudaFree(c->d_lg);
  c->d_lg = nullptr;
  c->lg_cap = 0;
  cudaFree(c->d_wtasks);
  cudaFree(c->d_wcta);
  c->d_wtasks = nullptr;
  c->d_wcta = nullptr;
  c->wtasks_cap = c->wcta_cap = 0;
  cudaFree(c->d_T2);
  cudaFree(c->d_lo);
  cudaFree(c->d_s);
  cudaFree(c->d_ptab);
  cudaFree(c->d_err);
  cudaFree(c->d_adj);
  c->d_adj = nullptr;
  c->adj_cap = 0;
  cudaFree(c->d_tune);
  c->d_tune = nullptr;
  cudaFree(c->d_adi_tasks);
  c->d_adi_tasks = nullptr;
  c->n_adi_tasks = 0;
  cudaFree(c->d_adi);
  c->d_adi = nullptr;
  c->adi_scratch = 0;
  c->d_inst = nullptr;
  c->d_rg = nullptr;
  c->d_zg = nullptr;
  c->d_T2 = nullptr;
  c->d_lo = nullptr;
  c->d_s = nullptr;
  c->d_ptab = nullptr;
  c->d_err = nullptr;
  c->s_cap = 0;
}

// Allocate device memory (first use) and upload the per-instance tables.
// Lanes per line of every instance from the rows-per-lane policy; when the
// lines of all instances give fewer than kMinWarpTasks warp tasks (32/G
// lines each), use more lanes per line (fewer rows per lane) so that every
// SM sub-partition has work.
void choose_instance_lanes(std::vector<Instance>& inst, int rows_policy) {
  constexpr long long kMinWarpTasks = 2048;
  for (int rows = rows_policy;; rows /= 2) {
    long long warp_tasks = 0;
    for (Instance& in : inst) {
      in.G = choose_lanes(in.d.nr, rows);
      const int lpw = 32 / in.G;
      warp_tasks += (in.d.nz - 2 + lpw - 1) / lpw;
    }
    if (warp_tasks >= kMinWarpTasks || rows <= 4) break;
  }
}

// Lines per CTA tile of every instance, (threads / 32) warps x 32/G lines,
// halved until the tile fits in shared memory; returns the largest tile's
// shared memory (above kMaxTileSmem if even one line does not fit).
int tile_lines(const std::vector<Instance>& inst, int threads, int precision,
               std::vector<int>& lpcs) {
  lpcs.assign(inst.size(), 1);
  int smem = 0;
  for (size_t k = 0; k < inst.size(); ++k) {
    const Instance& in = inst[k];
    int lpc = (threads / 32) * (32 / in.G);
    auto tile_smem = [&](int nl) {
      return precision == CC_FP64 ? fp64_tile_smem_bytes(nl, in.d.nr)
                                  : mixed_tile_smem_bytes(nl, in.d.nr);
    };
    // fewer lines per tile (idle lanes) if the tile would not fit
    while (lpc > 1 && tile_smem(lpc) > kMaxTileSmem) lpc /= 2;
    lpcs[k] = lpc;
    smem = std::max(smem, tile_smem(std::min(lpc, in.d.nz - 2)));
  }
  return smem;
}

// CTA tiles of the step kernels: lines of one instance, at most lpcs[k] of
// them.  With B > 0 blocks, block b takes an equal share of all interior
// nodes as the consecutive tiles [cta[b], cta[b+1]); with B = 0 the tiles
// are cut per instance and the blocks stride over them (cta stays empty).
void cut_tiles(const std::vector<Instance>& inst, const std::vector<int>& lpcs, int B,
               std::vector<TileTask>& tiles, std::vector<int>& cta) {
  const int n = (int)inst.size();
  tiles.clear();
  cta.clear();
  long long total_nodes = 0;  // of the interior lines
  for (const Instance& in : inst) total_nodes += (long long)in.d.nr * (in.d.nz - 2);
  if (B > 0) {
    cta.assign(B + 1, 0);
    int k = 0, jn = 1;  // next line of instance k
    long long g = 0;
    for (int b = 0; b < B; ++b) {
      cta[b] = (int)tiles.size();
      const long long g_end = (long long)(b + 1) * total_nodes / B;
      while (g < g_end && k < n) {
        const Instance& in = inst[k];
        const int take = (int)std::min<long long>((g_end - g + in.d.nr - 1) / in.d.nr,
                                                  in.d.nz - 1 - jn);
        // the fewest tiles of at most lpcs lines, of sizes that differ by at
        // most one (no short last tile that leaves consumer warps idle)
        const int nt = (take + lpcs[k] - 1) / lpcs[k];
        for (int t = 0, j = jn; t < nt; ++t) {
          const int e = jn + (int)((long long)(t + 1) * take / nt);
          tiles.push_back(TileTask{k, j, e - j, 0});
          j = e;
        }
        jn += take;
        g += (long long)take * in.d.nr;
        if (jn > in.d.nz - 2) {
          ++k;
          jn = 1;
        }
      }
    }
    cta[B] = (int)tiles.size();
  } else {
    for (int k = 0; k < n; ++k)
      for (int j0 = 1; j0 <= inst[k].d.nz - 2; j0 += lpcs[k])
        tiles.push_back(TileTask{k, j0, std::min(lpcs[k], inst[k].d.nz - 1 - j0), 0});
  }
}

// Copy a host vector into a device buffer, growing it when needed.
template <class V>
int put_grown(V** dev, size_t* cap, const std::vector<V>& h) {
  if (h.size() > *cap) {
    cudaFree(*dev);
    *dev = nullptr;
    *cap = 0;
    if (cudaMalloc(dev, sizeof(V) * h.size()) != cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
    *cap = h.size();
  }
  if (!h.empty() && cudaMemcpy(*dev, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice) !=
                        cudaSuccess)
    return CC_ECUDA;
  return CC_OK;
}

// Warp tasks of launch mode 2: all interior lines cut into equal node shares,
// one per warp of the resident grid.
int cut_warp_tasks(cc_ctx* c) {
  c->lines_ok = true;
  int if_slots = 1;
  for (const Instance& in : c->inst) {
    if (in.j_narrow < in.d.nz) c->lines_ok = false;
    int n_if = 0;
    for (int i = 0; i < in.d.nr; ++i) n_if += (in.cls[i] == RC_IFACE || in.cls[i] == RC_OUTER);
    if_slots = std::max(if_slots, (32 / in.G) * n_if);
  }
  if (!c->lines_ok) return CC_OK;
  c->lines_warp_doubles = lines_warp_doubles(if_slots);
  c->lines_smem = (c->threads / 32) * c->lines_warp_doubles * (int)sizeof(double);
  if (c->lines_smem > kMaxTileSmem) {
    c->lines_ok = false;
    return CC_OK;
  }
  const int B = c->precision == CC_FP64 ? fp64_lines_resident_blocks(c->threads, c->lines_smem)
                                        : mixed_lines_resident_blocks(c->threads, c->lines_smem);
  if (B < 0) return CC_ECUDA;
  // lane-major row tables for the lanes of each instance
  std::vector<LaneGeo> lg(c->inst.size());
  for (size_t k = 0; k < c->inst.size(); ++k) {
    const Instance& in = c->inst[k];
    std::vector<RowGeo> rg(in.d.nr);
    fill_row_geo(in.r.data(), in.cls.data(), in.seg.data(), in.d.nr, rg.data());
    fill_lane_geo(rg.data(), in.d.nr, in.G, lg[k]);
  }
  {
    const int rc = put_grown(&c->d_lg, &c->lg_cap, lg);
    if (rc != CC_OK) return rc;
  }
  std::vector<int> whole(c->inst.size());
  for (size_t k = 0; k < c->inst.size(); ++k) whole[k] = c->inst[k].d.nz;
  std::vector<TileTask> tasks;
  std::vector<int> first;
  cut_tiles(c->inst, whole, B * (c->threads / 32), tasks, first);
  int rc = put_grown(&c->d_wtasks, &c->wtasks_cap, tasks);
  if (rc == CC_OK) rc = put_grown(&c->d_wcta, &c->wcta_cap, first);
  c->lines_blocks = B;
  return rc;
}

// Tiles of launch modes 4 and 5: as many lines per tile as the block's
// consumer warps solve at once (halved until two row buffers fit), one launch
// grid of resident blocks taking equal node shares.
int cut_pipe_tiles(cc_ctx* c) {
  c->pipe_ok = false;
  const bool mixed = c->precision == CC_MIXED;
  // producer / consumer warps as measured fastest on GB300: for the mixed
  // step about half producers (9 of 16 warps at 512 threads; with the stores
  // also on the producers, mode 5, 7/16 of the warps consume), for the FP64
  // step three quarters producers (at least one of each)
  const int warps = c->threads / 32;
  const int prod = std::max(
      1, std::min(warps - 1, !mixed ? (3 * warps) / 4
                             : c->mode == 5 ? warps - (7 * warps) / 16 : warps / 2 + warps / 16));
  const int cons = warps - prod;
  const int elem = mixed ? (int)sizeof(float) : (int)sizeof(double);
  std::vector<int> lpcs(c->inst.size());
  for (size_t k = 0; k < c->inst.size(); ++k) lpcs[k] = cons * (32 / c->inst[k].G);
  for (;;) {
    int buf = 0;
    for (size_t k = 0; k < c->inst.size(); ++k) {
      const Instance& in = c->inst[k];
      const int nl = std::min(lpcs[k], in.d.nz - 2);
      buf = std::max(buf, mixed ? mixed_packed_buf_floats(nl, in.d.nr)
                                : fp64_buf_doubles(nl, in.d.nr));
    }
    const int smem = ((mixed ? kCarryFloats : 2 * kCarryStride) + 2 * buf) * elem;
    if (smem > kMaxTileSmem) {
      bool halved = false;
      for (int& l : lpcs)
        if (l > 1) {
          l /= 2;
          halved = true;
        }
      if (!halved) return CC_OK;  // does not fit: mode 0 runs instead
      continue;
    }
    const int B = mixed ? mixed_pipe_resident_blocks(c->threads, smem)
                        : fp64_pipe_resident_blocks(c->threads, smem);
    if (B < 0) return CC_ECUDA;
    std::vector<TileTask> tiles;
    std::vector<int> cta;
    cut_tiles(c->inst, lpcs, B, tiles, cta);
    int rc = put_grown(&c->d_ptiles, &c->ptiles_cap, tiles);
    if (rc == CC_OK) rc = put_grown(&c->d_pcta, &c->pcta_cap, cta);
    if (rc != CC_OK) return rc;
    c->pipe_blocks = B;
    c->pipe_smem = smem;
    c->pipe_buf = buf;
    c->pipe_producers = prod;
    c->pipe_ok = true;
    return CC_OK;
  }
}

// Tiles of launch mode 3: one block per SM (at most one per interior line),
// each holding its run of lines of the single instance resident in shared
// memory next to the scratch of one tile; the tile size is halved until both
// fit.  Leaves res_ok false when the context does not qualify (several
// instances, a stepped outline, mixed precision) or the field does not fit.
int cut_resident_tiles(cc_ctx* c) {
  c->res_ok = false;
  if (c->inst.size() != 1 || c->precision != CC_FP64) return CC_OK;
  const Instance& in = c->inst[0];
  if (in.j_narrow < in.d.nz) return CC_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CC_ECUDA;
  const int lines = in.d.nz - 2, nr = in.d.nr, nrp = smem_row_stride(nr);
  const int B = std::min(sms, lines);
  for (int lpc = (c->threads / 32) * (32 / in.G); lpc >= 1; lpc /= 2) {
    std::vector<TileTask> tiles;
    std::vector<int> cta;
    cut_tiles(c->inst, std::vector<int>{lpc}, B, tiles, cta);
    int max_lines = 0;
    bool empty = false;
    for (int b = 0; b < B; ++b) {
      if (cta[b + 1] == cta[b]) {
        empty = true;
        break;
      }
      const TileTask& f = tiles[cta[b]];
      const TileTask& l = tiles[cta[b + 1] - 1];
      max_lines = std::max(max_lines, l.j0 + l.nl - f.j0);
    }
    if (empty) return CC_OK;
    const int tile = fp64_tile_smem_bytes(std::min(lpc, lines), nr);
    const int smem = tile + (max_lines + 2) * nrp * (int)sizeof(double);
    if (smem > kMaxTileSmem) continue;
    const int resident = fp64_resident_kernel_blocks(c->threads, smem);
    if (resident < 0) return CC_ECUDA;
    if (resident < B) continue;
    int rc = put_grown(&c->d_rtiles, &c->rtiles_cap, tiles);
    if (rc == CC_OK) rc = put_grown(&c->d_rcta, &c->rcta_cap, cta);
    if (rc != CC_OK) return rc;
    const size_t xb = (size_t)B * 4 * nr;
    if (xb > c->xb_cap) {
      cudaFree(c->d_xb);
      c->d_xb = nullptr;
      c->xb_cap = 0;
      if (cudaMalloc(&c->d_xb, sizeof(double) * xb) != cudaSuccess) {
        cudaGetLastError();
        return CC_ENOMEM;
      }
      c->xb_cap = xb;
    }
    if ((size_t)B > c->rflags_cap) {
      cudaFree(c->d_rflags);
      c->d_rflags = nullptr;
      c->rflags_cap = 0;
      if (cudaMalloc(&c->d_rflags, sizeof(unsigned) * B) != cudaSuccess) {
        cudaGetLastError();
        return CC_ENOMEM;
      }
      c->rflags_cap = B;
    }
    c->res_blocks = B;
    c->res_smem = smem;
    c->res_offset = tile / (int)sizeof(double);
    c->res_ok = true;
    return CC_OK;
  }
  return CC_OK;
}

int upload(cc_ctx* c, const std::vector<double>& dts, cudaStream_t st) {
  const int n = (int)c->inst.size();
  if (c->device < 0) {
    if (cudaGetDevice(&c->device) != cudaSuccess) return CC_ECUDA;
    size_t nrow = 0, nz = 0;
    for (auto& in : c->inst) {
      nrow += in.d.nr;
      nz += in.d.nz;
    }
    const size_t elem = c->precision == CC_FP64 ? sizeof(double) : sizeof(float);
    if (cudaMalloc(&c->d_inst, sizeof(DevInst) * n) != cudaSuccess ||
        cudaMalloc(&c->d_rg, sizeof(RowGeo) * nrow) != cudaSuccess ||
        cudaMalloc(&c->d_zg, sizeof(ZGeo) * nz) != cudaSuccess ||
        cudaMalloc(&c->d_T2, elem * c->total_nodes) != cudaSuccess ||
        cudaMalloc(&c->d_ptab, sizeof(double) * kPowTabLen * CC_MAX_LAYERS * n) != cudaSuccess ||
        cudaMalloc(&c->d_err, 4 * sizeof(unsigned)) != cudaSuccess) {
      free_device(c);
      c->device = -1;
      cudaGetLastError();
      return CC_ENOMEM;
    }
    if (c->precision == CC_MIXED &&
        cudaMalloc(&c->d_lo, 2 * sizeof(float) * c->total_nodes) != cudaSuccess) {
      free_device(c);
      c->device = -1;
      cudaGetLastError();
      return CC_ENOMEM;
    }
    if (cudaMemset(c->d_err, 0, 4 * sizeof(unsigned)) != cudaSuccess) return CC_ECUDA;
    // geometry tables (do not change after creation)
    std::vector<RowGeo> rg(nrow);
    std::vector<ZGeo> zg(nz);
    size_t ro = 0, zo = 0;
    for (auto& in : c->inst) {
      fill_row_geo(in.r.data(), in.cls.data(), in.seg.data(), in.d.nr, rg.data() + ro);
      fill_z_geo(in.z.data(), in.d.nz, in.j_narrow, zg.data() + zo);
      ro += in.d.nr;
      zo += in.d.nz;
    }
    if (cudaMemcpy(c->d_rg, rg.data(), sizeof(RowGeo) * rg.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(c->d_zg, zg.data(), sizeof(ZGeo) * zg.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return CC_ECUDA;
    c->dirty = true;
  } else {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) return CC_EINVAL;
  }
  if (c->tasks_dirty) {
    choose_instance_lanes(c->inst, c->rows);
    std::vector<int> lpcs;
    const int smem = tile_lines(c->inst, c->threads, c->precision, lpcs);
    // the grid of the launch mode in use: per-step or cooperative kernels
    const int B = smem > kMaxTileSmem ? 0
                  : c->precision == CC_FP64
                      ? (c->mode == 1 ? fp64_persistent_resident_blocks(c->threads, smem)
                                      : fp64_resident_blocks(c->threads, smem))
                      : (c->mode == 1 ? mixed_persistent_resident_blocks(c->threads, smem)
                                      : mixed_resident_blocks(c->threads, smem));
    if (B < 0) return CC_ECUDA;  // current device unreadable
    std::vector<TileTask> tiles;
    std::vector<int> cta;
    cut_tiles(c->inst, lpcs, B, tiles, cta);
    if (smem > kMaxTileSmem) return CC_EUNSUPPORTED;
    if (tiles.size() > c->tiles_cap) {
      cudaFree(c->d_tiles);
      c->d_tiles = nullptr;
      c->tiles_cap = 0;
      if (cudaMalloc(&c->d_tiles, sizeof(TileTask) * tiles.size()) != cudaSuccess) {
        cudaGetLastError();
        return CC_ENOMEM;
      }
      c->tiles_cap = tiles.size();
    }
    if (cudaMemcpy(c->d_tiles, tiles.data(), sizeof(TileTask) * tiles.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return CC_ECUDA;
    c->n_tiles = (int)tiles.size();
    c->n_cta = B;
    if (B > 0) {
      if ((size_t)(B + 1) > c->cta_cap) {
        cudaFree(c->d_cta);
        c->d_cta = nullptr;
        c->cta_cap = 0;
        if (cudaMalloc(&c->d_cta, sizeof(int) * (B + 1)) != cudaSuccess) {
          cudaGetLastError();
          return CC_ENOMEM;
        }
        c->cta_cap = B + 1;
      }
      if (cudaMemcpy(c->d_cta, cta.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess)
        return CC_ECUDA;
    }
    c->smem_bytes = smem;
    c->lines_ok = false;
    c->res_ok = false;
    if (c->mode == 2) {
      const int rc = cut_warp_tasks(c);
      if (rc != CC_OK) return rc;
    }
    if (c->mode == 3) {
      const int rc = cut_resident_tiles(c);
      if (rc != CC_OK) return rc;
    }
    c->pipe_ok = false;
    if (c->mode == 4 || c->mode == 5) {
      const int rc = cut_pipe_tiles(c);
      if (rc != CC_OK) return rc;
    }
    c->tasks_dirty = false;
    c->dirty = true;
  }
  if (!c->dirty && dts == c->uploaded_dt) return CC_OK;
  std::vector<DevInst> h(n);
  std::vector<double> ptab((size_t)kPowTabLen * CC_MAX_LAYERS * n, 0.0);
  size_t rofs = 0, zofs = 0;
  for (int k = 0; k < n; ++k) {
    const Instance& in = c->inst[k];
    DevInst& D = h[k];
    fill_inst_scalars(in.d, in.src, dts[k], in.G, in.j_narrow, in.i_step, in.t_off,
                      in.cls.data(), D);
    D.rg = c->d_rg + rofs;
    D.zg = c->d_zg + zofs;
    D.lg = (c->lines_ok && c->d_lg) ? c->d_lg + k : nullptr;
    rofs += in.d.nr;
    zofs += in.d.nz;
    for (int m = 0; m < in.d.n_layers; ++m) {
      const cc_material& s = in.mat[m];
      DevMaterial& t = D.mat[m];
      fold_material(s, dts[k], t);
      if (s.lam_model == 1) {
        const size_t ofs = ((size_t)k * CC_MAX_LAYERS + m) * kPowTabLen;
        const double lam0s = s.lam0 * s.lam_scale;
        if (build_pow_table(s.lam_b, lam0s * std::pow(2.0 * s.t_ref, -s.lam_b),
                            lam0s * std::pow(s.t_ref, -s.lam_b), ptab.data() + ofs))
          t.ptab = c->d_ptab + ofs;
      }
    }
  }
  if (cudaMemcpyAsync(c->d_ptab, ptab.data(), sizeof(double) * ptab.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->d_inst, h.data(), sizeof(DevInst) * n, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return CC_ECUDA;
  c->uploaded_dt = dts;
  c->dirty = false;
  return CC_OK;
}

}  // namespace

namespace {

// One time step with the per-step kernel of the context's launch mode: the
// pipelined tiles (modes 4 and 5), the warp-owned lines (mode 2) or the CTA tiles
// (modes 0, 1 and 3, and any mode whose tiles the context could not use).
int launch_one_step(const cc_ctx* c, const StepArgs& a, void* stream) {
  if ((c->mode == 4 || c->mode == 5) && c->pipe_ok) {
    StepArgs p = a;
    p.pipe_stores = c->mode == 5;
    p.tiles = c->d_ptiles;
    p.cta_start = c->d_pcta;
    p.n_cta = c->pipe_blocks;
    p.smem_bytes = c->pipe_smem;
    p.pipe_buf = c->pipe_buf;
    p.pipe_producers = c->pipe_producers;
    return c->precision == CC_FP64 ? launch_step_fp64_pipe(p, stream)
                                   : launch_step_mixed_pipe(p, stream);
  }
  if (c->mode == 2 && c->lines_ok) {
    StepArgs w = a;
    w.tiles = c->d_wtasks;
    w.cta_start = c->d_wcta;
    w.n_cta = c->lines_blocks;
    w.smem_bytes = c->lines_smem;
    w.warp_doubles = c->lines_warp_doubles;
    return c->precision == CC_FP64 ? launch_step_fp64_lines(w, stream)
                                   : launch_step_mixed_lines(w, stream);
  }
  return c->precision == CC_FP64 ? launch_step_fp64(a, stream) : launch_step_mixed(a, stream);
}

}  // namespace

extern "C" {

int cc_create_geometry(const cc_geometry_desc* desc, int32_t n_instances, cc_ctx** out) {
  if (!desc || !out || n_instances < 1) return CC_EINVAL;
  *out = nullptr;
  cc_ctx* c = new (std::nothrow) cc_ctx();
  if (!c) return CC_ENOMEM;
  c->precision = desc[0].precision;
  // default launch: pipelined tiles, the block size measured fastest for the
  // precision on GB300 (FP64: 3 producer + 1 consumer warps, three blocks per
  // SM; mixed: 9 + 7 warps, one block per SM)
  c->mode = 4;
  c->threads = c->precision == CC_FP64 ? 128 : 512;
  long long off = 0;
  for (int k = 0; k < n_instances; ++k) {
    const int v = valid_desc(desc[k]);
    if (v != CC_OK || desc[k].precision != c->precision) {
      delete c;
      return v != CC_OK ? v : CC_EINVAL;
    }
    Instance in;
    in.d = desc[k];
    grid_of(in.d, in.r, in.z, in.cls, in.seg);
    if (build_outline(in.d, in.z.data(), in.cls.data(), in.i_step, in.j_narrow) != CC_OK) {
      delete c;
      return CC_EINVAL;
    }
    in.G = choose_lanes(in.d.nr);
    in.t_off = off;
    in.src.layer = -1;
    off += (long long)in.d.nr * in.d.nz;
    c->inst.push_back(std::move(in));
  }
  c->total_nodes = off;
  *out = c;
  return CC_OK;
}

int cc_set_materials(cc_ctx* c, int32_t instance, const cc_material* m) {
  if (!c || !m) return CC_EINVAL;
  if (instance < -1 || instance >= (int)c->inst.size()) return CC_EINVAL;
  const int k0 = instance < 0 ? 0 : instance;
  const int k1 = instance < 0 ? (int)c->inst.size() : instance + 1;
  for (int k = k0; k < k1; ++k)
    for (int q = 0; q < c->inst[k].d.n_layers; ++q)
      if (!valid_material(m[q])) return CC_EINVAL;
  for (int k = k0; k < k1; ++k) {
    std::memcpy(c->inst[k].mat, m, sizeof(cc_material) * c->inst[k].d.n_layers);
    c->inst[k].mat_set = true;
  }
  c->dirty = true;
  return CC_OK;
}

int cc_set_source(cc_ctx* c, int32_t instance, const cc_source* s) {
  if (!c || !s) return CC_EINVAL;
  if (instance < -1 || instance >= (int)c->inst.size()) return CC_EINVAL;
  const int k0 = instance < 0 ? 0 : instance;
  const int k1 = instance < 0 ? (int)c->inst.size() : instance + 1;
  for (int k = k0; k < k1; ++k)
    if (valid_source(*s, c->inst[k].d.n_layers) != CC_OK) return CC_EINVAL;
  for (int k = k0; k < k1; ++k) c->inst[k].src = *s;
  c->dirty = true;
  return CC_OK;
}

int cc_set_dt(cc_ctx* c, int32_t instance, double dt) {
  if (!c || !(dt > 0.0) || !std::isfinite(dt)) return CC_EINVAL;
  if (instance < -1 || instance >= (int)c->inst.size()) return CC_EINVAL;
  for (int k = 0; k < (int)c->inst.size(); ++k)
    if (instance < 0 || k == instance) c->inst[k].dt = dt;
  return CC_OK;
}

int cc_tau_stab(const cc_ctx* c, int32_t instance, double* out) {
  if (!c || !out || instance < 0 || instance >= (int)c->inst.size()) return CC_EINVAL;
  if (!c->inst[instance].mat_set) return CC_ESTATE;
  *out = tau_stab(c->inst[instance]);
  return CC_OK;
}

int cc_step_n(cc_ctx* c, void* T_dev, int64_t n_steps, double t0, double dt_s, double* trace_dev,
              double* energy_dev, void* stream) {
  if (!c || !T_dev || n_steps < 0 || !std::isfinite(t0)) return CC_EINVAL;
  if (c->failed) return CC_ESTATE;
  if (n_steps == 0) return CC_OK;
  const int n = (int)c->inst.size();
  std::vector<double> dts(n);
  for (int k = 0; k < n; ++k) {
    Instance& in = c->inst[k];
    if (!in.mat_set) return CC_ESTATE;
    dts[k] = dt_s > 0.0 ? dt_s : in.dt;
    if (!(dts[k] > 0.0) || !std::isfinite(dts[k])) return CC_EINVAL;
    if (dts[k] > tau_stab(in) * (1.0 + 1e-12) && !force_unstable()) return CC_EUNSTABLE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = upload(c, dts, st);
  if (rc != CC_OK) return rc;
  if (c->s_cap < n_steps * n) {
    cudaFree(c->d_s);
    c->d_s = nullptr;
    c->s_cap = 0;
    if (cudaMalloc(&c->d_s, sizeof(double) * n_steps * n) != cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
    c->s_cap = n_steps * n;
  }
  if (launch_waveform(c->d_inst, n, n_steps, t0, c->d_s, stream)) return CC_ECUDA;
  if (trace_dev &&
      cudaMemsetAsync(trace_dev, 0, sizeof(double) * 2 * n_steps * n, st) != cudaSuccess)
    return CC_ECUDA;
  const size_t elem = c->precision == CC_FP64 ? sizeof(double) : sizeof(float);
  StepArgs a{};
  a.insts = c->d_inst;
  a.tiles = c->d_tiles;
  a.n_tiles = c->n_tiles;
  a.cta_start = c->n_cta > 0 ? c->d_cta : nullptr;
  a.n_cta = c->n_cta;
  a.smem_bytes = c->smem_bytes;
  a.n_inst = n;
  a.s_tab = c->d_s;
  a.trace = trace_dev;
  a.n_steps = n_steps;
  a.energy = energy_dev;
  a.err = c->d_err;
  a.threads = c->threads;
  a.bar = c->d_err + 1;
  a.bar_extra = 0;
  a.spin_limit = 1LL << 24;
  if (const char* v = std::getenv("CC_TEST_BARRIER_TIMEOUT")) {
    if (v[0] == '1') {  // test hook: a barrier that can never complete, short wait
      a.bar_extra = 1;
      a.spin_limit = 1LL << 12;
    }
  }
  void* bufs[2] = {T_dev, c->d_T2};
  if (c->precision == CC_MIXED) {
    if (launch_mixed_init(c->d_lo, c->total_nodes, stream))
      return CC_ECUDA;
  }
  bool done = false, in_place = false;
  if (c->mode == 3 && c->res_ok) {
    // all steps in one cooperative launch, field resident in shared memory;
    // the result is written back to T_dev
    if (cudaMemsetAsync(c->d_rflags, 0, sizeof(unsigned) * c->res_blocks, st) != cudaSuccess)
      return CC_ECUDA;
    StepArgs r = a;
    r.tiles = c->d_rtiles;
    r.cta_start = c->d_rcta;
    r.n_cta = c->res_blocks;
    r.smem_bytes = c->res_smem;
    r.res_offset = c->res_offset;
    r.xb = c->d_xb;
    r.nbr_flags = c->d_rflags;
    r.step = 0;
    r.Tin = T_dev;
    r.Tout = T_dev;
    const int rc = launch_steps_fp64_resident(r, n_steps, stream);
    if (rc == 0) done = in_place = true;
    else if (rc != -3) return CC_ECUDA;  // -3: not co-resident, use per-step launches
  }
  if (!done && c->mode == 1) {
    // all steps in one cooperative launch with a bounded grid barrier per step
    if (cudaMemsetAsync(a.bar, 0, sizeof(unsigned), st) != cudaSuccess) return CC_ECUDA;
    a.step = 0;
    a.Tin = T_dev;
    a.Tout = c->d_T2;
    a.lo_in = c->d_lo;
    a.lo_out = c->d_lo + c->total_nodes;
    const int r = c->precision == CC_FP64 ? launch_steps_fp64_persistent(a, n_steps, stream)
                                          : launch_steps_mixed_persistent(a, n_steps, stream);
    if (r == 0) done = true;
    else if (r != -3) return CC_ECUDA;  // -3: grid cannot be co-resident, use per-step launches
  }
  for (long long s = 0; !done && s < n_steps; ++s) {
    a.step = s;
    a.Tin = bufs[s & 1];
    a.Tout = bufs[(s + 1) & 1];
    if (c->precision == CC_MIXED) {
      a.lo_in = c->d_lo + (s & 1) * c->total_nodes;
      a.lo_out = c->d_lo + ((s + 1) & 1) * c->total_nodes;
    }
    const int r = launch_one_step(c, a, stream);
    if (r) return CC_ECUDA;
  }
  if ((n_steps & 1) && !in_place) {
    if (cudaMemcpyAsync(T_dev, c->d_T2, elem * c->total_nodes, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return CC_ECUDA;
  }
  return CC_OK;
}

int cc_step_adi_n(cc_ctx* c, void* T_dev, int64_t n_steps, double t0, double dt_s,
                  double* trace_dev, void* stream) {
  if (!c || !T_dev || n_steps < 0 || !std::isfinite(t0)) return CC_EINVAL;
  if (c->failed) return CC_ESTATE;
  if (c->precision != CC_FP64) return CC_EUNSUPPORTED;
  if (n_steps == 0) return CC_OK;
  const int n = (int)c->inst.size();
  std::vector<double> half(n);
  for (int k = 0; k < n; ++k) {
    Instance& in = c->inst[k];
    if (in.j_narrow < in.d.nz) return CC_EUNSUPPORTED;  // rectangles only
    if (!in.mat_set) return CC_ESTATE;
    const double dt = dt_s > 0.0 ? dt_s : in.dt;
    if (!(dt > 0.0) || !std::isfinite(dt)) return CC_EINVAL;
    half[k] = 0.5 * dt;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = upload(c, half, st);  // the tables fold rho / (dt/2)
  if (rc != CC_OK) return rc;
  if (!c->d_adi_tasks) {  // columns of regular nodes, one warp each
    std::vector<AdiTask> tasks;
    int rows = 0;
    for (int k = 0; k < n; ++k) {
      const Instance& in = c->inst[k];
      const int L = in.d.nz - 2;
      int S = kAdiLanes;  // segments of a column
      while (S > 1 && L < 2 * S) S >>= 1;
      rows = std::max(rows, (L + S - 1) / S);
      for (int i = 0; i < in.d.nr; ++i)
        if (in.cls[i] == RC_REGULAR) tasks.push_back(AdiTask{k, i});
    }
    if (cudaMalloc(&c->d_adi_tasks, sizeof(AdiTask) * std::max<size_t>(1, tasks.size())) !=
        cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
    if (!tasks.empty() &&
        cudaMemcpy(c->d_adi_tasks, tasks.data(), sizeof(AdiTask) * tasks.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return CC_ECUDA;
    c->n_adi_tasks = (int)tasks.size();
    c->adi_rows = rows;
  }
  const size_t nodes = (size_t)c->total_nodes;
  const size_t need = 3 * nodes + 3 * (size_t)c->n_adi_tasks * c->adi_rows * kAdiLanes;
  if (need > c->adi_scratch) {
    cudaFree(c->d_adi);
    c->d_adi = nullptr;
    c->adi_scratch = 0;
    if (cudaMalloc(&c->d_adi, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
    c->adi_scratch = need;
  }
  // waveform at the half steps; step m uses entry 2m, t_m = t0 + m dt
  const long long n_half = 2 * n_steps;
  if (c->s_cap < n_half * n) {
    cudaFree(c->d_s);
    c->d_s = nullptr;
    c->s_cap = 0;
    if (cudaMalloc(&c->d_s, sizeof(double) * n_half * n) != cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
    c->s_cap = n_half * n;
  }
  if (launch_waveform(c->d_inst, n, n_half, t0, c->d_s, stream)) return CC_ECUDA;
  if (trace_dev &&
      cudaMemsetAsync(trace_dev, 0, sizeof(double) * 2 * n_steps * n, st) != cudaSuccess)
    return CC_ECUDA;
  StepArgs a{};
  a.insts = c->d_inst;
  a.tiles = c->d_tiles;
  a.n_tiles = c->n_tiles;
  a.cta_start = c->n_cta > 0 ? c->d_cta : nullptr;
  a.n_cta = c->n_cta;
  a.smem_bytes = c->smem_bytes;
  a.n_inst = n;
  a.s_tab = c->d_s;
  a.n_steps = n_half;
  a.err = c->d_err;
  a.threads = c->threads;
  a.adi_rct = c->d_adi;
  a.adi_lj = c->d_adi + nodes;
  a.adi_lamz = c->d_adi + 2 * nodes;
  AdiArgs z{};
  z.insts = c->d_inst;
  z.n_inst = n;
  z.tasks = c->d_adi_tasks;
  z.n_tasks = c->n_adi_tasks;
  z.rows_max = c->adi_rows;
  for (int k = 0; k < n; ++k) z.lines_max = std::max(z.lines_max, c->inst[k].d.nz - 2);
  z.rct = a.adi_rct;
  z.lj = a.adi_lj;
  z.lamz = a.adi_lamz;
  z.scr = c->d_adi + 3 * nodes;
  z.trace = trace_dev;
  z.n_steps = n_steps;
  z.err = c->d_err;
  void* bufs[2] = {T_dev, c->d_T2};
  for (long long m = 0; m < n_steps; ++m) {
    // half step 1: the step of cc_step_n at dt/2, T^n -> T*
    a.step = 2 * m;
    a.Tin = bufs[m & 1];
    a.Tout = bufs[(m + 1) & 1];
    if (launch_step_fp64(a, stream)) return CC_ECUDA;
    // half step 2: columns along z, T* -> T^n+1 in place; then the rest
    z.Tn = static_cast<const double*>(bufs[m & 1]);
    z.Tx = static_cast<double*>(bufs[(m + 1) & 1]);
    z.step = m;
    if (launch_adi_axial(z, stream) || launch_adi_finish(z, stream)) return CC_ECUDA;
  }
  if (n_steps & 1) {
    if (cudaMemcpyAsync(T_dev, c->d_T2, sizeof(double) * nodes, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return CC_ECUDA;
  }
  return CC_OK;
}

int cc_set_launch(cc_ctx* c, int32_t mode, int32_t threads, int32_t rows_per_lane) {
  if (!c || mode < 0 || mode > 5 || (mode == 5 && c->precision != CC_MIXED) ||
      (threads != 64 && threads != 128 && threads != 256 && !(threads == 384 && mode >= 4) &&
       !(threads == 512 && mode >= 4 && c->precision == CC_MIXED)) ||
      rows_per_lane < 2 || rows_per_lane > kRowsPerLane)
    return CC_EINVAL;
  if (rows_per_lane != c->rows || threads != c->threads || mode != c->mode) c->tasks_dirty = true;
  c->mode = mode;
  c->threads = threads;
  c->rows = rows_per_lane;
  return CC_OK;
}

int cc_get_launch(const cc_ctx* c, int32_t* mode, int32_t* threads, int32_t* rows_per_lane) {
  if (!c) return CC_EINVAL;
  if (mode) *mode = c->mode;
  if (threads) *threads = c->threads;
  if (rows_per_lane) *rows_per_lane = c->rows;
  return CC_OK;
}

int cc_autotune(cc_ctx* c, void* T_dev, int32_t n_trial, float* best_ms, void* stream) {
  if (!c || !T_dev || n_trial < 1) return CC_EINVAL;
  if (c->failed) return CC_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t elem = c->precision == CC_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = elem * (size_t)c->total_nodes;
  if (!c->d_tune) {
    if (cudaMalloc(&c->d_tune, bytes) != cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
  }
  if (cudaMemcpyAsync(c->d_tune, T_dev, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return CC_ECUDA;
  // candidate lane policies: only those that change G for some instance
  std::vector<int> rows_opts = {kRowsPerLane};
  for (int r : {8, 4}) {
    bool differs = false;
    for (auto& in : c->inst) differs |= choose_lanes(in.d.nr, r) != choose_lanes(in.d.nr, kRowsPerLane);
    if (differs) rows_opts.push_back(r);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CC_ECUDA;
  float best = 1e30f;
  int bm = c->mode, bt = c->threads, br = c->rows;
  int rc = CC_OK;
  bool rect = true;
  for (auto& in : c->inst) rect &= in.j_narrow == in.d.nz;
  // mode 2: rectangles; mode 3: one FP64 rectangle (others fall back to mode 0)
  std::vector<int> modes = {0, 1, 4};
  if (c->precision == CC_MIXED) modes.push_back(5);
  if (rect) modes.push_back(2);
  if (rect && c->inst.size() == 1 && c->precision == CC_FP64) modes.push_back(3);
  for (int mode : modes)
    for (int threads : {64, 128, 256, 384, 512})
      for (int rows : rows_opts) {
        if (threads >= 384 && mode < 4) continue;
        if (threads == 512 && c->precision != CC_MIXED) continue;
        cc_set_launch(c, mode, threads, rows);
        rc = cc_step_n(c, T_dev, 1, 0.0, 0.0, nullptr, nullptr, stream);  // warm and upload
        if (rc != CC_OK) break;
        cudaEventRecord(e0, st);
        rc = cc_step_n(c, T_dev, n_trial, 0.0, 0.0, nullptr, nullptr, stream);
        cudaEventRecord(e1, st);
        if (rc != CC_OK || cudaEventSynchronize(e1) != cudaSuccess) {
          rc = rc != CC_OK ? rc : CC_ECUDA;
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)n_trial;
        if (ms < best) {
          best = ms;
          bm = mode;
          bt = threads;
          br = rows;
        }
        cudaMemcpyAsync(T_dev, c->d_tune, bytes, cudaMemcpyDeviceToDevice, st);
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cc_set_launch(c, bm, bt, br);
  cudaMemcpyAsync(T_dev, c->d_tune, bytes, cudaMemcpyDeviceToDevice, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return CC_ECUDA;
  if (best_ms) *best_ms = best;
  return rc == CC_OK ? cc_sync(c, stream) : rc;
}

int cc_sync(cc_ctx* c, void* stream) {
  if (!c) return CC_EINVAL;
  if (c->failed) return c->failed;
  if (c->device < 0) return CC_OK;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    c->failed = CC_ECUDA;
    return CC_ECUDA;
  }
  unsigned e = 0;
  if (cudaMemcpy(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess) {
    c->failed = CC_ECUDA;
    return CC_ECUDA;
  }
  if (e & 1u) {
    c->failed = CC_ENONFINITE;
    return CC_ENONFINITE;
  }
  if (e & 2u) {
    c->failed = CC_ETIMEOUT;
    return CC_ETIMEOUT;
  }
  return CC_OK;
}

}  // extern "C"

namespace {

// Reverse sweep shared by cc_adjoint and cc_adjoint_vjp.  If target is not
// null the seeds are 2 tau (Sbar_n - target_n) and the loss is written; else
// seed_in holds dJ/dSbar_n for every instance and step.
int adjoint_impl(cc_ctx* c, const void* T0_dev, int64_t n_steps, double t0, double dt_s,
                 const double* target, const double* seed_in, int32_t ckpt, double* loss_dev,
                 double* grad_dev, void* dT0_dev, void* stream) {
  if (!c || !T0_dev || !grad_dev || n_steps < 1 || !std::isfinite(t0)) return CC_EINVAL;
  if (c->failed) return CC_ESTATE;
  if (c->precision != CC_FP64) return CC_EUNSUPPORTED;
  const int n = (int)c->inst.size();
  std::vector<double> dts(n);
  for (int k = 0; k < n; ++k) {
    Instance& in = c->inst[k];
    if (in.j_narrow < in.d.nz) return CC_EUNSUPPORTED;  // rectangles only
    if (!in.mat_set) return CC_ESTATE;
    dts[k] = dt_s > 0.0 ? dt_s : in.dt;
    if (!(dts[k] > 0.0)) return CC_EINVAL;
    if (dts[k] > tau_stab(in) * (1.0 + 1e-12) && !force_unstable()) return CC_EUNSTABLE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = upload(c, dts, st);
  if (rc != CC_OK) return rc;
  const long long K = ckpt > 0 ? ckpt : 256;
  const long long n_ck = (n_steps + K - 1) / K;
  const size_t nodes = (size_t)c->total_nodes;
  int max_nr = 0, max_nz = 0;
  std::vector<long long> goff(n);
  std::vector<int> nl(n);
  long long gsum = 0;
  for (int k = 0; k < n; ++k) {
    max_nr = std::max(max_nr, c->inst[k].d.nr);
    max_nz = std::max(max_nz, c->inst[k].d.nz);
    goff[k] = gsum;
    nl[k] = c->inst[k].d.n_layers;
    gsum += 2 + 2 * nl[k];
  }
  // scratch layout (doubles): checkpoints, segment states, lam x2, xi, the
  // five per-node values the tile kernel hands to the gather, trace, seed,
  // s, ds, grad offsets and layer counts
  const size_t need = nodes * (size_t)(n_ck + K + 1 + 3 + 5) + (size_t)n * n_steps * 5 + 2 * (size_t)n + 8;
  if (c->adj_cap < need) {
    cudaFree(c->d_adj);
    c->d_adj = nullptr;
    c->adj_cap = 0;
    if (cudaMalloc(&c->d_adj, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return CC_ENOMEM;
    }
    c->adj_cap = need;
  }
  double* p = c->d_adj;
  double* ck = p; p += nodes * n_ck;
  double* segs = p; p += nodes * (K + 1);
  double* lamA = p; p += nodes;
  double* lamB = p; p += nodes;
  double* xi = p; p += nodes;
  double* hand = p; p += nodes * 5;
  double* trace = p; p += (size_t)n * n_steps * 2;
  double* seed = p; p += (size_t)n * n_steps;
  double* s_tab = p; p += (size_t)n * n_steps;
  double* ds_tab = p; p += (size_t)n * n_steps;
  long long* d_goff = reinterpret_cast<long long*>(p); p += n;
  int* d_nl = reinterpret_cast<int*>(p);
  if (cudaMemcpyAsync(d_goff, goff.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_nl, nl.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) ||
      cudaMemsetAsync(trace, 0, sizeof(double) * 2 * n * n_steps, st) ||
      cudaMemsetAsync(lamA, 0, sizeof(double) * nodes, st) ||
      cudaMemsetAsync(grad_dev, 0, sizeof(double) * gsum, st) ||
      cudaMemcpyAsync(segs + nodes * ((n_ck - 1) * K & 1), T0_dev, sizeof(double) * nodes,
                      cudaMemcpyDeviceToDevice, st))
    return CC_ECUDA;
  if (launch_waveform(c->d_inst, n, n_steps, t0, s_tab, stream, ds_tab)) return CC_ECUDA;
  StepArgs a{};
  a.insts = c->d_inst;
  a.tiles = c->d_tiles;
  a.n_tiles = c->n_tiles;
  a.cta_start = c->n_cta > 0 ? c->d_cta : nullptr;
  a.n_cta = c->n_cta;
  a.smem_bytes = c->smem_bytes;
  a.n_inst = n;
  a.s_tab = s_tab;
  a.n_steps = n_steps;
  a.err = c->d_err;
  a.threads = c->threads;
  // forward sweep with checkpoints: slots 0 and 1 of the segment buffer in
  // turn, arranged so that the last segment starts in slot 0 and keeps all
  // its states (it needs no recompute)
  const long long lo_last = (n_ck - 1) * K;
  auto slot = [&](long long s) { return s >= lo_last ? s - lo_last : (s + lo_last) & 1; };
  for (long long s = 0; s < n_steps; ++s) {
    double* cur = segs + nodes * slot(s);
    if (s % K == 0 && s < lo_last &&
        cudaMemcpyAsync(ck + nodes * (s / K), cur, sizeof(double) * nodes, cudaMemcpyDeviceToDevice,
                        st))
      return CC_ECUDA;
    a.step = s;
    a.Tin = cur;
    a.Tout = segs + nodes * slot(s + 1);
    a.trace = trace;
    if (launch_one_step(c, a, stream)) return CC_ECUDA;
  }
  if (target) {
    if (launch_adj_seed(c->d_inst, n, trace, target, n_steps, seed, loss_dev, stream))
      return CC_ECUDA;
  } else if (cudaMemcpyAsync(seed, seed_in, sizeof(double) * n * n_steps, cudaMemcpyDeviceToDevice,
                             st)) {
    return CC_ECUDA;
  }
  // reverse sweep, one checkpoint segment at a time
  AdjArgs b{};
  b.insts = c->d_inst;
  b.tiles = c->d_tiles;
  b.n_tiles = c->n_tiles;
  b.threads = c->threads;
  b.smem_bytes = c->smem_bytes;  // FP64 tiles: five rows and more per line
  b.n_inst = n;
  b.xi = xi;
  b.st = hand;
  b.st_stride = (long long)nodes;
  {
    // lines per gather warp: 8 (one extra axial face evaluation per 8 lines),
    // halved while the gather would not fill one 256-thread block per SM
    // (small grids: one 256 x 1024 instance takes 4, measured fastest)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return CC_ECUDA;
    int gl = 8;
    for (; gl > 1; gl /= 2) {
      const long long warps = (long long)((max_nr - 1 + 30) / 31) * ((max_nz + gl - 1) / gl);
      if (((warps + 7) / 8) * n >= (long long)sms) break;
    }
    b.gather_lines = gl;
  }
  b.seed = seed;
  b.s_tab = s_tab;
  b.ds_tab = ds_tab;
  b.n_steps = n_steps;
  b.grad_off = d_goff;
  b.grad = grad_dev;
  b.n_layers = d_nl;
  a.trace = nullptr;
  for (long long k = n_ck - 1; k >= 0; --k) {
    const long long lo = k * K, hi = std::min(lo + K, (long long)n_steps);
    for (long long s = lo; s < hi && k < n_ck - 1; ++s) {  // recompute the segment
      if (s == lo && cudaMemcpyAsync(segs, ck + nodes * k, sizeof(double) * nodes,
                                     cudaMemcpyDeviceToDevice, st))
        return CC_ECUDA;
      a.step = s;
      a.Tin = segs + nodes * (s - lo);
      a.Tout = segs + nodes * (s - lo + 1);
      if (launch_one_step(c, a, stream)) return CC_ECUDA;
    }
    for (long long s = hi - 1; s >= lo; --s) {
      b.step = s;
      b.x = segs + nodes * (s - lo);
      b.y = segs + nodes * (s - lo + 1);
      b.lam = lamA;
      b.lam_out = lamB;
      if (launch_adj_tile(b, stream) || launch_adj_gather(b, max_nr, max_nz, stream)) return CC_ECUDA;
      std::swap(lamA, lamB);
    }
  }
  if (dT0_dev &&
      cudaMemcpyAsync(dT0_dev, lamA, sizeof(double) * nodes, cudaMemcpyDeviceToDevice, st))
    return CC_ECUDA;
  return CC_OK;
}

}  // namespace

extern "C" {

int cc_adjoint(cc_ctx* c, const void* T0_dev, int64_t n_steps, double t0, double dt_s,
               const double* target_dev, int32_t ckpt_every, double* loss_dev, double* grad_dev,
               void* dT0_dev, void* stream) {
  if (!target_dev || !loss_dev) return CC_EINVAL;
  return adjoint_impl(c, T0_dev, n_steps, t0, dt_s, target_dev, nullptr, ckpt_every, loss_dev,
                      grad_dev, dT0_dev, stream);
}

int cc_adjoint_vjp(cc_ctx* c, const void* T0_dev, int64_t n_steps, double t0, double dt_s,
                   const double* seed_dev, int32_t ckpt_every, double* grad_dev, void* dT0_dev,
                   void* stream) {
  if (!seed_dev) return CC_EINVAL;
  return adjoint_impl(c, T0_dev, n_steps, t0, dt_s, nullptr, seed_dev, ckpt_every, nullptr,
                      grad_dev, dT0_dev, stream);
}

int cc_destroy(cc_ctx* c) {
  if (!c) return CC_OK;
  if (c->device >= 0) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) cudaSetDevice(c->device);
    free_device(c);
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
  }
  delete c;
  return CC_OK;
}

int cc_query_grid(const cc_geometry_desc* d, double* r, double* z, int32_t* rclass) {
  if (!d) return CC_EINVAL;
  const int v = valid_desc(*d);
  if (v != CC_OK) return v;
  std::vector<double> rr, zz;
  std::vector<int> cls, seg;
  grid_of(*d, rr, zz, cls, seg);
  if (r) std::memcpy(r, rr.data(), sizeof(double) * rr.size());
  if (z) std::memcpy(z, zz.data(), sizeof(double) * zz.size());
  if (rclass)
    for (size_t i = 0; i < cls.size(); ++i) rclass[i] = cls[i];
  return CC_OK;
}

int cc_query_tiles(const cc_geometry_desc* descs, int32_t n_instances, int32_t threads,
                   int32_t rows_per_lane, int32_t n_blocks, int32_t* tiles, int32_t max_tiles,
                   int32_t* n_tiles, int32_t* cta, int32_t* lanes, int32_t* smem_bytes) {
  if (!descs || n_instances < 1 || !n_tiles || n_blocks < 0 || max_tiles < 0 ||
      (threads != 64 && threads != 128 && threads != 256) || rows_per_lane < 2 ||
      rows_per_lane > kRowsPerLane)
    return CC_EINVAL;
  std::vector<Instance> inst(n_instances);
  for (int k = 0; k < n_instances; ++k) {
    const int v = valid_desc(descs[k]);
    if (v != CC_OK) return v;
    if (descs[k].precision != descs[0].precision) return CC_EINVAL;
    inst[k].d = descs[k];
  }
  choose_instance_lanes(inst, rows_per_lane);
  std::vector<int> lpcs, cv;
  std::vector<TileTask> tv;
  const int smem = tile_lines(inst, threads, descs[0].precision, lpcs);
  cut_tiles(inst, lpcs, n_blocks, tv, cv);
  *n_tiles = (int32_t)tv.size();
  if (tiles)
    for (size_t t = 0; t < tv.size() && (int)t < max_tiles; ++t) {
      tiles[3 * t] = tv[t].inst;
      tiles[3 * t + 1] = tv[t].j0;
      tiles[3 * t + 2] = tv[t].nl;
    }
  if (cta && n_blocks > 0)
    for (int b = 0; b <= n_blocks; ++b) cta[b] = cv[b];
  if (lanes)
    for (int k = 0; k < n_instances; ++k) lanes[k] = inst[k].G;
  if (smem_bytes) *smem_bytes = smem;
  return (int)tv.size() > max_tiles && tiles ? CC_EINVAL : CC_OK;
}

int cc_query_outline(const cc_geometry_desc* d, int32_t* i_step, int32_t* j_narrow) {
  if (!d || !i_step || !j_narrow) return CC_EINVAL;
  const int v = valid_desc(*d);
  if (v != CC_OK) return v;
  std::vector<double> rr, zz;
  std::vector<int> cls, seg;
  grid_of(*d, rr, zz, cls, seg);
  int is = 0, jn = 0;
  const int o = build_outline(*d, zz.data(), cls.data(), is, jn);
  if (o != CC_OK) return o;
  *i_step = is;
  *j_narrow = jn;
  return CC_OK;
}

const char* cc_status_string(int s) {
  switch (s) {
    case CC_OK: return "ok";
    case CC_EINVAL: return "invalid argument";
    case CC_ENOMEM: return "out of memory";
    case CC_ECUDA: return "CUDA error";
    case CC_EUNSTABLE: return "time step above the axial stability bound";
    case CC_ETIMEOUT: return "bounded device wait expired";
    case CC_ENONFINITE: return "non-finite temperature";
    case CC_ESTATE: return "context not configured or unusable after a failure";
    case CC_EUNSUPPORTED: return "not supported by this build";
    default: return "unknown status";
  }
}

int64_t cc_kernel_launches(void) { return kernel_launch_count(); }

}  // extern "C"
