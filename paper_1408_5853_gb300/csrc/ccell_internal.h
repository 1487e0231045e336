// Internal layouts shared by the host side (ccell_api.cpp) and the kernels
// (ccell_step.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>

#include "../../include/ccell.h"

namespace ccell {

enum : int { RC_AXIS = 0, RC_REGULAR = 1, RC_IFACE = 2, RC_OUTER = 3, RC_OUTSIDE = 4 };

// Largest number of rows one lane eliminates sequentially; a line of nr rows
// is split over G lanes (G a power of two, G <= 32), so nr <= 32 * kRowsPerLane.
constexpr int kRowsPerLane = 16;
constexpr int kMaxNr = 32 * kRowsPerLane;

// Per radial node i of one instance (index i in [0, nr)).
struct RowGeo {
  double gA;   // r_{i-1/2} / (r_i hbar_i h_i)      (Eq. (ABC), coefficient of lambda_{i-1/2})
  double gC;   // r_{i+1/2} / (r_i hbar_i h_{i+1})  (coefficient of lambda_{i+1/2})
  double hw;   // h_i     = r_i - r_{i-1}
  double he;   // h_{i+1} = r_{i+1} - r_i
  double rw;   // r_{i-1/2}
  double re;   // r_{i+1/2}
  double V2;   // 2 pi r_i hbar_i (radial part of the control volume)
  float gA_f, gC_f, hw_f, he_f, rw_f, re_f, V2_f;  // FP32 copies (mixed precision)
  int cls;     // RC_*
  int seg;     // layer of the segment [r_i, r_{i+1}] (regular node: its layer)
  int segw;    // layer of the segment [r_{i-1}, r_i]
  int ifo;     // RC_IFACE / RC_OUTER: position of i in DevInst::if_i (else -1)
};

// Per axial node j (index j in [0, nz)).
struct ZGeo {
  double gzs;    // 1 / (etabar_j eta_j)
  double gzn;    // 1 / (etabar_j eta_{j+1})
  double etabar; // (eta_j + eta_{j+1}) / 2
  double wnorm;  // trapezoid weight of z_j divided by the sum of weights
  double eta_s;  // eta_j
  double eta_n;  // eta_{j+1}
  float gzs_f, gzn_f, etabar_f, pad_f;  // FP32 copies (mixed precision)
};

// Power-law tables: x^b = 2^(e b) * p_q(m - c_q) for x = m 2^e, m in [1, 2),
// with 2^kPowBits mantissa intervals q of centre c_q and degree-kPowDeg
// polynomials p_q; binary exponents e in [kPowEmin, kPowEmin + kPowNE).
constexpr int kPowBits = 8;
constexpr int kPowQ = 1 << kPowBits;
constexpr int kPowDeg = 4;
constexpr int kPowEmin = -2;
constexpr int kPowNE = 16;
// per layer: [face scale kPowNE][node scale kPowNE][kPowQ][kPowDeg + 1]
constexpr int kPowTabLen = 2 * kPowNE + kPowQ * (kPowDeg + 1);

// Material of one layer, with the user scales folded in.
struct DevMaterial {
  double rho;
  double lam0s;      // lam0 * lam_scale
  double lam_b;
  double inv_tref;
  double c0s;        // c0 * cap_scale
  double inv_theta;
  double lam_poly[5];  // * lam_scale
  double cap_poly[4];  // * cap_scale
  const double* ptab;  // power-law table (kPowTabLen doubles) or null: use pow()
  // rho c(T) / tau = rct_k T^3 / (1 + inv_theta3 T^3) (cap_model 1), rct_k
  // (cap_model 0), rho_tau * poly(T) (cap_model 2)
  double rct_k, inv_theta3, rho_tau;
  double inv_lam_scale, inv_cap_scale;  // adjoint: d/d scale = value / scale
  // FP32 copies (mixed precision)
  float rho_f, lam0s_f, lam_b_f, inv_tref_f, c0s_f, inv_theta_f;
  float lam_poly_f[5], cap_poly_f[4];
  int lam_model, cap_model;
};

// Row geometry of one instance in lane-major order for the warp-owned lines
// (launch mode 2): entry e = k G + l is row i = (l nr) / G + k, the k-th row
// of lane l, so the lanes of a group read consecutive entries.  meta packs
// the class (bits 0-3), the layer seg (bits 4-7) and the interface ordinal
// ifo + 1 (bits 8-15) of the row.
struct LaneGeo {
  double gA[kMaxNr], gC[kMaxNr], V2[kMaxNr];
  float gA_f[kMaxNr], gC_f[kMaxNr], V2_f[kMaxNr];
  int meta[kMaxNr];
};

struct DevInst {
  int nr, nz;            // nodes
  int G;                 // lanes per line
  int bc_rmax, bc_z0, bc_zmax;
  int face_rule, interface_rule;
  int src_layer, waveform, g_model;
  // stepped outline: the lines j >= j_narrow end at the radial node i_step
  // (class RC_OUTER there, RC_OUTSIDE beyond); a rectangle has j_narrow = nz
  int j_narrow, i_step;
  int pad0;
  int n_if;              // interface and r_max nodes (classes RC_IFACE, RC_OUTER) ...
  int if_i[CC_MAX_LAYERS];  // ... their radial indices, ascending
  long long t_off;       // element offset of this instance in T
  double t_d;            // Dirichlet temperature
  double tau, inv_tau;   // time step and its reciprocal
  double q0, t_period, t_on, t_start, edge_w, g_ref;
  float tau_f, inv_tau_f, q0_f, g_ref_f;  // FP32 copies (mixed precision)
  float td_hi, td_lo;    // Dirichlet temperature as an FP32 pair
  const RowGeo* rg;      // [nr]
  const ZGeo* zg;        // [nz]
  const LaneGeo* lg;     // lane-major rows for lanes G (launch mode 2), or null
  DevMaterial mat[CC_MAX_LAYERS];
};

// Class of radial node i on line j: the node's own class, except on the
// narrow lines of a stepped outline.
#ifdef __CUDACC__
__device__ __forceinline__ int line_class(const DevInst& I, int cls, int i, int j) {
  if (j >= I.j_narrow && i >= I.i_step) return i == I.i_step ? RC_OUTER : RC_OUTSIDE;
  return cls;
}
#endif

// One CTA's work in the FP64 step: nl consecutive lines starting at j0
// (nl <= warps per CTA x 32/G).
struct TileTask {
  int inst;
  int j0;
  int nl;
  int pad;
};

#ifdef __CUDACC__
#define CC_HOST_DEVICE __host__ __device__
#else
#define CC_HOST_DEVICE
#endif

// Shared-memory stride of one staged row of nr doubles: one pad double after
// every 16, so lanes reading rows 16 apart hit different banks.
CC_HOST_DEVICE inline int smem_row_stride(int nr) { return nr + (nr >> 4) + 1; }
CC_HOST_DEVICE inline int smem_col(int i) { return i + (i >> 4); }

// Shared memory of one FP64 CTA tile of nl lines: the four coefficient rows
// of every line's tridiagonal system and the heat capacities (nl padded rows
// each), two rows of axial face fluxes handed from one tile to the next, and
// four values per line and interface node.
CC_HOST_DEVICE inline int fp64_tile_smem_bytes(int nl, int nr) {
  return ((5 * nl + 2) * smem_row_stride(nr) + 4 * CC_MAX_LAYERS * nl) * (int)sizeof(double);
}
// Shared memory of one mixed-precision CTA tile: two rows of axial face
// fluxes handed from tile to tile (FP32), the four rows of every line's
// system (FP64), then in FP32 the heat capacities and kMixIf floats per line
// and interface node.
constexpr int kMixIf = 8;
CC_HOST_DEVICE inline int mixed_tile_smem_bytes(int nl, int nr) {
  return 4 * nl * smem_row_stride(nr) * (int)sizeof(double) +
         ((nl + 2) * smem_row_stride(nr) + kMixIf * CC_MAX_LAYERS * nl) * (int)sizeof(float);
}
// Warp-owned lines (launch mode 2): one padded row of a warp's shared memory
// holds the rows of all its lane groups' current lines (32/G lines of
// nr <= 16 G rows: at most 512 rows).  A warp's shared memory holds c', a',
// d' (then That), the energy factors and the south face fluxes carried from
// line to line, then four values per (lane group, interface node).
constexpr int kWarpRowStride = 512 + (512 >> 4) + 1;
CC_HOST_DEVICE inline int lines_warp_doubles(int if_slots) {
  return 5 * kWarpRowStride + 4 * if_slots;
}
// Row buffers of one tile of nl lines (the tile shared memory above without
// the two carry rows): doubles of an FP64 tile; floats of a mixed tile,
// rounded up to keep a following buffer's doubles aligned.
CC_HOST_DEVICE inline int fp64_buf_doubles(int nl, int nr) {
  return 5 * nl * smem_row_stride(nr) + 4 * CC_MAX_LAYERS * nl;
}
CC_HOST_DEVICE inline int mixed_buf_floats(int nl, int nr) {
  const int nrp = smem_row_stride(nr);
  return (8 * nl * nrp + nl * nrp + kMixIf * CC_MAX_LAYERS * nl + 1) & ~1;
}
// Floats of one packed mixed tile (float4 per node, then the interface
// values), a multiple of 4 so that a following buffer stays 16-byte aligned;
// and the carry rows ahead of the pipelined buffers, rounded the same way.
CC_HOST_DEVICE inline int mixed_packed_buf_floats(int nl, int nr) {
  return (4 * nl * smem_row_stride(nr) + kMixIf * CC_MAX_LAYERS * nl + 3) & ~3;
}
// Largest dynamic shared memory of an FP64 tile: the opt-in limit per block
// on sm_103 (227 KiB) less room for the kernels' static shared memory.
constexpr int kMaxTileSmem = 226 * 1024;

// Positions of the interface and r_max nodes in DevInst::if_i (RowGeo::ifo).
inline void number_ifaces(RowGeo* rg, int nr) {
  int n = 0;
  for (int i = 0; i < nr; ++i)
    rg[i].ifo = (rg[i].cls == RC_IFACE || rg[i].cls == RC_OUTER) ? n++ : -1;
}

// Everything one step launch needs.
struct StepArgs {
  const DevInst* insts;
  const TileTask* tiles; // FP64 step: CTA tiles
  int n_tiles;
  const int* cta_start;  // FP64 step: tiles [cta_start[b], cta_start[b+1]) of block b, or
                         // null (blocks stride over the tiles)
  int n_cta;             // blocks of the FP64 step launch when cta_start is set
  int smem_bytes;        // dynamic shared memory of the FP64 tile kernel
  int n_inst;
  const void* Tin;       // double* (FP64) or float* (mixed, high part)
  void* Tout;
  const float* lo_in;    // mixed: low-order part of the state (or null)
  float* lo_out;
  const double* s_tab;   // [n_steps][n_inst] waveform values
  long long step;        // step index within the call
  double* trace;         // [n_inst][n_steps][2] or null
  long long n_steps;
  double* energy;        // [n_inst][5] or null
  unsigned* err;         // error word: bit0 non-finite, bit1 barrier timeout
  // ADI variant, first half step (or null): rho c / tau, Lambda_j[T] and the
  // axial face conductivity lambda_{i,j+1/2} at the regular nodes, [node]
  double* adi_rct;
  double* adi_lj;
  double* adi_lamz;
  // launch shape
  int threads;           // threads per block (64, 128 or 256)
  int warp_doubles;      // warp-lines kernel: doubles of shared memory per warp
  // shared-memory-resident persistent launch: the field region starts
  // res_offset doubles into the dynamic shared memory; boundary rows are
  // exchanged through xb [block][2 step parities][first, last][nr] with
  // per-block step counters nbr_flags
  int res_offset;
  double* xb;
  unsigned* nbr_flags;
  // pipelined tiles (launch modes 4 and 5): elements (FP64: doubles, mixed: floats)
  // of one of the two row buffers after the two carry rows, and the number
  // of producer warps (the rest of the block's warps consume)
  int pipe_buf;
  int pipe_producers;
  int pipe_stores;       // mixed launch mode 5: the producers also store every tile
  // persistent launches: grid barrier state [count, generation], bounded wait
  unsigned* bar;
  unsigned bar_extra;    // extra arrivals expected (nonzero only to test the timeout)
  long long spin_limit;  // polls before a barrier wait gives up
};

// Reverse sweep of the adjoint (ccell_adjoint.cu).
#ifndef CC_ADJ_MAX_THREADS
#define CC_ADJ_MAX_THREADS 256
#endif
struct AdjArgs {
  const DevInst* insts;
  const TileTask* tiles;  // CTA tiles of lines (those of the step kernels)
  int n_tiles;
  int threads;            // block size the tiles were cut for
  int smem_bytes;         // >= 4 rows of nl x nrp doubles
  int n_inst;
  const double* x;       // T^n, all instances
  const double* y;       // T^{n+1}
  const double* lam;     // dJ/dT^{n+1} (without the seed of step n)
  double* lam_out;       // dJ/dT^n
  double* xi;            // M^{-T} mu, [node]
  // per node of the solved lines, from the tile kernel to the gather:
  // st[k * st_stride + node] = lambda_e, d lambda_e / dT_i, d lambda_e /
  // dT_{i+1} (face (i, i+1); zero at i = N), rho c / tau, d(rho c / tau)/dT
  double* st;
  long long st_stride;
  int gather_lines;      // lines per warp task of the gather (1..8)
  const double* seed;    // [n_inst][n_steps]: dJ/dSbar_n
  const double* s_tab;   // [n_steps][n_inst] waveform
  const double* ds_tab;  // [n_steps][n_inst] d waveform / d t_on
  long long step;
  long long n_steps;
  const long long* grad_off;  // per instance offset into grad
  double* grad;          // [sum_k (2 + 2 L_k)]
  const int* n_layers;   // per instance
};

// ADI variant, axial half step: one block of kAdiLanes threads per column of
// regular nodes, each thread a run of rows.
constexpr int kAdiLanes = 128;
struct AdiTask {
  int inst;
  int i;
};

struct AdiArgs {
  const DevInst* insts;
  int n_inst;
  const AdiTask* tasks;
  int n_tasks;
  int rows_max;          // rows per lane of the longest column segment
  int lines_max;         // largest nz - 2 over the instances
  const double* Tn;      // T^n, all instances
  double* Tx;            // T* in, T^{n+1} out
  const double* rct;     // rho c / (tau/2) at T^n, [node]
  const double* lj;      // Lambda_j[T^n], [node]
  const double* lamz;    // lambda_{i,j+1/2} at T^n, [node]
  double* scr;           // [3][n_tasks][rows_max][kAdiLanes]: c', a', d' of the column solves
  double* trace;         // [n_inst][n_steps][2] or null
  long long step;
  long long n_steps;
  unsigned* err;
};
int launch_adi_axial(const AdiArgs& a, void* stream);
int launch_adi_finish(const AdiArgs& a, void* stream);

// kernels (ccell_step.cu)
int launch_waveform(const DevInst* insts, int n_inst, long long n_steps, double t0,
                    double* s_tab, void* stream, double* ds_tab = nullptr);
// adjoint (ccell_adjoint.cu)
int launch_adj_tile(const AdjArgs& a, void* stream);
int launch_adj_gather(const AdjArgs& a, int max_nr, int max_nz, void* stream);
int launch_adj_seed(const DevInst* insts, int n_inst, const double* trace, const double* target,
                    long long n_steps, double* seed, double* loss, void* stream);
int launch_step_fp64(const StepArgs& a, void* stream);
// Resident blocks of the FP64 step kernels (all variants) for a block size and
// dynamic shared memory: the grid of launches with per-block tile ranges.
int fp64_resident_blocks(int threads, int smem);
int mixed_resident_blocks(int threads, int smem);
// The same for the persistent (cooperative) kernels.
int fp64_persistent_resident_blocks(int threads, int smem);
int mixed_persistent_resident_blocks(int threads, int smem);
int launch_step_mixed(const StepArgs& a, void* stream);
// n steps in one cooperative launch; buffers alternate Tin -> Tout -> Tin ...
// (and lo_in/lo_out for mixed).  Returns -3 if the grid cannot be co-resident.
int launch_steps_fp64_persistent(const StepArgs& a, long long n, void* stream);
int launch_steps_mixed_persistent(const StepArgs& a, long long n, void* stream);
int launch_mixed_init(float* lo, long long n_total, void* stream);
// FP64 step with warp-owned lines (ccell_step_lines.cu): a.tiles are warp
// tasks, a.cta_start[w] .. a.cta_start[w + 1] those of warp w, a.n_cta blocks.
int launch_step_fp64_lines(const StepArgs& a, void* stream);
int fp64_lines_resident_blocks(int threads, int smem);
// All n steps in one cooperative launch with the field resident in shared
// memory (ccell_step_resident.cu): block b holds the lines of its tiles
// [cta_start[b], cta_start[b+1]) of one instance; result in a.Tin.
int launch_steps_fp64_resident(const StepArgs& a, long long n, void* stream);
int fp64_resident_kernel_blocks(int threads, int smem);
// Pipelined CTA tiles, one launch per step (ccell_step_pipe.cu): the block's
// first a.pipe_producers warps assemble the rows of tile k+1 while the others
// solve and store tile k; a.tiles / a.cta_start / a.n_cta are the launch's
// tiles.
int launch_step_fp64_pipe(const StepArgs& a, void* stream);
int launch_step_mixed_pipe(const StepArgs& a, void* stream);
int fp64_pipe_resident_blocks(int threads, int smem);
int mixed_pipe_resident_blocks(int threads, int smem);
// Shared memory of the pipelined tiles: two carry rows and two row buffers
// (kCarryFloats: the mixed kernels' carry rows padded to 16 bytes).
constexpr int kCarryStride = kMaxNr + (kMaxNr >> 4) + 1;
constexpr int kCarryFloats = (2 * kCarryStride + 3) & ~3;
// The same for the mixed-precision step (ccell_step_lines_mixed.cu).
int launch_step_mixed_lines(const StepArgs& a, void* stream);
int mixed_lines_resident_blocks(int threads, int smem);
int launch_boundary_trace_zero(double* trace, long long n, void* stream);
long long kernel_launch_count();
// Host: fill one power-law table for exponent b and scales; returns false if
// the polynomial fit misses the accuracy bound (the kernel then calls pow).
bool build_pow_table(double b, double face_scale, double node_scale, double* tab);
void count_launch();

}  // namespace ccell
