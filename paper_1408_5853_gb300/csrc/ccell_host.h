// Host-side building blocks shared by every entry point that sets up a time
// step (cc_create_geometry / cc_step_n in ccell_api.cpp and the
// no-allocation entry point in ccell_noalloc.cu): descriptor checks, the grid
// of Eq. (uniform_grid), the stability bound of Eq. (stability_condition) and
// the device tables.  Nothing here allocates memory: every output goes to a
// caller-provided array.  Not part of the public ABI.
#pragma once

#include "ccell_internal.h"

namespace ccell {

// CC_OK or the status a descriptor / material / source is refused with.
int valid_desc(const cc_geometry_desc& d);
bool valid_material(const cc_material& m);
int valid_source(const cc_source& s, int n_layers);

// Radial cells per layer: proportional to thickness with the largest
// remainder method (ties to the lower layer), at least two per layer.
void layer_cells(const cc_geometry_desc& d, int* n);

// Node positions r[nr], z[nz], radial classes cls[nr] (RC_*) and the layer
// seg[nr] of the segment [r_i, r_{i+1}] of a valid descriptor.
void build_grid(const cc_geometry_desc& d, double* r, double* z, int* cls, int* seg);

// Stepped outline of Section 2 (see cc_geometry_desc): i_step, j_narrow.
int build_outline(const cc_geometry_desc& d, const double* z, const int* cls, int& i_step,
                  int& j_narrow);

// Material laws in plain host arithmetic (stability guard only).
double lam_host(const cc_material& m, double T);
double cap_host(const cc_material& m, double T);

// Eq. (stability_condition): (min_j eta_j^2 / 2) * min rho c / lambda over the
// layers and the guard range of d.
double tau_stab_of(const cc_geometry_desc& d, const cc_material* mat, const double* z);

// Per radial node tables of one instance (RowGeo::ifo numbered).
void fill_row_geo(const double* r, const int* cls, const int* seg, int nr, RowGeo* out);

// Lane-major copy of the row tables for G lanes per line (rows of lane l:
// [(l nr) / G, ((l+1) nr) / G)).
void fill_lane_geo(const RowGeo* rg, int nr, int G, LaneGeo& out);

// Per axial node tables; the surface-trace weights cover the lines j < j_narrow.
void fill_z_geo(const double* z, int nz, int j_narrow, ZGeo* out);

// Device constants of one layer at time step tau (ptab left null).
void fold_material(const cc_material& s, double tau, DevMaterial& t);

// Instance constants other than the tables' device pointers and materials.
void fill_inst_scalars(const cc_geometry_desc& d, const cc_source& src, double tau, int G,
                       int j_narrow, int i_step, long long t_off, const int* cls,
                       DevInst& D);

// Lanes per line: the smallest power of two giving at most `rows` rows per
// lane (rows <= kRowsPerLane), keeping at least two rows per lane.
int choose_lanes(int nr, int rows = kRowsPerLane);

}  // namespace ccell
