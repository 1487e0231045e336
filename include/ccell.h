/*
 * ccell.h -- C ABI of the GB300 solver for the explicit-implicit
 * finite-difference heat-conduction scheme of Ayriyan, Busa, Donets,
 * Grigorian, Pribis, "Algorithm and Simulation of Heat Conduction Process for
 * Design of a Thin Multilayer Technical Device" (arXiv:1408.5853).
 *
 * The solver advances the temperature T(r, z, t) of a multilayer
 * axisymmetric cylinder (Section 2, Eqs. (equation)-(sch)) with the scheme of
 * Section 3: every time step evaluates the temperature-dependent
 * conductivity and heat capacity, applies the explicit axial operator
 * Lambda_j (Eq. (Lambda_j)), and solves the implicit radial operator Lambda_i
 * (Eq. (Lambda_i)) as one tridiagonal system per axial line j (Eqs.
 * (front_sweep)-(back_sweep)) with the layer-interface rows of Eqs.
 * (cc_first_1)-(cc_first_3) and the closures of Eqs.
 * (first_oder_bc)-(T_ini_for_back_sweep); the periodic source enters through
 * Eqs. (source)-(period).
 *
 * Conventions for every entry point:
 *  - Return value: CC_OK (0) or a negative cc_status.  Nothing throws across
 *    the ABI, nothing calls exit/abort, no kernel traps.
 *  - Ownership: the caller owns every buffer it passes; descriptors are
 *    copied during the call.  The context owns its device tables and scratch
 *    memory and releases them in cc_destroy.
 *  - Device pointers ("_dev") are CUDA device addresses on the current device
 *    of the calling thread; host pointers are plain CPU memory.
 *  - Streams: all device work of a call is enqueued on the given CUDA stream
 *    (NULL = legacy default stream).  A context is not thread-safe; calls on
 *    one context must be serialised by the caller.
 *  - Asynchronous kernel failures (a CUDA error, a non-finite temperature)
 *    are reported by the next call that synchronises (cc_step_n with a host
 *    trace/energy, cc_sync, cc_adjoint); the context then refuses further
 *    work with CC_ESTATE until destroyed.
 *
 * Field layout: an instance with nr radial and nz axial nodes stores
 * T[j * nr + i] (i = 0..nr-1 radial, contiguous; j = 0..nz-1 axial), so one
 * axial line j is one contiguous row.  Instances are concatenated in the
 * order of cc_create_geometry.  Temperatures are in kelvin.
 */
#ifndef CCELL_H
#define CCELL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_ctx cc_ctx; /* opaque, owned by the library */

typedef enum {
  CC_OK = 0,
  CC_EINVAL = -1,        /* invalid argument or descriptor                   */
  CC_ENOMEM = -2,        /* host or device allocation failed                 */
  CC_ECUDA = -3,         /* a CUDA runtime call or kernel failed             */
  CC_EUNSTABLE = -4,     /* dt above the axial stability bound, Eq. (stability_condition) */
  CC_ETIMEOUT = -5,      /* a bounded device wait expired                    */
  CC_ENONFINITE = -6,    /* a non-finite temperature was produced            */
  CC_ESTATE = -7,        /* context unusable after an earlier failure, or not configured */
  CC_EUNSUPPORTED = -8   /* valid request this build does not implement      */
} cc_status;

#define CC_MAX_LAYERS 8

enum { CC_NEUMANN = 0, CC_DIRICHLET = 1 };
enum { CC_FP64 = 0, CC_MIXED = 1 };

/*
 * Geometry of one instance (Section 2; grid of Eq. (uniform_grid)).
 * Layers are listed from the axis outwards; radial nodes are placed
 * uniformly inside each layer with a node exactly on every layer border
 * (cells per layer proportional to thickness, largest remainder, at least
 * 2 per layer, ties to the lower layer); axial nodes are uniform.
 *   bc_*        boundary condition of the face r = r_max, z = 0, z = z_max
 *               (paper default, Eq. (boundcond): Neumann, Neumann,
 *               Dirichlet); the axis r = 0 is always a symmetry line.
 *   placement   0: nodes on the boundaries (paper).  1: a Neumann face lies
 *               half a cell inside its outermost node (second-order
 *               closures; single layer only; used for analytic checks).
 *   precision   CC_FP64: state, properties, stencil and elimination in
 *               FP64; T is double.  CC_MIXED: T is float; properties and the
 *               explicit stencil run in FP32, the tridiagonal elimination and
 *               the energy sums in FP64.
 *   face_rule   0: lambda_{i+1/2} = lambda((T_i + T_i+1)/2)  (reading of the
 *               face rule printed with Eq. (Lambda_j)); 1: mean of the nodal
 *               lambda values.
 *   interface_rule  0: Eq. (cc_first_3) with lambda* at the old interface
 *               temperature; 1: same row with the r-weighted face
 *               conductivities (conserves energy exactly).
 *   t_guard_lo_K, t_guard_hi_K  temperature range over which the stability
 *               guard minimises rho c / lambda (0, 0 = [t_dirichlet, 100 K]).
 *   step_layers, z_step_m  stepped outline r in [0, r_max(z)] of Section 2
 *               (the paper's cell has its outer layers on z in [0, z_0]
 *               only, Section 5).  0: rectangle.  k in [1, n_layers): the
 *               lines with z_j > z_step_m (a line on the step face counts
 *               as below it) hold only the k innermost layers; their outer
 *               node is the interface node that starts layer k and takes
 *               the r_max condition bc_rmax; no heat crosses the step face
 *               (Eq. (boundcond)); the nodes outside the domain keep their
 *               values and must be finite.  Vertex placement only; line 1
 *               must keep the full width (else CC_EINVAL).  The surface
 *               trace averages over the full-width lines (r = r_max).
 *               cc_step_adi_n and the adjoint take rectangles only
 *               (CC_EUNSUPPORTED).
 */
typedef struct {
  int32_t n_layers;
  double thickness_m[CC_MAX_LAYERS];
  int32_t nr, nz;
  double length_m;
  int32_t bc_rmax, bc_z0, bc_zmax;
  double t_dirichlet_K;
  int32_t placement;
  int32_t precision;
  int32_t face_rule;
  int32_t interface_rule;
  double t_guard_lo_K, t_guard_hi_K;
  int32_t step_layers;
  double z_step_m;
} cc_geometry_desc;

/*
 * Material of one layer (Section 5 models and the power-law workloads):
 *   lambda(T) = lam_scale * { lam0                      (lam_model 0)
 *                           { lam0 (T / t_ref)^lam_b    (lam_model 1)
 *                           { sum_k lam_poly[k] T^k     (lam_model 2, Eq. (poly_cond))
 *   c(T)      = cap_scale * { c0                        (cap_model 0)
 *                           { c0 (T/t_ref)^3 / (1 + (T/theta)^3)  (cap_model 1)
 *                           { sum_k cap_poly[k] T^k     (cap_model 2, Eq. (poly_cap))
 * rho is the constant density.  SI units (W/m/K, J/kg/K, kg/m^3).
 */
typedef struct {
  double rho;
  int32_t lam_model;
  double lam0, lam_b;
  int32_t cap_model;
  double c0, theta, t_ref;
  double lam_scale, cap_scale;
  double lam_poly[5];
  double cap_poly[4];
} cc_material;

/*
 * Heating source, Eqs. (source)-(period): X = q0 s(t) g(T) at the regular
 * nodes of layer `layer` (interface nodes carry no source).
 *   waveform 0: s = nu(t), 1 on [t_start + n t_period, ... + t_on), else 0.
 *   waveform 1: s = (tanh(phi/w) - tanh((phi - t_on)/w)) / 2 around the
 *               nearest pulse (phase phi), w = edge_w.
 *   waveform 2: s = nu(t) p^2(t), the transient turn-on of Section 3.1,
 *               Eq. (transient_function) with the exponent read as negative:
 *               p^2 = 1 - exp(-phi / (7 tau*)) for phase phi < tau, else 1,
 *               with tau = edge_w and tau* = tau / 100.  The paper advances
 *               the first tau of each period with steps tau* (a schedule of
 *               cc_step_n calls).
 *   g_model  0: g = 1;  1: g = g_ref / sqrt(T) (resistivity of the paper's
 *            conducting layer, Section 5).
 * layer = -1 disables the source.
 */
typedef struct {
  int32_t layer;
  double q0;
  double t_period, t_on, t_start;
  int32_t waveform;
  double edge_w;
  int32_t g_model;
  double g_ref;
} cc_source;

/* Create a context for n_instances instances; desc points to n_instances
 * descriptors.  Host work only: device memory is allocated on the first
 * call that needs it, on the device current at that time.
 * Errors: CC_EINVAL (bad descriptor), CC_ENOMEM. */
int cc_create_geometry(const cc_geometry_desc* desc, int32_t n_instances, cc_ctx** out);

/* Materials of instance `instance` (-1: all instances), m[n_layers]. */
int cc_set_materials(cc_ctx* ctx, int32_t instance, const cc_material* m);

/* Source of instance `instance` (-1: all instances). */
int cc_set_source(cc_ctx* ctx, int32_t instance, const cc_source* s);

/* Per-instance time step [s], used by cc_step_n when its dt_s is 0. */
int cc_set_dt(cc_ctx* ctx, int32_t instance, double dt_s);

/*
 * Advance every instance by n_steps steps of Eq. (scheme_eq) starting at
 * t0_s; step n uses t_n = t0_s + n dt (dt = dt_s if dt_s > 0, else the
 * per-instance value of cc_set_dt).
 *   T_dev       in/out field of all instances (double for CC_FP64, float
 *               for CC_MIXED), layout above.  Caller-owned device memory.
 *   trace_dev   NULL or device double[n_instances][n_steps][2]: after step n,
 *               T(r_max, z_0) and the trapezoid-weighted mean over z of
 *               T(r_max, z) (the surface temperature of Section 5.1).
 *   energy_dev  NULL or device double[n_instances][5], ADDED to: stored heat
 *               sum V rho c (That - T), injected heat tau sum V X, heat through
 *               Dirichlet edges, through interface edges, through Neumann
 *               edges (V = 2 pi r_i hbar_i etabar_j).  The scheme satisfies
 *               stored = injected + the three edge terms up to rounding.
 *   stream      cudaStream_t or NULL.
 * Errors: CC_EINVAL, CC_EUNSTABLE (dt above the bound of Eq.
 * (stability_condition) over the guard range; set CC_FORCE_UNSTABLE=1 in the
 * environment to run anyway), CC_ESTATE, CC_ECUDA, CC_ENOMEM.
 * The call is asynchronous with respect to the host. */
int cc_step_n(cc_ctx* ctx, void* T_dev, int64_t n_steps, double t0_s, double dt_s,
              double* trace_dev, double* energy_dev, void* stream);

/*
 * ADI variant (Peaceman-Rachford), the scheme the paper names as the
 * unconditionally stable alternative to its own (Section 3, after
 * Eq. (stability_condition)): each step is two half steps of dt/2 with the
 * material properties and the source frozen at (T^n, t_n),
 *   rho c (T* - T^n)/(dt/2)    = Lambda_i[T*] + Lambda_j[T^n]   + X   (implicit in r)
 *   rho c (T^n+1 - T*)/(dt/2)  = Lambda_i[T*] + Lambda_j[T^n+1] + X   (implicit in z)
 * The first is the step of cc_step_n at dt/2; the second is one tridiagonal
 * system along z per column of regular nodes, after which the axis, r_max
 * and interface columns take their radial relations (interface: Eq.
 * (cc_first_3) with lambda* at T^n) and the axial boundary rows are set.
 * There is no stability bound on dt (no CC_EUNSTABLE); accuracy is second
 * order in dt for frozen coefficients.
 *   T_dev      in/out double field of all instances (FP64 contexts only).
 *   trace_dev  NULL or double[n_instances][n_steps][2] as in cc_step_n.
 * No energy terms.  The first call sizes the ADI scratch (about 24 bytes
 * per node plus 24 bytes per node of the column solves).
 * Errors: CC_EINVAL, CC_EUNSUPPORTED (CC_MIXED context or a stepped
 * outline), CC_ESTATE,
 * CC_ECUDA, CC_ENOMEM.  Asynchronous; cc_sync reports deferred failures. */
int cc_step_adi_n(cc_ctx* ctx, void* T_dev, int64_t n_steps, double t0_s, double dt_s,
                  double* trace_dev, void* stream);

/* Launch shape of cc_step_n (the numerics do not depend on it):
 *   mode 0: one kernel launch per time step; mode 1: all steps of a call in
 *   one cooperative (co-resident) launch with a grid barrier between steps
 *   (bounded wait: a barrier that does not complete within ~seconds ends the
 *   kernel and cc_sync reports CC_ETIMEOUT; if the grid cannot be
 *   co-resident the call falls back to mode 0).  Modes 0 and 1 work on CTA
 *   tiles: the warps of a block assemble the rows of a few lines into shared
 *   memory, then solve them, then store, with block barriers in between.
 *   mode 2: one launch per time step in which every warp owns a run of
 *   consecutive lines and takes each line from its rows to its stored
 *   values without block barriers (rectangles; a context with a stepped
 *   outline runs mode 0).
 *   mode 3: all steps of a call in one cooperative launch with the field
 *   resident in shared memory: each block (one per SM) keeps its run of
 *   lines on chip for the whole call and exchanges only its first and last
 *   lines with its two neighbours between steps, through global memory and
 *   per-block step counters (bounded waits, reported as CC_ETIMEOUT).  For
 *   FP64 contexts of one rectangular instance whose field fits in the SMs'
 *   shared memory (e.g. 512 x 4096); other contexts, or a grid that cannot
 *   be co-resident, run mode 0.
 *   mode 4: one launch per time step with pipelined CTA tiles: producer
 *   warps (three quarters of the block for CC_FP64, about half for
 *   CC_MIXED) assemble the rows of the next tile while the consumer warps
 *   solve and store the current one, two row buffers changing hands through
 *   named barriers (every context).
 *   mode 5 (CC_MIXED contexts only): mode 4 with the stores, trace and
 *   energy sums of every tile done by the producer warps, so the consumers
 *   only solve; faster when the line solves dominate (long lines, e.g.
 *   512 x 4096), slower when the rows do (short lines of a ragged batch).
 *   threads: 64, 128 or 256 per block; 384 with modes 4 and 5 only; 512
 *   with modes 4 and 5 in CC_MIXED contexts only.
 *   Default (a new context): mode 4 with 128 threads per block for CC_FP64,
 *   512 for CC_MIXED, rows_per_lane 16.
 *   rows_per_lane: 2..16, target rows per lane of the line solve; a line of
 *   nr rows is split over the smallest power-of-two number of lanes G <= 32
 *   that meets it (at least 2 rows per lane, at most 16).
 * After a first call has sized the context's buffers, cc_step_n performs no
 * allocation and no host synchronisation, so a call can be captured in a
 * CUDA graph (its t0 is then part of the graph). */
int cc_set_launch(cc_ctx* ctx, int32_t mode, int32_t threads, int32_t rows_per_lane);
int cc_get_launch(const cc_ctx* ctx, int32_t* mode, int32_t* threads, int32_t* rows_per_lane);

/* Autotuner: times n_trial steps of every launch shape (mode x threads x the
 * row policies that change G for some instance) on the caller's field T_dev,
 * keeps the fastest (cc_get_launch), restores T_dev, and returns its time per
 * step in best_ms (may be NULL).  Synchronous. */
int cc_autotune(cc_ctx* ctx, void* T_dev, int32_t n_trial, float* best_ms, void* stream);

/* Wait for the context's work on `stream`, then report a deferred kernel
 * failure (CC_ENONFINITE, CC_ETIMEOUT, CC_ECUDA) or CC_OK. */
int cc_sync(cc_ctx* ctx, void* stream);

/*
 * Reverse-time discrete adjoint of n_steps steps (Section 3 scheme) for the
 * loss J = sum_n dt (Sbar_n - target_n)^2, Sbar_n the z-mean surface
 * temperature after step n (trace column 1).  Returns J and dJ/dtheta for
 * theta = (q0, t_on, lam_scale[0..L-1], cap_scale[0..L-1]) per instance,
 * plus dJ/dT0 if dT0_dev is not NULL.  Checkpoints every ckpt_every steps
 * (<= 0: 256) and recomputes in between; the forward sweep keeps every state
 * of the last segment, which needs no recompute.  Device scratch, owned by
 * the context: ceil(n_steps / ckpt_every) + ckpt_every + 9 fields plus 5 doubles
 * per instance and step.
 *   T0_dev      initial field (not modified); target_dev double[n_inst][n_steps]
 *   loss_dev    double[n_inst]; grad_dev: for each instance in order, 2 + 2 n_layers
 *               doubles (q0, t_on, lam_scale[0..L-1], cap_scale[0..L-1])
 *   dT0_dev     NULL or double field like T0: dJ/dT0
 * Each step of the reverse sweep rebuilds the rows of the forward step at the
 * recomputed state, solves the transposed line systems, and gathers the
 * derivatives through lambda(T), c(T), X and the interface rows.  The
 * t_on derivative is nonzero only for the smoothed waveform (waveform 1).
 * Errors as cc_step_n; CC_EUNSUPPORTED for CC_MIXED contexts and for a
 * stepped outline (step_layers > 0 with a narrow line). */
int cc_adjoint(cc_ctx* ctx, const void* T0_dev, int64_t n_steps, double t0_s, double dt_s,
               const double* target_dev, int32_t ckpt_every, double* loss_dev,
               double* grad_dev, void* dT0_dev, void* stream);

/* Same reverse sweep as cc_adjoint for a loss that is any function of the
 * surface traces: seed_dev is device double[n_inst][n_steps] holding
 * dJ/dSbar_n (Sbar_n = trace column 1 after step n).  Fills grad_dev
 * (layout of cc_adjoint) and, if not NULL, dT0_dev.  Used by the autograd
 * binding.  Errors as cc_adjoint. */
int cc_adjoint_vjp(cc_ctx* ctx, const void* T0_dev, int64_t n_steps, double t0_s, double dt_s,
                   const double* seed_dev, int32_t ckpt_every, double* grad_dev, void* dT0_dev,
                   void* stream);

/* Release the context and everything it owns.  NULL is accepted. */
int cc_destroy(cc_ctx* ctx);

/* ---- no-allocation variant --------------------------------------------- */

/* Limits of cc_step_n_noalloc (they size its static device scratch array). */
#define CC_NOALLOC_MAX_NR 512
#define CC_NOALLOC_MAX_NZ 16384
#define CC_NOALLOC_MAX_NODES (1 << 20)   /* nr * nz */
#define CC_NOALLOC_MAX_STEPS 65536       /* n_steps per call */

/*
 * cc_step_n for one FP64 instance, for callers that cannot allocate device
 * memory.  The paper has no counterpart to this entry point; it exists
 * because some callers cannot call cudaMalloc (an embedding framework whose
 * allocator owns the device memory, loops that forbid allocation after
 * start-up), while cc_step_n allocates its context tables and scratch on
 * first use.  This call allocates nothing, on the device or the host: its
 * scratch (tables, work list, waveform table, power-law tables, error word,
 * and the ping-pong partner of T_dev) lives in a file-scope static device
 * array of about 9.5 MiB that every GPU loading the library holds until the
 * process exits.  The grid, checks, stability guard and device tables are
 * those of cc_create_geometry / cc_step_n (same host code), including the
 * tabulated power law, so the results equal cc_step_n's up to the FMA
 * contraction of a different block size (CTA tiles of 128 threads).
 *   desc        geometry (precision must be CC_FP64, a rectangle:
 *               step_layers 0, else CC_EUNSUPPORTED); materials[n_layers];
 *               source (layer -1 for none; waveforms 0, 1 and 2).  Same
 *               meaning and checks as cc_create_geometry, cc_set_materials and
 *               cc_set_source.
 *   T_dev       caller-owned device double[nz][nr], advanced in place.
 *   trace_dev, energy_dev  as in cc_step_n (one instance), or NULL.
 *   dt_s        time step, > 0.
 * Limits: nr <= CC_NOALLOC_MAX_NR, nz <= CC_NOALLOC_MAX_NZ,
 * nr * nz <= CC_NOALLOC_MAX_NODES, n_steps <= CC_NOALLOC_MAX_STEPS; larger
 * requests return CC_EINVAL before any device work.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current).  Every call copies its
 * tables from pageable host memory and waits for its own work on `stream`
 * before returning (so that it can report CC_ENONFINITE): it cannot be called
 * while a stream is being captured into a CUDA graph.  All calls share the
 * array and it keeps the last call's contents: calls whose work overlaps on
 * the GPU (different streams or host threads) race and must be serialised by
 * the caller.  Errors: CC_EINVAL, CC_EUNSTABLE, CC_EUNSUPPORTED, CC_ECUDA,
 * CC_ENONFINITE.
 */
int cc_step_n_noalloc(const cc_geometry_desc* desc, const cc_material* materials,
                      const cc_source* source, double* T_dev, int64_t n_steps, double t0_s,
                      double dt_s, double* trace_dev, double* energy_dev, void* stream);

/* ---- measurement -------------------------------------------------------- */

/*
 * FP64 FMA rate of the current GPU, the denominator of the FP64-pipe roofline
 * that bounds this scheme (the paper has no counterpart: it reports wall
 * times only).  Runs one warm-up and one timed launch of a kernel in which
 * every thread advances 8 independent chains of `iters` dependent FP64 FMAs,
 * four blocks of 256 threads per SM, timed with CUDA events on `stream`.
 *   scratch_dev  device double[scratch_len], scratch_len >= 1024 x the SM
 *                count (one result per thread; overwritten).
 *   fma_per_s    out: thread-level FP64 FMAs per second (x2 = FLOP/s).
 *   seconds      out (or NULL): duration of the timed launch.
 * Synchronous.  Errors: CC_EINVAL (null output, iters < 1, scratch too short),
 * CC_ECUDA. */
int cc_measure_fp64_rate(double* scratch_dev, int64_t scratch_len, int32_t iters,
                         double* fma_per_s, double* seconds, void* stream);

/* ---- host-only queries (no GPU needed) ---------------------------------- */

/* Node positions and radial classes of one descriptor: r[nr], z[nz],
 * rclass[nr] (0 axis, 1 regular, 2 layer interface, 3 outer boundary). */
int cc_query_grid(const cc_geometry_desc* desc, double* r, double* z, int32_t* rclass);

/* CTA tiles the step kernels use for a set of instances (all of one
 * precision) with `threads` per block and the rows-per-lane policy of
 * cc_set_launch: tiles[3 t .. 3 t + 2] = (instance, first line j0, lines nl)
 * for t < min(*n_tiles, max_tiles); with n_blocks > 0 blocks, cta[b] ..
 * cta[b+1] (cta: int32[n_blocks + 1] or NULL) are the tiles of block b, an
 * equal share of all interior nodes (a launch uses its resident block
 * count), and a block's run of lines of one instance is cut into the fewest
 * tiles that fit, of sizes that differ by at most one; lanes[k] (or NULL): lanes G per line of instance k; *smem_bytes
 * (or NULL): dynamic shared memory of the largest tile.  CC_EINVAL for
 * invalid arguments or when max_tiles is too small (*n_tiles is then set). */
int cc_query_tiles(const cc_geometry_desc* descs, int32_t n_instances, int32_t threads,
                   int32_t rows_per_lane, int32_t n_blocks, int32_t* tiles, int32_t max_tiles,
                   int32_t* n_tiles, int32_t* cta, int32_t* lanes, int32_t* smem_bytes);

/* Stepped outline of one descriptor: the lines j >= *j_narrow end at the
 * radial node *i_step (a rectangle gives nr - 1 and nz).  CC_EINVAL for an
 * outline the scheme does not take. */
int cc_query_outline(const cc_geometry_desc* desc, int32_t* i_step, int32_t* j_narrow);

/* Stability bound of Eq. (stability_condition) for one instance:
 * (min_j eta_j^2 / 2) * min over layers and the guard range of rho c/lambda. */
int cc_tau_stab(const cc_ctx* ctx, int32_t instance, double* tau_out);

/* Static description of a status code. */
const char* cc_status_string(int status);

/* Number of this library's kernel launches issued so far by this process. */
int64_t cc_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* CCELL_H */
