/*
 * rt.h — C ABI of the B300 radiation-step library (librt_b300.so).
 *
 * The library advances the gray, angle-resolved covariant radiative transfer
 * equation of Wallace, Begue & Pe'er (cuHARM radiation module): the tetrad-
 * frame intensity I-hat on every spatial cell x every direction of a geodesic
 * (subdivided icosahedron) angular grid, eq. (covariant_radiative_transfer)
 * in the finite-volume form eq. (radiative_transfer_discrete), with the
 * implicit radiation-gas coupling of section 3.5.2 and the predictor-corrector
 * update of section 3.6.
 *
 * Conventions (all entry points):
 *  - Cell index: cell = (k*nx[1] + j)*nx[0] + i for logical indices (i, j, k)
 *    along (x1, x2, x3).  Intensities are cell-major with the direction index
 *    fastest: I[cell*n_dir + s], in the storage type of rt_config.precision
 *    (double, float, or bfloat16 stored as uint16).
 *  - Array arguments may be host or device pointers (the library copies with
 *    cudaMemcpyDefault on the context's stream); they are caller-owned and
 *    never freed or retained by the library.  rt_set_* copy into
 *    library-owned device buffers.
 *  - All work is ordered on the CUDA stream given to rt_create; calls that
 *    return data to a host pointer synchronise that stream.
 *  - Errors: every call returns an rt_status; rt_last_error() gives a message.
 *    Calling out of order (e.g. rt_step before rt_set_fluid) is RT_ESTATE.
 *    No call traps or hangs: temperature roots that fail to converge leave
 *    the cell at its bracketed best estimate and are counted (RT_ENOCONV).
 */
#ifndef RT_B300_H
#define RT_B300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0, RT_EINVAL = 1, RT_ENOMEM = 2, RT_ECUDA = 3, RT_ENOCONV = 4,
    RT_ESTATE = 5, RT_ETIMEOUT = 6
} rt_status;

typedef enum { RT_FP64 = 0, RT_FP32 = 1, RT_BF16 = 2 } rt_precision;
/* RT_SNAKE: flat space in snake coordinates (w, y, z), w = x - A sin(k pi y)
 * (App. A.1; params {A, k}); RT_CART_CYLTETRAD: flat space in Cartesian
 * coordinates with the tetrad aligned with the cylindrical unit vectors
 * (r-hat, phi-hat, z-hat), phi = atan2(y, x) (section 4.5; no params; the
 * box must not contain the axis x = y = 0). */
typedef enum { RT_MINKOWSKI_CART = 0, RT_KERR_SCHILD = 1, RT_SNAKE = 2, RT_CART_CYLTETRAD = 3 } rt_metric_kind;
typedef enum { RT_BC_PERIODIC = 0, RT_BC_OUTFLOW = 1, RT_BC_POLE = 2, RT_BC_BEAM = 3, RT_BC_HALO = 4 } rt_bc;
typedef enum { RT_LIM_MC = 0, RT_LIM_MINMOD = 1, RT_LIM_DONOR = 2 } rt_limiter;

typedef struct rt_grid rt_grid;   /* opaque, library-owned */
typedef struct rt_ctx rt_ctx;     /* opaque, library-owned */

/* Problem description.  Units are scale-free (G = c = a_rad = k_B/(mu m_p) = 1
 * by default), as in the paper's equilibration test (section 4.10). */
typedef struct {
    int nx[3];          /* cells per logical axis; an axis with one cell carries no flux */
    double x0[3];       /* logical coordinate of the lower face of cell 0 */
    double dx[3];       /* logical cell widths (Kerr-Schild: x1 = ln r, x2 = theta, x3 = phi) */
    int bc[3][2];       /* rt_bc at the lower/upper face of each axis */
    int beam_dir;       /* RT_BC_BEAM (x1-lower face only): injected direction */
    int beam_lo, beam_hi;  /* ghost rows j in [beam_lo, beam_hi) carry the beam */
    double beam_I;      /* injected intensity; every other ghost value is 0 */
    int n_pole_zero;    /* theta cells zeroed next to each pole (section 5); 0 = none */
    double gam;         /* adiabatic index Gamma */
    double arad;        /* radiation constant */
    double rho_exp;     /* absorption alpha^a = kappa rho^rho_exp T^-T_exp (comoving) */
    double T_exp;       /* 0 <= T_exp < 4 */
    double rho_floor;   /* rho below it: no interaction, vacuum fluxes (section 3.7) */
    double abar;        /* signal-speed coefficient (eq. rad_speeds), 1 in the paper */
    int tau_dt;         /* 0: tau = abar alpha dl (proper cell length); 1: abar alpha dt */
    int order;          /* 2: predictor-corrector (section 3.6); 1: one Euler stage */
    int limiter;        /* rt_limiter of the piecewise-linear reconstruction */
    int ang_recon;      /* 0: minimum-angle plane reconstruction; 1: donor cell */
    int transport;      /* 0 disables transport */
    int source;         /* 0 disables the radiation-gas interaction */
    double n0_cut;      /* intensities zeroed where |n_0| < n0_cut (section 3.5) */
    int precision;      /* rt_precision of the stored intensities */
    int coupling;       /* temperature solve of section 3.5.2: 3 (or 0) the
                           semi-implicit method 3 (eq. T_almost_fully_implicit);
                           1 and 2 the explicit-opacity methods (eqs.
                           semi_implicit_T, implicit_T), whose A1, A2 and total
                           absorption use T_-, with the Planck absorption of the
                           emission at T_- (1) or T_+ (2).  Methods 1 and 2 run
                           on the general stage kernel and have no reverse mode;
                           a cell whose equation has no positive temperature is
                           left unchanged and counted as unconverged. */
} rt_config;

/* Geodesic angular grid, section 3.3: icosahedron, log2(n) edge bisections
 * with projection to the sphere, Voronoi cells of the Delaunay triangulation.
 * n: edge subdivisions, a power of two in [1, 32]; n_dir = 10 n^2 + 2.
 * Directions are in the canonical order (ascending -n_z rounded to 1e-9,
 * then ascending atan2(n_y, n_x)).  Needs a CUDA device (the per-direction
 * geometry is computed there).  RT_EINVAL for a bad n. */
rt_status rt_create_geodesic_grid(int n, rt_grid **out);
/* Sizes and (optionally, host pointers) directions [n_dir*3] and solid angles [n_dir]. */
rt_status rt_grid_query(const rt_grid *g, int *n_dir, int *n_edge, double *dirs, double *weights);
void rt_destroy_grid(rt_grid *g);
/* Message of the last failed rt_create_geodesic_grid on this thread. */
const char *rt_grid_last_error(void);

/* Context for one problem on the current CUDA device.  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  The grid must outlive the
 * context.  RT_EINVAL for inconsistent configs, RT_ENOMEM if device memory
 * runs out. */
rt_status rt_create(const rt_grid *g, const rt_config *cfg, void *cuda_stream, rt_ctx **out);
void rt_destroy(rt_ctx *c);
const char *rt_last_error(const rt_ctx *c);

/* Metric and tetrad cache, sections 2.1 and App. A.2: kind = rt_metric_kind;
 * params = {M, a} for Kerr-Schild, {A, k} for snake coordinates (ignored
 * otherwise).  Computes, in FP64
 * on the device, the metric, the normal-observer tetrad (eq.
 * tetrad_restriction), the Ricci rotation coefficients (eq.
 * ricci_rotation_coefficients) with exact derivatives, and the per-direction
 * and per-edge tables the step uses.  Must precede rt_set_fluid. */
rt_status rt_set_metric(rt_ctx *c, int kind, const double *params);

/* Fluid (sections 3.5.1-3.5.2), each [n_cell] except ucon [n_cell*4]
 * (coordinate u^mu): density rho, gas internal energy u_g, absorption
 * prefactor kappa, scattering coefficient alpha_s_coef (alpha^s = coef*rho),
 * emission multiplier eta (NULL = 1).  Copied. */
rt_status rt_set_fluid(rt_ctx *c, const double *rho, const double *u_gas, const double *ucon,
                       const double *kappa, const double *alpha_s_coef, const double *eta);
/* Tetrad-frame intensities [n_cell*n_dir] in the configured storage type.
 * rt_set_intensity also sets the force on the gas (rt_moments' G) to zero:
 * no interaction has acted on the new state. */
rt_status rt_set_intensity(rt_ctx *c, const void *I);
rt_status rt_get_intensity(rt_ctx *c, void *I);
rt_status rt_set_ugas(rt_ctx *c, const double *u_gas);
rt_status rt_get_ugas(rt_ctx *c, double *u_gas);

/* Time-step bound of section 3.7: cfl times the shortest coordinate light
 * crossing dx^a n^0/|n^a| over cells (pole-zeroed cells excluded), axes and
 * directions.  Written to *dt. */
rt_status rt_cfl_dt(rt_ctx *c, double cfl, double *dt);

/* rt_cfl_dt without device allocation (the paper has no counterpart: this is
 * an interface for callers that cannot allocate).  rt_cfl_dt obtains its
 * reduction word with cudaMalloc/cudaFree on every call; a host code whose
 * memory manager owns the device (a caching allocator or a fixed pool) or a
 * time loop that must not synchronise the device between steps cannot allow
 * that.  This variant reduces in a file-scope static device array of 8193
 * doubles (64 KB) that every GPU loading the library holds until exit.
 * Same result as rt_cfl_dt.  Runs on the current device, which must be the
 * context's.  Limit: nx[0]*nx[1]*n_dir (point, direction) items, or n_dir for
 * flat geometry, at most 8192*2048 = 16,777,216; beyond it returns RT_EINVAL
 * with a message naming the limit.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  Every call on a device shares the one array:
 * calls whose kernels overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  Nothing needs clearing between calls:
 * each slot read is written earlier in the same call.  Synchronises the
 * context's stream; allocates nothing. */
rt_status rt_cfl_dt_noalloc(rt_ctx *c, double cfl, double *dt);

/* nsteps steps of size dt (dt <= 0: the cfl bound with cfl 0.4), section 3.6:
 * predictor transport over dt/2 + interaction over dt/2, corrector transport
 * over dt with the predictor fluxes + interaction over dt.  *n_fail (may be
 * NULL) receives the number of unconverged temperature solves (then
 * RT_ENOCONV).  Asynchronous unless n_fail is non-NULL.  Grids of up to 1024
 * directions step (n <= 8 of rt_create_geodesic_grid: 642 directions; n = 16
 * and 32 return RT_EINVAL from the first stage). */
rt_status rt_step(rt_ctx *c, double dt, int nsteps, double *dt_used, long long *n_fail);

/* One stage of a step (section 3.6): stage 0 is the predictor (transport
 * over dt/2 and the interaction over dt/2; for order 1 the single Euler
 * stage), stage 1 the corrector; the stages of a step run in order, and the
 * state takes the step's result after its last stage.  rt_step is the loop of
 * these stages.  dt <= 0: the cfl bound with cfl 0.4.  *n_fail as for
 * rt_step.  RT_ESTATE for a stage out of order.  This is how a context with
 * x3 halo faces steps: before each stage its caller fills the ghost planes
 * (rt_halo_pack / rt_halo_unpack). */
rt_status rt_step_stage(rt_ctx *c, double dt, int stage, long long *n_fail);

/* x3 slab decomposition (spatial domain decomposition of the box along x3;
 * the paper plans the transfer between GPUs as further work, section 5.2).
 * A context whose config has RT_BC_HALO on an x3 face owns a slab of a larger
 * box: its nx[2] planes, x0[2] the slab's own origin.  The transport reads two
 * cells on each side of a face (the piecewise-linear reconstruction of section
 * 3.4), so before every stage the two planes beyond each halo face must hold
 * the neighbouring slab's values of that stage's source: its intensities and
 * the opacity of its flux stage (the interaction and the angular flux are
 * cell-local).  Cells are x1-fastest, so a plane is contiguous.
 * Limits: x3 faces only, nx[2] >= 2, no pole boundary on x2 (its ghost is the
 * cell at phi + pi, on another slab) and no beam; rt_step, rt_step_record and
 * rt_step_adjoint refuse such a context (RT_EINVAL).
 *
 * rt_halo_bytes: bytes of one side's halo block, 2 P n_dir S + 8 P for P =
 * nx[0] nx[1] cells per plane and S bytes per stored intensity (0 without a
 * halo face).
 * rt_halo_pack: copies the halo blocks of the source of `stage` (which must be
 * the next stage to run) into the caller's buffers lo and hi (host or device,
 * rt_halo_bytes each): the intensities of the first two owned planes then
 * the flux opacity of the first plane (lo), and those of the last two planes
 * and of the last plane (hi).  Stream-ordered; a host buffer is complete
 * after the stream synchronises.
 * rt_halo_unpack: takes the neighbours' blocks as this context's ghost planes
 * for `stage`: lo is the lower neighbour's hi block, hi the upper
 * neighbour's lo block; a side that is the box's own boundary is ignored
 * (may be NULL).  Stream-ordered.
 * rt_set_fluid_halo: the fluid of the ghost planes, per halo side [2 P * 7]
 * doubles (rho, kappa, alpha_s coefficient, u^0, u^1, u^2, u^3 per cell,
 * lower side's plane -2 first, upper side's plane nx[2] first), of which the
 * advective face term uses the velocity.  Needed (after every rt_set_fluid)
 * unless the fluid is at rest in flat space; otherwise rt_step_stage returns
 * RT_ESTATE. */
rt_status rt_halo_bytes(const rt_ctx *c, size_t *bytes);
rt_status rt_halo_pack(rt_ctx *c, int stage, void *lo, void *hi);
rt_status rt_halo_unpack(rt_ctx *c, int stage, const void *lo, const void *hi);
rt_status rt_set_fluid_halo(rt_ctx *c, const double *lo, const double *hi);

/* Moments, eq. (R): R [n_cell*10] = coordinate R^{mu nu} (00,01,02,03,11,12,
 * 13,22,23,33) = sum_s n^mu n^nu I_s dOmega_s; Ebar [n_cell] comoving energy
 * density sum_s D_s^2 I_s dOmega_s; G [n_cell*4] coordinate force on the gas
 * -Delta R^{0 mu}/dt of the last interaction (section 3.5.3).  Any may be NULL. */
rt_status rt_moments(rt_ctx *c, double *R, double *Ebar, double *G);

/* Reverse mode of nsteps steps of size dt (dt <= 0: the cfl bound with cfl
 * 0.4) started from the checkpoint (I_ckpt [n_cell*n_dir], u_g ckpt
 * [n_cell]), with the fluid of rt_set_fluid.  Given the cotangents of the
 * final state, dL_dI_out [n_cell*n_dir] and dL_dug_out [n_cell] (NULL = 0),
 * writes dL_dI_in and dL_dug_in (the cotangents of the checkpoint) and ADDS
 * the gradients with respect to the absorption prefactor kappa and the
 * emission multiplier eta to dL_dkappa and dL_deta [n_cell].  The paper
 * (section 5.2) asks for gradients through the solver; this is the hand-derived
 * reverse of section 3.6's predictor-corrector, eq. radiative_transfer_discrete
 * with eqs. rad_speeds / flux_Jiang, and method 3 of section 3.5.2 (implicit
 * function theorem at the temperature root).  The forward is recomputed from
 * the checkpoint by the stage kernels of rt_step into a library-owned arena of
 * (2 nsteps + 3) intensity arrays (order 2; nsteps + 3 for order 1) plus a few
 * per-cell arrays per stage, kept for the next call; the reverse then takes
 * one kernel per stage.  With FP64 intensities the reverse pass is FP64
 * throughout; with FP32 intensities (I_ckpt in FP32) the recompute is stored
 * in FP32 and the per-element reverse arithmetic and intensity cotangents are
 * FP32, while per-cell sums and per-cell cotangents stay FP64.
 * Scope: flat Cartesian geometry, fluid at rest, FP64 or FP32 intensities,
 * at most 672 directions (G3 = 642 of section 3.3), periodic (>= 4 cells) or
 * outflow boundaries;
 * anything else is RT_EINVAL.
 * All pointers are device pointers; dL_dI_in may alias dL_dI_out.  The
 * recompute reads I_ckpt in place (a 256-byte aligned checkpoint that does
 * not overlap dL_dI_in; otherwise it is first copied into the arena), so it
 * must not change until the call's work on the stream is done.
 * Stream-ordered. */
rt_status rt_step_adjoint(rt_ctx *c, const void *I_ckpt, const double *ug_ckpt, double dt, int nsteps,
                          const double *dL_dI_out, const double *dL_dug_out, double *dL_dI_in,
                          double *dL_dug_in, double *dL_dkappa, double *dL_deta);

/* Forward steps that keep their stage states for the reverse pass.  Same
 * steps, results and end state as rt_step (dt <= 0: the cfl bound with cfl
 * 0.4; *dt_used, may be NULL, receives the step size), with the scope of
 * rt_step_adjoint.  Every stage's states (the ones rt_step_adjoint recomputes
 * from its checkpoint) are written to the library-owned reverse-mode arena,
 * and *rec_id receives a positive id of that recording.  Checkpointing
 * schemes keep the states of their last segment this way, so that its reverse
 * (rt_step_adjoint_recorded) needs no recompute; the paper has no counterpart.
 * A later rt_step_record, rt_step_adjoint or rt_set_fluid replaces the
 * recording.  Stream-ordered; the states cost the arena of rt_step_adjoint
 * for nsteps. */
rt_status rt_step_record(rt_ctx *c, double dt, int nsteps, double *dt_used, long long *rec_id);

/* rt_step_adjoint for the steps of the recording rec_id (rt_step_record),
 * without the recompute: same arguments and results as rt_step_adjoint from
 * the recording's start state, with its nsteps and dt.  RT_ESTATE if rec_id
 * is not the context's current recording. */
rt_status rt_step_adjoint_recorded(rt_ctx *c, long long rec_id, const double *dL_dI_out,
                                   const double *dL_dug_out, double *dL_dI_in, double *dL_dug_in,
                                   double *dL_dkappa, double *dL_deta);

/* Launch timing of the stage kernel (no counterpart in the paper: a
 * measurement hook).  rt_set_timing(c, 1) makes rt_step record a CUDA event
 * pair around every stage launch on the context's stream; rt_get_timing
 * synchronises the stream and returns the summed device time in ms and the
 * number of launches since the last call, then clears them. */
rt_status rt_set_timing(rt_ctx *c, int on);
rt_status rt_get_timing(rt_ctx *c, double *ms, long long *launches);

#ifdef __cplusplus
}
#endif
#endif
