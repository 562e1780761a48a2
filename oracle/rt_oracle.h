/*
 * rt_oracle.h — plain FP64 CPU oracle for the gray radiation step of
 * Wallace, Begue & Pe'er, "Direct Solution of the Time-Dependent Covariant
 * Radiative Transfer Equation and its Coupling to GRMHD with cuHARM".
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or
 * call this code: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it. It shares no source with the CUDA library.
 *
 * Everything is double precision, written loop-by-loop in the order the paper
 * states the method (no blocking, fusion or reordering).  Arrays are
 * cell-major with the direction index fastest: I[cell*nd + s], where
 * cell = (k*ny + j)*nx + i for logical indices (i, j, k) along (x1, x2, x3).
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds per logical face */
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1, OR_BC_POLE = 2, OR_BC_BEAM = 3, OR_BC_HALO = 4 };
/* coordinates */
/* OR_SNAKE: flat space in snake coordinates (w, y, z), w = x - A sin(k pi y)
   (App. A.1); OR_CART_CYLTETRAD: flat space in Cartesian coordinates with the
   tetrad aligned with the cylindrical unit vectors (r-hat, phi-hat, z-hat)
   (section 4.5, eq. cylindrical_alignment) */
enum { OR_MINKOWSKI_CART = 0, OR_KERR_SCHILD = 1, OR_SNAKE = 2, OR_CART_CYLTETRAD = 3 };

typedef struct {
    int n_geo;            /* icosahedron edge subdivisions n (1,2,4,...): 10n^2+2 directions */
    int nx[3];            /* cells per logical axis; an axis with one cell carries no flux */
    double x0[3];         /* logical coordinate of the lower face of cell 0 */
    double dx[3];         /* logical cell widths */
    int coords;           /* OR_MINKOWSKI_CART or OR_KERR_SCHILD (x1 = ln r, x2 = theta, x3 = phi) */
    double M, a;          /* black-hole mass and spin parameter (Kerr-Schild only) */
    int bc[3][2];         /* boundary kind at the lower/upper face of each axis */
    int beam_dir;         /* OR_BC_BEAM: injected direction index */
    int beam_lo, beam_hi; /* OR_BC_BEAM on axis 0: ghost rows j in [lo, hi) carry the beam */
    double beam_I;        /* OR_BC_BEAM: injected intensity */
    int n_pole_zero;      /* theta cells zeroed next to each pole (0 = none) */
    double gam;           /* adiabatic index Gamma */
    double arad;          /* radiation constant (scale-free units: 1) */
    double rho_exp;       /* absorption opacity alpha^a = kappa * rho^rho_exp * T^-T_exp */
    double T_exp;
    double rho_floor;     /* below this density: no interaction, vacuum fluxes */
    double abar;          /* signal-speed coefficient a-bar */
    int tau_dt;           /* 0: tau = abar*alpha*proper cell length; 1: tau = abar*alpha*dt */
    int order;            /* 2: predictor-corrector; 1: single Euler stage */
    int limiter;          /* 0 MC, 1 minmod, 2 donor cell */
    int ang_recon;        /* 0 minimum-angle plane reconstruction, 1 donor cell */
    int transport;        /* 0 disables transport (source only) */
    int source;           /* 0 disables the interaction step */
    double n0_cut;        /* |n_0| below this: intensity zeroed */
    int coupling;         /* temperature solve of section 3.5.2: 1, 2 or 3 (0 = 3) */
    double snake_A, snake_k;   /* OR_SNAKE: amplitude and wave number of the coordinate wiggle */
} or_config;

typedef struct or_ctx or_ctx;

or_ctx *or_create(const or_config *cfg);
void or_destroy(or_ctx *c);
const char *or_error(void);

/* geodesic grid (section 3.3) */
int or_grid_sizes(const or_ctx *c, int *nd, int *ne);
int or_grid_get(const or_ctx *c, double *dir, double *w, int *nnb, int *nbr,
                int *edge, double *dlam, double *emid, double *eu);
int or_grid_mirror(const or_ctx *c, int *mirror);

/* fluid and intensity (copied in) */
int or_set_fluid(or_ctx *c, const double *rho, const double *ug, const double *ucon,
                 const double *kappa, const double *alpha_s_coef, const double *eta);
int or_set_intensity(or_ctx *c, const double *I);
int or_get_intensity(const or_ctx *c, double *I);
int or_get_ug(const or_ctx *c, double *ug);
int or_set_ug(or_ctx *c, const double *ug);

double or_cfl_dt(const or_ctx *c, double cfl);
/* nsteps full steps; returns the number of cells whose temperature root was
   not bracketed (-1 for a context with x3 halos, which steps by stages) */
long or_step(or_ctx *c, double dt, int nsteps);
/* one stage of a step of size dt (section 3.6): stage 0 is the predictor
   (order 2) or the single Euler stage (order 1), stage 1 the corrector; the
   state takes the step's result after its last stage.  Returns the unconverged
   temperature solves of the stage (-1 for a stage out of order). */
long or_step_stage(or_ctx *c, double dt, int stage);

/* x3 slab decomposition (section 8 of the design: spatial domain
   decomposition).  With OR_BC_HALO on an x3 face the two ghost planes on
   that side come from the caller: per side, 2 planes of nx0*nx1 cells, the
   stage source's intensities [2*P*nd] followed by its gas energies [2*P]
   (or_halo_doubles of them).  or_halo_pack writes the first two (lo) and last
   two (hi) owned planes of the source of `stage`; or_halo_unpack takes the
   neighbours' packs as this context's ghost planes for the next stage.
   or_set_fluid_halo: the ghost planes' fluid, per side [2*P*7] as (rho, kappa,
   alpha_s coefficient, u^0, u^1, u^2, u^3) per cell. */
size_t or_halo_doubles(const or_ctx *c);
int or_halo_pack(const or_ctx *c, int stage, double *lo, double *hi);
int or_halo_unpack(or_ctx *c, const double *lo, const double *hi);
int or_set_fluid_halo(or_ctx *c, const double *lo, const double *hi);
/* one interaction step only (no transport) */
long or_source_only(or_ctx *c, double dt);
/* R[cell*10] coordinate R^{mu nu} (00,01,02,03,11,12,13,22,23,33), Ebar[cell],
   G[cell*4] coordinate force on the gas from the last interaction (or NULL) */
int or_moments(const or_ctx *c, double *R, double *Ebar, double *G);

/* geometry at one logical point: g_{mu nu}[16], e^mu_a[16] (row a), omega^a_{bc}[64]
   (index (a*4+b)*4+c), sqrt(-g) */
int or_geometry_at(const or_ctx *c, const double x[3], double *g, double *e,
                   double *omega, double *sqrtg);
/* the ghosted copy of I that the transport stage reads: Ig[(gk*gn1 + gj)*gn0 + gi]
   over the extents gn_a = nx_a + 4 (2 ghost layers on each side of an active
   axis; inactive axes: nx_a), direction fastest; beam ghosts hold the beam */
int or_ghost_fill(const or_ctx *c, const double *I, double *Ig, int gn[3]);
/* angular speed coefficient n_0(m) (v(m).u) for every edge at a cell centre */
int or_edge_speeds(const or_ctx *c, int cell, double *wspeed);

/* spatial numerical flux (per unit n_0) for one face and direction */
double or_face_flux(double n, double IL, double IR, double Il, double Ir,
                    double tau, double vL, double vR);
/* minimum-angle plane reconstruction of a single angular field at every
   (direction, ring slot): out[s*6+k] is the value reconstructed from s at the
   midpoint of the edge to nbr[s*6+k] */
int or_mapr(const or_ctx *c, const double *Icell, double *out);

/* reverse mode: gradient of L with respect to initial I, kappa and eta over a
   rollout of nsteps from (I0, ug0).  dL_dI_out and dL_dug_out are the cotangents
   of the final state; results are written (not accumulated). */
int or_adjoint(or_ctx *c, const double *I0, const double *ug0, int nsteps, double dt,
               const double *dL_dI_out, const double *dL_dug_out,
               double *dL_dI0, double *dL_dkappa, double *dL_deta);

#ifdef __cplusplus
}
#endif
#endif
