/* or_internal.h — private structures of the FP64 CPU oracle (test infrastructure only). */
#ifndef OR_INTERNAL_H
#define OR_INTERNAL_H
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "rt_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int nd, ne;
    double *dir;       /* [nd*3] unit directions n-hat_s (tetrad components 1,2,3) */
    double *w;         /* [nd] solid angle of the Voronoi cell */
    int *nnb;          /* [nd] 5 or 6 */
    int *nbr;          /* [nd*6] counter-clockwise neighbour ring */
    int *ring_edge;    /* [nd*6] edge index of ring slot */
    int *ring_back;    /* [nd*6] slot of s in the ring of nbr */
    double *vor;       /* [nd*6*3] Voronoi vertex between ring slots q and q+1 */
    int *edge;         /* [ne*2] (s, s') with s < s' */
    double *dlam;      /* [ne] arc length of the Voronoi edge */
    double *emid;      /* [ne*3] edge midpoint */
    double *eu;        /* [ne*3] unit normal of the edge, from s towards s' */
    int *mirror;       /* [nd] direction with components (n1, -n2, -n3) */
} or_grid;

int or_build_grid(or_grid *G, int n);
void or_free_grid(or_grid *G);

/* geometry of one spacetime point (static metric) */
typedef struct {
    double g[4][4];      /* g_{mu nu} */
    double gi[4][4];     /* g^{mu nu} */
    double sqrtg;        /* sqrt(-g) */
    double e[4][4];      /* e[a][mu] = e^mu_(a): tetrad legs in coordinate components */
    double ei[4][4];     /* ei[a][mu] = e^(a)_mu */
    double om[4][4][4];  /* om[a][b][c] = omega^(a)_(b)(c) (cell centres only) */
} or_geom;

void or_geometry(const or_config *c, const double x[3], int want_omega, or_geom *out);

struct or_ctx {
    or_config c;
    or_grid G;
    int ncell;
    int ng[3];            /* ghost width per axis (2 if active, 0 otherwise) */
    int active[3];
    int gn[3];            /* ghosted extents */
    /* geometry: one record (flat Cartesian) or an (i, j) table over the
       ghosted index space (Kerr-Schild does not depend on x3): cell centres
       and the lower face of each cell along each axis */
    or_geom *gc;
    or_geom *gf[3];
    /* state */
    double *I, *ug;
    double *rho, *ucon, *kap, *cs, *eta;
    double *G4;           /* [ncell*4] force on the gas from the last interaction */
    /* stage states of the step in progress: predictor (Is, ugs), step result (I2, ug2) */
    double *Is, *ugs, *I2, *ug2;
    int next_stage;
    /* x3 halo (OR_BC_HALO): ghost planes k = -2, -1 (side 0) and nx2, nx2 + 1
       (side 1), plane-major like the cells; intensities and gas energy of the
       stage source, fluid of the ghost cells */
    int halo;
    double *hI[2], *hug[2], *hrho[2], *hkap[2], *hcs[2], *hucon[2];
};

static inline int or_gidx(const or_ctx *c, int i, int j, int k) {
    return ((k + c->ng[2]) * c->gn[1] + (j + c->ng[1])) * c->gn[0] + (i + c->ng[0]);
}
static inline int or_cidx(const or_ctx *c, int i, int j, int k) {
    return (k * c->c.nx[1] + j) * c->c.nx[0] + i;
}
static inline const or_geom *or_gcen(const or_ctx *c, int i, int j) {
    return c->c.coords == OR_MINKOWSKI_CART ? &c->gc[0] : &c->gc[(j + c->ng[1]) * c->gn[0] + (i + c->ng[0])];
}
static inline const or_geom *or_gface(const or_ctx *c, int a, int i, int j) {
    return c->c.coords == OR_MINKOWSKI_CART ? &c->gf[a][0] : &c->gf[a][(j + c->ng[1]) * c->gn[0] + (i + c->ng[0])];
}
static inline int or_pole_zero(const or_ctx *c, int j) {
    int nz = c->c.n_pole_zero;
    return nz > 0 && (j < nz || j >= c->c.nx[1] - nz);
}

void or_set_err(const char *msg);

/* physics pieces (or_physics.c) */
void or_tetrad_dir(const or_geom *g, const double nh[3], double n_up[4], double *n_lo0);
double or_cell_alpha(const or_ctx *c, double rho, double ug, double kap, double cs);
void or_transport_stage(or_ctx *c, const double *Isrc, const double *ug_src,
                        const double *Ibase, double dtk, double *Iout);
long or_source_step(or_ctx *c, double *I, const double *ug_in, double *ug_out, double dtk, double *G4);
double or_limiter(int kind, double dl, double dr);
int or_map_cell(const or_ctx *c, int idx[3], int *mir, int *fixed_row);
/* ghost fluid and gas energy of the ghosted cell (i, j, k) of a transport
   stage whose source gas energy is ug_src: the cell it copies, or the caller's
   halo plane */
void or_ghost_fluid(const or_ctx *c, int i, int j, int k, const double *ug_src, double *rho, double *ug,
                    double *kap, double *cs, const double **ucon);
void or_fill_ghosts(const or_ctx *c, const double *I, double *Ig);

#endif
