/*
 * or_api.c — context, state, time step and moments of the oracle.
 * TEST INFRASTRUCTURE ONLY (see rt_oracle.h).
 */
#include "or_internal.h"

static char g_err[256];
void or_set_err(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
const char *or_error(void) { return g_err; }

or_ctx *or_create(const or_config *cfg) {
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd)
            if (cfg->bc[a][sd] == OR_BC_HALO && (a != 2 || cfg->nx[2] < 2 ||
                                                  cfg->bc[1][0] == OR_BC_POLE || cfg->bc[1][1] == OR_BC_POLE)) {
                or_set_err("halo boundaries: x3 faces only, at least 2 x3 cells, no pole boundary on x2");
                return NULL;
            }
    or_ctx *c = calloc(1, sizeof(or_ctx));
    c->c = *cfg;
    if (or_build_grid(&c->G, cfg->n_geo) != 0) { or_set_err("grid: n must be a power of two"); free(c); return NULL; }
    c->ncell = cfg->nx[0] * cfg->nx[1] * cfg->nx[2];
    for (int a = 0; a < 3; ++a) {
        c->active[a] = cfg->nx[a] > 1;
        c->ng[a] = c->active[a] ? 2 : 0;
        c->gn[a] = cfg->nx[a] + 2 * c->ng[a];
    }
    int npts = cfg->coords == OR_MINKOWSKI_CART ? 1 : c->gn[0] * c->gn[1];
    c->gc = malloc(sizeof(or_geom) * npts);
    for (int a = 0; a < 3; ++a) c->gf[a] = malloc(sizeof(or_geom) * npts);
    for (int p = 0; p < npts; ++p) {
        int i = p % c->gn[0] - c->ng[0], j = p / c->gn[0] - c->ng[1];
        double xc[3] = {cfg->x0[0] + (i + 0.5) * cfg->dx[0], cfg->x0[1] + (j + 0.5) * cfg->dx[1], cfg->x0[2] + 0.5 * cfg->dx[2]};
        or_geometry(cfg, xc, 1, &c->gc[p]);
        for (int a = 0; a < 3; ++a) {
            double xf[3] = {xc[0], xc[1], xc[2]};
            xf[a] -= 0.5 * cfg->dx[a];
            or_geometry(cfg, xf, 0, &c->gf[a][p]);
        }
    }
    size_t n = (size_t)c->ncell;
    c->I = calloc(n * c->G.nd, sizeof(double));
    c->ug = calloc(n, sizeof(double)); c->rho = calloc(n, sizeof(double));
    c->ucon = calloc(4 * n, sizeof(double)); c->kap = calloc(n, sizeof(double));
    c->cs = calloc(n, sizeof(double)); c->eta = calloc(n, sizeof(double));
    c->G4 = calloc(4 * n, sizeof(double));
    for (size_t i = 0; i < n; ++i) { c->ucon[4 * i] = 1.0; c->eta[i] = 1.0; }
    c->Is = calloc(n * c->G.nd, sizeof(double)); c->I2 = calloc(n * c->G.nd, sizeof(double));
    c->ugs = calloc(n, sizeof(double)); c->ug2 = calloc(n, sizeof(double));
    c->halo = cfg->bc[2][0] == OR_BC_HALO || cfg->bc[2][1] == OR_BC_HALO;
    if (c->halo) {
        size_t P2 = 2 * (size_t)cfg->nx[0] * cfg->nx[1];
        for (int sd = 0; sd < 2; ++sd) {
            c->hI[sd] = calloc(P2 * c->G.nd, sizeof(double)); c->hug[sd] = calloc(P2, sizeof(double));
            c->hrho[sd] = calloc(P2, sizeof(double)); c->hkap[sd] = calloc(P2, sizeof(double));
            c->hcs[sd] = calloc(P2, sizeof(double)); c->hucon[sd] = calloc(4 * P2, sizeof(double));
            for (size_t q = 0; q < P2; ++q) c->hucon[sd][4 * q] = 1.0;
        }
    }
    return c;
}

void or_destroy(or_ctx *c) {
    if (!c) return;
    or_free_grid(&c->G);
    free(c->gc); for (int a = 0; a < 3; ++a) free(c->gf[a]);
    free(c->I); free(c->ug); free(c->rho); free(c->ucon); free(c->kap); free(c->cs); free(c->eta); free(c->G4);
    free(c->Is); free(c->I2); free(c->ugs); free(c->ug2);
    for (int sd = 0; sd < 2; ++sd) {
        free(c->hI[sd]); free(c->hug[sd]); free(c->hrho[sd]); free(c->hkap[sd]); free(c->hcs[sd]); free(c->hucon[sd]);
    }
    free(c);
}

int or_grid_sizes(const or_ctx *c, int *nd, int *ne) { *nd = c->G.nd; *ne = c->G.ne; return 0; }

int or_grid_get(const or_ctx *c, double *dir, double *w, int *nnb, int *nbr,
                int *edge, double *dlam, double *emid, double *eu) {
    const or_grid *G = &c->G;
    if (dir) memcpy(dir, G->dir, sizeof(double) * 3 * G->nd);
    if (w) memcpy(w, G->w, sizeof(double) * G->nd);
    if (nnb) memcpy(nnb, G->nnb, sizeof(int) * G->nd);
    if (nbr) memcpy(nbr, G->nbr, sizeof(int) * 6 * G->nd);
    if (edge) memcpy(edge, G->edge, sizeof(int) * 2 * G->ne);
    if (dlam) memcpy(dlam, G->dlam, sizeof(double) * G->ne);
    if (emid) memcpy(emid, G->emid, sizeof(double) * 3 * G->ne);
    if (eu) memcpy(eu, G->eu, sizeof(double) * 3 * G->ne);
    return 0;
}

int or_grid_mirror(const or_ctx *c, int *mirror) { memcpy(mirror, c->G.mirror, sizeof(int) * c->G.nd); return 0; }

int or_set_fluid(or_ctx *c, const double *rho, const double *ug, const double *ucon,
                 const double *kappa, const double *alpha_s_coef, const double *eta) {
    size_t n = (size_t)c->ncell;
    memcpy(c->rho, rho, sizeof(double) * n); memcpy(c->ug, ug, sizeof(double) * n);
    memcpy(c->ucon, ucon, sizeof(double) * 4 * n); memcpy(c->kap, kappa, sizeof(double) * n);
    memcpy(c->cs, alpha_s_coef, sizeof(double) * n);
    if (eta) memcpy(c->eta, eta, sizeof(double) * n); else for (size_t i = 0; i < n; ++i) c->eta[i] = 1.0;
    return 0;
}

int or_set_intensity(or_ctx *c, const double *I) { memcpy(c->I, I, sizeof(double) * (size_t)c->ncell * c->G.nd); return 0; }
int or_get_intensity(const or_ctx *c, double *I) { memcpy(I, c->I, sizeof(double) * (size_t)c->ncell * c->G.nd); return 0; }
int or_get_ug(const or_ctx *c, double *ug) { memcpy(ug, c->ug, sizeof(double) * (size_t)c->ncell); return 0; }
int or_set_ug(or_ctx *c, const double *ug) { memcpy(c->ug, ug, sizeof(double) * (size_t)c->ncell); return 0; }

/* time step bound of section 3.7: a fraction cfl of the shortest coordinate
   crossing time dx^a n^0 / |n^a| over cells, axes and directions (pole-zeroed
   cells carry no radiation and are left out) */
double or_cfl_dt(const or_ctx *c, double cfl) {
    double best = 1e300;
    for (int j = 0; j < c->c.nx[1]; ++j) {
        if (or_pole_zero(c, j)) continue;
        for (int i = 0; i < c->c.nx[0]; ++i) {
            const or_geom *g = or_gcen(c, i, j);
            for (int s = 0; s < c->G.nd; ++s) {
                double nup[4], n0;
                or_tetrad_dir(g, c->G.dir + 3 * s, nup, &n0);
                for (int a = 0; a < 3; ++a) {
                    if (!c->active[a] || nup[a + 1] == 0.0) continue;
                    double t = c->c.dx[a] * nup[0] / fabs(nup[a + 1]);
                    if (t < best) best = t;
                }
            }
        }
    }
    return cfl * best;
}

/* one stage of a step, section 3.6: the predictor (transport over dt/2 from
   I^n, then the implicit interaction over dt/2) and the corrector (transport
   over dt from I^n with the fluxes of the predictor state, then the
   interaction over dt); the gas enters each interaction with u_g^n.  Order 1
   is a single Euler stage.  The state takes the step's result after its last
   stage. */
long or_step_stage(or_ctx *c, double dt, int stage) {
    size_t n = (size_t)c->ncell, ni = n * c->G.nd;
    int last = c->c.order == 1 ? 0 : 1;
    if (stage != c->next_stage || stage > last) { or_set_err("or_step_stage: stage out of order"); return -1; }
    long fails = 0;
    if (stage == 0 && last == 1) {
        if (c->c.transport) or_transport_stage(c, c->I, c->ug, c->I, 0.5 * dt, c->Is); else memcpy(c->Is, c->I, sizeof(double) * ni);
        if (c->c.source) fails += or_source_step(c, c->Is, c->ug, c->ugs, 0.5 * dt, NULL); else memcpy(c->ugs, c->ug, sizeof(double) * n);
        c->next_stage = 1;
        return fails;
    }
    const double *Isrc = stage == 0 ? c->I : c->Is, *usrc = stage == 0 ? c->ug : c->ugs;
    if (c->c.transport) or_transport_stage(c, Isrc, usrc, c->I, dt, c->I2); else memcpy(c->I2, c->I, sizeof(double) * ni);
    if (c->c.source) fails += or_source_step(c, c->I2, c->ug, c->ug2, dt, c->G4); else memcpy(c->ug2, c->ug, sizeof(double) * n);
    memcpy(c->I, c->I2, sizeof(double) * ni);
    memcpy(c->ug, c->ug2, sizeof(double) * n);
    c->next_stage = 0;
    return fails;
}

long or_step(or_ctx *c, double dt, int nsteps) {
    if (c->halo) { or_set_err("or_step: a context with x3 halos steps by stages (or_step_stage)"); return -1; }
    long fails = 0;
    for (int st = 0; st < nsteps; ++st)
        for (int stage = 0; stage <= (c->c.order == 1 ? 0 : 1); ++stage) fails += or_step_stage(c, dt, stage);
    return fails;
}

size_t or_halo_doubles(const or_ctx *c) {
    size_t P2 = 2 * (size_t)c->c.nx[0] * c->c.nx[1];
    return P2 * c->G.nd + P2;
}

int or_halo_pack(const or_ctx *c, int stage, double *lo, double *hi) {
    if (!c->halo) { or_set_err("or_halo_pack: no x3 halo"); return -1; }
    size_t P = (size_t)c->c.nx[0] * c->c.nx[1], nd = c->G.nd, n = (size_t)c->ncell;
    const double *I = stage == 0 ? c->I : c->Is, *u = stage == 0 ? c->ug : c->ugs;
    double *dst[2] = {lo, hi};
    size_t first[2] = {0, n - 2 * P};
    for (int sd = 0; sd < 2; ++sd) {
        memcpy(dst[sd], I + first[sd] * nd, sizeof(double) * 2 * P * nd);
        memcpy(dst[sd] + 2 * P * nd, u + first[sd], sizeof(double) * 2 * P);
    }
    return 0;
}

int or_halo_unpack(or_ctx *c, const double *lo, const double *hi) {
    if (!c->halo) { or_set_err("or_halo_unpack: no x3 halo"); return -1; }
    size_t P = (size_t)c->c.nx[0] * c->c.nx[1], nd = c->G.nd;
    const double *src[2] = {lo, hi};
    for (int sd = 0; sd < 2; ++sd) {
        memcpy(c->hI[sd], src[sd], sizeof(double) * 2 * P * nd);
        memcpy(c->hug[sd], src[sd] + 2 * P * nd, sizeof(double) * 2 * P);
    }
    return 0;
}

int or_set_fluid_halo(or_ctx *c, const double *lo, const double *hi) {
    if (!c->halo) { or_set_err("or_set_fluid_halo: no x3 halo"); return -1; }
    size_t P2 = 2 * (size_t)c->c.nx[0] * c->c.nx[1];
    const double *src[2] = {lo, hi};
    for (int sd = 0; sd < 2; ++sd)
        for (size_t q = 0; q < P2; ++q) {
            const double *f = src[sd] + 7 * q;
            c->hrho[sd][q] = f[0]; c->hkap[sd][q] = f[1]; c->hcs[sd][q] = f[2];
            for (int m = 0; m < 4; ++m) c->hucon[sd][4 * q + m] = f[3 + m];
        }
    return 0;
}

long or_source_only(or_ctx *c, double dt) {
    size_t n = (size_t)c->ncell;
    double *ug2 = malloc(sizeof(double) * n);
    long f = or_source_step(c, c->I, c->ug, ug2, dt, c->G4);
    memcpy(c->ug, ug2, sizeof(double) * n);
    free(ug2);
    return f;
}

/* moments, eq. (R): R^{mu nu} = sum_s n^mu n^nu I_s dOmega_s in coordinate
   components, and the comoving energy density E-bar = sum_s D^2 I_s dOmega_s */
int or_moments(const or_ctx *c, double *R, double *Ebar, double *G) {
    int nd = c->G.nd;
    for (int k = 0; k < c->c.nx[2]; ++k)
        for (int j = 0; j < c->c.nx[1]; ++j)
            for (int i = 0; i < c->c.nx[0]; ++i) {
                int ci = or_cidx(c, i, j, k);
                const or_geom *g = or_gcen(c, i, j);
                const double *u = c->ucon + 4 * (size_t)ci;
                double uh[4];
                for (int a = 0; a < 4; ++a) { double s = 0.0; for (int m = 0; m < 4; ++m) s += g->ei[a][m] * u[m]; uh[a] = s; }
                double r[10] = {0}, E = 0.0;
                for (int s = 0; s < nd; ++s) {
                    const double *nh = c->G.dir + 3 * s;
                    double nup[4], n0;
                    or_tetrad_dir(g, nh, nup, &n0);
                    double Iw = c->I[(size_t)ci * nd + s] * c->G.w[s];
                    int q = 0;
                    for (int m = 0; m < 4; ++m) for (int n = m; n < 4; ++n) r[q++] += nup[m] * nup[n] * Iw;
                    double D = uh[0] - (uh[1] * nh[0] + uh[2] * nh[1] + uh[3] * nh[2]);
                    E += D * D * Iw;
                }
                if (R) for (int q = 0; q < 10; ++q) R[10 * (size_t)ci + q] = r[q];
                if (Ebar) Ebar[ci] = E;
                if (G) for (int m = 0; m < 4; ++m) G[4 * (size_t)ci + m] = c->G4[4 * (size_t)ci + m];
            }
    return 0;
}

int or_ghost_fill(const or_ctx *c, const double *I, double *Ig, int gn[3]) {
    for (int a = 0; a < 3; ++a) gn[a] = c->gn[a];
    if (Ig) or_fill_ghosts(c, I, Ig);
    return 0;
}
