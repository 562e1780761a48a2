/*
 * or_api.c — context, state, time step and moments of the oracle.
 * TEST INFRASTRUCTURE ONLY (see rt_oracle.h).
 */
#include "or_internal.h"

static char g_err[256];
void or_set_err(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
const char *or_error(void) { return g_err; }

or_ctx *or_create(const or_config *cfg) {
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
    return c;
}

void or_destroy(or_ctx *c) {
    if (!c) return;
    or_free_grid(&c->G);
    free(c->gc); for (int a = 0; a < 3; ++a) free(c->gf[a]);
    free(c->I); free(c->ug); free(c->rho); free(c->ucon); free(c->kap); free(c->cs); free(c->eta); free(c->G4);
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

/* one full step, section 3.6: predictor (transport over dt/2 from I^n, then
   the implicit interaction over dt/2) and corrector (transport over dt from
   I^n with the fluxes of the predictor state, then the interaction over dt);
   the gas enters each interaction with u_g^n */
long or_step(or_ctx *c, double dt, int nsteps) {
    size_t n = (size_t)c->ncell, ni = n * c->G.nd;
    double *Is = malloc(sizeof(double) * ni), *I2 = malloc(sizeof(double) * ni);
    double *ugs = malloc(sizeof(double) * n), *ug2 = malloc(sizeof(double) * n);
    long fails = 0;
    for (int st = 0; st < nsteps; ++st) {
        if (c->c.order == 1) {
            if (c->c.transport) or_transport_stage(c, c->I, c->ug, c->I, dt, I2); else memcpy(I2, c->I, sizeof(double) * ni);
            if (c->c.source) fails += or_source_step(c, I2, c->ug, ug2, dt, c->G4); else memcpy(ug2, c->ug, sizeof(double) * n);
        } else {
            if (c->c.transport) or_transport_stage(c, c->I, c->ug, c->I, 0.5 * dt, Is); else memcpy(Is, c->I, sizeof(double) * ni);
            if (c->c.source) fails += or_source_step(c, Is, c->ug, ugs, 0.5 * dt, NULL); else memcpy(ugs, c->ug, sizeof(double) * n);
            if (c->c.transport) or_transport_stage(c, Is, ugs, c->I, dt, I2); else memcpy(I2, c->I, sizeof(double) * ni);
            if (c->c.source) fails += or_source_step(c, I2, c->ug, ug2, dt, c->G4); else memcpy(ug2, c->ug, sizeof(double) * n);
        }
        memcpy(c->I, I2, sizeof(double) * ni);
        memcpy(c->ug, ug2, sizeof(double) * n);
    }
    free(Is); free(I2); free(ugs); free(ug2);
    return fails;
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
