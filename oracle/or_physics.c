/*
 * or_physics.c — transport and interaction of the oracle.
 * TEST INFRASTRUCTURE ONLY (see rt_oracle.h).
 *
 * Every function follows one passage of the paper and is written as plain
 * loops in FP64.  The readings taken where the paper is silent or garbled are
 * named at the point of use.
 */
#include "or_internal.h"

/* OR_MUTANT (default 0) plants one known mistake, for the test that shows the
   pins of the angular flux and the pole boundary catch it; builds with it are
   kept apart (oracle/build.py, liboracle_m<k>.so) and never serve as oracle:
   1 drift sign flipped, 2 angular upwind side taken from the sign of the
   weighted speed n_0 v.u (downwind wherever n_0 < 0), 3 pole ghost without
   the phi + pi shift, 4 pole ghost without the direction mirror, 6 angular
   flux without the n_0 weight */
#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

/* n^mu = e^mu_(a) nhat^(a) with nhat^(0) = 1 (eq. n_vector_definition mapped by
   eq. tetrad_transform) and the covariant time component n_0 = g_{0 mu} n^mu */
void or_tetrad_dir(const or_geom *g, const double nh[3], double n_up[4], double *n_lo0) {
    for (int m = 0; m < 4; ++m) n_up[m] = g->e[0][m] + nh[0] * g->e[1][m] + nh[1] * g->e[2][m] + nh[2] * g->e[3][m];
    double s = 0.0;
    for (int m = 0; m < 4; ++m) s += g->g[0][m] * n_up[m];
    *n_lo0 = s;
}

/* comoving total opacity alpha = alpha^a + alpha^s (section 3.5.2) with the
   density floor of section 3.7 (below it: no interaction, free streaming) */
double or_cell_alpha(const or_ctx *c, double rho, double ug, double kap, double cs) {
    if (!(rho >= c->c.rho_floor) || rho <= 0.0) return 0.0;
    double T = (c->c.gam - 1.0) * ug / rho;
    double aa = kap * pow(rho, c->c.rho_exp) * pow(T, -c->c.T_exp);
    return aa + cs * rho;
}

/* slope limiter of the piecewise-linear reconstruction (section 3.4) */
double or_limiter(int kind, double dl, double dr) {
    if (kind == 2) return 0.0;
    if (dl * dr <= 0.0) return 0.0;
    double s = dl > 0.0 ? 1.0 : -1.0;
    double al = fabs(dl), ar = fabs(dr);
    if (kind == 1) return s * (al < ar ? al : ar);
    double m = 2.0 * al;
    if (2.0 * ar < m) m = 2.0 * ar;
    if (0.5 * fabs(dl + dr) < m) m = 0.5 * fabs(dl + dr);
    return s * m;
}

/* spatial flux per unit n_0: eq. (spatial_fluxes_vacuum) for tau = 0, else the
   exponentially cut HLL form eq. (flux_Jiang) with the signal speeds of eq.
   (rad_speeds).  Readings: S+ multiplies the left state and S- the right one,
   the advected state is the upwind one of the fluid velocity, and the
   diffusive term carries no extra n factor — the only orientation for which
   tau -> 0 gives the vacuum upwind flux and tau -> infinity gives the
   -|n|/(2 tau) (I_{l+1} - I_l) flux of App. B.  Unequal left/right fluid
   velocities use the one-sided split max(vL,0) I_L + min(vR,0) I_R.  A
   direction with n = 0 keeps only the advective term. */
double or_face_flux(double n, double IL, double IR, double Il, double Ir,
                    double tau, double vL, double vR) {
    double adv = 0.0;
    if (tau > 0.0) adv = -expm1(-tau) * ((vL > 0.0 ? vL : 0.0) * IL + (vR < 0.0 ? vR : 0.0) * IR);
    if (n == 0.0) return adv;
    if (!(tau > 0.0)) return n * (n > 0.0 ? IL : IR);
    double f = sqrt(-expm1(-tau * tau)) / tau;
    double g = sqrt(-expm1(-tau * tau * tau * tau)) / tau;
    double Sp, Sm;
    if (n > 0.0) { Sp = n * f; Sm = -n * g; } else { Sp = -n * g; Sm = n * f; }
    double et = exp(-tau);
    return (Sp * n * IL - Sm * n * IR) * et / (Sp - Sm) + Sp * Sm / (Sp - Sm) * (Ir - Il) + adv;
}

/* ---------------------------------------------------------------- ghosts */
/* map a ghosted index to the interior cell it copies; returns 0 for a fixed
   (beam) value, 1 otherwise; *mir toggles the pole direction mirror.
   Pole boundary: the ghost at theta < 0 is the cell across the pole
   (theta -> -theta, phi -> phi + pi), seen with theta-hat and phi-hat reversed. */
int or_map_cell(const or_ctx *c, int idx[3], int *mir, int *fixed_row) {
    *mir = 0; *fixed_row = -1;
    int halo = -1;
    for (int a = 0; a < 3; ++a) {
        int n = c->c.nx[a];
        if (idx[a] >= 0 && idx[a] < n) continue;
        int side = idx[a] < 0 ? 0 : 1;
        int bc = c->c.bc[a][side];
        if (bc == OR_BC_HALO) {            /* x3 only: plane 0, 1 of the caller's ghost planes */
            halo = side;
            idx[a] = side ? idx[a] - n : idx[a] + 2;
        } else if (bc == OR_BC_PERIODIC) idx[a] = ((idx[a] % n) + n) % n;
        else if (bc == OR_BC_OUTFLOW) idx[a] = side ? n - 1 : 0;
        else if (bc == OR_BC_POLE) {
            idx[a] = side ? 2 * n - 1 - idx[a] : -1 - idx[a];
#if OR_MUTANT != 4
            *mir ^= 1;
#endif
#if OR_MUTANT != 3
            if (a == 1 && c->c.nx[2] > 1) idx[2] = (idx[2] + c->c.nx[2] / 2) % c->c.nx[2];
#endif
        } else {   /* beam: fixed inflow on axis 0, lower side */
            *fixed_row = (a == 0 && side == 0) ? idx[1] : -2;
            idx[a] = side ? n - 1 : 0;
        }
    }
    if (halo >= 0) { *fixed_row = -3 - halo; return 2; }
    return *fixed_row == -1 ? 1 : 0;
}

/* cell of the caller's halo plane p (0, 1) at (i, j) */
static size_t halo_cell(const or_ctx *c, int p, int i, int j) {
    return ((size_t)p * c->c.nx[1] + j) * c->c.nx[0] + i;
}

void or_ghost_fluid(const or_ctx *c, int i, int j, int k, const double *ug_src, double *rho, double *ug,
                    double *kap, double *cs, const double **ucon) {
    int idx[3] = {i, j, k}, mir, row;
    int r = or_map_cell(c, idx, &mir, &row);
    if (r == 2) {
        int side = -3 - row;
        size_t h = halo_cell(c, idx[2], idx[0], idx[1]);
        *rho = c->hrho[side][h]; *ug = c->hug[side][h]; *kap = c->hkap[side][h]; *cs = c->hcs[side][h];
        *ucon = c->hucon[side] + 4 * h;
        return;
    }
    int ci = or_cidx(c, idx[0], idx[1], idx[2]);
    *rho = c->rho[ci]; *ug = ug_src[ci]; *kap = c->kap[ci]; *cs = c->cs[ci];
    *ucon = c->ucon + 4 * (size_t)ci;
}

void or_fill_ghosts(const or_ctx *c, const double *I, double *Ig) {
    int nd = c->G.nd;
    for (int k = -c->ng[2]; k < c->c.nx[2] + c->ng[2]; ++k)
        for (int j = -c->ng[1]; j < c->c.nx[1] + c->ng[1]; ++j)
            for (int i = -c->ng[0]; i < c->c.nx[0] + c->ng[0]; ++i) {
                int idx[3] = {i, j, k}, mir, row;
                int ok = or_map_cell(c, idx, &mir, &row);
                double *dst = Ig + (size_t)or_gidx(c, i, j, k) * nd;
                if (ok == 2) {
                    const double *src = c->hI[-3 - row] + halo_cell(c, idx[2], idx[0], idx[1]) * nd;
                    for (int s = 0; s < nd; ++s) dst[s] = src[s];
                    continue;
                }
                if (!ok) {
                    for (int s = 0; s < nd; ++s)
                        dst[s] = (row >= c->c.beam_lo && row < c->c.beam_hi && s == c->c.beam_dir) ? c->c.beam_I : 0.0;
                    continue;
                }
                const double *src = I + (size_t)or_cidx(c, idx[0], idx[1], idx[2]) * nd;
                for (int s = 0; s < nd; ++s) dst[s] = mir ? src[c->G.mirror[s]] : src[s];
            }
}

/* minimum-angle plane reconstruction on the geodesic grid (section 3.4).
   Reading: in the gnomonic tangent plane of direction s, the planes through s
   and each pair of consecutive ring neighbours are formed; the one whose
   gradient has the smallest norm (smallest tilt; norms within a relative 1e-6
   of the smallest tie, and the first in ring order wins) is evaluated at the
   edge midpoints.  out[q] is the value at the
   midpoint of the edge to ring slot q. */
static void mapr_dir(const or_ctx *c, const double *Ic, int s, double out[6]) {
    const or_grid *G = &c->G;
    int k = G->nnb[s];
    const double *ns = G->dir + 3 * s;
    if (c->c.ang_recon == 1) { for (int q = 0; q < k; ++q) out[q] = Ic[s]; return; }
    double x[6][3], dI[6];
    for (int q = 0; q < k; ++q) {
        int t = G->nbr[6 * s + q];
        const double *nt = G->dir + 3 * t;
        double d = nt[0] * ns[0] + nt[1] * ns[1] + nt[2] * ns[2];
        for (int m = 0; m < 3; ++m) x[q][m] = nt[m] / d - ns[m];
        dI[q] = Ic[t] - Ic[s];
    }
    double al[6] = {0}, be[6] = {0}, nrm[6] = {0}, mn = 0.0;
    for (int q = 0; q < k; ++q) {
        int q1 = (q + 1) % k;
        double g00 = x[q][0]*x[q][0] + x[q][1]*x[q][1] + x[q][2]*x[q][2];
        double g01 = x[q][0]*x[q1][0] + x[q][1]*x[q1][1] + x[q][2]*x[q1][2];
        double g11 = x[q1][0]*x[q1][0] + x[q1][1]*x[q1][1] + x[q1][2]*x[q1][2];
        double det = g00 * g11 - g01 * g01;
        al[q] = (g11 * dI[q] - g01 * dI[q1]) / det;
        be[q] = (g00 * dI[q1] - g01 * dI[q]) / det;
        nrm[q] = al[q] * dI[q] + be[q] * dI[q1];
        if (q == 0 || nrm[q] < mn) mn = nrm[q];
    }
    /* planes within a relative 1e-6 of the smallest norm count as equal (mirror
       symmetric neighbourhoods tie exactly); the first in ring order wins */
    int best = 0;
    while (!(nrm[best] <= mn + 1e-6 * fabs(mn))) ++best;
    double ba = al[best], bb = be[best];
    int b1 = (best + 1) % k;
    for (int q = 0; q < k; ++q) {
        int e = G->ring_edge[6 * s + q];
        const double *m = G->emid + 3 * e;
        double d = m[0] * ns[0] + m[1] * ns[1] + m[2] * ns[2];
        double xm[3];
        for (int r = 0; r < 3; ++r) xm[r] = m[r] / d - ns[r];
        double p0 = x[best][0]*xm[0] + x[best][1]*xm[1] + x[best][2]*xm[2];
        double p1 = x[b1][0]*xm[0] + x[b1][1]*xm[1] + x[b1][2]*xm[2];
        out[q] = Ic[s] + ba * p0 + bb * p1;
    }
}

int or_mapr(const or_ctx *c, const double *Icell, double *out) {
    for (int s = 0; s < c->G.nd; ++s) {
        double v[6];
        mapr_dir(c, Icell, s, v);
        for (int q = 0; q < 6; ++q) out[6*s+q] = q < c->G.nnb[s] ? v[q] : 0.0;
    }
    return 0;
}

/* angular speed coefficient of every edge at a cell centre: n_0(m) (v(m) . u_e)
   with the tangent drift v^i = -(omega^i_{bc} - m^i omega^0_{bc}) m^b m^c of a
   photon direction m (the geodesic equation in the tetrad frame; it gives
   r^nu, r^zeta, r^psi of eq. angular_n_vectors as components, without a
   polar chart), evaluated at the edge midpoint as in eq. (angular_fluxes). */
static void edge_speeds(const or_ctx *c, const or_geom *g, double *wsp, double *vu) {
    const or_grid *G = &c->G;
    for (int e = 0; e < G->ne; ++e) {
        const double *mm = G->emid + 3 * e, *u = G->eu + 3 * e;
        double m4[4] = {1.0, mm[0], mm[1], mm[2]};
        double q[4];
        for (int a = 0; a < 4; ++a) {
            double s = 0.0;
            for (int b = 0; b < 4; ++b) for (int cc = 0; cc < 4; ++cc) s += g->om[a][b][cc] * m4[b] * m4[cc];
            q[a] = s;
        }
        double v[3];
        for (int i = 0; i < 3; ++i) v[i] = -(q[i + 1] - mm[i] * q[0]);
#if OR_MUTANT == 1
        for (int i = 0; i < 3; ++i) v[i] = -v[i];
#endif
        double nup[4], n0;
        or_tetrad_dir(g, mm, nup, &n0);
#if OR_MUTANT == 6
        n0 = 1.0;
#endif
        wsp[e] = n0 * (v[0] * u[0] + v[1] * u[1] + v[2] * u[2]);
        if (vu) vu[e] = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
    }
}

int or_edge_speeds(const or_ctx *c, int cell, double *wspeed) {
    int i = cell % c->c.nx[0], j = (cell / c->c.nx[0]) % c->c.nx[1];
    edge_speeds(c, or_gcen(c, i, j), wspeed, NULL);
    return 0;
}

/* one explicit transport stage of the finite-volume form eq.
   (radiative_transfer_discrete), beta = 0, conserved variable n^0 n_0 I:
   Iout = [U(Ibase) - dtk (sum_a [dA F_a]/dV + sum_e dlam F_e / dOmega)] / (n^0 n_0)
   with the fluxes taken from Isrc, then the |n_0| < n0_cut zeroing (section
   3.5, last paragraph) and the pole-cell zeroing of section 5.  No flux
   crosses a face where n_0 changes sign between the two cells, nor a face of
   zero area (a coordinate pole). */
void or_transport_stage(or_ctx *c, const double *Isrc, const double *ug_src,
                        const double *Ibase, double dtk, double *Iout) {
    int nd = c->G.nd;
    size_t ngc = (size_t)c->gn[0] * c->gn[1] * c->gn[2];
    double *Ig = malloc(sizeof(double) * ngc * nd);
    double *alg = malloc(sizeof(double) * ngc), *vg = malloc(sizeof(double) * ngc * 3);
    or_fill_ghosts(c, Isrc, Ig);
    /* ghost fluid: the cell a ghost copies (beam ghosts: the adjacent cell) */
    for (int k = -c->ng[2]; k < c->c.nx[2] + c->ng[2]; ++k)
        for (int j = -c->ng[1]; j < c->c.nx[1] + c->ng[1]; ++j)
            for (int i = -c->ng[0]; i < c->c.nx[0] + c->ng[0]; ++i) {
                int gi = or_gidx(c, i, j, k);
                double rho, ug, kap, cs;
                const double *u;
                or_ghost_fluid(c, i, j, k, ug_src, &rho, &ug, &kap, &cs, &u);
                alg[gi] = or_cell_alpha(c, rho, ug, kap, cs);
                for (int a = 0; a < 3; ++a) vg[3 * (size_t)gi + a] = u[a + 1] / u[0];
            }
    int stride[3] = {1, c->gn[0], c->gn[0] * c->gn[1]};
    int angular = c->c.coords != OR_MINKOWSKI_CART;
    /* cells are independent: OpenMP over (k, j) rows, per-thread scratch */
#pragma omp parallel
    {
    double *wsp = malloc(sizeof(double) * c->G.ne), *vu = malloc(sizeof(double) * c->G.ne);
    double *Icell = malloc(sizeof(double) * nd), *rec = malloc(sizeof(double) * 6 * nd);
#pragma omp for collapse(2) schedule(static)
    for (int k = 0; k < c->c.nx[2]; ++k)
        for (int j = 0; j < c->c.nx[1]; ++j)
            for (int i = 0; i < c->c.nx[0]; ++i) {
                int ci = or_cidx(c, i, j, k), gi = or_gidx(c, i, j, k);
                const or_geom *gcc = or_gcen(c, i, j);
                if (angular) {
                    edge_speeds(c, gcc, wsp, vu);
                    for (int s = 0; s < nd; ++s) Icell[s] = Ig[(size_t)gi * nd + s];
                    for (int s = 0; s < nd; ++s) mapr_dir(c, Icell, s, rec + 6 * s);
                }
                for (int s = 0; s < nd; ++s) {
                    const double *nh = c->G.dir + 3 * s;
                    double nc[4], n0c;
                    or_tetrad_dir(gcc, nh, nc, &n0c);
                    double U = nc[0] * n0c * Ibase[(size_t)ci * nd + s];
                    double div = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        if (!c->active[a]) continue;
                        double fl[2];
                        for (int side = 0; side < 2; ++side) {
                            int gl = gi + (side - 1) * stride[a], gr = gl + stride[a];
                            int fi[3] = {i, j, k}; fi[a] += side;
                            const or_geom *gf = or_gface(c, a, fi[0], fi[1]);
                            if (!(gf->sqrtg > 0.0)) { fl[side] = 0.0; continue; }
                            int li[3] = {i, j, k}, ri[3] = {i, j, k};
                            li[a] += side - 1; ri[a] += side;
                            double t4[4], n0L, n0R, nf[4], n0f;
                            or_tetrad_dir(or_gcen(c, li[0], li[1]), nh, t4, &n0L);
                            or_tetrad_dir(or_gcen(c, ri[0], ri[1]), nh, t4, &n0R);
                            if ((n0L > 0.0) != (n0R > 0.0)) { fl[side] = 0.0; continue; }
                            or_tetrad_dir(gf, nh, nf, &n0f);
                            double Im = Ig[(size_t)(gl - stride[a]) * nd + s], Il = Ig[(size_t)gl * nd + s];
                            double Ir = Ig[(size_t)gr * nd + s], Ip = Ig[(size_t)(gr + stride[a]) * nd + s];
                            double sl = or_limiter(c->c.limiter, Ir - Il, Il - Im);
                            double sr = or_limiter(c->c.limiter, Ip - Ir, Ir - Il);
                            double IL = Il + 0.5 * sl, IR = Ir - 0.5 * sr;
                            double len = c->c.tau_dt ? dtk : sqrt(gf->g[a + 1][a + 1]) * c->c.dx[a];
                            double tau = c->c.abar * 0.5 * (alg[gl] + alg[gr]) * len;
                            double F = or_face_flux(nf[a + 1], IL, IR, Il, Ir, tau, vg[3 * (size_t)gl + a], vg[3 * (size_t)gr + a]);
                            double dA = gf->sqrtg;
                            for (int b = 0; b < 3; ++b) if (b != a) dA *= c->c.dx[b];
                            fl[side] = dA * n0f * F;
                        }
                        double dV = gcc->sqrtg * c->c.dx[0] * c->c.dx[1] * c->c.dx[2];
                        div += (fl[1] - fl[0]) / dV;
                    }
                    double ang = 0.0;
                    if (angular) {
                        for (int q = 0; q < c->G.nnb[s]; ++q) {
                            int e = c->G.ring_edge[6 * s + q], t = c->G.nbr[6 * s + q];
                            int back = c->G.ring_back[6 * s + q];
                            int s0 = c->G.edge[2 * e];
                            double w = wsp[e];
                            /* reconstructed values on the s0 side (L) and the s1 side (R) */
                            double Iown = rec[6 * s + q], Ioth = rec[6 * t + back];
                            double IL = (s == s0) ? Iown : Ioth, IR = (s == s0) ? Ioth : Iown;
                            /* eq. (angular_fluxes): the upwind side follows the sign of the
                               drift v.u itself, not of the flux weight n_0 v.u (n_0 < 0 for
                               future-directed photons wherever d_t is timelike) */
#if OR_MUTANT == 2
                            double F = w * (w > 0.0 ? IL : IR);
#else
                            double F = w * (vu[e] > 0.0 ? IL : IR);
#endif
                            ang += c->G.dlam[e] * (s == s0 ? F : -F);
                        }
                        ang /= c->G.w[s];
                    }
                    double Un = U - dtk * (div + ang);
                    double In = Un / (nc[0] * n0c);
                    if (fabs(n0c) < c->c.n0_cut || or_pole_zero(c, j)) In = 0.0;
                    Iout[(size_t)ci * nd + s] = In;
                }
            }
    free(wsp); free(vu); free(Icell); free(rec);
    }
    free(Ig); free(alg); free(vg);
}

/* Method 3 (eq. T_almost_fully_implicit) with A'_1 = B1, A'_2 = B2 taken
   without the 1/(alpha_+ dt) prefactor (the only reading under which eq.
   T_almost_fully_implicit follows from eqs. ideal_gas_difference and
   energy_integral), and the emission multiplier eta.  Divided by T^p it reads
     (alpha(T) dt - B2 alpha^s) E* - B1 - B2 eta alpha^a(T) a T^4 = 0,
   with E* = W - Y T the radiation energy after the interaction (eq.
   ideal_gas_difference).  It is solved for E* (T = T_- + (E-bar_- - E*)/Y):
   where the gas holds far more energy than the radiation, W - Y T cancels
   catastrophically, while E* itself is well conditioned.  h increases
   strictly with E* on [0, W), so the root is unique. */
typedef struct { double B1, B2, W, Y, Tm, Em, au, as, eta, arad, dt, p; } teq;
static double teq_T(const teq *q, double X) { return q->Tm + (q->Em - X) / q->Y; }
static double teq_h(const teq *q, double X) {
    double T = teq_T(q, X);
    if (!(T > 0.0)) return INFINITY;
    double aa = q->au * pow(T, -q->p);
    return ((aa + q->as) * q->dt - q->B2 * q->as) * X - q->B1 - q->B2 * q->eta * aa * q->arad * T * T * T * T;
}

/* root of h(E*) on [0, W) by bisection to adjacent doubles */
static int solve_E(const teq *q, double *X) {
    double lo = 0.0, hi = q->W;
    if (!(teq_h(q, lo) < 0.0)) { *X = 0.0; return teq_h(q, lo) == 0.0; }
    for (int n = 0; n < 2000; ++n) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (teq_h(q, mid) > 0.0) hi = mid; else lo = mid;
    }
    *X = fabs(teq_h(q, lo)) <= fabs(teq_h(q, hi)) ? lo : hi;
    return 1;
}

/* Methods 1 and 2 of section 3.5.2 (eqs. semi_implicit_T and implicit_T):
   the angular sums A1, A2 (eqs. A1, A2) with the explicit alpha_-, and
   eq. energy_integral, E-bar_+ = A1 + A2 (alpha^a_P a T_+^4 + alpha^s E-bar_+),
   with the Planck absorption alpha^a_P at T_- (method 1) or at T_+ (method 2)
   and the emission multiplier eta.  Solved, like method 3, for
   X = E-bar_+ with T_+ = T_- + (E-bar_- - X)/Y (eq. ideal_gas_difference):
     h(X) = (1 - A2 alpha^s) X - A1 - A2 eta alpha^a_P a T(X)^4 = 0,
   the paper's quartic (method 1) and its T^(4-p) form (method 2) rewritten
   for X.  h increases strictly on [0, W), h(0) < 0, and h(W) = (1 - A2 alpha^s)
   W - A1, which need not be positive: then no positive temperature solves the
   equations (the instability the paper reports for these methods). */
typedef struct { double A1, A2, W, Y, Tm, Em, au, as, eta, arad, p; int method; } meq;
static double meq_T(const meq *q, double X) { return q->Tm + (q->Em - X) / q->Y; }
static double meq_aaP(const meq *q, double T) { return q->au * pow(q->method == 1 ? q->Tm : T, -q->p); }
static double meq_h(const meq *q, double X) {
    double T = meq_T(q, X);
    if (!(T >= 0.0)) return INFINITY;
    return (1.0 - q->A2 * q->as) * X - q->A1 - q->A2 * q->eta * meq_aaP(q, T) * q->arad * T * T * T * T;
}
/* root by bisection to adjacent doubles; 0 if there is none in [0, W) */
static int solve_meq(const meq *q, double *X) {
    double lo = 0.0, hi = q->W;
    if (!((1.0 - q->A2 * q->as) * q->W - q->A1 > 0.0)) return 0;
    for (int n = 0; n < 2000; ++n) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (meq_h(q, mid) > 0.0) hi = mid; else lo = mid;
    }
    *X = fabs(meq_h(q, lo)) <= fabs(meq_h(q, hi)) ? lo : hi;
    return 1;
}

/* the implicit interaction of section 3.5.2 for every cell:
   boost to the fluid frame (I-bar = D^4 I-hat, dOmega-bar = dOmega-hat / D^2,
   D = nbar^0 = u^0 - u.n in the tetrad frame), the angular sums of eqs.
   (A1, A2) with the explicit alpha_-, the temperature from method 3, the
   intensity update eq. (fluid_interaction_discrete) with alpha(T_+), emission
   at T_+ and E-bar_+ from eq. (ideal_gas_difference), the back transform,
   and the exchange ledger: u_g,+ = u_g,- - (E-bar(I_+) - E-bar_-) and the
   force on the gas G = -Delta R^{0 mu} / dt (section 3.5.3). */
long or_source_step(or_ctx *c, double *I, const double *ug_in, double *ug_out, double dtk, double *G4) {
    int nd = c->G.nd;
    long fails = 0;
    const double fourpi = 4.0 * M_PI;
#pragma omp parallel for collapse(2) schedule(static) reduction(+:fails)
    for (int k = 0; k < c->c.nx[2]; ++k)
        for (int j = 0; j < c->c.nx[1]; ++j)
            for (int i = 0; i < c->c.nx[0]; ++i) {
                int ci = or_cidx(c, i, j, k);
                double *Ic = I + (size_t)ci * nd;
                const or_geom *g = or_gcen(c, i, j);
                double rho = c->rho[ci], ugm = ug_in[ci];
                if (G4) for (int m = 0; m < 4; ++m) G4[4 * (size_t)ci + m] = 0.0;
                ug_out[ci] = ugm;
                if (!(rho >= c->c.rho_floor) || rho <= 0.0) continue;
                double Y = rho / (c->c.gam - 1.0);
                double Tm = ugm / Y;
                double au = c->kap[ci] * pow(rho, c->c.rho_exp), as = c->cs[ci] * rho, eta = c->eta[ci];
                if (!(Tm > 0.0)) { if (au + as > 0.0) ++fails; continue; }
                double aam = au * pow(Tm, -c->c.T_exp), atm = aam + as;
                if (!(atm > 0.0)) continue;
                /* fluid velocity in the tetrad frame */
                const double *u = c->ucon + 4 * (size_t)ci;
                double uh[4];
                for (int a = 0; a < 4; ++a) { double s = 0.0; for (int m = 0; m < 4; ++m) s += g->ei[a][m] * u[m]; uh[a] = s; }
                double Em = 0.0, B1 = 0.0, B2 = 0.0, A1 = 0.0, A2 = 0.0;
                double *Dd = malloc(sizeof(double) * nd), *n0 = malloc(sizeof(double) * nd), *Iold = malloc(sizeof(double) * nd);
                for (int s = 0; s < nd; ++s) {
                    const double *nh = c->G.dir + 3 * s;
                    double nup[4], nlo;
                    or_tetrad_dir(g, nh, nup, &nlo);
                    n0[s] = nup[0];
                    Dd[s] = uh[0] - (uh[1] * nh[0] + uh[2] * nh[1] + uh[3] * nh[2]);
                    Iold[s] = Ic[s];
                    double Ib = Dd[s] * Dd[s] * Dd[s] * Dd[s] * Ic[s];
                    double wb = c->G.w[s] / (Dd[s] * Dd[s]);
                    double K = 1.0 / (n0[s] / (atm * dtk) + Dd[s]);
                    Em += Ib * wb;
                    B1 += n0[s] * K * Ib * wb;
                    B2 += Dd[s] * K * wb;
                    A1 += n0[s] / (n0[s] + Dd[s] * atm * dtk) * Ib * wb;
                    A2 += Dd[s] / (n0[s] + Dd[s] * atm * dtk) * wb;
                }
                B2 *= dtk / fourpi;
                A2 *= dtk / fourpi;
                double Estar, Tp, aap, atp;
                if (c->c.coupling == 1 || c->c.coupling == 2) {
                    meq q = {A1, A2, Em + Y * Tm, Y, Tm, Em, au, as, eta, c->c.arad, c->c.T_exp, c->c.coupling};
                    if (!solve_meq(&q, &Estar)) {   /* no positive temperature: the cell is left as it was */
                        ++fails;
                        free(Dd); free(n0); free(Iold);
                        continue;
                    }
                    Tp = meq_T(&q, Estar);
                    aap = meq_aaP(&q, Tp);
                    atp = atm;                      /* the total absorption stays explicit */
                } else {
                    teq q = {B1, B2, Em + Y * Tm, Y, Tm, Em, au, as, eta, c->c.arad, dtk, c->c.T_exp};
                    if (!solve_E(&q, &Estar)) ++fails;
                    Tp = teq_T(&q, Estar);
                    aap = au * pow(Tp, -c->c.T_exp);
                    atp = aap + as;
                }
                double em = eta * aap * c->c.arad * Tp * Tp * Tp * Tp + as * Estar;
                double Ep = 0.0, dR[4] = {0, 0, 0, 0};
                for (int s = 0; s < nd; ++s) {
                    double D4 = Dd[s] * Dd[s] * Dd[s] * Dd[s];
                    double Ib = D4 * Ic[s];
                    double Ibp = (n0[s] * Ib + Dd[s] * dtk * em / fourpi) / (n0[s] + Dd[s] * atp * dtk);
                    double In = Ibp / D4;
                    const double *nh = c->G.dir + 3 * s;
                    double nup[4], nlo;
                    or_tetrad_dir(g, nh, nup, &nlo);
                    if (fabs(nlo) < c->c.n0_cut || or_pole_zero(c, j)) In = 0.0;
                    Ic[s] = In;
                    Ep += Dd[s] * Dd[s] * In * c->G.w[s];
                    double dI = (In - Iold[s]) * c->G.w[s];
                    dR[0] += dI; dR[1] += nh[0] * dI; dR[2] += nh[1] * dI; dR[3] += nh[2] * dI;
                }
                ug_out[ci] = ugm - (Ep - Em);
                if (G4) for (int m = 0; m < 4; ++m) {
                    double s = 0.0;
                    for (int a = 0; a < 4; ++a) s += g->e[a][m] * dR[a];
                    G4[4 * (size_t)ci + m] = -s / dtk;
                }
                free(Dd); free(n0); free(Iold);
            }
    return fails;
}
