/*
 * or_adjoint.c — reverse mode of the oracle's step, hand-derived (test
 * infrastructure only).
 *
 * Scope: flat Cartesian geometry with the fluid at rest (D = 1, n^0 = 1,
 * no fluid advection), any limiter, order 1 or 2.  The gradient of a scalar
 * L(I_N, u_g,N) with respect to the initial intensity, the per-cell absorption
 * prefactor kappa and the emission multiplier eta is accumulated by running
 * every stage backwards:
 *  - interaction (section 3.5.2, method 3): the reverse of the explicit
 *    pieces, and the implicit function theorem at the temperature root,
 *    d(E*)/d(theta) = -(dh/d(theta)) / (dh/d(E*));
 *  - transport (eq. radiative_transfer_discrete): the transpose of the
 *    linearised face fluxes, with the limiter branches of the forward state
 *    and the derivative of the face coefficients c1, c2, c3 with respect to
 *    the optical depth (eqs. rad_speeds, flux_Jiang), which carries the
 *    gradient into kappa and u_g through the opacity.
 */
#include "or_internal.h"

/* derivative of the limited slope with respect to (dl, dr), same branches as
   or_limiter */
static void lim_grad(int kind, double dl, double dr, double *gl, double *gr) {
    *gl = 0.0; *gr = 0.0;
    if (kind == 2 || dl * dr <= 0.0) return;
    double al = fabs(dl), ar = fabs(dr);
    if (kind == 1) { if (al < ar) *gl = 1.0; else *gr = 1.0; return; }
    double m = 2.0 * al;
    int which = 0;
    if (2.0 * ar < m) { m = 2.0 * ar; which = 1; }
    if (0.5 * fabs(dl + dr) < m) which = 2;
    if (which == 0) *gl = 2.0;
    else if (which == 1) *gr = 2.0;
    else { *gl = 0.5; *gr = 0.5; }
}

/* face coefficients c1 = f e/(f+g), c2 = g e/(f+g), c3 = f g/(f+g) and their
   derivatives with respect to tau; f = sqrt(1 - e^-tau^2)/tau,
   g = sqrt(1 - e^-tau^4)/tau, e = e^-tau (the flux of eq. flux_Jiang per unit
   n: n (cL I_L + cR I_R) - |n| c3 (I_{l+1} - I_l)) */
static void face_coeffs(double tau, double c[3], double dc[3]) {
    if (!(tau > 0.0)) {
        c[0] = 1.0; c[1] = 0.0; c[2] = 0.0;
        dc[0] = -2.0; dc[1] = 1.0; dc[2] = 1.0;
        return;
    }
    double F = -expm1(-tau * tau), G = -expm1(-tau * tau * tau * tau);
    double f = sqrt(F) / tau, g = sqrt(G) / tau, e = exp(-tau);
    double fp = exp(-tau * tau) / sqrt(F) - f / tau;
    double gp = G > 0.0 ? 2.0 * tau * tau * exp(-tau * tau * tau * tau) / sqrt(G) - g / tau : 1.0;
    double ep = -e, S = f + g, Sp = fp + gp;
    c[0] = f * e / S; c[1] = g * e / S; c[2] = f * g / S;
    dc[0] = ((fp * e + f * ep) * S - f * e * Sp) / (S * S);
    dc[1] = ((gp * e + g * ep) * S - g * e * Sp) / (S * S);
    dc[2] = ((fp * g + f * gp) * S - f * g * Sp) / (S * S);
}

static int check_scope(const or_ctx *c) {
    if (c->c.coords != OR_MINKOWSKI_CART) { or_set_err("adjoint: flat Cartesian geometry only"); return 0; }
    for (int ci = 0; ci < c->ncell; ++ci) {
        const double *u = c->ucon + 4 * (size_t)ci;
        if (u[0] != 1.0 || u[1] != 0.0 || u[2] != 0.0 || u[3] != 0.0) { or_set_err("adjoint: fluid at rest only"); return 0; }
    }
    return 1;
}

/* reverse of one transport stage Iout = Ibase - dtk sum_a [Phi]/dx_a:
   Ib_out (cotangent of Iout) -> accumulate Ib_src, Ib_base, ub_src (through
   the opacity of the flux), kb */
static void transport_adj(or_ctx *c, const double *Isrc, const double *ug_src, double dtk, const double *Ib_out,
                          double *Ib_src, double *Ib_base, double *ub_src, double *kb) {
    int nd = c->G.nd;
    size_t ncell = (size_t)c->ncell, ngc = (size_t)c->gn[0] * c->gn[1] * c->gn[2];
    for (size_t q = 0; q < ncell * nd; ++q) Ib_base[q] += Ib_out[q];
    double *Ig = malloc(sizeof(double) * ngc * nd), *Gb = calloc(ngc * nd, sizeof(double));
    double *alg = malloc(sizeof(double) * ngc), *abar_g = calloc(ngc, sizeof(double));
    int *gmap = malloc(sizeof(int) * ngc), *gmir = malloc(sizeof(int) * ngc), *gfix = malloc(sizeof(int) * ngc);
    int *ginterior = malloc(sizeof(int) * ngc);
    or_fill_ghosts(c, Isrc, Ig);
    for (int k = -c->ng[2]; k < c->c.nx[2] + c->ng[2]; ++k)
        for (int j = -c->ng[1]; j < c->c.nx[1] + c->ng[1]; ++j)
            for (int i = -c->ng[0]; i < c->c.nx[0] + c->ng[0]; ++i) {
                int idx[3] = {i, j, k}, mir, row;
                int ok = or_map_cell(c, idx, &mir, &row);
                int gi = or_gidx(c, i, j, k), ci = or_cidx(c, idx[0], idx[1], idx[2]);
                gmap[gi] = ci; gmir[gi] = mir; gfix[gi] = !ok;
                ginterior[gi] = (i >= 0 && i < c->c.nx[0] && j >= 0 && j < c->c.nx[1] && k >= 0 && k < c->c.nx[2]);
                alg[gi] = or_cell_alpha(c, c->rho[ci], ug_src[ci], c->kap[ci], c->cs[ci]);
            }
    int stride[3] = {1, c->gn[0], c->gn[0] * c->gn[1]};
    for (int a = 0; a < 3; ++a) {
        if (!c->active[a]) continue;
        double dxa = c->c.dx[a];
        /* faces between cells idx-1 and idx along a, idx in [0, nx_a] */
        for (int k = 0; k < c->c.nx[2] + (a == 2); ++k)
            for (int j = 0; j < c->c.nx[1] + (a == 1); ++j)
                for (int i = 0; i < c->c.nx[0] + (a == 0); ++i) {
                    int gr = or_gidx(c, i, j, k), gl = gr - stride[a];
                    double len = c->c.tau_dt ? dtk : dxa;
                    double tau = c->c.abar * 0.5 * (alg[gl] + alg[gr]) * len;
                    double cf[3], dcf[3];
                    face_coeffs(tau, cf, dcf);
                    double cb[3] = {0.0, 0.0, 0.0};
                    int lin = ginterior[gl], rin = ginterior[gr];
                    for (int s = 0; s < nd; ++s) {
                        double n = c->G.dir[3 * s + a];
                        double ol = lin ? Ib_out[(size_t)gmap[gl] * nd + s] : 0.0;
                        double orr = rin ? Ib_out[(size_t)gmap[gr] * nd + s] : 0.0;
                        double phib = dtk / dxa * (orr - ol);
                        if (phib == 0.0 || n == 0.0) continue;
                        double Ill = Ig[(size_t)(gl - stride[a]) * nd + s], Il = Ig[(size_t)gl * nd + s];
                        double Ir = Ig[(size_t)gr * nd + s], Irr = Ig[(size_t)(gr + stride[a]) * nd + s];
                        double sl = or_limiter(c->c.limiter, Ir - Il, Il - Ill);
                        double sr = or_limiter(c->c.limiter, Irr - Ir, Ir - Il);
                        double IL = Il + 0.5 * sl, IR = Ir - 0.5 * sr;
                        double cL = n > 0.0 ? cf[0] : cf[1], cR = n > 0.0 ? cf[1] : cf[0];
                        double an = fabs(n);
                        double ILb = phib * n * cL, IRb = phib * n * cR;
                        double *Gl = Gb + (size_t)gl * nd, *Gr = Gb + (size_t)gr * nd;
                        double *Gll = Gb + (size_t)(gl - stride[a]) * nd, *Grr = Gb + (size_t)(gr + stride[a]) * nd;
                        Gl[s] += phib * an * cf[2];
                        Gr[s] -= phib * an * cf[2];
                        double gla, glb;
                        Gl[s] += ILb;
                        lim_grad(c->c.limiter, Ir - Il, Il - Ill, &gla, &glb);
                        Gr[s] += 0.5 * ILb * gla; Gl[s] -= 0.5 * ILb * gla;
                        Gl[s] += 0.5 * ILb * glb; Gll[s] -= 0.5 * ILb * glb;
                        Gr[s] += IRb;
                        lim_grad(c->c.limiter, Irr - Ir, Ir - Il, &gla, &glb);
                        Grr[s] -= 0.5 * IRb * gla; Gr[s] += 0.5 * IRb * gla;
                        Gr[s] -= 0.5 * IRb * glb; Gl[s] += 0.5 * IRb * glb;
                        double cLb = phib * n * IL, cRb = phib * n * IR;
                        cb[0] += n > 0.0 ? cLb : cRb;
                        cb[1] += n > 0.0 ? cRb : cLb;
                        cb[2] += -phib * an * (Ir - Il);
                    }
                    double taub = cb[0] * dcf[0] + cb[1] * dcf[1] + cb[2] * dcf[2];
                    double ab = taub * c->c.abar * 0.5 * len;
                    abar_g[gl] += ab; abar_g[gr] += ab;
                }
    }
    /* ghost cotangents back to the cells they copy */
    for (size_t gi = 0; gi < ngc; ++gi) {
        size_t ci = (size_t)gmap[gi];
        if (!gfix[gi]) for (int s = 0; s < nd; ++s) Ib_src[ci * nd + (gmir[gi] ? c->G.mirror[s] : s)] += Gb[gi * nd + s];
        /* opacity of the cell (ghost fluid is the copied cell's) */
        double rho = c->rho[ci];
        if (abar_g[gi] != 0.0 && rho >= c->c.rho_floor && rho > 0.0) {
            double T = (c->c.gam - 1.0) * ug_src[ci] / rho;
            double rm = pow(rho, c->c.rho_exp), tp = pow(T, -c->c.T_exp);
            kb[ci] += abar_g[gi] * rm * tp;
            ub_src[ci] += abar_g[gi] * c->kap[ci] * rm * (-c->c.T_exp) * tp / T * (c->c.gam - 1.0) / rho;
        }
    }
    free(Ig); free(Gb); free(alg); free(abar_g); free(gmap); free(gmir); free(gfix); free(ginterior);
}

/* a stage of section 3.6 with the transport switched off (a source-only
   configuration) leaves its base unchanged: Iout = Ibase, whose reverse adds
   Ib_out to the base's cotangent */
static void stage_fwd(or_ctx *c, const double *Isrc, const double *ug_src, const double *Ibase, double dtk,
                      double *Iout) {
    if (c->c.transport) or_transport_stage(c, Isrc, ug_src, Ibase, dtk, Iout);
    else memcpy(Iout, Ibase, sizeof(double) * (size_t)c->ncell * c->G.nd);
}
static void stage_adj(or_ctx *c, const double *Isrc, const double *ug_src, double dtk, const double *Ib_out,
                      double *Ib_src, double *Ib_base, double *ub_src, double *kb) {
    if (c->c.transport) { transport_adj(c, Isrc, ug_src, dtk, Ib_out, Ib_src, Ib_base, ub_src, kb); return; }
    const size_t ni = (size_t)c->ncell * c->G.nd;
    for (size_t e = 0; e < ni; ++e) Ib_base[e] += Ib_out[e];
}

/* reverse of one interaction step (fluid at rest): Iin = transported
   intensities, ugin = gas energy entering; Ib_out, ub_out = cotangents of the
   outputs -> accumulate Ib_in, ub_in, kb, eb */
static void source_adj(or_ctx *c, const double *Iin, const double *ugin, double dtk, const double *Ib_out,
                       const double *ub_out, double *Ib_in, double *ub_in, double *kb, double *eb) {
    int nd = c->G.nd;
    const double fourpi = 4.0 * M_PI, a_ = c->c.arad, p = c->c.T_exp;
    double S = 0.0;
    for (int s = 0; s < nd; ++s) S += c->G.w[s];
    for (int ci = 0; ci < c->ncell; ++ci) {
        const double *I = Iin + (size_t)ci * nd;
        const double *Ibo = Ib_out + (size_t)ci * nd;
        double *Ibi = Ib_in + (size_t)ci * nd;
        double rho = c->rho[ci], u = ugin[ci];
        double Y = rho / (c->c.gam - 1.0), Tm = u / Y;
        double au = c->kap[ci] * pow(rho, c->c.rho_exp), as = c->cs[ci] * rho, eta = c->eta[ci];
        int on = c->c.source && rho >= c->c.rho_floor && rho > 0.0 && Tm > 0.0 && (au + as) > 0.0;
        if (!on) {
            for (int s = 0; s < nd; ++s) Ibi[s] += Ibo[s];
            ub_in[ci] += ub_out[ci];
            continue;
        }
        /* forward (the same operations as or_source_step with D = 1, n^0 = 1) */
        double am = au * pow(Tm, -p) + as;
        double Em = 0.0;
        for (int s = 0; s < nd; ++s) Em += I[s] * c->G.w[s];
        double K = am * dtk / (1.0 + am * dtk);
        double B1 = K * Em, B2 = K * S * dtk / fourpi;
        /* root E* of h (monotone; bisection as in the forward) */
        double lo = 0.0, hi = Em + Y * Tm;
        for (int it = 0; it < 2000; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double T = Tm + (Em - mid) / Y;
            double h;
            if (!(T > 0.0)) h = INFINITY;
            else { double aa = au * pow(T, -p); h = ((aa + as) * dtk - B2 * as) * mid - B1 - B2 * eta * aa * a_ * T * T * T * T; }
            if (h > 0.0) hi = mid; else lo = mid;
        }
        double X = 0.5 * (lo + hi);
        double Tp = Tm + (Em - X) / Y;
        double aap = au * pow(Tp, -p), atp = aap + as;
        double cc = dtk * (eta * aap * a_ * Tp * Tp * Tp * Tp + as * X) / fourpi;
        double A = 1.0 + atp * dtk;
        /* reverse */
        double ub = ub_out[ci];
        ub_in[ci] += ub;
        double Epb = -ub, Emb = ub;
        double ccb = 0.0, Ab = 0.0;
        for (int s = 0; s < nd; ++s) {
            double Ipb = Ibo[s] + Epb * c->G.w[s];
            double Ip = (I[s] + cc) / A;
            Ibi[s] += Ipb / A;
            ccb += Ipb / A;
            Ab += -Ipb * Ip / A;
        }
        double aapb = Ab * dtk;                           /* A = 1 + (aap + as) dt */
        double Tp4 = Tp * Tp * Tp * Tp;
        eb[ci] += ccb * dtk * aap * a_ * Tp4 / fourpi;
        aapb += ccb * dtk * eta * a_ * Tp4 / fourpi;
        double Tpb = ccb * dtk * eta * aap * a_ * 4.0 * Tp * Tp * Tp / fourpi;
        double Xb = ccb * dtk * as / fourpi;
        double aub = aapb * pow(Tp, -p);
        Tpb += aapb * (-p) * aap / Tp;
        double Tmb = Tpb;
        Emb += Tpb / Y;
        Xb += -Tpb / Y;
        /* implicit root: h(X; B1, B2, Tm, Em, au, eta) = 0 */
        double aa = aap, lin = (aa + as) * dtk - B2 * as;
        double hT = -p * aa / Tp * dtk * X - B2 * eta * a_ * (4.0 - p) * aa * Tp * Tp * Tp;
        double hX = lin - hT / Y;
        double lam = -Xb / hX;
        double B1b = -lam;
        double B2b = lam * (-as * X - eta * a_ * aa * Tp4);
        Tmb += lam * hT;
        Emb += lam * hT / Y;
        aub += lam * (pow(Tp, -p) * dtk * X - B2 * eta * a_ * pow(Tp, -p) * Tp4);
        eb[ci] += lam * (-B2 * a_ * aa * Tp4);
        double Kb = B2b * S * dtk / fourpi + B1b * Em;
        Emb += B1b * K;
        double amb = Kb * dtk / ((1.0 + am * dtk) * (1.0 + am * dtk));
        aub += amb * pow(Tm, -p);
        Tmb += amb * (-p) * au * pow(Tm, -p) / Tm;
        ub_in[ci] += Tmb / Y;
        for (int s = 0; s < nd; ++s) Ibi[s] += Emb * c->G.w[s];
        kb[ci] += aub * pow(rho, c->c.rho_exp);
    }
}

int or_adjoint(or_ctx *c, const double *I0, const double *ug0, int nsteps, double dt,
               const double *dL_dI_out, const double *dL_dug_out,
               double *dL_dI0, double *dL_dkappa, double *dL_deta) {
    if (!check_scope(c)) return -1;
    size_t n = (size_t)c->ncell, ni = n * c->G.nd;
    double *In = malloc(sizeof(double) * ni * (nsteps + 1)), *un = malloc(sizeof(double) * n * (nsteps + 1));
    double *Is = malloc(sizeof(double) * ni), *Ist = malloc(sizeof(double) * ni), *I2 = malloc(sizeof(double) * ni);
    double *us = malloc(sizeof(double) * n), *tmpu = malloc(sizeof(double) * n);
    memcpy(In, I0, sizeof(double) * ni);
    memcpy(un, ug0, sizeof(double) * n);
    /* forward, keeping every step's state */
    for (int st = 0; st < nsteps; ++st) {
        const double *I = In + ni * st, *u = un + n * st;
        double *Inext = In + ni * (st + 1), *unext = un + n * (st + 1);
        if (c->c.order == 1) {
            stage_fwd(c, I, u, I, dt, Inext);
            or_source_step(c, Inext, u, unext, dt, NULL);
        } else {
            stage_fwd(c, I, u, I, 0.5 * dt, Ist);
            or_source_step(c, Ist, u, us, 0.5 * dt, NULL);
            stage_fwd(c, Ist, us, I, dt, Inext);
            or_source_step(c, Inext, u, unext, dt, NULL);
        }
    }
    double *Ib = malloc(sizeof(double) * ni), *ub = malloc(sizeof(double) * n);
    double *Ib2 = calloc(ni, sizeof(double)), *Ibs = calloc(ni, sizeof(double)), *Ibn = calloc(ni, sizeof(double));
    double *ubs = calloc(n, sizeof(double)), *ubn = calloc(n, sizeof(double));
    memcpy(Ib, dL_dI_out, sizeof(double) * ni);
    memcpy(ub, dL_dug_out, sizeof(double) * n);
    memset(dL_dkappa, 0, sizeof(double) * n);
    memset(dL_deta, 0, sizeof(double) * n);
    for (int st = nsteps - 1; st >= 0; --st) {
        const double *I = In + ni * st, *u = un + n * st;
        memset(Ibn, 0, sizeof(double) * ni); memset(ubn, 0, sizeof(double) * n);
        if (c->c.order == 1) {
            stage_fwd(c, I, u, I, dt, I2);
            memset(Ib2, 0, sizeof(double) * ni);
            source_adj(c, I2, u, dt, Ib, ub, Ib2, ubn, dL_dkappa, dL_deta);
            stage_adj(c, I, u, dt, Ib2, Ibn, Ibn, ubn, dL_dkappa);
        } else {
            /* recompute the stage intermediates */
            stage_fwd(c, I, u, I, 0.5 * dt, Is);
            memcpy(Ist, Is, sizeof(double) * ni);
            or_source_step(c, Ist, u, us, 0.5 * dt, NULL);
            stage_fwd(c, Ist, us, I, dt, I2);
            /* corrector interaction and transport */
            memset(Ib2, 0, sizeof(double) * ni);
            source_adj(c, I2, u, dt, Ib, ub, Ib2, ubn, dL_dkappa, dL_deta);
            memset(Ibs, 0, sizeof(double) * ni); memset(ubs, 0, sizeof(double) * n);
            stage_adj(c, Ist, us, dt, Ib2, Ibs, Ibn, ubs, dL_dkappa);
            /* predictor interaction and transport */
            memset(Ib2, 0, sizeof(double) * ni);
            source_adj(c, Is, u, 0.5 * dt, Ibs, ubs, Ib2, ubn, dL_dkappa, dL_deta);
            stage_adj(c, I, u, 0.5 * dt, Ib2, Ibn, Ibn, ubn, dL_dkappa);
        }
        memcpy(Ib, Ibn, sizeof(double) * ni);
        memcpy(ub, ubn, sizeof(double) * n);
    }
    memcpy(dL_dI0, Ib, sizeof(double) * ni);
    (void)tmpu;
    free(In); free(un); free(Is); free(Ist); free(I2); free(us); free(tmpu);
    free(Ib); free(ub); free(Ib2); free(Ibs); free(Ibn); free(ubs); free(ubn);
    return 0;
}
