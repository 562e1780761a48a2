/*
 * or_geom.c — metric, tetrad and Ricci rotation coefficients of the oracle.
 * TEST INFRASTRUCTURE ONLY (see rt_oracle.h).
 *
 *  - Tetrad: orthonormality eq. (tetrad_def); the time leg is the unit normal
 *    to t = const, eq. (tetrad_restriction); the spatial legs are Gram-Schmidt
 *    of (d_3, d_2, d_1) under the spatial metric, giving (3,2,1) = (phi, theta, r)
 *    hats in Kerr-Schild (section 2.1.1 and App. A.2; the appendix's printed
 *    components are garbled, the normal-observer legs reproduce its legible
 *    entries).
 *  - Ricci rotation coefficients eq. (ricci_rotation_coefficients):
 *    omega^a_{bc} = e^a_beta e^mu_b (d_mu e^beta_c + Gamma^beta_{mu nu} e^nu_c).
 *    All derivatives are exact: the metric and the tetrad are evaluated on
 *    forward-mode dual numbers, one run per coordinate direction.
 *  - Kerr-Schild metric in logical coordinates x1 = ln r, x2 = theta, x3 = phi
 *    (the textbook Kerr-Schild form with dr = r dx1).
 *  - Snake coordinates (App. A.1): (w, y, z) with w = x - A sin(k pi y), the
 *    metric of dx = dw + delta dy, delta = A k pi cos(k pi y); the tetrad is the
 *    same Gram-Schmidt construction.  (The appendix prints a tetrad that is not
 *    orthonormal under its own metric; this reading keeps eq. tetrad_def.)
 *  - Flat space in Cartesian coordinates with the tetrad aligned with the
 *    cylindrical unit vectors (section 4.5): e_1 = r-hat, e_2 = phi-hat,
 *    e_3 = z-hat, phi = atan2(y, x).  (The printed matrix of
 *    eq. cylindrical_alignment is garbled; this is the frame the text names.)
 */
#include "or_internal.h"

typedef struct { double v, d; } dn;
static dn D(double v) { dn o = {v, 0.0}; return o; }
static dn dadd(dn a, dn b) { dn o = {a.v + b.v, a.d + b.d}; return o; }
static dn dsub(dn a, dn b) { dn o = {a.v - b.v, a.d - b.d}; return o; }
static dn dmul(dn a, dn b) { dn o = {a.v * b.v, a.d * b.v + a.v * b.d}; return o; }
static dn ddiv(dn a, dn b) { dn o = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; return o; }
static dn dsqrt(dn a) { double s = sqrt(a.v); dn o = {s, a.d / (2.0 * s)}; return o; }
static dn dneg(dn a) { dn o = {-a.v, -a.d}; return o; }
static dn dsin(dn a) { dn o = {sin(a.v), cos(a.v) * a.d}; return o; }
static dn dcos(dn a) { dn o = {cos(a.v), -sin(a.v) * a.d}; return o; }
static dn dexp(dn a) { double e = exp(a.v); dn o = {e, e * a.d}; return o; }

/* g_{mu nu}(x) with derivative along coordinate wrt (1 or 2; 0 = none) */
static void metric(const or_config *c, const double x[3], int wrt, dn g[4][4]) {
    for (int m = 0; m < 4; ++m) for (int n = 0; n < 4; ++n) g[m][n] = D(0.0);
    if (c->coords == OR_MINKOWSKI_CART || c->coords == OR_CART_CYLTETRAD) {
        g[0][0] = D(-1.0); g[1][1] = D(1.0); g[2][2] = D(1.0); g[3][3] = D(1.0);
        return;
    }
    if (c->coords == OR_SNAKE) {
        dn y = {x[1], wrt == 2 ? 1.0 : 0.0};
        dn kp = D(c->snake_k * M_PI);
        dn del = dmul(D(c->snake_A), dmul(kp, dcos(dmul(kp, y))));
        g[0][0] = D(-1.0); g[1][1] = D(1.0); g[3][3] = D(1.0);
        g[1][2] = g[2][1] = del;
        g[2][2] = dadd(D(1.0), dmul(del, del));
        return;
    }
    dn x1 = {x[0], wrt == 1 ? 1.0 : 0.0}, th = {x[1], wrt == 2 ? 1.0 : 0.0};
    dn r = dexp(x1);
    dn ct = dcos(th), st = dsin(th);
    dn a = D(c->a), M = D(c->M);
    dn sig = dadd(dmul(r, r), dmul(dmul(a, a), dmul(ct, ct)));
    dn z = ddiv(dmul(D(2.0), dmul(M, r)), sig);
    dn s2 = dmul(st, st);
    dn opz = dadd(D(1.0), z);
    g[0][0] = dneg(dsub(D(1.0), z));
    g[0][1] = g[1][0] = dmul(z, r);
    g[0][3] = g[3][0] = dneg(dmul(z, dmul(a, s2)));
    g[1][1] = dmul(opz, dmul(r, r));
    g[1][3] = g[3][1] = dneg(dmul(dmul(a, s2), dmul(opz, r)));
    g[2][2] = sig;
    g[3][3] = dmul(s2, dadd(sig, dmul(dmul(a, a), dmul(s2, opz))));
}

/* inverse by Gauss-Jordan elimination with partial pivoting (on values) */
static void inverse4(dn A[4][4], dn B[4][4]) {
    dn M[4][8];
    for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) { M[i][j] = A[i][j]; M[i][4 + j] = D(i == j ? 1.0 : 0.0); }
    for (int col = 0; col < 4; ++col) {
        int p = col;
        for (int r = col + 1; r < 4; ++r) if (fabs(M[r][col].v) > fabs(M[p][col].v)) p = r;
        if (p != col) for (int j = 0; j < 8; ++j) { dn t = M[col][j]; M[col][j] = M[p][j]; M[p][j] = t; }
        dn piv = M[col][col];
        for (int j = 0; j < 8; ++j) M[col][j] = ddiv(M[col][j], piv);
        for (int r = 0; r < 4; ++r) if (r != col) {
            dn f = M[r][col];
            for (int j = 0; j < 8; ++j) M[r][j] = dsub(M[r][j], dmul(f, M[col][j]));
        }
    }
    for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) B[i][j] = M[i][4 + j];
}

static double det4(const double A[4][4]) {
    double M[4][4]; memcpy(M, A, sizeof(M));
    double det = 1.0;
    for (int col = 0; col < 4; ++col) {
        int p = col;
        for (int r = col + 1; r < 4; ++r) if (fabs(M[r][col]) > fabs(M[p][col])) p = r;
        if (p != col) { for (int j = 0; j < 4; ++j) { double t = M[col][j]; M[col][j] = M[p][j]; M[p][j] = t; } det = -det; }
        det *= M[col][col];
        if (M[col][col] == 0.0) return 0.0;
        for (int r = col + 1; r < 4; ++r) {
            double f = M[r][col] / M[col][col];
            for (int j = col; j < 4; ++j) M[r][j] -= f * M[col][j];
        }
    }
    return det;
}

/* spatial inner product gamma(u, v) of purely spatial vectors */
static dn sdot(dn g[4][4], const dn u[4], const dn v[4]) {
    dn s = D(0.0);
    for (int i = 1; i < 4; ++i) for (int j = 1; j < 4; ++j) s = dadd(s, dmul(g[i][j], dmul(u[i], v[j])));
    return s;
}

/* tetrad legs e[a][mu] = e^mu_(a) on dual numbers */
static void tetrad(dn g[4][4], dn gi[4][4], dn e[4][4]) {
    dn lapse_inv = dsqrt(dneg(gi[0][0]));           /* sqrt(-g^00) */
    for (int m = 0; m < 4; ++m) e[0][m] = dneg(ddiv(gi[0][m], lapse_inv));
    dn b[4][4];   /* coordinate basis d_0..d_3 as 4-vectors */
    for (int i = 0; i < 4; ++i) for (int m = 0; m < 4; ++m) b[i][m] = D(i == m ? 1.0 : 0.0);
    dn n3 = dsqrt(sdot(g, b[3], b[3]));
    for (int m = 0; m < 4; ++m) e[3][m] = ddiv(b[3][m], n3);
    dn p = sdot(g, b[2], e[3]), v[4];
    for (int m = 0; m < 4; ++m) v[m] = dsub(b[2][m], dmul(p, e[3][m]));
    dn n2 = dsqrt(sdot(g, v, v));
    for (int m = 0; m < 4; ++m) e[2][m] = ddiv(v[m], n2);
    dn p3 = sdot(g, b[1], e[3]), p2 = sdot(g, b[1], e[2]);
    for (int m = 0; m < 4; ++m) v[m] = dsub(dsub(b[1][m], dmul(p3, e[3][m])), dmul(p2, e[2][m]));
    dn n1 = dsqrt(sdot(g, v, v));
    for (int m = 0; m < 4; ++m) e[1][m] = ddiv(v[m], n1);
}

/* tetrad (r-hat, phi-hat, z-hat) of Cartesian coordinates at (x, y) */
static void tetrad_cyl(const double x[3], int wrt, dn e[4][4]) {
    for (int a = 0; a < 4; ++a) for (int m = 0; m < 4; ++m) e[a][m] = D(0.0);
    dn X = {x[0], wrt == 1 ? 1.0 : 0.0}, Y = {x[1], wrt == 2 ? 1.0 : 0.0};
    dn r = dsqrt(dadd(dmul(X, X), dmul(Y, Y)));
    dn c = ddiv(X, r), s = ddiv(Y, r);
    e[0][0] = D(1.0);
    e[1][1] = c; e[1][2] = s;
    e[2][1] = dneg(s); e[2][2] = c;
    e[3][3] = D(1.0);
}

void or_geometry(const or_config *c, const double x[3], int want_omega, or_geom *out) {
    dn g[3][4][4], gi[3][4][4], e[3][4][4];
    for (int w = 0; w < 3; ++w) {
        metric(c, x, w, g[w]);
        inverse4(g[w], gi[w]);
        if (c->coords == OR_CART_CYLTETRAD) tetrad_cyl(x, w, e[w]);
        else tetrad(g[w], gi[w], e[w]);
        if (!want_omega) break;
    }
    for (int m = 0; m < 4; ++m) for (int n = 0; n < 4; ++n) {
        out->g[m][n] = g[0][m][n].v; out->gi[m][n] = gi[0][m][n].v; out->e[m][n] = e[0][m][n].v;
    }
    double dt = det4(out->g);
    out->sqrtg = dt < 0.0 ? sqrt(-dt) : 0.0;
    /* inverse tetrad e^(a)_mu = eta^{ab} g_{mu nu} e^nu_(b) */
    for (int a = 0; a < 4; ++a) for (int m = 0; m < 4; ++m) {
        double s = 0.0;
        for (int n = 0; n < 4; ++n) s += out->g[m][n] * out->e[a][n];
        out->ei[a][m] = (a == 0 ? -s : s);
    }
    memset(out->om, 0, sizeof(out->om));
    if (!want_omega) return;
    /* derivatives: index 0 and 3 vanish (static, axisymmetric / flat) */
    double dg[4][4][4] = {{{0}}};     /* dg[mu][a][b] = d_mu g_ab */
    double de[4][4][4] = {{{0}}};     /* de[mu][c][beta] = d_mu e^beta_(c) */
    for (int mu = 1; mu <= 2; ++mu)
        for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) {
            dg[mu][a][b] = g[mu][a][b].d; de[mu][a][b] = e[mu][a][b].d;
        }
    double Gam[4][4][4];   /* Gam[beta][mu][nu] */
    for (int be = 0; be < 4; ++be) for (int mu = 0; mu < 4; ++mu) for (int nu = 0; nu < 4; ++nu) {
        double s = 0.0;
        for (int la = 0; la < 4; ++la)
            s += out->gi[be][la] * (dg[mu][la][nu] + dg[nu][la][mu] - dg[la][mu][nu]);
        Gam[be][mu][nu] = 0.5 * s;
    }
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int cc = 0; cc < 4; ++cc) {
        double s = 0.0;
        for (int be = 0; be < 4; ++be) for (int mu = 0; mu < 4; ++mu) {
            double cov = de[mu][cc][be];
            for (int nu = 0; nu < 4; ++nu) cov += Gam[be][mu][nu] * out->e[cc][nu];
            s += out->ei[a][be] * out->e[b][mu] * cov;
        }
        out->om[a][b][cc] = s;
    }
}

int or_geometry_at(const or_ctx *c, const double x[3], double *g, double *e, double *omega, double *sqrtg) {
    or_geom G;
    or_geometry(&c->c, x, 1, &G);
    for (int m = 0; m < 16; ++m) { g[m] = G.g[m / 4][m % 4]; e[m] = G.e[m / 4][m % 4]; }
    for (int m = 0; m < 64; ++m) omega[m] = G.om[m / 16][(m / 4) % 4][m % 4];
    *sqrtg = G.sqrtg;
    return 0;
}
