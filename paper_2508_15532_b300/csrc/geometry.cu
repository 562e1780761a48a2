// geometry.cu — metric, tetrad and Ricci rotation coefficient cache (FP64).
//
// Section 2.1 / App. A.2.  One thread per (x1, x2) point of the ghosted
// geometry table (Kerr-Schild does not depend on x3 = phi; the paper keeps
// the same independence to cut its metric loads, section 5.2):
//   g_{mu nu}: Kerr-Schild in x1 = ln r, x2 = theta, x3 = phi;
//   g^{mu nu}: adjugate / determinant (Laplace expansion in 2x2 minors);
//   tetrad: time leg -g^{0 mu}/sqrt(-g^{00}) (eq. tetrad_restriction),
//     e_3 = d_3/|d_3|, e_2 = the part of d_2 orthogonal to d_3,
//     e_1 = the gradient of x1 raised with the spatial metric, normalised;
//   omega^a_{bc} = e^a_beta e^mu_b (d_mu e^beta_c + Gamma^beta_{mu nu} e^nu_c)
//     (eq. ricci_rotation_coefficients) with d_mu from forward-mode duals.
// Derived per (point, direction) and per (point, edge) tables feed the step.
#include "stage_common.cuh"
#include <cmath>

struct Dl {
    double v, d;
};
__device__ inline Dl mk(double v, double d = 0.0) { return {v, d}; }
__device__ inline Dl operator+(Dl a, Dl b) { return {a.v + b.v, a.d + b.d}; }
__device__ inline Dl operator-(Dl a, Dl b) { return {a.v - b.v, a.d - b.d}; }
__device__ inline Dl operator-(Dl a) { return {-a.v, -a.d}; }
__device__ inline Dl operator*(Dl a, Dl b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ inline Dl operator/(Dl a, Dl b) { double q = a.v / b.v; return {q, (a.d - q * b.d) / b.v}; }
__device__ inline Dl dl_sqrt(Dl a) { double r = sqrt(a.v); return {r, 0.5 * a.d / r}; }
__device__ inline Dl dl_sin(Dl a) { return {sin(a.v), cos(a.v) * a.d}; }
__device__ inline Dl dl_cos(Dl a) { return {cos(a.v), -sin(a.v) * a.d}; }
__device__ inline Dl dl_exp(Dl a) { double e = exp(a.v); return {e, e * a.d}; }

struct GeoPoint {
    Dl g[4][4], gi[4][4], e[4][4];   // e[a][mu] = e^mu_(a)
    Dl det;
};

// (M, a) are Kerr-Schild's mass and spin, or (A, k) of snake coordinates
__device__ void metric_ks(int kind, double M, double a, double x1, double x2, int wrt, Dl g[4][4]) {
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) g[m][n] = mk(0.0);
    if (kind == RT_MINKOWSKI_CART || kind == RT_CART_CYLTETRAD) {
        g[0][0] = mk(-1.0); g[1][1] = mk(1.0); g[2][2] = mk(1.0); g[3][3] = mk(1.0);
        return;
    }
    if (kind == RT_SNAKE) {
        // dx = dw + delta dy, delta = A k pi cos(k pi y), y = x2
        const Dl y = mk(x2, wrt == 2 ? 1.0 : 0.0), kp = mk(a * 3.14159265358979323846);
        const Dl del = mk(M) * kp * dl_cos(kp * y);
        g[0][0] = mk(-1.0); g[1][1] = mk(1.0); g[3][3] = mk(1.0);
        g[1][2] = g[2][1] = del;
        g[2][2] = mk(1.0) + del * del;
        return;
    }
    Dl r = dl_exp(mk(x1, wrt == 1 ? 1.0 : 0.0));
    Dl th = mk(x2, wrt == 2 ? 1.0 : 0.0);
    Dl s = dl_sin(th), c = dl_cos(th);
    Dl A = mk(a), A2 = mk(a * a);
    Dl sig = r * r + A2 * c * c;
    Dl z = mk(2.0 * M) * r / sig;
    Dl s2 = s * s;
    g[0][0] = z - mk(1.0);
    g[0][1] = g[1][0] = z * r;
    g[0][3] = g[3][0] = -(z * A * s2);
    g[1][1] = (mk(1.0) + z) * r * r;
    g[1][3] = g[3][1] = -(A * s2 * (mk(1.0) + z) * r);
    g[2][2] = sig;
    g[3][3] = s2 * (sig + A2 * s2 * (mk(1.0) + z));
}

__device__ void inverse_adj(const Dl a[4][4], Dl inv[4][4], Dl *det_out) {
    Dl s01 = a[0][0] * a[1][1] - a[0][1] * a[1][0], s02 = a[0][0] * a[1][2] - a[0][2] * a[1][0];
    Dl s03 = a[0][0] * a[1][3] - a[0][3] * a[1][0], s12 = a[0][1] * a[1][2] - a[0][2] * a[1][1];
    Dl s13 = a[0][1] * a[1][3] - a[0][3] * a[1][1], s23 = a[0][2] * a[1][3] - a[0][3] * a[1][2];
    Dl c01 = a[2][0] * a[3][1] - a[2][1] * a[3][0], c02 = a[2][0] * a[3][2] - a[2][2] * a[3][0];
    Dl c03 = a[2][0] * a[3][3] - a[2][3] * a[3][0], c12 = a[2][1] * a[3][2] - a[2][2] * a[3][1];
    Dl c13 = a[2][1] * a[3][3] - a[2][3] * a[3][1], c23 = a[2][2] * a[3][3] - a[2][3] * a[3][2];
    Dl C[4][4];
    C[0][0] = a[1][1] * c23 - a[1][2] * c13 + a[1][3] * c12;
    C[0][1] = -(a[1][0] * c23 - a[1][2] * c03 + a[1][3] * c02);
    C[0][2] = a[1][0] * c13 - a[1][1] * c03 + a[1][3] * c01;
    C[0][3] = -(a[1][0] * c12 - a[1][1] * c02 + a[1][2] * c01);
    C[1][0] = -(a[0][1] * c23 - a[0][2] * c13 + a[0][3] * c12);
    C[1][1] = a[0][0] * c23 - a[0][2] * c03 + a[0][3] * c02;
    C[1][2] = -(a[0][0] * c13 - a[0][1] * c03 + a[0][3] * c01);
    C[1][3] = a[0][0] * c12 - a[0][1] * c02 + a[0][2] * c01;
    C[2][0] = a[3][1] * s23 - a[3][2] * s13 + a[3][3] * s12;
    C[2][1] = -(a[3][0] * s23 - a[3][2] * s03 + a[3][3] * s02);
    C[2][2] = a[3][0] * s13 - a[3][1] * s03 + a[3][3] * s01;
    C[2][3] = -(a[3][0] * s12 - a[3][1] * s02 + a[3][2] * s01);
    C[3][0] = -(a[2][1] * s23 - a[2][2] * s13 + a[2][3] * s12);
    C[3][1] = a[2][0] * s23 - a[2][2] * s03 + a[2][3] * s02;
    C[3][2] = -(a[2][0] * s13 - a[2][1] * s03 + a[2][3] * s01);
    C[3][3] = a[2][0] * s12 - a[2][1] * s02 + a[2][2] * s01;
    Dl det = a[0][0] * C[0][0] + a[0][1] * C[0][1] + a[0][2] * C[0][2] + a[0][3] * C[0][3];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) inv[i][j] = C[j][i] / det;
    *det_out = det;
}

__device__ void build_point(int kind, double M, double a, double x1, double x2, int wrt, GeoPoint &P) {
    metric_ks(kind, M, a, x1, x2, wrt, P.g);
    inverse_adj(P.g, P.gi, &P.det);
    if (kind == RT_CART_CYLTETRAD) {
        // (r-hat, phi-hat, z-hat) of the Cartesian (x, y) = (x1, x2)
        const Dl X = mk(x1, wrt == 1 ? 1.0 : 0.0), Y = mk(x2, wrt == 2 ? 1.0 : 0.0);
        const Dl r = dl_sqrt(X * X + Y * Y), c = X / r, s = Y / r;
        for (int b = 0; b < 4; ++b)
            for (int m = 0; m < 4; ++m) P.e[b][m] = mk(0.0);
        P.e[0][0] = mk(1.0);
        P.e[1][1] = c; P.e[1][2] = s;
        P.e[2][1] = -s; P.e[2][2] = c;
        P.e[3][3] = mk(1.0);
        return;
    }
    Dl root = dl_sqrt(-P.gi[0][0]);
    for (int m = 0; m < 4; ++m) P.e[0][m] = -P.gi[0][m] / root;
    for (int b = 1; b < 4; ++b)
        for (int m = 0; m < 4; ++m) P.e[b][m] = mk(0.0);
    P.e[3][3] = mk(1.0) / dl_sqrt(P.g[3][3]);
    Dl r23 = P.g[2][3] / P.g[3][3];
    Dl n2 = dl_sqrt(P.g[2][2] - P.g[2][3] * r23);
    P.e[2][2] = mk(1.0) / n2;
    P.e[2][3] = -r23 / n2;
    Dl gam1[4];
    for (int j = 1; j < 4; ++j) gam1[j] = P.gi[1][j] - P.gi[0][1] * P.gi[0][j] / P.gi[0][0];
    Dl n1 = dl_sqrt(gam1[1]);
    for (int j = 1; j < 4; ++j) P.e[1][j] = gam1[j] / n1;
}

// One thread per ghosted (i, j) point: centre tetrad, inverse tetrad, volume,
// n^0, rotation coefficients; lower faces along each axis: tetrad, g_{0 mu},
// area and proper length.
__global__ void k_points(int kind, double M, double a, int gn0, int gn1, int ng0, int ng1, double x00, double x01,
                         double x02, double dx0, double dx1, double dx2, double *__restrict__ pe,
                         double *__restrict__ pei, double *__restrict__ pV, double *__restrict__ pn0,
                         double *__restrict__ pom, double *__restrict__ pg0, double *__restrict__ fe,
                         double *__restrict__ fg0, double *__restrict__ fA, double *__restrict__ plen) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int npt = gn0 * gn1;
    if (p >= npt) return;
    int i = p % gn0 - ng0, j = p / gn0 - ng1;
    double xc1 = x00 + (i + 0.5) * dx0, xc2 = x01 + (j + 0.5) * dx1;
    (void)x02;
    GeoPoint P[3];
    for (int w = 0; w < 3; ++w) build_point(kind, M, a, xc1, xc2, w, P[w]);
    for (int b = 0; b < 4; ++b)
        for (int m = 0; m < 4; ++m) pe[p * 16 + b * 4 + m] = P[0].e[b][m].v;
    for (int m = 0; m < 4; ++m) pg0[p * 4 + m] = P[0].g[0][m].v;
    double ei[4][4];
    for (int b = 0; b < 4; ++b)
        for (int m = 0; m < 4; ++m) {
            double s = 0.0;
            for (int n = 0; n < 4; ++n) s += P[0].g[m][n].v * P[0].e[b][n].v;
            ei[b][m] = b == 0 ? -s : s;
            pei[p * 16 + b * 4 + m] = ei[b][m];
        }
    double det = P[0].det.v;
    pV[p] = (det < 0.0 ? sqrt(-det) : 0.0) * dx0 * dx1 * dx2;
    pn0[p] = P[0].e[0][0].v;
    // Christoffel symbols and rotation coefficients (derivatives along x1, x2 only)
    double Gam[4][4][4];
    for (int be = 0; be < 4; ++be)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                double s = 0.0;
                for (int la = 0; la < 4; ++la) {
                    double d1 = (mu == 1 || mu == 2) ? P[mu].g[la][nu].d : 0.0;
                    double d2 = (nu == 1 || nu == 2) ? P[nu].g[la][mu].d : 0.0;
                    double d3 = (la == 1 || la == 2) ? P[la].g[mu][nu].d : 0.0;
                    s += P[0].gi[be][la].v * (d1 + d2 - d3);
                }
                Gam[be][mu][nu] = 0.5 * s;
            }
    for (int al = 0; al < 4; ++al)
        for (int b = 0; b < 4; ++b)
            for (int cc = 0; cc < 4; ++cc) {
                double s = 0.0;
                for (int mu = 0; mu < 4; ++mu) {
                    double emu = P[0].e[b][mu].v;
                    if (emu == 0.0) continue;
                    for (int be = 0; be < 4; ++be) {
                        double cov = (mu == 1 || mu == 2) ? P[mu].e[cc][be].d : 0.0;
                        for (int nu = 0; nu < 4; ++nu) cov += Gam[be][mu][nu] * P[0].e[cc][nu].v;
                        s += ei[al][be] * emu * cov;
                    }
                }
                pom[p * 64 + al * 16 + b * 4 + cc] = s;
            }
    // lower faces
    double dxs[3] = {dx0, dx1, dx2};
    for (int ax = 0; ax < 3; ++ax) {
        double f1 = xc1 - (ax == 0 ? 0.5 * dx0 : 0.0), f2 = xc2 - (ax == 1 ? 0.5 * dx1 : 0.0);
        GeoPoint F;
        build_point(kind, M, a, f1, f2, 0, F);
        size_t q = (size_t)ax * npt + p;
        for (int b = 0; b < 4; ++b)
            for (int m = 0; m < 4; ++m) fe[q * 16 + b * 4 + m] = F.e[b][m].v;
        for (int m = 0; m < 4; ++m) fg0[q * 4 + m] = F.g[0][m].v;
        double fd = F.det.v;
        double area = fd < 0.0 ? sqrt(-fd) : 0.0;
        for (int b = 0; b < 3; ++b) if (b != ax) area *= dxs[b];
        fA[q] = area;
        plen[q] = sqrt(F.g[ax + 1][ax + 1].v) * dxs[ax];
    }
}

// Per (point, direction): n^0 n_0 and masks at the centre; n^a and
// dA_a n_0 at each lower face (zero on faces of zero area).
__global__ void k_dir_tables(int npt, int nd, double n0cut, const double *__restrict__ dir,
                             const double *__restrict__ pe, const double *__restrict__ pg0,
                             const double *__restrict__ fe, const double *__restrict__ fg0,
                             const double *__restrict__ fA, double *__restrict__ cU, float *__restrict__ cUf,
                             uint8_t *__restrict__ mask, double *__restrict__ fn, float *__restrict__ fnf,
                             double *__restrict__ fP, float *__restrict__ fPf) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)npt * nd) return;
    int p = (int)(idx / nd), s = (int)(idx % nd);
    const double *nh = dir + 3 * s;
    auto nvec = [&](const double *e, double *n) {
        for (int m = 0; m < 4; ++m) n[m] = e[m] + nh[0] * e[4 + m] + nh[1] * e[8 + m] + nh[2] * e[12 + m];
    };
    double n[4];
    nvec(pe + (size_t)p * 16, n);
    const double *g0 = pg0 + (size_t)p * 4;
    double n0lo = g0[0] * n[0] + g0[1] * n[1] + g0[2] * n[2] + g0[3] * n[3];
    cU[idx] = n[0] * n0lo;
    cUf[idx] = (float)(n[0] * n0lo);
    mask[idx] = (uint8_t)((fabs(n0lo) < n0cut ? 1 : 0) | (n0lo > 0.0 ? 2 : 0));
    for (int ax = 0; ax < 3; ++ax) {
        size_t q = (size_t)ax * npt + p;
        double nf[4];
        nvec(fe + q * 16, nf);
        const double *h0 = fg0 + q * 4;
        double n0f = h0[0] * nf[0] + h0[1] * nf[1] + h0[2] * nf[2] + h0[3] * nf[3];
        double A = fA[q];
        bool ok = A > 0.0 && isfinite(nf[ax + 1]) && isfinite(n0f);
        double na = ok ? nf[ax + 1] : 0.0, P = ok ? A * n0f : 0.0;
        size_t o = (size_t)ax * npt * nd + idx;
        fn[o] = na; fnf[o] = (float)na;
        fP[o] = P; fPf[o] = (float)P;
    }
}

// Per (point, edge): dlam_e n_0(m) v(m).u_e, with the tangent drift of a
// photon direction m, v^i = -(omega^i_{bc} - m^i omega^0_{bc}) m^b m^c
// (geodesic equation in the tetrad frame; its components are the r^zeta,
// r^psi of eq. angular_n_vectors), taken at the edge midpoint (eq. angular_fluxes).
// eneg records where n_0(m) < 0: the flux takes its upwind value from the
// sign of v.u_e (eq. angular_fluxes), which there is the opposite of the sign
// of the tabulated product.
__global__ void k_edge_tables(int npt, int ne, const double *__restrict__ emid, const double *__restrict__ eu,
                              const double *__restrict__ dlam, const double *__restrict__ pe,
                              const double *__restrict__ pg0, const double *__restrict__ pom,
                              double *__restrict__ ew, float *__restrict__ ewf, uint8_t *__restrict__ eneg) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)npt * ne) return;
    int p = (int)(idx / ne), e = (int)(idx % ne);
    const double *m3 = emid + 3 * e, *u = eu + 3 * e, *om = pom + (size_t)p * 64, *E = pe + (size_t)p * 16;
    double m[4] = {1.0, m3[0], m3[1], m3[2]};
    double q[4];
    for (int al = 0; al < 4; ++al) {
        double s = 0.0;
        for (int b = 0; b < 4; ++b) {
            double t = 0.0;
            for (int cc = 0; cc < 4; ++cc) t += om[al * 16 + b * 4 + cc] * m[cc];
            s += t * m[b];
        }
        q[al] = s;
    }
    double vu = 0.0;
    for (int i = 0; i < 3; ++i) vu += -(q[i + 1] - m[i + 1] * q[0]) * u[i];
    double nup[4];
    for (int mu = 0; mu < 4; ++mu) nup[mu] = E[mu] + m[1] * E[4 + mu] + m[2] * E[8 + mu] + m[3] * E[12 + mu];
    const double *g0 = pg0 + (size_t)p * 4;
    double n0lo = g0[0] * nup[0] + g0[1] * nup[1] + g0[2] * nup[2] + g0[3] * nup[3];
    double v = dlam[e] * n0lo * vu;
    ew[idx] = v;
    ewf[idx] = (float)v;
    eneg[idx] = n0lo < 0.0;
}

rt_status rt_build_geometry(rt_ctx *c) {
    const rt_config &cf = c->cfg;
    int ng0 = c->active[0] ? 2 : 0, ng1 = c->active[1] ? 2 : 0;
    c->gn[0] = cf.nx[0] + 2 * ng0;
    c->gn[1] = cf.nx[1] + 2 * ng1;
    int npt = c->gn[0] * c->gn[1];
    int nd = c->nd, ne = c->ne;
    double *pg0 = nullptr, *fe = nullptr, *fg0 = nullptr, *fA = nullptr;
    auto A = [&](void **p, size_t bytes) { return cudaMalloc(p, bytes); };
    RT_CUDA_TRY(c, A((void **)&c->pt_e, sizeof(double) * 16 * npt));
    RT_CUDA_TRY(c, A((void **)&c->pt_ei, sizeof(double) * 16 * npt));
    RT_CUDA_TRY(c, A((void **)&c->pt_V, sizeof(double) * npt));
    RT_CUDA_TRY(c, A((void **)&c->pt_n0, sizeof(double) * npt));
    RT_CUDA_TRY(c, A((void **)&c->pt_len, sizeof(double) * 3 * npt));
    RT_CUDA_TRY(c, A((void **)&c->pt_om, sizeof(double) * 64 * npt));
    RT_CUDA_TRY(c, A((void **)&pg0, sizeof(double) * 4 * npt));
    RT_CUDA_TRY(c, A((void **)&fe, sizeof(double) * 16 * 3 * npt));
    RT_CUDA_TRY(c, A((void **)&fg0, sizeof(double) * 4 * 3 * npt));
    RT_CUDA_TRY(c, A((void **)&fA, sizeof(double) * 3 * npt));
    size_t nPD = (size_t)npt * nd, nPE = (size_t)npt * ne;
    RT_CUDA_TRY(c, A((void **)&c->cenU_d, sizeof(double) * nPD));
    RT_CUDA_TRY(c, A((void **)&c->cenU_f, sizeof(float) * nPD));
    RT_CUDA_TRY(c, A((void **)&c->mask, nPD));
    RT_CUDA_TRY(c, A((void **)&c->fn_d, sizeof(double) * 3 * nPD));
    RT_CUDA_TRY(c, A((void **)&c->fn_f, sizeof(float) * 3 * nPD));
    RT_CUDA_TRY(c, A((void **)&c->fP_d, sizeof(double) * 3 * nPD));
    RT_CUDA_TRY(c, A((void **)&c->fP_f, sizeof(float) * 3 * nPD));
    RT_CUDA_TRY(c, A((void **)&c->ew_d, sizeof(double) * nPE));
    RT_CUDA_TRY(c, A((void **)&c->ew_f, sizeof(float) * nPE));
    RT_CUDA_TRY(c, A((void **)&c->eneg, nPE));
    k_points<<<(npt + 63) / 64, 64, 0, c->stream>>>(c->metric, c->M, c->a, c->gn[0], c->gn[1], ng0, ng1, cf.x0[0],
                                                    cf.x0[1], cf.x0[2], cf.dx[0], cf.dx[1], cf.dx[2], c->pt_e, c->pt_ei,
                                                    c->pt_V, c->pt_n0, c->pt_om, pg0, fe, fg0, fA, c->pt_len);
    RT_CUDA_TRY(c, cudaGetLastError());
    k_dir_tables<<<(unsigned)((nPD + 255) / 256), 256, 0, c->stream>>>(npt, nd, cf.n0_cut, c->g->dir, c->pt_e, pg0,
                                                                      fe, fg0, fA, c->cenU_d, c->cenU_f, c->mask,
                                                                      c->fn_d, c->fn_f, c->fP_d, c->fP_f);
    RT_CUDA_TRY(c, cudaGetLastError());
    k_edge_tables<<<(unsigned)((nPE + 255) / 256), 256, 0, c->stream>>>(npt, ne, c->g->emid, c->g->eu, c->g->dlam,
                                                                       c->pt_e, pg0, c->pt_om, c->ew_d, c->ew_f,
                                                                       c->eneg);
    RT_CUDA_TRY(c, cudaGetLastError());
    RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    cudaFree(pg0); cudaFree(fe); cudaFree(fg0); cudaFree(fA);
    return RT_OK;
}

// tetrad-frame fluid velocity u-hat^(a) = e^(a)_mu u^mu and coordinate velocity u^a/u^0
__global__ void k_uhat(int ncell, int nx0, int nx1, int gn0, int ng0, int ng1, int flat,
                       const double *__restrict__ ucon, const double *__restrict__ pei, double *__restrict__ uhat,
                       double *__restrict__ vel) {
    int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= ncell) return;
    const double *u = ucon + 4 * (size_t)cidx;
    if (flat) {
        for (int m = 0; m < 4; ++m) uhat[4 * (size_t)cidx + m] = u[m];
    } else {
        int i = cidx % nx0, j = (cidx / nx0) % nx1;
        const double *E = pei + 16 * (size_t)((j + ng1) * gn0 + (i + ng0));
        for (int b = 0; b < 4; ++b)
            uhat[4 * (size_t)cidx + b] = E[b * 4] * u[0] + E[b * 4 + 1] * u[1] + E[b * 4 + 2] * u[2] + E[b * 4 + 3] * u[3];
    }
    for (int a = 0; a < 3; ++a) vel[3 * (size_t)cidx + a] = u[a + 1] / u[0];
}

// per cell sum_s w_s / D_s^2 (FP64), D_s = u-hat^0 - u-hat.n_s; the solid
// angles are the stage kernels' (FP32-rounded for FP32 math)
__global__ void k_wbar(int ncell, int nd, const double *__restrict__ uhat, const double *__restrict__ dir,
                       const double *__restrict__ w, const float *__restrict__ wf, double *__restrict__ wbar) {
    int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= ncell) return;
    const double *u = uhat + 4 * (size_t)cidx;
    double sum = 0.0;
    const bool rest = u[0] == 1.0 && u[1] == 0.0 && u[2] == 0.0 && u[3] == 0.0;   // D = 1
    for (int s = 0; s < nd; ++s) {
        const double ws = wf ? (double)wf[s] : w[s];
        if (rest) { sum += ws; continue; }
        const double D = u[0] - (u[1] * dir[3 * s] + u[2] * dir[3 * s + 1] + u[3] * dir[3 * s + 2]);
        const double r = rtk::rcp64(D);
        sum += ws * r * r;
    }
    wbar[cidx] = sum;
}

rt_status rt_compute_uhat(rt_ctx *c) {
    int ng0 = c->active[0] ? 2 : 0, ng1 = c->active[1] ? 2 : 0;
    k_uhat<<<(c->ncell + 255) / 256, 256, 0, c->stream>>>(c->ncell, c->cfg.nx[0], c->cfg.nx[1], c->gn[0], ng0, ng1,
                                                         c->metric == RT_MINKOWSKI_CART, c->ucon, c->pt_ei, c->uhat,
                                                         c->vel);
    RT_CUDA_TRY(c, cudaGetLastError());
    k_wbar<<<(c->ncell + 127) / 128, 128, 0, c->stream>>>(c->ncell, c->nd, c->uhat, c->g->dir, c->g->w,
                                                         c->cfg.precision == RT_FP64 ? nullptr : c->g->wf, c->wbar);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}
