// stage_common.cuh — pieces shared by the stage kernels (stage.cu, stage_flat.cu).
#pragma once
#include "rt_internal.cuh"
#include <cmath>

namespace rtk {

constexpr int NCELL = 32;    // cells per CTA
constexpr int MAXNT = 256;
constexpr int MAXNT_BIG = 1024;     // general stage kernel on finer grids: one direction per thread
constexpr int CURV_NT = 192, CURV_MINB = 4;   // general stage kernel, curved geometry, up to 192 directions
constexpr size_t SMEM_MAX = 227 * 1024;   // shared memory of one CTA (opt-in maximum)
constexpr double FOURPI = 12.566370614359172953850573533118;
constexpr int F_MIR = 1 << 29, F_FIX = 1 << 30, F_MASK = (1 << 29) - 1;

struct StageArgs {
    int nx0, nx1, nx2, nd, ne;
    int act0, act1, act2;
    int bc[3][2];
    int beam_dir, beam_lo, beam_hi;
    double beam_I;
    int n_pole_zero;
    double dx0, dx1, dx2;
    double gam, arad, T_exp, abar, sumw, sumwf;
    double sumnw[3];           // sum of n-hat_s dOmega_s (0 to rounding)
    int tau_dt, limiter, ang_recon, transport, source;
    // x3 slab (RT_BC_HALO): the row descriptors of the general and the flat
    // kernel count cells from plane -kb (the first ghost plane), and Isrc,
    // alpha_in and vel point there, so that descriptors stay non-negative;
    // the packed kernel takes kb = 0 with pointers at the owned origin and
    // signed offsets
    int kb;
    int coupling;              // temperature solve of section 3.5.2: 1, 2 or 3
    double dtk;
    const void *Isrc; const void *Ibase; void *Iout;
    const double *ug_in; double *ug_out;
    const double *alpha_in;    // opacity of the flux stage (neighbours)
    const double *alpha_int;   // opacity at the interaction's initial gas state
    double *alpha_out;         // opacity after the interaction
    const double *cc_au, *cc_as, *cc_Y, *eta, *vel, *uhat;
    const double *wbar;        // per cell sum_s w_s / D_s^2 in FP64 (the FP32 paths' solid angles)
    const uint8_t *cc_on;
    double *G;
    float2 *gac;               // packed FP32 path: per-cell (a, c) of the interaction, for a deferred G
    unsigned long long *fail;
    double *sv_Em, *sv_X;      // optional per-cell E-bar_- and root X of the interaction (reverse-pass recompute)
    const int *mirror, *nnb, *nbr, *ring_edge, *ring_back, *edge;
    const void *dirT, *wT, *mxT, *mgT, *mmT;   // math-type copies of the grid tables
    const void *mdT;                            // MAPR dual-basis dot products [nd][6][6][2]
    int gn0, ng0, ng1;
    const void *cenU, *fn, *fP, *ew;           // math-type geometry tables (curved)
    const uint8_t *mask;
    const uint8_t *eneg;       // per (point, edge): n_0(m) < 0 (see k_edge_tables)
    const double *pt_V, *pt_n0, *pt_e;
    const double *pt_len;
};

template <typename TS, typename TM> struct IO;
template <> struct IO<double, double> {
    __device__ static double ld(const void *p, size_t i) { return __ldg((const double *)p + i); }
    __device__ static double st(void *p, size_t i, double v) { ((double *)p)[i] = v; return v; }
};
template <> struct IO<float, float> {
    __device__ static float ld(const void *p, size_t i) { return __ldg((const float *)p + i); }
    __device__ static float st(void *p, size_t i, float v) { __stcs((float *)p + i, v); return v; }
};
template <> struct IO<__nv_bfloat16, float> {
    __device__ static float ld(const void *p, size_t i) {
        return __bfloat162float(__ldg((const __nv_bfloat16 *)p + i));
    }
    __device__ static float st(void *p, size_t i, float v) {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        ((__nv_bfloat16 *)p)[i] = b;
        return __bfloat162float(b);
    }
};

template <typename TM> __device__ __forceinline__ TM ldT(const void *p, size_t i) { return __ldg((const TM *)p + i); }
template <typename TM> __device__ __forceinline__ TM qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000ll); }
// elements 2i and 2i + 1 in one load
__device__ __forceinline__ void ldT2(const void *p, size_t i, float &a, float &b) {
    const float2 v = __ldg((const float2 *)p + i);
    a = v.x; b = v.y;
}
__device__ __forceinline__ void ldT2(const void *p, size_t i, double &a, double &b) {
    const double2 v = __ldg((const double2 *)p + i);
    a = v.x; b = v.y;
}

template <typename TM> __device__ __forceinline__ TM dv(TM a, TM b);
template <> __device__ __forceinline__ float dv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double dv<double>(double a, double b) { return a / b; }

template <typename TM> __device__ __forceinline__ TM limiter(int kind, TM dl, TM dr) {
    if (kind == RT_LIM_DONOR) return TM(0);
    if (dl * dr <= TM(0)) return TM(0);
    TM al = fabs(dl), ar = fabs(dr);
    TM m = (kind == RT_LIM_MINMOD) ? fmin(al, ar) : fmin(fmin(TM(2) * al, TM(2) * ar), TM(0.5) * fabs(dl + dr));
    return dl > TM(0) ? m : -m;
}

// per-unit-n_0 flux through one face for one direction: the exponentially cut
// HLL form (eqs. rad_speeds, flux_Jiang; see the oracle for the orientation
// reading); rec = (c1, c2, c3, kL, kR) of the face
template <typename TM>
__device__ __forceinline__ TM face_phi(TM n, const TM *rec, TM IL, TM IR, TM Il, TM Ir) {
    TM cL = n > TM(0) ? rec[0] : rec[1];
    TM cR = n > TM(0) ? rec[1] : rec[0];
    // explicit multiply-adds: the general kernel's file is compiled without
    // contraction, so that every brick shape rounds alike
    const TM a = fma(cL, IL, cR * IR), b = fma(rec[3], IL, rec[4] * IR);
    return fma(n, a, fma(-fabs(n) * rec[2], Ir - Il, b));
}

// boundary resolution of one index along one axis (setup only)
__device__ inline int map_axis(const StageArgs &A, int ax, int q, int *flags, int *kshift) {
    int n = ax == 0 ? A.nx0 : (ax == 1 ? A.nx1 : A.nx2);
    if (q >= 0 && q < n) return q;
    int side = q < 0 ? 0 : 1, bc = A.bc[ax][side];
    if (bc == RT_BC_HALO) return q;     // the caller's ghost planes (x3 only)
    if (bc == RT_BC_PERIODIC) return (q + n) % n;
    if (bc == RT_BC_POLE) {
        *flags ^= F_MIR;
        if (ax == 1 && A.nx2 > 1 && kshift) *kshift = A.nx2 / 2;
        return side ? 2 * n - 1 - q : -1 - q;
    }
    if (bc == RT_BC_BEAM) *flags |= F_FIX;
    return side ? n - 1 : 0;
}

// row descriptor: base cell index of row (j, k) at x1 = 0, with flags
__device__ inline int row_desc(const StageArgs &A, int j, int k) {
    int fl = 0, ks = 0;
    int jm = map_axis(A, 1, j, &fl, &ks);
    int km = map_axis(A, 2, k, &fl, nullptr);
    if (ks) km = (km + ks) % A.nx2;
    return (((km + A.kb) * A.nx1 + jm) * A.nx0) | fl;
}

// ------------------------------------------------------------ temperature
// Method 3 solved for the post-interaction radiation energy X = E* (see the
// oracle): h(X) = (alpha(T) dt - B2 alpha^s) X - B1 - B2 eta alpha^a(T) a T^4,
// T = T_- + (E-bar_- - X)/Y; h increases strictly on [0, W).
template <typename R> struct Teq { R B1, B2, W, Y, Tm, Em, au, as, eta, arad, dt, p, iY; };

// (iY = 1/Y, so that an evaluation of h divides only for T^-p and the step)
template <typename R>
__device__ __forceinline__ Teq<R> make_teq(R B1, R B2, R W, R Y, R Tm, R Em, R au, R as, R eta, R arad, R dt, R p) {
    return Teq<R>{B1, B2, W, Y, Tm, Em, au, as, eta, arad, dt, p, R(1) / Y};
}

template <typename R> __device__ __forceinline__ R tpow_neg(R T, R p) {
    if (p == R(3.5)) { R r = sqrt(T); return R(1) / (T * T * T * r); }
    if (p == R(0)) return R(1);
    return pow(T, -p);
}

// *hs: the size of the terms that make up h, so that |h| <= eps * hs is h at
// the level of its own rounding (with alpha^s dt >> 1, h is the difference of
// two terms ~alpha^s dt X that cancel to ~X)
template <typename R> __device__ __forceinline__ void teq_eval(const Teq<R> &q, R X, R *h, R *dh, R *hs) {
    R T = q.Tm + (q.Em - X) * q.iY;
    if (!(T > R(0))) { *h = R(1e30); *dh = R(1); *hs = R(0); return; }
    // T^-p and 1/T with one division (p = 3.5: 1/T = T^2 sqrt(T) T^-3.5)
    R tp, iT;
    if (q.p == R(3.5)) {
        const R r = sqrt(T);
        tp = R(1) / (T * T * T * r);
        iT = T * T * r * tp;
    } else {
        tp = tpow_neg(T, q.p);
        iT = R(1) / T;
    }
    R aa = q.au * tp;
    R T4 = T * T * T * T;
    R em = q.B2 * q.eta * q.arad * aa * T4;
    R lin = (aa + q.as) * q.dt - q.B2 * q.as;
    *h = lin * X - q.B1 - em;
    *hs = ((aa + q.as) * q.dt + q.B2 * q.as) * X + q.B1 + em;
    // dh/dX with dT/dX = -1/Y
    *dh = lin + (q.p * aa * iT) * q.dt * X * q.iY + em * (R(4) - q.p) * iT * q.iY;
}

// safeguarded Newton on [lo, hi] with h(lo) <= 0 < h(hi); returns converged
// flag.  Converged: a Newton step below tol X, a bracket below tol hi, or a
// residual at its rounding level (|h| <= tol hs), where no step can do better
template <typename R> __device__ bool newton_E(const Teq<R> &q, R X, R &lo, R &hi, int maxit, R tol, R *Xout) {
    R h, dh, hs;
    for (int it = 0; it < maxit; ++it) {
        teq_eval(q, X, &h, &dh, &hs);
        if (fabs(h) <= tol * hs) { *Xout = X; return true; }   // exact root or rounding-level residual
        if (h > R(0)) hi = fmin(hi, X); else lo = fmax(lo, X);
        R d = h / dh;
        if (fabs(d) <= tol * X) { *Xout = fmin(fmax(X - d, lo), hi); return true; }   // converged Newton step
        R Xn = X - d;
        bool newton = Xn > lo && Xn < hi;
        if (!newton) Xn = R(0.5) * (lo + hi);
        R step = fabs(Xn - X);
        X = Xn;
        if ((newton && step <= tol * X) || hi - lo <= tol * hi) { *Xout = X; return true; }
    }
    *Xout = X;
    return false;
}

// 1/x in FP64 without the FP64 division sequence (long on this part's FP64
// pipe): an FP32 reciprocal refined by two Newton-Raphson steps
// y <- y + y (1 - x y), each of which squares the relative error (1e-7 ->
// 1e-14 -> rounding level); the exact division outside the FP32 range
// |x| within [2^-99, 2^99) (nonzero, finite, well inside the FP32 range),
// tested on the exponent bits with integer instructions: a comparison in
// FP64 would occupy this part's slow FP64 pipe
__device__ __forceinline__ bool in_fp32_range(double x) {
    const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    return e - (1023u - 99u) < 198u;
}
// 1/x from the correctly rounded FP32 reciprocal (relative error <= 2^-24)
// and one FP64 Newton step, which squares that error (~4e-15)
__device__ __forceinline__ double rcp64(double x) {
    if (!in_fp32_range(x)) return 1.0 / x;
    const double y = (double)__frcp_rn((float)x);
    return fma(y, fma(-x, y, 1.0), y);
}

// T^-p in FP64 for the mixed path: for p = 3.5 an FP32 reciprocal square
// root refined by one FP64 Newton step for 1/sqrt (relative error ~1e-14)
__device__ __forceinline__ double tneg_mixed(double T, double p) {
    if (p == 3.5 && T > 0.0 && in_fp32_range(T)) {
        double y = (double)rsqrtf((float)T);
        y = y * (1.5 - 0.5 * T * y * y);
        double y2 = y * y;
        return y2 * y2 * y2 * y;
    }
    return tpow_neg<double>(T, p);
}

// Methods 1 and 2 of section 3.5.2 (eqs. semi_implicit_T, implicit_T) for the
// post-interaction energy X = E-bar_+ with T = T_- + (E-bar_- - X)/Y:
//   h(X) = (1 - A2 alpha^s) X - A1 - A2 eta alpha^a_P a T^4,
// A1, A2 of eqs. A1, A2 (explicit alpha_-), alpha^a_P = kappa rho^m T_-^-p
// (method 1) or kappa rho^m T^-p (method 2).  h increases strictly on [0, W);
// without a sign change there (h(W) = (1 - A2 alpha^s) W - A1 <= 0) no
// positive temperature solves the equations and the solve reports failure.
struct M12 { double A1, A2, W, Y, iY, Tm, Em, au, as, eta, arad, p, aam; int method; };
__device__ inline bool solve_m12(const M12 &q, double *Xout) {
    const double lin = 1.0 - q.A2 * q.as;
    if (!(lin * q.W - q.A1 > 0.0)) return false;
    double lo = 0.0, hi = q.W, X = fmin(fmax(q.Em, 0.0), 0.5 * q.W);
    const double pe = q.method == 1 ? 0.0 : q.p;
    for (int it = 0; it < 200; ++it) {
        const double T = q.Tm + (q.Em - X) * q.iY;
        const double aa = q.method == 1 ? q.aam : q.au * tpow_neg<double>(T, q.p);
        const double e4 = q.A2 * q.eta * aa * q.arad * T * T * T * T;
        const double h = lin * X - q.A1 - e4;
        if (h > 0.0) hi = X; else lo = X;
        if (fabs(h) <= 4.0 * 2.220446049250313e-16 * (fabs(lin * X) + q.A1 + e4)) break;
        const double dh = lin + (4.0 - pe) * e4 / T * q.iY;
        double Xn = X - h / dh;
        if (!(Xn > lo && Xn < hi)) Xn = 0.5 * (lo + hi);
        if (fabs(Xn - X) <= 4.0 * 2.220446049250313e-16 * fabs(X) || hi - lo <= 4.0 * 2.220446049250313e-16 * hi) {
            X = Xn;
            break;
        }
        X = Xn;
    }
    *Xout = X;
    return true;
}

// Temperature solve of the mixed (FP32-storage) path: FP32 Newton from E-bar_-,
// then FP64 residual iterations X <- X - h_64(X) / h'_32(X) (the residual is
// FP64, the slope FP32, so each iteration gains ~7 digits; one suffices after
// a converged FP32 Newton, up to three otherwise).  Returns X = E*.
__device__ inline bool solve_mixed(const Teq<double> &q, double *Xout) {
    Teq<float> qf{(float)q.B1, (float)q.B2, (float)q.W, (float)q.Y, (float)q.Tm, (float)q.Em, (float)q.au,
                  (float)q.as, (float)q.eta, (float)q.arad, (float)q.dt, (float)q.p, (float)q.iY};
    float flo = 0.0f, fhi = (float)q.W, fx;
    bool okf = newton_E<float>(qf, (float)q.Em, flo, fhi, 40, 2e-7f, &fx);
    const double invY = q.iY, B2ea = q.B2 * q.eta * q.arad, B2as = q.B2 * q.as;
    double X = (double)fx;
    for (int it = 0; it < 3; ++it) {
        double T = q.Tm + (q.Em - X) * invY;
        if (!(T > 0.0)) return false;
        double aa = q.au * tneg_mixed(T, q.p);
        double T2 = T * T;
        double h = ((aa + q.as) * q.dt - B2as) * X - q.B1 - B2ea * aa * T2 * T2;
        float Tf = (float)T, aaf = (float)aa, Xf = (float)X;
        float lin = (aaf + qf.as) * qf.dt - qf.B2 * qf.as;
        float emf = qf.B2 * qf.eta * qf.arad * aaf * Tf * Tf * Tf * Tf;
        float dh = lin + (qf.p * aaf / Tf) * qf.dt * Xf / qf.Y + emf * (4.0f - qf.p) / (Tf * qf.Y);
        double d = h * (double)(1.0f / dh);
        X -= d;
        // each iteration multiplies the error by the slope's FP32 error (~1e-7):
        // a correction below 1e-6 X leaves an error below ~1e-13 X
        if (fabs(d) <= 1e-6 * fabs(X)) break;
    }
    *Xout = X;
    return okf && X >= 0.0 && X < q.W;
}

}  // namespace rtk

// fast path of the stage (stage_flat.cu): flat Cartesian geometry, a fluid at
// rest in every cell, MC limiter, fewer than 2^31 stored intensities
bool rt_stage_fast_ok(const rt_ctx *c);
// method 3 of section 3.5.2 (the fast paths and the reverse pass implement it only)
inline bool rt_coupling3(const rt_ctx *c) { return c->cfg.coupling == 0 || c->cfg.coupling == 3; }
rt_status rt_launch_stage_fs(rt_ctx *c, const rtk::StageArgs &A, int NT);
