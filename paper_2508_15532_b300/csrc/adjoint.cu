// adjoint.cu — reverse mode of the radiation step for flat Cartesian geometry
// with the fluid at rest, FP64 or FP32 intensities (section 5.2 motivates gradients
// through the step; the reverse pass is derived by hand from eq.
// radiative_transfer_discrete, eqs. rad_speeds / flux_Jiang and method 3 of
// section 3.5.2).
//
// One call reverses nsteps steps from a checkpoint (I^0, u_g^0):
//  1. forward recompute with the ordinary stage kernels, which also save each
//     cell's E-bar_- and temperature root X; every stage's input intensities,
//     gas energies and opacities are kept in a library-owned arena;
//  2. reverse sweep, one kernel per stage (k_rev): the transport adjoint of
//     the stage, computed face by face (each face's flux derivatives once,
//     each cell's limited slope and its derivatives once), fused with the
//     interaction adjoint of the stage before it, whose output is this
//     stage's input.  The interaction adjoint is written in terms of its
//     output I_+ = (I_* + c)/(1 + a), so I_* is never stored, and its root
//     enters through the implicit function theorem.
#include <atomic>
#include <cstdint>
#include "stage_common.cuh"
#include "f32x2.cuh"
#include <algorithm>

using namespace rtk;

namespace {

// ------------------------------------------------------------ lane types
// FP32 pass: a thread owns two adjacent directions (n_dir is even) and works
// on both with f32x2 arithmetic.  FP64 pass: one direction per thread.
__device__ __forceinline__ double fma2(double a, double b, double c) { return fma(a, b, c); }

struct LaneF {
    using S = float;
    using V = F2;
    // five CTAs per SM (128 registers), measured 5% faster than four; bricks of
    // 2 x 1 cells across x2/x3 (the 2 x 2 brick spills even at four CTAs)
    static constexpr int L = 2, NT = 96, MINB = 5;
    static constexpr bool BRICK22 = false;
    __device__ static V splat(float a) { return f2(a); }
    __device__ static V ld(const float *p) { float2 v = __ldg(reinterpret_cast<const float2 *>(p)); return F2{v.x, v.y}; }
    __device__ static void st(float *p, V v) { *reinterpret_cast<float2 *>(p) = make_float2(v.x, v.y); }
    __device__ static void st64(double *p, V v) { *reinterpret_cast<double2 *>(p) = make_double2(v.x, v.y); }
    __device__ static V ld64(const double *p) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        return F2{(float)v.x, (float)v.y};
    }
    __device__ static float hsum(V v) { return v.x + v.y; }
    __device__ static V vabs(V v) { return F2{fabsf(v.x), fabsf(v.y)}; }
    __device__ static V dirv(const double *dir, int d, int a) { return F2{(float)dir[3 * d + a], (float)dir[3 * d + 3 + a]}; }
    __device__ static V wv(const double *w, int d) { return F2{(float)w[d], (float)w[d + 1]}; }
};
struct LaneD {
    using S = double;
    using V = double;
    static constexpr int L = 1, NT = 192, MINB = 2;
    static constexpr bool BRICK22 = true;     // measured 7% faster than 2 x 1 (FP64-pipe bound)
    __device__ static V splat(double a) { return a; }
    __device__ static V ld(const double *p) { return __ldg(p); }
    __device__ static void st(double *p, V v) { *p = v; }
    __device__ static void st64(double *p, V v) { *p = v; }
    __device__ static V ld64(const double *p) { return __ldg(p); }
    __device__ static double hsum(V v) { return v; }
    __device__ static V vabs(V v) { return fabs(v); }
    __device__ static V dirv(const double *dir, int d, int a) { return dir[3 * d + a]; }
    __device__ static V wv(const double *w, int d) { return w[d]; }
};

// finer geodesic grids (G3 = 642 directions): the same lanes in one CTA of up
// to 704 (FP32 pairs) or 672 (FP64) threads, one per SM
struct LaneF3 : LaneF {
    static constexpr int NT = 352, MINB = 1;
};
struct LaneD3 : LaneD {
    static constexpr int NT = 672, MINB = 1;
};
constexpr int REV_MAX_DIRS = LaneD3::NT;   // 672

// Half of the limited slope, hs = s/2 (the reconstruction offset of eq.
// radiative_transfer_discrete's face states), and its derivatives in the
// forward difference dl = I_{p+1} - I_p and the backward difference
// dr = I_p - I_{p-1}.  Values as rtk::limiter / 2 (halving is exact).  The
// branch taken at ties follows the MC rule of the forward scan: 2|dl| first,
// 2|dr| only when strictly smaller, (dl + dr)/2 only when strictly below both.
// Every kind has zero derivatives where dl dr <= 0 (in particular where one
// difference is zero), which the outflow ghost folding below relies on.
template <typename S> __device__ __forceinline__ void lim_half(int kind, S dl, S dr, S &hs, S &gl, S &gr, S &gd) {
    const S al = fabs(dl), ar = fabs(dr);
    const bool ok = dl * dr > S(0);
    if (kind == RT_LIM_MC) {
        const S q = S(0.25) * fabs(dl + dr);
        const bool w1 = ar < al;                    // |dr| strictly smaller
        const S m1 = w1 ? ar : al;
        const bool w2 = q < m1;
        const S m = w2 ? q : m1;
        hs = ok ? copysign(m, dl) : S(0);
        gl = ok ? (w2 ? S(0.25) : (w1 ? S(0) : S(1))) : S(0);
        gr = ok ? (w2 ? S(0.25) : (w1 ? S(1) : S(0))) : S(0);
        gd = ok ? (w2 ? S(0) : (w1 ? S(1) : S(-1))) : S(0);
    } else if (kind == RT_LIM_MINMOD) {
        const bool wl = al < ar;
        hs = ok ? copysign(S(0.5) * (wl ? al : ar), dl) : S(0);
        gl = (ok && wl) ? S(0.5) : S(0);
        gr = (ok && !wl) ? S(0.5) : S(0);
        gd = ok ? (wl ? S(-0.5) : S(0.5)) : S(0);
    } else {
        hs = S(0); gl = S(0); gr = S(0); gd = S(0);
    }
}
// FP64: the magnitude comparisons and minima on the integer pipe (the bit
// patterns of non-negative doubles order as their values), which leaves the
// FP64 pipe - 1/64 of the FP32 rate on this part - the sign test, dl + dr and
// its quarter.  Same values and branches as the generic form.
template <> __device__ __forceinline__ void lim_half<double>(int kind, double dl, double dr, double &hs, double &gl,
                                                            double &gr, double &gd) {
    constexpr long long MAG = 0x7fffffffffffffffLL;
    const long long sl = __double_as_longlong(dl), al = sl & MAG, ar = __double_as_longlong(dr) & MAG;
    const bool ok = dl * dr > 0.0;
    if (kind == RT_LIM_MC) {
        const long long q = __double_as_longlong(0.25 * fabs(dl + dr));
        const bool w1 = ar < al;
        const long long m1 = w1 ? ar : al;
        const bool w2 = q < m1;
        const long long m = w2 ? q : m1;
        hs = ok ? __longlong_as_double(m | (sl & ~MAG)) : 0.0;
        gl = ok ? (w2 ? 0.25 : (w1 ? 0.0 : 1.0)) : 0.0;
        gr = ok ? (w2 ? 0.25 : (w1 ? 1.0 : 0.0)) : 0.0;
        gd = ok ? (w2 ? 0.0 : (w1 ? 1.0 : -1.0)) : 0.0;
    } else if (kind == RT_LIM_MINMOD) {
        const bool wl = al < ar;
        hs = ok ? 0.5 * __longlong_as_double((wl ? al : ar) | (sl & ~MAG)) : 0.0;
        gl = (ok && wl) ? 0.5 : 0.0;
        gr = (ok && !wl) ? 0.5 : 0.0;
        gd = ok ? (wl ? -0.5 : 0.5) : 0.0;
    } else {
        hs = 0.0; gl = 0.0; gr = 0.0; gd = 0.0;
    }
}
// per lane type, with gd = gr - gl: one packed subtraction for FP32 pairs;
// selects for FP64, which keeps the subtraction off the FP64 pipe
// FP32 pairs: dl dr and (dl + dr)/4 as packed operations, the rest per lane
__device__ __forceinline__ void lim_pre(int kind, float dl, float dr, float prod, float q4, float &hs, float &gl, float &gr) {
    const float al = fabsf(dl), ar = fabsf(dr);
    const bool ok = prod > 0.0f;
    if (kind == RT_LIM_MC) {
        const float q = fabsf(q4);
        const bool w1 = ar < al;
        const float m1 = w1 ? ar : al;
        const bool w2 = q < m1;
        const float m = w2 ? q : m1;
        hs = ok ? copysignf(m, dl) : 0.0f;
        gl = ok ? (w2 ? 0.25f : (w1 ? 0.0f : 1.0f)) : 0.0f;
        gr = ok ? (w2 ? 0.25f : (w1 ? 1.0f : 0.0f)) : 0.0f;
    } else if (kind == RT_LIM_MINMOD) {
        const bool wl = al < ar;
        hs = ok ? copysignf(0.5f * (wl ? al : ar), dl) : 0.0f;
        gl = (ok && wl) ? 0.5f : 0.0f;
        gr = (ok && !wl) ? 0.5f : 0.0f;
    } else {
        hs = 0.0f; gl = 0.0f; gr = 0.0f;
    }
}
// MC for a pair of lanes: the value from the min/max form (mc_half_xs, the
// forward kernel's); the branch from exact equalities, since hs equals dl
// bit for bit exactly when |dl| is a minimum (taken first at ties) and dr when
// |dr| is (and |dl| is not); otherwise the quarter sum.  The branch masks are
// 1/0 per lane, combined with packed arithmetic:
//   gl = ok (e_l + e_q / 4), gr = ok (e_r + e_q / 4), e_q = 1 - e_l - e_r
__device__ __forceinline__ void limv_mc(F2 dl, F2 dr, F2 &hs, F2 &gl, F2 &gr, F2 &gd) {
    const F2 prod = dl * dr, q4 = f2(0.25f) * (dl + dr);
    hs = F2{mc_half_xs(dl.x, dr.x, q4.x), mc_half_xs(dl.y, dr.y, q4.y)};
    const F2 ok = F2{prod.x > 0.0f ? 1.0f : 0.0f, prod.y > 0.0f ? 1.0f : 0.0f};
    const F2 el = F2{hs.x == dl.x ? 1.0f : 0.0f, hs.y == dl.y ? 1.0f : 0.0f};
    const F2 er0 = F2{hs.x == dr.x ? 1.0f : 0.0f, hs.y == dr.y ? 1.0f : 0.0f};
    const F2 er = fma2(F2{-er0.x, -er0.y}, el, er0);
    gl = ok * fma2(f2(-0.25f), er, fma2(f2(0.75f), el, f2(0.25f)));
    gr = ok * fma2(f2(-0.25f), el, fma2(f2(0.75f), er, f2(0.25f)));
    gd = gr - gl;
}
__device__ __forceinline__ void limv(int kind, F2 dl, F2 dr, F2 &hs, F2 &gl, F2 &gr, F2 &gd) {
    if (kind == RT_LIM_MC) { limv_mc(dl, dr, hs, gl, gr, gd); return; }
    const F2 prod = dl * dr, q4 = f2(0.25f) * (dl + dr);
    lim_pre(kind, dl.x, dr.x, prod.x, q4.x, hs.x, gl.x, gr.x);
    lim_pre(kind, dl.y, dr.y, prod.y, q4.y, hs.y, gl.y, gr.y);
    gd = gr - gl;
}
__device__ __forceinline__ void limv(int kind, double dl, double dr, double &hs, double &gl, double &gr, double &gd) {
    lim_half<double>(kind, dl, dr, hs, gl, gr, gd);
}

// Face record of the exponentially cut flux (eqs. rad_speeds, flux_Jiang):
// with (cL, cR) = (c1, c2) for n > 0 and (c2, c1) for n < 0,
//   n cL = n P + |n| D,  n cR = n P - |n| D,  P = (c1 + c2)/2, D = (c1 - c2)/2,
// and the same for the derivatives in tau.  Stored: P, D, -D, c3, dP, dD, -dc3.
template <typename S> __device__ void face_record(S tau, S *r) {
    S c1, c2, c3, d1, d2, d3;
    if (tau > S(0)) {
        const S t2 = tau * tau, t4 = t2 * t2;
        const S F = -expm1(-t2), G = -expm1(-t4);
        const S f = sqrt(F) / tau, g = sqrt(G) / tau, e = exp(-tau), Sg = f + g;
        const S fp = exp(-t2) / sqrt(F) - f / tau;
        const S gp = G > S(0) ? S(2) * t2 * exp(-t4) / sqrt(G) - g / tau : S(1);
        const S ep = -e, Sp = fp + gp, iS2 = S(1) / (Sg * Sg);
        c1 = f * e / Sg; c2 = g * e / Sg; c3 = f * g / Sg;
        d1 = ((fp * e + f * ep) * Sg - f * e * Sp) * iS2;
        d2 = ((gp * e + g * ep) * Sg - g * e * Sp) * iS2;
        d3 = ((fp * g + f * gp) * Sg - f * g * Sp) * iS2;
    } else {
        c1 = S(1); c2 = S(0); c3 = S(0);
        d1 = S(-2); d2 = S(1); d3 = S(1);
    }
    r[0] = S(0.5) * (c1 + c2); r[1] = S(0.5) * (c1 - c2); r[2] = -r[1]; r[3] = c3;
    r[4] = S(0.5) * (d1 + d2); r[5] = S(0.5) * (d1 - d2); r[6] = -d3; r[7] = S(0);
}

// cotangents of a face's states from the cotangent phib of its flux:
// ILb = phib n cL, IRb = phib n cR, c3t = phib |n| c3
template <typename V> struct FaceCot { V ILb, IRb, c3t; };
template <class LT>
__device__ __forceinline__ FaceCot<typename LT::V> face_cot(typename LT::V phib, typename LT::V n, typename LT::V an,
                                                           const typename LT::S *r) {
    using V = typename LT::V;
    const V nP = n * LT::splat(r[0]);
    const V ncL = fma2(an, LT::splat(r[1]), nP), ncR = fma2(an, LT::splat(r[2]), nP);
    return FaceCot<V>{phib * ncL, phib * ncR, phib * (an * LT::splat(r[3]))};
}
// d flux / d tau times phib, for face states IL, IR and cells Il, Ir:
// phib (n dcL IL + n dcR IR - |n| dc3 (Ir - Il))
template <class LT>
__device__ __forceinline__ typename LT::V face_tau(typename LT::V phib, typename LT::V n, typename LT::V an,
                                                   typename LT::V IL, typename LT::V IR, typename LT::V dI,
                                                   const typename LT::S *r) {
    using V = typename LT::V;
    V u = LT::splat(r[5]) * (IL - IR);
    u = fma2(LT::splat(r[6]), dI, u);
    V v = an * u;
    v = fma2(n * LT::splat(r[4]), IL + IR, v);
    return phib * v;
}

// Per-cell FP64 arithmetic without FP64 divisions or square roots, which are
// long instruction sequences on this part's FP64 pipe (1/64 of the FP32 rate):
// an FP32 estimate refined by one FP64 Newton step (Newton's method squares
// the relative error: ~1e-14 from the FP32 estimates' ~1e-7), with the exact
// operation outside the FP32 range (tested on the exponent bits).
__device__ __forceinline__ double rcp_nr(double x) { return rcp64(x); }
__device__ __forceinline__ double rsqrt_nr(double x) {   // x > 0
    if (!in_fp32_range(x)) return 1.0 / sqrt(x);
    const double y = (double)rsqrtf((float)x);
    return y * fma(-0.5 * x * y, y, 1.5);
}
// T^-p and 1/T (T > 0); for p = 3.5 both from r = T^-1/2: T^-3.5 = r^7, 1/T = r^2
__device__ __forceinline__ void tpow_inv(double T, double p, double &tp, double &iT) {
    if (p == 3.5) {
        const double r = rsqrt_nr(T), r2 = r * r, r6 = r2 * r2 * r2;
        tp = r6 * r; iT = r2;
    } else {
        tp = tpow_neg<double>(T, p); iT = rcp_nr(T);
    }
}

// rho^m = (kappa rho^m) / kappa, the derivative of alpha^a's prefactor in
// kappa, without an FP64 pow where kappa is nonzero
__device__ __forceinline__ double rho_m(double au, double kap, double rho, double m) {
    return kap != 0.0 ? au * rcp_nr(kap) : pow(rho, m);
}

// Reverse of the interaction of section 3.5.2 (method 3) in one cell at rest,
// from its output: I_+ = (I_* + c)/A in every direction, A = 1 + a,
// E-bar_+ = sum w I_+, u_g+ = u_g- - (E-bar_+ - E-bar_-), with a = alpha(T_+) dt,
// c = dt (eta alpha^a(T_+) a_R T_+^4 + alpha^s X)/(4 pi), T_+ = T_- + (E-bar_- - X)/Y
// and X the root of h(X; B1, B2, T_-, E-bar_-) = 0 (B1 = K E-bar_-,
// B2 = K sum w dt/(4 pi), K = alpha(T_-) dt / (1 + alpha(T_-) dt)).
// Given P = sum Ibo, Q = sum Ibo I_+ (Ibo: cotangent of I_+) and ub (cotangent
// of u_g+), the cotangent of I_* in direction s is (Ibo_s - ub w_s) inv + Emb w_s.
struct SrcRev { double inv, ub, Emb, ugb, kb, eb; };
// iY = 1/Y, (tm, iTm) = (T_-^-p, 1/T_-) and rhom = rho^m come from the caller,
// which needs them for the opacity chain too.
__device__ SrcRev src_rev(bool on, double iY, double ugm, double au, double as, double eta, double tm, double iTm,
                          double rhom, double Em, double X, double P, double Q, double ub, double dt, double S,
                          double p, double ar) {
    SrcRev o{1.0, 0.0, 0.0, ub, 0.0, 0.0};
    if (!on) return o;
    constexpr double i4pi = 1.0 / FOURPI;
    const double Tm = ugm * iY;
    double tp, iTp;
    const double am = au * tm + as;
    const double adt = am * dt, i1a = rcp_nr(1.0 + adt), K = adt * i1a, B2 = K * S * dt * i4pi;
    const double Tp = Tm + (Em - X) * iY;
    tpow_inv(Tp, p, tp, iTp);
    const double aap = au * tp;
    const double Tp4 = Tp * Tp * Tp * Tp;
    const double a = (aap + as) * dt;
    const double cc = dt * (eta * aap * ar * Tp4 + as * X) * i4pi;
    const double inv = rcp_nr(1.0 + a);
    const double Ep = (Em + cc * S) * inv;
    const double sIpb = P - ub * S;                 // sum_s Ipb_s, Ipb_s = Ibo_s - ub w_s
    const double ccb = sIpb * inv;
    const double Ab = -(Q - ub * Ep) * inv;         // d/dA of sum_s Ipb_s I_+s = -sum_s Ipb_s I_+s / A
    double aapb = Ab * dt;
    const double ccbd = ccb * dt * i4pi;
    double etab = ccbd * aap * ar * Tp4;
    aapb += ccbd * eta * ar * Tp4;
    double Tpb = ccbd * eta * aap * ar * 4.0 * Tp * Tp * Tp;
    double Xb = ccbd * as;
    double aub = aapb * tp;
    Tpb += aapb * (-p) * aap * iTp;
    double Tmb = Tpb, Emb = ub + Tpb * iY;
    Xb -= Tpb * iY;
    // the root: h(X) = (alpha(T_+) dt - B2 alpha^s) X - B1 - B2 eta alpha^a(T_+) a_R T_+^4
    const double lin = (aap + as) * dt - B2 * as;
    const double hT = -p * aap * iTp * dt * X - B2 * eta * ar * (4.0 - p) * aap * Tp * Tp * Tp;
    const double hX = lin - hT * iY;
    const double lam = -Xb * rcp_nr(hX);
    const double B1b = -lam;
    const double B2b = lam * (-as * X - eta * ar * aap * Tp4);
    Tmb += lam * hT;
    Emb += lam * hT * iY;
    aub += lam * (tp * dt * X - B2 * eta * ar * tp * Tp4);
    etab += lam * (-B2 * ar * aap * Tp4);
    const double Kb = B2b * S * dt * i4pi + B1b * Em;
    Emb += B1b * K;
    const double amb = Kb * dt * i1a * i1a;
    aub += amb * tm;
    Tmb += amb * (-p) * au * tm * iTm;
    o.inv = inv; o.ub = ub; o.Emb = Emb;
    o.ugb = ub + Tmb * iY;
    o.kb = aub * rhom;
    o.eb = etab;
    return o;
}

// asynchronous 8-byte global -> shared copy; waiting for all but the newest group
__device__ __forceinline__ void cp_async8f(float *smem, const float *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// N values per lane -> every lane l holds the warp sum of value l % N
// (N a power of two <= 32; N - 1 + 5 - log2 N shuffles)
template <int N, typename R> __device__ __forceinline__ R tsum_n(R (&v)[N], int lane) {
#pragma unroll
    for (int n = N / 2; n >= 1; n >>= 1) {
        const bool hi = (lane & n) != 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const R keep = hi ? v[i + n] : v[i], send = hi ? v[i] : v[i + n];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, n);
        }
    }
#pragma unroll
    for (int m = N; m < 32; m <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    return v[0];
}

// ------------------------------------------------------ reverse stage kernel
constexpr int RNC = 32;                        // cells per CTA: a TXC x BY x BZ brick
constexpr int F_OUT = 1 << 30, F_IDX = F_OUT - 1;   // index flag: ghost beyond an outflow boundary

// One stage of the reverse sweep.  The stage maps its input I to
// base - dtk div F(I) (eq. radiative_transfer_discrete; base = I for the
// predictor and for first-order steps, I^n for the corrector); Zg is the
// cotangent of that transported state.  The kernel forms, per own element,
//   Ibar = sum over faces of Zg's flux cotangents through dF/dI  (+ Zg if the
//          base is the input) (+ Zown),
// and the opacity cotangent of every own cell (the face coefficients depend
// on tau = abar alpha len).  FUSE: the stage before this one ended with an
// interaction whose output is I; its reverse (src_rev) turns Ibar into the
// cotangent of that interaction's input, written to Zout.  Otherwise Ibar is
// written to Zout.  Cotangents of the gas energies and of kappa and eta go
// to per-cell arrays.
struct RevArgs {
    int nx[3], act[3], per[3], nd, limiter, transport, source;
    int add_base;                 // the stage's base intensities are its input
    int out_f64;                  // !FUSE: Zout is FP64 whatever the storage type
    int rev_order;                // bricks in reverse launch order
    int zg_f64;                   // Zg is FP64 whatever the storage type (read at own elements only:
                                  // the transport-free launch takes the caller's cotangent as it is)
    int ub_dst_acc;               // FUSE: add to ub_dst instead of writing it
    double coef[3];               // dtk / dx_a
    double hl[3];                 // d tau / d alpha of one side of an a-face: abar len_a / 2
    double taulen[3];             // the length in tau: dtk (tau_dt) or dx_a
    double abar, dts, sumw, T_exp, arad, rho_exp;
    const double *dir, *w;        // [3 nd], [nd]
    const void *I;                // stage input (storage type)
    const void *Zg;               // cotangent of the transported state (storage type)
    const void *Zown;             // extra cotangent of I at own elements, or null
    void *Zout;
    const double *alpha;          // opacity of the stage's faces
    const double *ug_a;           // the gas energy that alpha belongs to
    const double *ubA;            // cotangent of ug_a gathered so far, or null
    double *ubA_out;              // !FUSE: the complete cotangent of ug_a, or null
    const double *ugm, *Em, *X;   // FUSE: the interaction's gas energy in, saved E-bar_- and root
    double *ub_dst;               // FUSE: cotangent of ugm
    double *kb, *eb;              // added
    const double *cc_au, *cc_as, *cc_Y, *kap, *rho, *eta;
    const uint8_t *cc_on;
};

// LK: the limiter kind fixed at compile time (RT_LIM_MC, the limiter of every
// workload here), or -1 to read it from the arguments.  PER: every active axis
// is periodic, so no stencil row lies beyond an outflow boundary and the ghost
// folding drops out at compile time
// NOTR: an instance for launches without transport, whose x1 loop is only
// loads and a reduction (kept apart, so that the transport instances compile
// as they would without it)
template <class LT, int BY, int BZ, bool FUSE, int LK, bool PER, bool NOTR = false>
__global__ void __launch_bounds__(LT::NT, LT::MINB) k_rev(const RevArgs A) {
    using S = typename LT::S;
    using V = typename LT::V;
    constexpr int NT = LT::NT, L = LT::L, NW = NT / 32;
    constexpr int TXC = RNC / (BY * BZ), NOWN = BY * BZ;
    constexpr int NRED = FUSE ? 2 * NOWN : NOWN;   // per x position: alpha-bar (and Q) of the own cells
    __shared__ int xmap[TXC + 4];                  // x1 window: positions i0 - 2 .. i0 + TXC + 1
    __shared__ int rowY[BZ * (BY + 4)], rowZ[BY * (BZ + 4)];
    // the same positions and rows as element offsets (times n_dir), resolved once
    __shared__ int xoff[TXC + 4], rowYo[BZ * (BY + 4)], rowZo[BY * (BZ + 4)];
    __shared__ __align__(16) S recX[NOWN][TXC + 3][8];   // x1 faces between window positions f, f + 1
    __shared__ __align__(16) S recY[BZ][BY + 3][TXC][8];
    __shared__ __align__(16) S recZ[BY][BZ + 3][TXC][8];
    __shared__ S part[NW][NRED][TXC];
    __shared__ S partP[NW][RNC];
    __shared__ S cInv[RNC], cUb[RNC], cEmb[RNC];   // rounded to the pass's type once, at the solve
    // FP32 pass: the x1 pipeline's next own-row values (I and Zg at x1 = i + 3)
    // are copied one position ahead with cp.async (double-buffered)
    constexpr bool PFX = L == 2;
    __shared__ __align__(16) S pfb[2][2 * NOWN][PFX ? NT * L : 2];
    extern __shared__ __align__(16) unsigned char dsm[];   // FUSE: cotangents of I_+ [RNC][NT L]
    S *sIt = reinterpret_cast<S *>(dsm);

    const int p = threadIdx.x, lane = p & 31, warp = p >> 5;
    const int nd = A.nd;
    const bool act = L * p < nd;
    const int d0 = act ? L * p : 0;        // idle lanes shadow direction 0; their results are dropped
    const int nx0 = A.nx[0], nx1 = A.nx[1], nx2 = A.nx[2];
    const int nseg = (nx0 + TXC - 1) / TXC;
    // every other launch walks the bricks in reverse: it starts where the launch
    // before it ended, on the part of that launch's output still in L2
    const int bid = A.rev_order ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int seg = bid % nseg, rest = bid / nseg, nyb = nx1 / BY;
    const int j0 = (rest % nyb) * BY, k0 = (rest / nyb) * BZ, i0 = seg * TXC;
    const int nc = min(TXC, nx0 - i0);
    auto mapq = [](int q, int n, int per) -> int {
        if (q >= 0 && q < n) return q;
        if (per) return ((q % n) + n) % n;
        return (q < 0 ? 0 : n - 1) | F_OUT;
    };
    for (int t = p; t < TXC + 4; t += NT) {
        xmap[t] = mapq(i0 - 2 + t, nx0, A.per[0]);
        xoff[t] = (xmap[t] & F_IDX) * nd;
    }
    for (int t = p; t < BZ * (BY + 4); t += NT) {
        const int q = t % (BY + 4), r = t / (BY + 4);
        const int my = mapq(j0 - 2 + q, nx1, A.per[1]);
        rowY[t] = (((k0 + r) * nx1 + (my & F_IDX)) * nx0) | (my & F_OUT);
        rowYo[t] = ((k0 + r) * nx1 + (my & F_IDX)) * nx0 * nd;
    }
    for (int t = p; t < BY * (BZ + 4); t += NT) {
        const int r = t % (BZ + 4), q = t / (BZ + 4);
        const int mz = mapq(k0 - 2 + r, nx2, A.per[2]);
        rowZ[t] = (((mz & F_IDX) * nx1 + j0 + q) * nx0) | (mz & F_OUT);
        rowZo[t] = ((mz & F_IDX) * nx1 + j0 + q) * nx0 * nd;
    }
    __syncthreads();
    if (A.transport) {
        const int nX = A.act[0] ? NOWN * (nc + 3) : 0;
        const int nY = A.act[1] ? BZ * (BY + 3) * nc : 0;
        const int nZ = A.act[2] ? BY * (BZ + 3) * nc : 0;
        for (int t = p; t < nX + nY + nZ; t += NT) {
            int cl, cr;
            S *dst;
            double len;
            if (t < nX) {
                const int o = t / (nc + 3), f = t % (nc + 3);
                const int rb = rowY[(o / BY) * (BY + 4) + o % BY + 2] & F_IDX;
                cl = rb + (xmap[f] & F_IDX); cr = rb + (xmap[f + 1] & F_IDX);
                dst = recX[o][f]; len = A.taulen[0];
            } else if (t < nX + nY) {
                const int u = t - nX, ii = u % nc, v = u / nc, f = v % (BY + 3), r = v / (BY + 3);
                cl = (rowY[r * (BY + 4) + f] & F_IDX) + i0 + ii;
                cr = (rowY[r * (BY + 4) + f + 1] & F_IDX) + i0 + ii;
                dst = recY[r][f][ii]; len = A.taulen[1];
            } else {
                const int u = t - nX - nY, ii = u % nc, v = u / nc, f = v % (BZ + 3), q = v / (BZ + 3);
                cl = (rowZ[q * (BZ + 4) + f] & F_IDX) + i0 + ii;
                cr = (rowZ[q * (BZ + 4) + f + 1] & F_IDX) + i0 + ii;
                dst = recZ[q][f][ii]; len = A.taulen[2];
            }
            face_record<S>((S)(A.abar * 0.5 * (A.alpha[cl] + A.alpha[cr]) * len), dst);
        }
    }
    __syncthreads();

    V n[3], an[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { n[a] = LT::dirv(A.dir, d0, a); an[a] = LT::vabs(n[a]); }
    const S cfs[3] = {(S)A.coef[0], (S)A.coef[1], (S)A.coef[2]};
    const S hvs[3] = {(S)A.hl[0], (S)A.hl[1], (S)A.hl[2]};
    auto cf = [&](int a) { return LT::splat(cfs[a]); };
    auto hv = [&](int a) { return LT::splat(hvs[a]); };
    const V zero = LT::splat(S(0));
    const int lim = LK >= 0 ? LK : A.limiter;
    auto beyond = [](int desc) -> bool {   // a stencil row beyond an outflow boundary
        if constexpr (PER) return false;
        else return (desc & F_OUT) != 0;
    };
    const S *Ip = (const S *)A.I, *Zp = (const S *)A.Zg, *Zo = (const S *)A.Zown;
    auto ldI = [&](int off) -> V { return LT::ld(Ip + off); };
    auto ldZ = [&](int off) -> V { return LT::ld(Zp + off); };
    // element offsets (32 bits: the host checks n_cell n_dir < 2^31) of the
    // stencil rows at x1 = 0, and which of them lie beyond an outflow boundary
    int ownv[NOWN];
#pragma unroll
    for (int o = 0; o < NOWN; ++o) ownv[o] = rowYo[(o / BY) * (BY + 4) + o % BY + 2] + d0;
    auto own = [&](int o) -> int { return ownv[o]; };

    // x1 pipeline per own row, at own position p: xE = the part of p's
    // cotangent known before face p + 3/2 (faces p -+ 1/2 and the slope terms
    // of p - 1 and p), xCa = S~_p gl_p, xIRb / xR1 / xPh = IRb, IRb - c3t and
    // phib of face p + 1/2, xI0 / xI1 = I_p / I_{p+1}, xH0 = hs_p,
    // xB0 / xB1 = Zg_p / Zg_{p+1}, xAb = alpha-bar share of face p - 1/2.
    // (S~_p = ILb_{p+1/2} - IRb_{p-1/2}; the cotangent of I_p along one axis is
    //  ILb_{p+1/2} + c3t_{p+1/2} + IRb_{p-1/2} - c3t_{p-1/2}
    //  + S~_p (gr_p - gl_p) + S~_{p-1} gl_{p-1} - S~_{p+1} gr_{p+1},
    //  with gl, gr the derivatives of the half slopes.)
    const bool xon = A.transport && A.act[0];
    const bool lowX = !PER && xon && i0 == 0 && !A.per[0];
    V xE[NOWN], xCa[NOWN], xIRb[NOWN], xR1[NOWN], xPh[NOWN], xI0[NOWN], xI1[NOWN], xH0[NOWN], xB0[NOWN], xB1[NOWN],
        xAb[NOWN];
    if (xon) {
#pragma unroll
        for (int o = 0; o < NOWN; ++o) {
            const int ob = own(o);
            V Iw[4], Zw[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xd = xmap[u], off = ob + xoff[u];
                Iw[u] = ldI(off);
                Zw[u] = beyond(xd) ? zero : ldZ(off);
            }
            const V d01 = Iw[1] - Iw[0], d12 = Iw[2] - Iw[1], d23 = Iw[3] - Iw[2];
            V hs1, gl1, gr1, gd1, hs2, gl2, gr2, gd2;
            limv(lim, d12, d01, hs1, gl1, gr1, gd1);
            limv(lim, d23, d12, hs2, gl2, gr2, gd2);
            const V ph0 = cf(0) * (Zw[1] - Zw[0]), ph1 = cf(0) * (Zw[2] - Zw[1]), ph2 = cf(0) * (Zw[3] - Zw[2]);
            const FaceCot<V> f0 = face_cot<LT>(ph0, n[0], an[0], recX[o][0]);
            const FaceCot<V> f1 = face_cot<LT>(ph1, n[0], an[0], recX[o][1]);
            const FaceCot<V> f2c = face_cot<LT>(ph2, n[0], an[0], recX[o][2]);
            const V St1 = f1.ILb - f0.IRb, St2 = f2c.ILb - f1.IRb;
            const V tb1 = face_tau<LT>(ph1, n[0], an[0], Iw[1] + hs1, Iw[2] - hs2, d12, recX[o][1]) * hv(0);
            V e = St2 * gd2 + St1 * gl1 + (f2c.ILb + f2c.c3t) + (f1.IRb - f1.c3t);
            if (lowX) e = e + (f1.ILb + f1.c3t);            // ghost I_{-1} is I_0
            xE[o] = e; xCa[o] = St2 * gl2;
            xIRb[o] = f2c.IRb; xR1[o] = f2c.IRb - f2c.c3t; xPh[o] = ph2;
            xI0[o] = Iw[2]; xI1[o] = Iw[3]; xH0[o] = hs2; xB0[o] = Zw[2]; xB1[o] = Zw[3];
            xAb[o] = lowX ? tb1 + tb1 : tb1;                  // tau of face -1/2 is 2 x (alpha_0 abar len / 2)
        }
    }

    const V wdir = LT::wv(A.w, d0);
    (void)wdir;
    // copies of position ii + 2 of the window (x1 = i0 + ii + 2) into stage ii & 1
    auto pf_issue = [&](int ii) {
        if constexpr (PFX) {
            if (!act) return;
            const int xd = xmap[ii + 4], st = ii & 1, xo = xoff[ii + 4];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                const int off = own(o) + xo;
                cp_async8f(&pfb[st][o][d0], (const float *)Ip + off);
                if (!beyond(xd)) cp_async8f(&pfb[st][NOWN + o][d0], (const float *)Zp + off);
            }
        }
    };
    if constexpr (PFX) {
        if (xon) { pf_issue(0); cp_commit(); }
    }
    // without transport (the launch that reverses the interaction ending a
    // reversed run, or a source-only configuration) a position's work is two
    // loads and a reduction: unrolled, so that several positions' loads are in
    // flight at once (rolled, the launch waits on one DRAM round trip per
    // position)
    if constexpr (NOTR) {
#pragma unroll 4
        for (int ii = 0; ii < nc; ++ii) {
            const int ie = (i0 + ii) * nd;
            S red[NRED];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                const V Ic = ldI(own(o) + ie);
                const V Zc = A.zg_f64 ? LT::ld64((const double *)A.Zg + own(o) + ie) : ldZ(own(o) + ie);
                V ib = zero;
                if (A.add_base) ib = ib + Zc;
                if (Zo) ib = ib + LT::ld(Zo + own(o) + ie);
                red[o] = act ? LT::hsum(zero) : S(0);
                if constexpr (FUSE) {
                    if (act) LT::st(sIt + (o * TXC + ii) * (NT * L) + d0, ib);
                    red[NOWN + o] = act ? LT::hsum(ib * Ic) : S(0);
                } else if (act) {
                    if (A.out_f64) LT::st64((double *)A.Zout + own(o) + ie, ib);
                    else LT::st((S *)A.Zout + own(o) + ie, ib);
                }
            }
            const S rs = tsum_n<NRED, S>(red, lane);
            if (lane < NRED) part[warp][lane][ii] = rs;
        }
    } else {
#pragma unroll 1
    for (int ii = 0; ii < nc; ++ii) {
        const int i = i0 + ii, ie = i * nd;
        V Ic[NOWN], Zc[NOWN], acc[NOWN], ab[NOWN];
        if (xon) {
            const int xd = xmap[ii + 4];
            const bool hiE = !PER && !A.per[0] && i == nx0 - 1;
            if constexpr (PFX) {
                if (ii + 1 < nc) pf_issue(ii + 1);
                cp_commit();
                cp_wait1();
            }
            const int xo = xoff[ii + 4];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                const int off = own(o) + xo;
                V I2, Z2;
                if constexpr (PFX) {
                    const float2 a = *reinterpret_cast<const float2 *>(&pfb[ii & 1][o][d0]);
                    const float2 b = *reinterpret_cast<const float2 *>(&pfb[ii & 1][NOWN + o][d0]);
                    I2 = LT::splat(0); Z2 = zero;
                    if constexpr (L == 2) { I2 = F2{a.x, a.y}; if (!beyond(xd)) Z2 = F2{b.x, b.y}; }
                    (void)off;
                } else {
                    I2 = ldI(off); Z2 = beyond(xd) ? zero : ldZ(off);
                }
                const V dr = xI1[o] - xI0[o], dl = I2 - xI1[o];
                V hsN, glN, grN, gdN;
                limv(lim, dl, dr, hsN, glN, grN, gdN);
                const V phN = cf(0) * (Z2 - xB1[o]);
                const FaceCot<V> fN = face_cot<LT>(phN, n[0], an[0], recX[o][ii + 3]);
                const V StN = fN.ILb - xIRb[o];
                V g = xE[o] - StN * grN;
                const V tb = face_tau<LT>(xPh[o], n[0], an[0], xI0[o] + xH0[o], xI1[o] - hsN, dr, recX[o][ii + 2]) * hv(0);
                if (hiE) g = g + xR1[o];                        // ghost I_{n} is I_{n-1}
                acc[o] = g;
                ab[o] = xAb[o] + (hiE ? tb + tb : tb);
                Ic[o] = xI0[o]; Zc[o] = xB0[o];
                xE[o] = StN * gdN + xCa[o] + (fN.ILb + fN.c3t) + xR1[o];
                xCa[o] = StN * glN; xIRb[o] = fN.IRb; xR1[o] = fN.IRb - fN.c3t; xPh[o] = phN;
                xI0[o] = xI1[o]; xI1[o] = I2; xH0[o] = hsN; xB0[o] = xB1[o]; xB1[o] = Z2; xAb[o] = tb;
            }
        } else {
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                Ic[o] = ldI(own(o) + ie);
                Zc[o] = A.zg_f64 ? LT::ld64((const double *)A.Zg + own(o) + ie) : ldZ(own(o) + ie);
                acc[o] = zero; ab[o] = zero;
            }
        }
        // one column of NB own cells along x2 or x3 (window rows k = 0 .. NB + 3,
        // own rows k = 2 .. NB + 1)
        auto column = [&](auto NBc, const int *rows, const int *rowso, int ax, auto ownidx, auto recp) {
            constexpr int NB = decltype(NBc)::value;
            V Yv[NB + 4], Bv[NB + 4];
            unsigned out = 0u;
#pragma unroll
            for (int k = 0; k < NB + 4; ++k) {
                const int d = rows[k];
                out |= (unsigned)beyond(d) << k;
                if (k >= 2 && k < NB + 2) { Yv[k] = Ic[ownidx(k - 2)]; Bv[k] = Zc[ownidx(k - 2)]; }
                else {
                    const int off = rowso[k] + d0 + ie;
                    Yv[k] = ldI(off);
                    Bv[k] = beyond(d) ? zero : ldZ(off);
                }
            }
            V dI[NB + 3];
#pragma unroll
            for (int k = 0; k < NB + 3; ++k) dI[k] = Yv[k + 1] - Yv[k];
            V hs[NB + 4], gl[NB + 4], gr[NB + 4], gd[NB + 4];
#pragma unroll
            for (int k = 1; k < NB + 3; ++k) limv(lim, dI[k], dI[k - 1], hs[k], gl[k], gr[k], gd[k]);
            V ph[NB + 3];
            FaceCot<V> fc[NB + 3];
#pragma unroll
            for (int f = 0; f < NB + 3; ++f) {
                ph[f] = cf(ax) * (Bv[f + 1] - Bv[f]);
                fc[f] = face_cot<LT>(ph[f], n[ax], an[ax], recp(f));
            }
            V St[NB + 4];
#pragma unroll
            for (int k = 1; k < NB + 3; ++k) St[k] = fc[k].ILb - fc[k - 1].IRb;
            V tb[NB + 2];   // d flux / d tau of the faces next to own cells (f = 1 .. NB + 1)
#pragma unroll
            for (int f = 1; f <= NB + 1; ++f)
                tb[f] = face_tau<LT>(ph[f], n[ax], an[ax], Yv[f] + hs[f], Yv[f + 1] - hs[f + 1], dI[f], recp(f));
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int k = q + 2, o = ownidx(q);
                const bool loE = (out >> (k - 1)) & 1u, hiE = (out >> (k + 1)) & 1u;
                V g = (fc[k].ILb + fc[k].c3t) + (fc[k - 1].IRb - fc[k - 1].c3t) + St[k] * gd[k] +
                      St[k - 1] * gl[k - 1] - St[k + 1] * gr[k + 1];
                if (loE) g = g + (fc[k - 1].ILb + fc[k - 1].c3t);
                if (hiE) g = g + (fc[k].IRb - fc[k].c3t);
                acc[o] = acc[o] + g;
                const V tl = tb[k - 1], tr = tb[k];
                ab[o] = fma2(hv(ax), (loE ? tl + tl : tl) + (hiE ? tr + tr : tr), ab[o]);
            }
        };
        if (A.transport && A.act[1]) {
#pragma unroll
            for (int r = 0; r < BZ; ++r)
                column(std::integral_constant<int, BY>{}, rowY + r * (BY + 4), rowYo + r * (BY + 4), 1,
                       [&](int q) { return r * BY + q; },
                       [&](int f) -> const S * { return recY[r][f][ii]; });
        }
        if (A.transport && A.act[2]) {
#pragma unroll
            for (int q = 0; q < BY; ++q)
                column(std::integral_constant<int, BZ>{}, rowZ + q * (BZ + 4), rowZo + q * (BZ + 4), 2,
                       [&](int r) { return r * BY + q; },
                       [&](int f) -> const S * { return recZ[q][f][ii]; });
        }
        S red[NRED];
#pragma unroll
        for (int o = 0; o < NOWN; ++o) {
            V ib = acc[o];
            if (A.add_base) ib = ib + Zc[o];
            if (Zo) ib = ib + LT::ld(Zo + own(o) + ie);
            red[o] = act ? LT::hsum(ab[o]) : S(0);
            if constexpr (FUSE) {
                if (act) LT::st(sIt + (o * TXC + ii) * (NT * L) + d0, ib);
                red[NOWN + o] = act ? LT::hsum(ib * Ic[o]) : S(0);
            } else if (act) {
                if (A.out_f64) LT::st64((double *)A.Zout + own(o) + ie, ib);
                else LT::st((S *)A.Zout + own(o) + ie, ib);
            }
        }
        const S rs = tsum_n<NRED, S>(red, lane);
        if (lane < NRED) part[warp][lane][ii] = rs;
    }
    }
    __syncthreads();
    if constexpr (FUSE) {
        // P = sum over directions of the cotangent of I_+, per own cell
        S v[RNC];
#pragma unroll
        for (int c = 0; c < RNC; ++c) {
            S t = S(0);
            if (act && c % TXC < nc) {
                if constexpr (L == 2) {
                    const float2 x = *reinterpret_cast<const float2 *>(sIt + c * (NT * L) + d0);
                    t = x.x + x.y;
                } else {
                    t = sIt[c * (NT * L) + d0];
                }
            }
            v[c] = t;
        }
        const S ps = tsum_n<RNC, S>(v, lane);
        partP[warp][lane] = ps;
        __syncthreads();
    }
    // one lane of warp 0 per own cell: the opacity chain and the interaction
    if (warp == 0) {
        const int lc = lane, o = lc / TXC, ii = lc % TXC;
        if (ii < nc) {
            const int c = ((k0 + o / BY) * nx1 + j0 + o % BY) * nx0 + i0 + ii;
            double abar = 0.0;
            for (int g = 0; g < NW; ++g) abar += (double)part[g][o][ii];
            const double Y = A.cc_Y[c], au = A.cc_au[c];
            const double iY = Y > 0.0 ? rcp_nr(Y) : 0.0;
            double t = A.ubA ? A.ubA[c] : 0.0, kbv = 0.0, rhom = -1.0;   // rho^m, formed on first use
            // alpha = kappa rho^m T^-p + alpha^s with T = u_g / Y
            if (A.transport && A.cc_on[c] && abar != 0.0) {
                const double Ta = A.ug_a[c] * iY;
                if (Ta > 0.0) {
                    double tp, iTa;
                    tpow_inv(Ta, A.T_exp, tp, iTa);
                    rhom = rho_m(au, A.kap[c], A.rho[c], A.rho_exp);
                    kbv = abar * rhom * tp;
                    t += abar * au * (-A.T_exp) * tp * iTa * iY;
                }
            }
            if constexpr (!FUSE) {
                if (A.ubA_out) A.ubA_out[c] = t;
                A.kb[c] += kbv;
            } else {
                const double ugm = A.ugm[c], as = A.cc_as[c];
                const double Tm = ugm * iY;
                double tmv = 0.0, iTmv = 0.0;
                if (Tm > 0.0) tpow_inv(Tm, A.T_exp, tmv, iTmv);
                const double am = (A.cc_on[c] && Tm > 0.0) ? au * tmv + as : 0.0;
                const bool on = A.source && A.cc_on[c] && am > 0.0 && Y > 0.0 && ugm > 0.0;
                if (on && rhom < 0.0) rhom = rho_m(au, A.kap[c], A.rho[c], A.rho_exp);
                double P = 0.0, Q = 0.0;
                for (int g = 0; g < NW; ++g) { P += (double)partP[g][lc]; Q += (double)part[g][NOWN + o][ii]; }
                const SrcRev r = src_rev(on, iY, ugm, au, as, A.eta[c], tmv, iTmv, rhom, on ? A.Em[c] : 0.0,
                                         on ? A.X[c] : 0.0, P, Q, t, A.dts, A.sumw, A.T_exp, A.arad);
                A.ub_dst[c] = (A.ub_dst_acc ? A.ub_dst[c] : 0.0) + r.ugb;
                A.kb[c] += kbv + r.kb;
                A.eb[c] += r.eb;
                cInv[lc] = (S)r.inv; cUb[lc] = (S)r.ub; cEmb[lc] = (S)r.Emb;
            }
        }
    }
    if constexpr (FUSE) {
        __syncthreads();
        if (act) {
            const V wv = LT::wv(A.w, d0);
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
#pragma unroll 4
                for (int ii = 0; ii < TXC; ++ii) {
                    if (ii >= nc) break;
                    const int lc = o * TXC + ii;
                    V ib;
                    if constexpr (L == 2) {
                        const float2 x = *reinterpret_cast<const float2 *>(sIt + lc * (NT * L) + d0);
                        ib = F2{x.x, x.y};
                    } else {
                        ib = sIt[lc * (NT * L) + d0];
                    }
                    const V out = (ib - LT::splat(cUb[lc]) * wv) * LT::splat(cInv[lc]) + LT::splat(cEmb[lc]) * wv;
                    LT::st((S *)A.Zout + own(o) + (i0 + ii) * nd, out);
                }
            }
        }
    }
}

// element-wise type conversion (the FP32 pass keeps its cotangents in FP32)
template <typename A, typename B> __global__ void k_cvt(const A *__restrict__ x, B *__restrict__ y, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (B)x[i];
}

static rt_status adj_fail(rt_ctx *c, rt_status st, const std::string &msg) {
    c->err = msg;
    return st;
}

template <class LT, int BY, int BZ, bool FUSE>
rt_status launch_rev_t(rt_ctx *c, const RevArgs &A) {
    constexpr int TXC = RNC / (BY * BZ);
    const size_t nblk = (size_t)((A.nx[0] + TXC - 1) / TXC) * (A.nx[1] / BY) * (A.nx[2] / BZ);
    const int dyn = FUSE ? (int)(RNC * LT::NT * LT::L * sizeof(typename LT::S)) : 0;
    bool per = true;   // every active axis periodic
    for (int a = 0; a < 3; ++a) per = per && (!A.act[a] || A.per[a]);
    auto kern = k_rev<LT, BY, BZ, FUSE, -1, false>;
    if constexpr (LT::NT <= LaneD::NT)       // the finer-grid lanes keep one instance per brick
        kern = A.limiter == RT_LIM_MC ? (per ? k_rev<LT, BY, BZ, FUSE, RT_LIM_MC, true> : k_rev<LT, BY, BZ, FUSE, RT_LIM_MC, false>)
                                      : (per ? k_rev<LT, BY, BZ, FUSE, -1, true> : kern);
    if (!A.transport) kern = k_rev<LT, BY, BZ, FUSE, -1, false, true>;   // neither limiter nor boundaries enter
    RT_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    kern<<<(unsigned)nblk, LT::NT, dyn, c->stream>>>(A);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}
template <class LT, bool FUSE> rt_status launch_rev_b(rt_ctx *c, const RevArgs &A) {
    // brick shapes as the forward stage kernel picks them (2 x 1 in place of 2 x 2 where the lane type asks)
    const bool by = A.act[1] && A.nx[1] % 2 == 0, bz = A.act[2] && A.nx[2] % 2 == 0;
    (void)bz;
    if constexpr (LT::BRICK22) {
        if (by && bz) return launch_rev_t<LT, 2, 2, FUSE>(c, A);
    }
    if (by) return launch_rev_t<LT, 2, 1, FUSE>(c, A);
    return launch_rev_t<LT, 1, 1, FUSE>(c, A);
}
static rt_status launch_rev(rt_ctx *c, const RevArgs &A, bool fuse) {
    if (c->nd > LaneD::NT) {       // finer grids: 1 x 1 bricks
        if (c->cfg.precision == RT_FP64)
            return fuse ? launch_rev_t<LaneD3, 1, 1, true>(c, A) : launch_rev_t<LaneD3, 1, 1, false>(c, A);
        return fuse ? launch_rev_t<LaneF3, 1, 1, true>(c, A) : launch_rev_t<LaneF3, 1, 1, false>(c, A);
    }
    if (c->cfg.precision == RT_FP64) return fuse ? launch_rev_b<LaneD, true>(c, A) : launch_rev_b<LaneD, false>(c, A);
    return fuse ? launch_rev_b<LaneF, true>(c, A) : launch_rev_b<LaneF, false>(c, A);
}

// The reverse pass's arena: the states of every stage of a run of N steps
// (the stage inputs I^0..I^N and the predictor outputs I*, u_g^0..u_g^N and
// u_g*, the stages' face opacities, the saved E-bar_- and roots), two
// cotangent buffers in the storage type and two gas-energy cotangents.  The
// layout depends only on N and the configuration, so a later call with the
// same N finds the same pointers.
struct AdjArena {
    int N = 0;
    std::vector<void *> In, Bs;
    std::vector<double *> un, us, aln, als, sE, sX;
    void *Z[2] = {nullptr, nullptr};
    double *ubc = nullptr, *ubp = nullptr;
};

// ids of forward recordings (rt_step_record); contexts may record from several host threads
static std::atomic<long long> g_rec_counter{0};

static rt_status adj_check(rt_ctx *c, const char *who) {
    const std::string w(who);
    if (c->metric < 0 || !c->have_fluid) return adj_fail(c, RT_ESTATE, "rt_set_metric and rt_set_fluid must precede " + w);
    if (rt_status d = rt_check_device(c)) return d;
    if (c->metric != RT_MINKOWSKI_CART || !c->static_fluid)
        return adj_fail(c, RT_EINVAL, w + ": flat Cartesian geometry with the fluid at rest only");
    if (c->cfg.precision == RT_BF16) return adj_fail(c, RT_EINVAL, w + ": FP64 or FP32 intensities only");
    if (!rt_coupling3(c)) return adj_fail(c, RT_EINVAL, w + ": coupling method 3 only");
    if (c->nd > REV_MAX_DIRS || c->nd % 2) return adj_fail(c, RT_EINVAL, w + ": at most 672 directions");
    if ((double)c->ncell * c->nd >= 2147483647.0)
        return adj_fail(c, RT_EINVAL, w + ": n_cell * n_dir must be below 2^31");
    for (int a = 0; a < 3; ++a) {
        if (!c->active[a]) continue;
        int b0 = c->cfg.bc[a][0], b1 = c->cfg.bc[a][1];
        bool per = b0 == RT_BC_PERIODIC && b1 == RT_BC_PERIODIC, out = b0 == RT_BC_OUTFLOW && b1 == RT_BC_OUTFLOW;
        if (!per && !out) return adj_fail(c, RT_EINVAL, w + ": periodic or outflow boundaries on both sides of an axis only");
        if (per && c->cfg.nx[a] < 4) return adj_fail(c, RT_EINVAL, w + ": periodic axes need at least 4 cells");
    }
    return RT_OK;
}

static rt_status adj_dt(rt_ctx *c, double &dt) {
    if (!(dt > 0.0)) {
        if (c->dt_cfl <= 0.0) {
            rt_status st = rt_cfl_dt(c, 0.4, &c->dt_cfl);
            if (st != RT_OK) return st;
        }
        dt = c->dt_cfl;
    }
    return RT_OK;
}

static rt_status adj_layout(rt_ctx *c, int N, AdjArena &ar) {
    const size_t nc = (size_t)c->ncell, ni = nc * c->nd, es = c->esize;
    const int order = c->cfg.order, ns = order == 2 ? 2 : 1;   // stages per step
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t bI = up(ni * es), bC = up(nc * 8);
    const size_t nI = (size_t)(N + 1) + (order == 2 ? N : 0) + 2;
    const size_t nCell = (size_t)(N + 1) * 2 + (order == 2 ? 2 * (size_t)N : 0) + 2 * (size_t)N * ns + 2;
    const size_t need = nI * bI + nCell * bC;
    if (c->adj_bytes < need) {
        c->rec_id = 0;
        if (c->adj) cudaFree(c->adj);
        c->adj = nullptr; c->adj_bytes = 0;
        RT_CUDA_TRY(c, cudaMalloc(&c->adj, need));
        c->adj_bytes = need;
    }
    char *p = (char *)c->adj;
    auto take = [&](size_t b) { char *r = p; p += b; return r; };
    ar.N = N;
    ar.In.assign(N + 1, nullptr); ar.Bs.assign(N, nullptr);
    ar.un.assign(N + 1, nullptr); ar.aln.assign(N + 1, nullptr); ar.us.assign(N, nullptr); ar.als.assign(N, nullptr);
    ar.sE.assign(N * ns, nullptr); ar.sX.assign(N * ns, nullptr);
    for (int n = 0; n <= N; ++n) ar.In[n] = take(bI);
    if (order == 2) for (int n = 0; n < N; ++n) ar.Bs[n] = take(bI);
    ar.Z[0] = take(bI); ar.Z[1] = take(bI);
    for (int n = 0; n <= N; ++n) { ar.un[n] = (double *)take(bC); ar.aln[n] = (double *)take(bC); }
    if (order == 2) for (int n = 0; n < N; ++n) { ar.us[n] = (double *)take(bC); ar.als[n] = (double *)take(bC); }
    for (int s = 0; s < N * ns; ++s) { ar.sE[s] = (double *)take(bC); ar.sX[s] = (double *)take(bC); }
    ar.ubc = (double *)take(bC); ar.ubp = (double *)take(bC);
    return RT_OK;
}

// forward run from (In[0], un[0]) with the stage kernels, saving every
// stage's state; G_last (may be null) receives the force of the last stage
static rt_status adj_forward(rt_ctx *c, const AdjArena &ar, double dt, double *G_last) {
    struct SaveGuard {
        rt_ctx *c;
        ~SaveGuard() { c->sv_Em = nullptr; c->sv_X = nullptr; }
    } guard{c};
    const int N = ar.N;
    rt_status st;
    if ((st = rt_launch_alpha(c, ar.un[0], ar.aln[0])) != RT_OK) return st;
    for (int n = 0; n < N; ++n) {
        double *G = n == N - 1 ? G_last : nullptr;
        if (c->cfg.order == 2) {
            c->sv_Em = ar.sE[2 * n]; c->sv_X = ar.sX[2 * n];
            st = rt_launch_stage(c, ar.In[n], ar.In[n], ar.Bs[n], ar.un[n], ar.us[n], ar.aln[n], ar.aln[n], ar.als[n],
                                 0.5 * dt, nullptr);
            if (st != RT_OK) return st;
            c->sv_Em = ar.sE[2 * n + 1]; c->sv_X = ar.sX[2 * n + 1];
            st = rt_launch_stage(c, ar.Bs[n], ar.In[n], ar.In[n + 1], ar.un[n], ar.un[n + 1], ar.als[n], ar.aln[n],
                                 ar.aln[n + 1], dt, G);
        } else {
            c->sv_Em = ar.sE[n]; c->sv_X = ar.sX[n];
            st = rt_launch_stage(c, ar.In[n], ar.In[n], ar.In[n + 1], ar.un[n], ar.un[n + 1], ar.aln[n], ar.aln[n],
                                 ar.aln[n + 1], dt, G);
        }
        if (st != RT_OK) return st;
    }
    return RT_OK;
}

// reverse sweep over the arena's N steps
// the reverse sweep's launches alternate their brick order (see k_rev)
static rt_status launch_rev_alt(rt_ctx *c, RevArgs &A, bool fuse, int &nlaunch) {
    A.rev_order = nlaunch++ & 1;
    return launch_rev(c, A, fuse);
}

static rt_status adj_reverse(rt_ctx *c, const AdjArena &ar, double dt, const double *dL_dI_out,
                             const double *dL_dug_out, double *dL_dI_in, double *dL_dug_in, double *dL_dkappa,
                             double *dL_deta) {
    const rt_config &f = c->cfg;
    const int order = f.order, ns = order == 2 ? 2 : 1, N = ar.N;
    const auto &In = ar.In, &Bs = ar.Bs;
    const auto &un = ar.un, &us = ar.us, &aln = ar.aln, &als = ar.als, &sE = ar.sE, &sX = ar.sX;
    void *const Z[2] = {ar.Z[0], ar.Z[1]};
    double *ubc = ar.ubc, *ubp = ar.ubp;
    rt_status st;
    int nl = 0;
    RevArgs B{};
    for (int a = 0; a < 3; ++a) {
        B.nx[a] = f.nx[a]; B.act[a] = c->active[a]; B.per[a] = f.bc[a][0] == RT_BC_PERIODIC;
    }
    B.nd = c->nd; B.limiter = f.limiter; B.source = f.source; B.abar = f.abar; B.sumw = c->sumw;
    B.T_exp = f.T_exp; B.arad = f.arad; B.rho_exp = f.rho_exp;
    B.dir = c->g->dir; B.w = c->g->w;
    B.cc_au = c->cc_au; B.cc_as = c->cc_as; B.cc_Y = c->cc_Y; B.kap = c->kap; B.rho = c->rho; B.eta = c->eta;
    B.cc_on = c->cc_on; B.kb = dL_dkappa; B.eb = dL_deta;
    auto stage_args = [&](double dtk) {
        RevArgs A = B;
        A.transport = f.transport;
        for (int a = 0; a < 3; ++a) {
            A.coef[a] = dtk / f.dx[a];
            A.taulen[a] = f.tau_dt ? dtk : f.dx[a];
            A.hl[a] = f.abar * 0.5 * A.taulen[a];
        }
        return A;
    };
    const bool f64 = f.precision == RT_FP64;
    {   // the interaction that ends the last step, alone (reading the caller's
        // FP64 cotangent directly in both passes)
        RevArgs A = B;
        A.transport = 0; A.add_base = 1;
        A.I = In[N]; A.Zg = dL_dI_out; A.zg_f64 = f64 ? 0 : 1; A.ubA = dL_dug_out;
        A.dts = dt; A.ugm = un[N - 1]; A.Em = sE[N * ns - 1]; A.X = sX[N * ns - 1];
        A.ub_dst = ubc; A.ub_dst_acc = 0; A.Zout = Z[0];
        if ((st = launch_rev_alt(c, A, true, nl)) != RT_OK) return st;
    }
    int zr = 0;   // Z[zr]: cotangent of the current stage's transported state
    for (int n = N - 1; n >= 0; --n) {
        if (order == 2) {
            // corrector: fluxes of I* (faces from u_g*), base I^n; fused with the
            // predictor's interaction (gas u_g^n -> u_g*, over dt/2)
            RevArgs A = stage_args(dt);
            A.I = Bs[n]; A.Zg = Z[0]; A.Zown = nullptr; A.add_base = 0;
            A.alpha = als[n]; A.ug_a = us[n]; A.ubA = nullptr;
            A.dts = 0.5 * dt; A.ugm = un[n]; A.Em = sE[2 * n]; A.X = sX[2 * n];
            A.ub_dst = ubc; A.ub_dst_acc = 1; A.Zout = Z[1];
            if ((st = launch_rev_alt(c, A, true, nl)) != RT_OK) return st;
            // predictor: fluxes of I^n, base I^n; the corrector's base cotangent Z[0] adds
            RevArgs P = stage_args(0.5 * dt);
            P.I = In[n]; P.Zg = Z[1]; P.Zown = Z[0]; P.add_base = 1;
            P.alpha = aln[n]; P.ug_a = un[n]; P.ubA = ubc;
            if (n > 0) {
                P.dts = dt; P.ugm = un[n - 1]; P.Em = sE[2 * n - 1]; P.X = sX[2 * n - 1];
                P.ub_dst = ubp; P.ub_dst_acc = 0; P.Zout = Z[0];   // Z[0] is read at own elements only
                if ((st = launch_rev_alt(c, P, true, nl)) != RT_OK) return st;
                std::swap(ubc, ubp);
            } else {
                P.ubA_out = dL_dug_in; P.Zout = dL_dI_in; P.out_f64 = 1;
                if ((st = launch_rev_alt(c, P, false, nl)) != RT_OK) return st;
            }
        } else {
            RevArgs A = stage_args(dt);
            A.I = In[n]; A.Zg = Z[zr]; A.Zown = nullptr; A.add_base = 1;
            A.alpha = aln[n]; A.ug_a = un[n]; A.ubA = ubc;
            if (n > 0) {
                A.dts = dt; A.ugm = un[n - 1]; A.Em = sE[n - 1]; A.X = sX[n - 1];
                A.ub_dst = ubp; A.ub_dst_acc = 0; A.Zout = Z[1 - zr];
                if ((st = launch_rev_alt(c, A, true, nl)) != RT_OK) return st;
                zr ^= 1;
                std::swap(ubc, ubp);
            } else {
                A.ubA_out = dL_dug_in; A.Zout = dL_dI_in; A.out_f64 = 1;
                if ((st = launch_rev_alt(c, A, false, nl)) != RT_OK) return st;
            }
        }
    }
    return RT_OK;
}

}  // namespace

extern "C" rt_status rt_step_adjoint(rt_ctx *c, const void *I_ckpt, const double *ug_ckpt, double dt, int nsteps,
                                     const double *dL_dI_out, const double *dL_dug_out, double *dL_dI_in,
                                     double *dL_dug_in, double *dL_dkappa, double *dL_deta) {
    if (!c) return RT_EINVAL;
    if (!I_ckpt || !ug_ckpt || !dL_dI_out || !dL_dI_in || !dL_dug_in || !dL_dkappa || !dL_deta || nsteps < 1)
        return adj_fail(c, RT_EINVAL, "rt_step_adjoint: null pointer or nsteps < 1");
    rt_status st;
    if ((st = adj_check(c, "rt_step_adjoint")) != RT_OK) return st;
    if ((st = adj_dt(c, dt)) != RT_OK) return st;
    // the recompute overwrites the arena, and with it any recording
    c->rec_id = 0;
    AdjArena ar;
    if ((st = adj_layout(c, nsteps, ar)) != RT_OK) return st;
    const size_t nc = (size_t)c->ncell, ni = nc * c->nd;
    // 1. forward recompute from the checkpoint with the stage kernels; the
    // stages only read their first input, so the checkpoint serves in place;
    // it is copied into the arena first where it overlaps the gradient this
    // call writes, or is not aligned as the arena's buffers (the stage kernels
    // load intensities in pairs, 8 bytes at a time)
    const char *ck = (const char *)I_ckpt, *gi = (const char *)dL_dI_in;
    if ((ck < gi + ni * sizeof(double) && gi < ck + ni * c->esize) || ((uintptr_t)ck & 255u) != 0)
        RT_CUDA_TRY(c, cudaMemcpyAsync(ar.In[0], I_ckpt, ni * c->esize, cudaMemcpyDeviceToDevice, c->stream));
    else
        ar.In[0] = const_cast<void *>(I_ckpt);
    RT_CUDA_TRY(c, cudaMemcpyAsync(ar.un[0], ug_ckpt, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if ((st = adj_forward(c, ar, dt, nullptr)) != RT_OK) return st;
    // 2. reverse sweep
    return adj_reverse(c, ar, dt, dL_dI_out, dL_dug_out, dL_dI_in, dL_dug_in, dL_dkappa, dL_deta);
}

extern "C" rt_status rt_step_record(rt_ctx *c, double dt, int nsteps, double *dt_used, long long *rec_id) {
    if (!c) return RT_EINVAL;
    if (!rec_id || nsteps < 1) return adj_fail(c, RT_EINVAL, "rt_step_record: null rec_id or nsteps < 1");
    *rec_id = 0;
    if (!c->have_I) return adj_fail(c, RT_ESTATE, "the intensity must be set before rt_step_record");
    rt_status st;
    if ((st = adj_check(c, "rt_step_record")) != RT_OK) return st;
    if ((st = adj_dt(c, dt)) != RT_OK) return st;
    if (dt_used) *dt_used = dt;
    c->rec_id = 0;
    AdjArena ar;
    if ((st = adj_layout(c, nsteps, ar)) != RT_OK) return st;
    const size_t nc = (size_t)c->ncell, ni = nc * c->nd;
    RT_CUDA_TRY(c, cudaMemcpyAsync(ar.In[0], c->I[0], ni * c->esize, cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(ar.un[0], c->ug[0], nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if ((st = adj_forward(c, ar, dt, c->G)) != RT_OK) return st;
    // the context's state becomes the end state, as after rt_step
    const int N = nsteps;
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->I[0], ar.In[N], ni * c->esize, cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->ug[0], ar.un[N], nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->alpha[0], ar.aln[N], nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->rec_id = g_rec_counter.fetch_add(1) + 1;
    c->rec_N = N;
    c->rec_dt = dt;
    *rec_id = c->rec_id;
    return RT_OK;
}

extern "C" rt_status rt_step_adjoint_recorded(rt_ctx *c, long long rec_id, const double *dL_dI_out,
                                              const double *dL_dug_out, double *dL_dI_in, double *dL_dug_in,
                                              double *dL_dkappa, double *dL_deta) {
    if (!c) return RT_EINVAL;
    if (!dL_dI_out || !dL_dI_in || !dL_dug_in || !dL_dkappa || !dL_deta)
        return adj_fail(c, RT_EINVAL, "rt_step_adjoint_recorded: null pointer");
    if (rec_id <= 0 || rec_id != c->rec_id)
        return adj_fail(c, RT_ESTATE, "rt_step_adjoint_recorded: no valid recording with this id (a later "
                                      "rt_step_record, rt_step_adjoint, rt_set_fluid or rt_set_metric replaced it)");
    rt_status st;
    if ((st = adj_check(c, "rt_step_adjoint_recorded")) != RT_OK) return st;
    AdjArena ar;
    if ((st = adj_layout(c, c->rec_N, ar)) != RT_OK) return st;
    return adj_reverse(c, ar, c->rec_dt, dL_dI_out, dL_dug_out, dL_dI_in, dL_dug_in, dL_dkappa, dL_deta);
}
