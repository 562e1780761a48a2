// adjoint.cu — reverse mode of the radiation step for flat Cartesian geometry
// with the fluid at rest, FP64 or FP32 intensities (section 5.2 motivates gradients
// through the step; the reverse pass is derived by hand from eq.
// radiative_transfer_discrete, eqs. rad_speeds / flux_Jiang and method 3 of
// section 3.5.2).
//
// One call reverses nsteps steps from a checkpoint (I^0, u_g^0):
//  1. forward recompute: every stage's transported intensities (the stage
//     kernel with the interaction switched off) and the interaction applied to
//     them, all kept in a library-owned arena;
//  2. reverse sweep, per stage from the last: the interaction adjoint (the
//     explicit pieces in reverse and the implicit function theorem at the
//     temperature root), then the transport adjoint, a gather over the faces
//     whose fluxes read each cell, with the limiter branches of the forward
//     state and the optical-depth dependence of the face coefficients, which
//     carries gradient into kappa and u_g through the opacity.
#include "stage_common.cuh"
#include <algorithm>

using namespace rtk;

namespace {

constexpr int ADJ_NT = 192;   // threads of a block = directions (n_dir <= 192)
constexpr int TXA = 8;        // cells per transport-adjoint block along x1
constexpr int NFACE = 9 * TXA + 3;

// ------------------------------------------------------------ interaction
struct SrcArgs {
    int ncell, nd, source;
    double dtk, sumw, T_exp, arad, rho_exp;
    const double *w, *ug_in, *cc_au, *cc_as, *cc_Y, *eta, *rho, *kap;
    const void *I;                           // storage type of the context
    const uint8_t *cc_on;
    void *I_out;                             // forward (storage type)
    double *ug_out;
    const void *Ibo;                         // reverse: cotangent of the output intensities (type R)
    const double *ubo;                       // cotangent of the output u_g
    void *Ibi;                               // cotangent of I (written, type R)
    double *ubi;                             // cotangent of u_g entering (ub_acc: added)
    int ub_acc;
    double *kb, *eb;                         // added
    unsigned long long *fail;
};

// rho^m = (kappa rho^m) / kappa, the derivative of alpha^a's prefactor in
// kappa, without an FP64 pow where kappa is nonzero
__device__ __forceinline__ double rho_m(double au, double kap, double rho, double m) {
    return kap != 0.0 ? au / kap : pow(rho, m);
}

// N (16 or 32) values per lane -> lane l holds the warp sum of value l % N
template <int N, typename R> __device__ __forceinline__ R tsum(R (&v)[N], int lane) {
#pragma unroll
    for (int n = N / 2; n >= 1; n >>= 1) {
        const bool hi = (lane & n) != 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            R keep = hi ? v[i + n] : v[i];
            R send = hi ? v[i] : v[i + n];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, n);
        }
    }
    if (N == 16) return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
    return v[0];
}

// cells per interaction block (one lane of warp 0 per cell in the solve):
// 32 for the FP32 pass, 16 for FP64 (register arrays of 16 doubles)
template <typename R> struct CellsPerBlock { static constexpr int v = sizeof(R) == 4 ? 32 : 16; };

// REV = false: I_out = interaction(I), u_g out.  REV = true: the reverse.
// R is the storage and per-element arithmetic type of intensities and their
// cotangents (FP64, or FP32 for the mixed pass); warp partial sums are in R,
// the sums over warps and the per-cell arithmetic in FP64.
template <bool REV, typename R>
__global__ void __launch_bounds__(ADJ_NT) k_src(const SrcArgs A) {
    constexpr int SC = CellsPerBlock<R>::v;
    constexpr int NW = ADJ_NT / 32;
    __shared__ double part[NW][3][SC];
    __shared__ double sh_a[SC], sh_b[SC], sh_c[SC];
    __shared__ int sh_on[SC];
    const int s = threadIdx.x, lane = s & 31, warp = s >> 5;
    const bool act = s < A.nd;
    const size_t c0 = (size_t)blockIdx.x * SC;
    const int nc = (int)min((size_t)SC, (size_t)A.ncell - c0);
    const R w = act ? (R)A.w[s] : R(0);
    const R *Isrc = (const R *)A.I, *Bsrc = (const R *)A.Ibo;
    R Iv[SC], Bv[SC], v[SC];
#pragma unroll
    for (int k = 0; k < SC; ++k) Iv[k] = (act && k < nc) ? __ldg(Isrc + (c0 + k) * A.nd + s) : R(0);
    if (REV) {
#pragma unroll
        for (int k = 0; k < SC; ++k) Bv[k] = (act && k < nc) ? __ldg(Bsrc + (c0 + k) * A.nd + s) : R(0);
    }
#pragma unroll
    for (int k = 0; k < SC; ++k) v[k] = Iv[k] * w;
    R r0 = tsum<SC, R>(v, lane);
    if (lane < SC) part[warp][0][lane] = (double)r0;
    if (REV) {
#pragma unroll
        for (int k = 0; k < SC; ++k) v[k] = Bv[k];
        R r1 = tsum<SC, R>(v, lane);
#pragma unroll
        for (int k = 0; k < SC; ++k) v[k] = Bv[k] * Iv[k];
        R r2 = tsum<SC, R>(v, lane);
        if (lane < SC) { part[warp][1][lane] = (double)r1; part[warp][2][lane] = (double)r2; }
    }
    __syncthreads();
    if (warp == 0 && lane < SC) {
        int on = 0;
        double a0 = 0.0, b0 = 0.0, cc0 = 0.0;
        if (lane < nc) {
            const size_t c = c0 + lane;
            const double Y = A.cc_Y[c], ugm = A.ug_in[c], au = A.cc_au[c], as = A.cc_as[c];
            // FP64 divisions are costly on this part: reciprocals once per cell
            const double iY = Y > 0.0 ? 1.0 / Y : 0.0, Tm = ugm * iY;
            const double tm = Tm > 0.0 ? tpow_neg<double>(Tm, A.T_exp) : 0.0;
            const double am = (A.cc_on[c] && Tm > 0.0) ? au * tm + as : 0.0;
            on = A.source && A.cc_on[c] && am > 0.0 && Y > 0.0 && ugm > 0.0;
            const double ub = (REV && A.ubo) ? A.ubo[c] : 0.0;
            if (on) {
                double Em = 0.0, P = 0.0, Q = 0.0;
                for (int g = 0; g < NW; ++g) Em += part[g][0][lane];
                if (REV)
                    for (int g = 0; g < NW; ++g) { P += part[g][1][lane]; Q += part[g][2][lane]; }
                constexpr double i4pi = 1.0 / FOURPI;
                const double dt = A.dtk, adt = am * dt, i1a = 1.0 / (1.0 + adt), K = adt * i1a, S = A.sumw;
                const double eta = A.eta[c], p = A.T_exp, ar = A.arad;
                Teq<double> q{K * Em, K * S * dt * i4pi, Em + ugm, Y, Tm, Em, au, as, eta, ar, dt, p, iY};
                double X, lo = 0.0, hi = q.W;
                bool ok;
                if constexpr (sizeof(R) == 4) ok = solve_mixed(q, &X);   // as the FP32 forward solves it
                else ok = newton_E<double>(q, Em, lo, hi, 200, 4.0 * 2.220446049250313e-16, &X);
                if (!ok && A.fail) atomicAdd(A.fail, 1ull);
                const double Tp = Tm + (Em - X) * iY;
                const double tp = tpow_neg<double>(Tp, p), aap = au * tp;
                const double Tp4 = Tp * Tp * Tp * Tp;
                const double a = (aap + as) * dt;
                const double cc = dt * (eta * aap * ar * Tp4 + as * X) * i4pi;
                const double inv = 1.0 / (1.0 + a);
                if (!REV) {
                    const double Ep = (Em + cc * S) * inv;
                    A.ug_out[c] = ugm - (Ep - Em);
                    a0 = cc; b0 = inv;
                } else {
                    // I_+ = (I + cc)/A, E_+ = sum w I_+, u_g+ = u_g - (E_+ - E_-)
                    const double sIpb = P - ub * S;                 // sum_s Ipb_s, Ipb_s = Ibo_s - ub w_s
                    const double sIpbI = Q - ub * Em;               // sum_s Ipb_s I_s
                    const double ccb = sIpb * inv;
                    const double Ab = -(sIpbI + cc * sIpb) * inv * inv;
                    double aapb = Ab * dt;
                    // 1/Tp without a division for p = 3.5: Tp^2 sqrt(Tp) Tp^-3.5
                    const double iTpx = p == 3.5 ? Tp * Tp * sqrt(Tp) * tp : 1.0 / Tp;
                    const double ccbd = ccb * dt * i4pi;
                    double etab = ccbd * aap * ar * Tp4;
                    aapb += ccbd * eta * ar * Tp4;
                    double Tpb = ccbd * eta * aap * ar * 4.0 * Tp * Tp * Tp;
                    double Xb = ccbd * as;
                    double aub = aapb * tp;
                    Tpb += aapb * (-p) * aap * iTpx;
                    double Tmb = Tpb, Emb = ub + Tpb * iY;
                    Xb -= Tpb * iY;
                    // root of h(X; B1, B2, T_-, E_-, au, eta) = 0
                    const double lin = (aap + as) * dt - q.B2 * as;
                    const double hT = -p * aap * iTpx * dt * X - q.B2 * eta * ar * (4.0 - p) * aap * Tp * Tp * Tp;
                    const double hX = lin - hT * iY;
                    const double lam = -Xb / hX;
                    const double B1b = -lam;
                    const double B2b = lam * (-as * X - eta * ar * aap * Tp4);
                    Tmb += lam * hT;
                    Emb += lam * hT * iY;
                    aub += lam * (tp * dt * X - q.B2 * eta * ar * tp * Tp4);
                    etab += lam * (-q.B2 * ar * aap * Tp4);
                    const double Kb = B2b * S * dt * i4pi + B1b * Em;
                    Emb += B1b * K;
                    const double amb = Kb * dt * i1a * i1a;
                    aub += amb * tm;
                    Tmb += amb * (-p) * au * tm * (p == 3.5 ? Tm * Tm * tm * sqrt(Tm) : 1.0 / Tm);
                    const double ugb = ub + Tmb * iY;
                    A.ubi[c] = A.ub_acc ? A.ubi[c] + ugb : ugb;
                    A.kb[c] += aub * rho_m(au, A.kap[c], A.rho[c], A.rho_exp);
                    A.eb[c] += etab;
                    a0 = inv; b0 = ub; cc0 = Emb;
                }
            } else {
                if (!REV) A.ug_out[c] = ugm;
                else A.ubi[c] = A.ub_acc ? A.ubi[c] + ub : ub;
            }
        }
        sh_on[lane] = on; sh_a[lane] = a0; sh_b[lane] = b0; sh_c[lane] = cc0;
    }
    __syncthreads();
    if (!act) return;
#pragma unroll
    for (int k = 0; k < SC; ++k) {
        if (k >= nc) break;
        const size_t i = (c0 + k) * A.nd + s;
        if (!REV) ((R *)A.I_out)[i] = sh_on[k] ? (Iv[k] + (R)sh_a[k]) * (R)sh_b[k] : Iv[k];
        else ((R *)A.Ibi)[i] = sh_on[k] ? (Bv[k] - (R)sh_b[k] * w) * (R)sh_a[k] + (R)sh_c[k] * w : Bv[k];
    }
}

// --------------------------------------------------------------- transport
struct TrArgs {
    int nx[3], act[3], per[3], nd, limiter, tau_dt;
    double dx[3], abar, dtk, T_exp, rho_exp;
    double coef[3], hl[3];                   // dtk/dx_a, and d tau/d alpha of one side of an a-face
    const double *dir, *alpha;
    const void *I;                           // intensities (type R)
    const void *Ibo;                         // cotangent of the stage output (type R)
    void *out_src, *base_out;                // cotangents written (type R)
    int src_acc, add_base;
    const double *ug, *cc_au, *cc_Y, *rho, *kap;
    const uint8_t *cc_on;
    double *ub, *kb;
    int ub_acc;
};

__device__ __forceinline__ int amap(int q, int n, int per) {
    if (q >= 0 && q < n) return q;
    if (per) return ((q % n) + n) % n;
    return q < 0 ? 0 : n - 1;
}

// c1, c2, c3 of the face and their derivatives in tau (in the pass's type)
template <typename TM> __device__ void face_cd(TM tau, TM *fc) {
    if (tau > TM(0)) {
        TM t2 = tau * tau, t4 = t2 * t2;
        TM F = -expm1(-t2), G = -expm1(-t4);
        TM f = sqrt(F) / tau, g = sqrt(G) / tau, e = exp(-tau), S = f + g;
        TM fp = exp(-t2) / sqrt(F) - f / tau;
        TM gp = G > TM(0) ? TM(2) * t2 * exp(-t4) / sqrt(G) - g / tau : TM(1);
        TM ep = -e, Sp = fp + gp, iS2 = TM(1) / (S * S);
        fc[0] = f * e / S; fc[1] = g * e / S; fc[2] = f * g / S;
        fc[3] = ((fp * e + f * ep) * S - f * e * Sp) * iS2;
        fc[4] = ((gp * e + g * ep) * S - g * e * Sp) * iS2;
        fc[5] = ((fp * g + f * gp) * S - f * g * Sp) * iS2;
    } else {
        fc[0] = TM(1); fc[1] = TM(0); fc[2] = TM(0);
        fc[3] = TM(-2); fc[4] = TM(1); fc[5] = TM(1);
    }
}

// the six face coefficients from a 16-byte aligned shared record, with vector loads
__device__ __forceinline__ void ldfc6(const float *p, float (&f)[6]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float2 b = *reinterpret_cast<const float2 *>(p + 4);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y;
}
__device__ __forceinline__ void ldfc6(const double *p, double (&f)[6]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2),
                  c = *reinterpret_cast<const double2 *>(p + 4);
    f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y; f[4] = c.x; f[5] = c.y;
}
__device__ __forceinline__ void ldfc2(const float *p, float (&f)[2]) {
    const float2 a = *reinterpret_cast<const float2 *>(p);
    f[0] = a.x; f[1] = a.y;
}
__device__ __forceinline__ void ldfc2(const double *p, double (&f)[2]) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    f[0] = a.x; f[1] = a.y;
}

// derivative of the limited slope in (dl, dr), branches of rtk::limiter
template <typename TM> __device__ __forceinline__ void lim_d(int kind, TM dl, TM dr, TM &gl, TM &gr) {
    gl = TM(0); gr = TM(0);
    if (kind == RT_LIM_DONOR || dl * dr <= TM(0)) return;
    const TM al = fabs(dl), ar = fabs(dr);
    if (kind == RT_LIM_MINMOD) { if (al < ar) gl = TM(1); else gr = TM(1); return; }
    TM m = TM(2) * al;
    int which = 0;
    if (TM(2) * ar < m) { m = TM(2) * ar; which = 1; }
    if (TM(0.5) * fabs(dl + dr) < m) which = 2;
    if (which == 0) gl = TM(2);
    else if (which == 1) gr = TM(2);
    else { gl = TM(0.5); gr = TM(0.5); }
}

// One axis of the gather for one (cell, direction).  V: intensities at
// offsets -3..3 along the axis (index o + 3), B: output cotangents at -2..2
// (index o + 2, zero outside an outflow boundary), eq: bit o + 3 set when
// offset o maps to this cell, fc[m + 2]: coefficients of the face between
// offsets m and m + 1 (m = -2..1).  Adds the cotangent of this cell's
// intensity to g and the cotangent of tau of the two adjacent faces to tb.
template <typename TM>
__device__ __forceinline__ void axis_adj(const TM (&V)[7], const TM (&B)[5], unsigned eq, const TM *const (&fc)[4],
                                         TM n, TM coef, int lim, TM &g, TM (&tb)[2]) {
    if (n == TM(0)) return;
    const TM an = fabs(n), h = TM(0.5), one = TM(1);
#pragma unroll
    for (int m = -2; m <= 1; ++m) {
        const TM phib = coef * (B[m + 3] - B[m + 2]);
        if (phib == TM(0)) continue;
        const TM Ill = V[m + 2], Il = V[m + 3], Ir = V[m + 4], Irr = V[m + 5];
        TM f[6];
        ldfc6(fc[m + 2], f);
        TM gla, glb, gra, grb;
        lim_d<TM>(lim, Ir - Il, Il - Ill, gla, glb);
        lim_d<TM>(lim, Irr - Ir, Ir - Il, gra, grb);
        const TM cL = n > TM(0) ? f[0] : f[1], cR = n > TM(0) ? f[1] : f[0];
        const TM ILb = phib * n * cL, IRb = phib * n * cR;
        const TM c3t = phib * an * f[2];
        const TM dIll = -h * ILb * glb;
        const TM dIl = c3t + ILb * (one - h * gla + h * glb) + h * IRb * grb;
        const TM dIr = -c3t + h * ILb * gla + IRb * (one + h * gra - h * grb);
        const TM dIrr = -h * IRb * gra;
        if (eq & (1u << (m + 2))) g += dIll;
        if (eq & (1u << (m + 3))) g += dIl;
        if (eq & (1u << (m + 4))) g += dIr;
        if (eq & (1u << (m + 5))) g += dIrr;
        if (m == -1 || m == 0) {
            TM sl = limiter<TM>(lim, Ir - Il, Il - Ill), sr = limiter<TM>(lim, Irr - Ir, Ir - Il);
            const TM IL = Il + h * sl, IR = Ir - h * sr;
            const TM cLb = phib * n * IL, cRb = phib * n * IR;
            const TM c1b = n > TM(0) ? cLb : cRb, c2b = n > TM(0) ? cRb : cLb;
            const TM c3b = -phib * an * (Ir - Il);
            tb[m + 1] += c1b * f[3] + c2b * f[4] + c3b * f[5];
        }
    }
}

// limited slope of a cell and its derivatives in (dl, dr); the MC case with
// selects only (same branches as lim_d: 0.5|dl+dr| wins when it is below
// both 2|dl| and 2|dr|, 2|dr| wins over 2|dl| when strictly smaller)
template <typename TM> __device__ __forceinline__ TM lim_dv(int kind, TM dl, TM dr, TM &gl, TM &gr) {
    if (kind == RT_LIM_MC) {
        const TM a2l = TM(2) * fabs(dl), a2r = TM(2) * fabs(dr), ah = TM(0.5) * fabs(dl + dr);
        const bool ok = dl * dr > TM(0);
        const TM mlr = fmin(a2l, a2r);
        const bool w2 = ah < mlr, w1 = !w2 && a2r < a2l;
        gl = ok ? (w2 ? TM(0.5) : (w1 ? TM(0) : TM(2))) : TM(0);
        gr = ok ? (w2 ? TM(0.5) : (w1 ? TM(2) : TM(0))) : TM(0);
        return ok ? copysign(fmin(mlr, ah), dl) : TM(0);
    }
    lim_d<TM>(kind, dl, dr, gl, gr);
    return limiter<TM>(kind, dl, dr);
}

// axis_adj for a cell whose stencil maps to seven distinct cells (every
// interior cell, and every cell of a periodic axis): only offset 0 is this
// cell, so face m needs only the derivative at its own stencil position 0 -
// the right neighbour's slope for m = -2, the full pair for m = -1 and 0, the
// left cell's slope for m = 1 - and the slopes of offsets -1, 0, 1.
template <typename TM>
__device__ __forceinline__ void axis_adj_int(const TM (&V)[7], const TM (&B)[5], const TM *const (&fc)[4], TM n, TM coef,
                                             int lim, TM &g, TM (&tb)[2]) {
    if (n == TM(0)) return;
    const TM an = fabs(n), h = TM(0.5), one = TM(1);
    const bool pos = n > TM(0);
    TM ga[3], gb[3], sv[3];
#pragma unroll
    for (int q = -1; q <= 1; ++q) sv[q + 1] = lim_dv<TM>(lim, V[q + 4] - V[q + 3], V[q + 3] - V[q + 2], ga[q + 1], gb[q + 1]);
    const TM ph[4] = {coef * (B[1] - B[0]), coef * (B[2] - B[1]), coef * (B[3] - B[2]), coef * (B[4] - B[3])};
    // m = -2: this cell is I_{r+1}; IR = I_r - s_r/2 with s_r the slope of offset -1
    {
        TM f[2];
        ldfc2(fc[0], f);
        const TM IRb = ph[0] * n * (pos ? f[1] : f[0]);
        g += -h * IRb * ga[0];
    }
    // m = -1: this cell is I_r
    {
        TM f[6];
        ldfc6(fc[1], f);
        const TM cL = pos ? f[0] : f[1], cR = pos ? f[1] : f[0];
        const TM ILb = ph[1] * n * cL, IRb = ph[1] * n * cR, c3t = ph[1] * an * f[2];
        g += -c3t + h * ILb * ga[0] + IRb * (one + h * ga[1] - h * gb[1]);
        const TM IL = V[2] + h * sv[0], IR = V[3] - h * sv[1];
        const TM cLb = ph[1] * n * IL, cRb = ph[1] * n * IR;
        tb[0] += (pos ? cLb : cRb) * f[3] + (pos ? cRb : cLb) * f[4] - ph[1] * an * (V[3] - V[2]) * f[5];
    }
    // m = 0: this cell is I_l
    {
        TM f[6];
        ldfc6(fc[2], f);
        const TM cL = pos ? f[0] : f[1], cR = pos ? f[1] : f[0];
        const TM ILb = ph[2] * n * cL, IRb = ph[2] * n * cR, c3t = ph[2] * an * f[2];
        g += c3t + ILb * (one - h * ga[1] + h * gb[1]) + h * IRb * gb[2];
        const TM IL = V[3] + h * sv[1], IR = V[4] - h * sv[2];
        const TM cLb = ph[2] * n * IL, cRb = ph[2] * n * IR;
        tb[1] += (pos ? cLb : cRb) * f[3] + (pos ? cRb : cLb) * f[4] - ph[2] * an * (V[4] - V[3]) * f[5];
    }
    // m = 1: this cell is I_{l-1}; IL = I_l + s_l/2 with s_l the slope of offset 1
    {
        TM f[2];
        ldfc2(fc[3], f);
        const TM ILb = ph[3] * n * (pos ? f[0] : f[1]);
        g += -h * ILb * gb[2];
    }
}

// TM: storage and per-element arithmetic of intensities and their cotangents
// (FP64, or FP32 for the mixed pass); the opacity cotangents are summed over
// warps and chained to u_g and kappa in FP64
template <typename TM>
__global__ void __launch_bounds__(ADJ_NT) k_tr_adj(const TrArgs A) {
    constexpr int NW = ADJ_NT / 32;
    __shared__ __align__(16) TM fcs[NFACE][8];   // c1 c2 c3 dc1 dc2 dc3 (padded for vector loads)
    __shared__ double abw[NW][TXA];
    const int s = threadIdx.x, lane = s & 31, warp = s >> 5;
    const bool act = s < A.nd;
    const int nx0 = A.nx[0], nx1 = A.nx[1], nx2 = A.nx[2];
    const int nseg = (nx0 + TXA - 1) / TXA;
    const int seg = blockIdx.x % nseg, row = blockIdx.x / nseg;
    const int j = row % nx1, k = row / nx1, x0 = seg * TXA;
    const int nc = min(TXA, nx0 - x0);
    auto cell = [&](int i, int jj, int kk) { return ((size_t)kk * nx1 + jj) * nx0 + i; };
    auto len = [&](int a) { return A.tau_dt ? A.dtk : A.dx[a]; };

    // face coefficients: x1 faces with left cell x0 + m, m = -2..TXA (slot m + 2);
    // x2 / x3 faces of cell t with left offset m = -2..1 (slot TXA + 3 + (axis - 1) 4 TXA + 4 t + m + 2)
    for (int f = s; f < NFACE; f += ADJ_NT) {
        int a, t, m;
        if (f < TXA + 3) { a = 0; t = 0; m = f - 2; }
        else { int u = f - (TXA + 3); a = 1 + u / (4 * TXA); t = (u % (4 * TXA)) / 4; m = u % 4 - 2; }
        if (!A.act[a] || (a > 0 && t >= nc)) continue;
        size_t cl, cr;
        if (a == 0) {
            cl = cell(amap(x0 + m, nx0, A.per[0]), j, k); cr = cell(amap(x0 + m + 1, nx0, A.per[0]), j, k);
        } else if (a == 1) {
            cl = cell(x0 + t, amap(j + m, nx1, A.per[1]), k); cr = cell(x0 + t, amap(j + m + 1, nx1, A.per[1]), k);
        } else {
            cl = cell(x0 + t, j, amap(k + m, nx2, A.per[2])); cr = cell(x0 + t, j, amap(k + m + 1, nx2, A.per[2]));
        }
        face_cd<TM>(TM(A.abar * 0.5 * (A.alpha[cl] + A.alpha[cr]) * len(a)), fcs[f]);
    }
    __syncthreads();

    TM n[3] = {TM(0), TM(0), TM(0)};
    if (act) for (int a = 0; a < 3; ++a) n[a] = (TM)A.dir[3 * s + a];
    // (host-computed: FP64 divisions per thread would cost more than the cell's work)
    const TM coef[3] = {TM(A.coef[0]), TM(A.coef[1]), TM(A.coef[2])};
    const TM hl[3] = {TM(A.hl[0]), TM(A.hl[1]), TM(A.hl[2])};
    const int nd = A.nd;
    // 32-bit element offsets (the host checks n_cell * n_dir < 2^31)
    const TM *Ip = (const TM *)A.I + s, *Bp = (const TM *)A.Ibo + s;
    auto ldI = [&](int off) -> TM { return act ? __ldg(Ip + off) : TM(0); };
    auto ldB = [&](int off) -> TM { return act ? __ldg(Bp + off) : TM(0); };
    auto eo = [&](int i, int jj, int kk) -> int { return ((kk * nx1 + jj) * nx0 + i) * nd; };

    // x2 / x3 stencils of the block's row (j, k): mapped indices, which
    // offsets are this cell, and which cotangent positions exist
    int ry[7], rz[7];   // element offsets of the stencil rows at x1 = 0
    unsigned eqa[3] = {0u, 0u, 0u}, ina[3] = {0u, 0u, 0u};
#pragma unroll
    for (int o = -3; o <= 3; ++o) {
        const int my = amap(j + o, nx1, A.per[1]), mz = amap(k + o, nx2, A.per[2]);
        ry[o + 3] = eo(0, my, k);
        rz[o + 3] = eo(0, j, mz);
        eqa[1] |= (unsigned)(my == j) << (o + 3);
        eqa[2] |= (unsigned)(mz == k) << (o + 3);
        ina[1] |= (unsigned)(A.per[1] || (j + o >= 0 && j + o < nx1)) << (o + 3);
        ina[2] |= (unsigned)(A.per[2] || (k + o >= 0 && k + o < nx2)) << (o + 3);
    }

    // sliding x1 window
    TM WX[7], BX[5];
    if (A.act[0]) {
#pragma unroll
        for (int o = -3; o <= 3; ++o) WX[o + 3] = ldI(eo(amap(x0 + o, nx0, A.per[0]), j, k));
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
            int q = x0 + o;
            BX[o + 2] = (A.per[0] || (q >= 0 && q < nx0)) ? ldB(eo(amap(q, nx0, A.per[0]), j, k)) : TM(0);
        }
    }
#pragma unroll 1
    for (int t = 0; t < nc; ++t) {
        const int i = x0 + t;
        const int ce = eo(i, j, k), ie = i * nd;
        const TM Ic = ldI(ce), Bc = ldB(ce);
        TM g = TM(0), abt = TM(0);
        if (A.act[0]) {
            unsigned eq = 0;
#pragma unroll
            for (int o = -3; o <= 3; ++o) eq |= (unsigned)(amap(i + o, nx0, A.per[0]) == i) << (o + 3);
            const TM *fc[4] = {fcs[t], fcs[t + 1], fcs[t + 2], fcs[t + 3]};
            TM tb[2] = {TM(0), TM(0)};
            if (eq == (1u << 3)) axis_adj_int<TM>(WX, BX, fc, n[0], coef[0], A.limiter, g, tb);
            else axis_adj<TM>(WX, BX, eq, fc, n[0], coef[0], A.limiter, g, tb);
            abt += hl[0] * (tb[0] * TM(1 + ((eq >> 2) & 1)) + tb[1] * TM(1 + ((eq >> 4) & 1)));
        }
#pragma unroll
        for (int a = 1; a < 3; ++a) {
            if (!A.act[a]) continue;
            const int *rr = a == 1 ? ry : rz;
            TM V[7], B[5];
#pragma unroll
            for (int o = -3; o <= 3; ++o) V[o + 3] = o == 0 ? Ic : ldI(rr[o + 3] + ie);
#pragma unroll
            for (int o = -2; o <= 2; ++o)
                B[o + 2] = o == 0 ? Bc : (((ina[a] >> (o + 3)) & 1u) ? ldB(rr[o + 3] + ie) : TM(0));
            const int base = TXA + 3 + (a - 1) * 4 * TXA + 4 * t;
            const TM *fc[4] = {fcs[base], fcs[base + 1], fcs[base + 2], fcs[base + 3]};
            TM tb[2] = {TM(0), TM(0)};
            const unsigned eq = eqa[a];
            if (eq == (1u << 3)) axis_adj_int<TM>(V, B, fc, n[a], coef[a], A.limiter, g, tb);
            else axis_adj<TM>(V, B, eq, fc, n[a], coef[a], A.limiter, g, tb);
            abt += hl[a] * (tb[0] * TM(1 + ((eq >> 2) & 1)) + tb[1] * TM(1 + ((eq >> 4) & 1)));
        }
        if (act) {
            const size_t ix = (size_t)ce + s;
            TM v = g + (A.add_base ? Bc : TM(0));
            if (A.src_acc) v += ((TM *)A.out_src)[ix];
            ((TM *)A.out_src)[ix] = v;
            if (A.base_out) ((TM *)A.base_out)[ix] = Bc;
        }
        // opacity cotangent of this cell: warp sum now, block sum below
        for (int o = 16; o > 0; o >>= 1) abt += __shfl_xor_sync(0xffffffffu, abt, o);
        if (lane == 0) abw[warp][t] = (double)abt;
        // slide the x1 window
        if (A.act[0] && t + 1 < nc) {
#pragma unroll
            for (int o = 0; o < 6; ++o) WX[o] = WX[o + 1];
#pragma unroll
            for (int o = 0; o < 4; ++o) BX[o] = BX[o + 1];
            WX[6] = ldI(eo(amap(i + 4, nx0, A.per[0]), j, k));
            const int q = i + 3;
            BX[4] = (A.per[0] || q < nx0) ? ldB(eo(amap(q, nx0, A.per[0]), j, k)) : TM(0);
        }
    }
    // through alpha = kappa rho^m T^-p + alpha^s (T = u_g/Y) to u_g and kappa
    __syncthreads();
    if (s < nc) {
        const size_t c = cell(x0 + s, j, k);
        double ab = 0.0;
        for (int g = 0; g < NW; ++g) ab += abw[g][s];
        const double Y = A.cc_Y[c], T = Y > 0.0 ? A.ug[c] / Y : 0.0;
        double ubv = 0.0;
        if (A.cc_on[c] && T > 0.0 && ab != 0.0) {
            const double tp = tpow_neg<double>(T, A.T_exp);
            A.kb[c] += ab * rho_m(A.cc_au[c], A.kap[c], A.rho[c], A.rho_exp) * tp;
            ubv = ab * A.cc_au[c] * (-A.T_exp) * tp / T / Y;
        }
        A.ub[c] = A.ub_acc ? A.ub[c] + ubv : ubv;
    }
}

// element-wise type conversion (the mixed pass keeps its cotangents in FP32)
template <typename A, typename B> __global__ void k_cvt(const A *__restrict__ x, B *__restrict__ y, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (B)x[i];
}

}  // namespace

// ----------------------------------------------------------------- host side
static rt_status adj_fail(rt_ctx *c, rt_status st, const std::string &msg) {
    c->err = msg;
    return st;
}

static rt_status launch_src(rt_ctx *c, bool rev, const void *I, const double *ug_in, double dtk, void *I_out,
                            double *ug_out, const void *Ibo, const double *ubo, void *Ibi, double *ubi, int ub_acc,
                            double *kb, double *eb) {
    SrcArgs A{};
    const rt_config &f = c->cfg;
    A.ncell = c->ncell; A.nd = c->nd; A.source = f.source;
    A.dtk = dtk; A.sumw = c->sumw; A.T_exp = f.T_exp; A.arad = f.arad; A.rho_exp = f.rho_exp;
    A.w = c->g->w; A.I = I; A.ug_in = ug_in; A.cc_au = c->cc_au; A.cc_as = c->cc_as; A.cc_Y = c->cc_Y;
    A.eta = c->eta; A.rho = c->rho; A.kap = c->kap; A.cc_on = c->cc_on;
    A.I_out = I_out; A.ug_out = ug_out; A.Ibo = Ibo; A.ubo = ubo; A.Ibi = Ibi; A.ubi = ubi; A.ub_acc = ub_acc;
    A.kb = kb; A.eb = eb; A.fail = c->fail;
    const bool f64 = c->cfg.precision == RT_FP64;
    const int SC = f64 ? CellsPerBlock<double>::v : CellsPerBlock<float>::v;
    unsigned nblk = (unsigned)((c->ncell + SC - 1) / SC);
    if (rev) {
        if (f64) k_src<true, double><<<nblk, ADJ_NT, 0, c->stream>>>(A);
        else k_src<true, float><<<nblk, ADJ_NT, 0, c->stream>>>(A);
    } else {
        if (f64) k_src<false, double><<<nblk, ADJ_NT, 0, c->stream>>>(A);
        else k_src<false, float><<<nblk, ADJ_NT, 0, c->stream>>>(A);
    }
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

static rt_status launch_tr(rt_ctx *c, const void *I, const double *ug, const double *alpha, double dtk,
                           const void *Ibo, void *out_src, int src_acc, int add_base, void *base_out, double *ub,
                           int ub_acc, double *kb) {
    TrArgs A{};
    const rt_config &f = c->cfg;
    for (int a = 0; a < 3; ++a) {
        A.nx[a] = f.nx[a]; A.act[a] = c->active[a]; A.per[a] = f.bc[a][0] == RT_BC_PERIODIC; A.dx[a] = f.dx[a];
    }
    A.nd = c->nd; A.limiter = f.limiter; A.tau_dt = f.tau_dt; A.abar = f.abar; A.dtk = dtk;
    A.T_exp = f.T_exp; A.rho_exp = f.rho_exp;
    A.dir = c->g->dir; A.I = I; A.alpha = alpha; A.Ibo = Ibo; A.out_src = out_src; A.base_out = base_out;
    A.src_acc = src_acc; A.add_base = add_base; A.ug = ug; A.cc_au = c->cc_au; A.cc_Y = c->cc_Y; A.rho = c->rho;
    A.kap = c->kap;
    for (int a = 0; a < 3; ++a) {
        A.coef[a] = dtk / f.dx[a];
        A.hl[a] = f.abar * 0.5 * (f.tau_dt ? dtk : f.dx[a]);
    }
    A.cc_on = c->cc_on; A.ub = ub; A.kb = kb; A.ub_acc = ub_acc;
    const int nseg = (f.nx[0] + TXA - 1) / TXA;
    unsigned nblk = (unsigned)((size_t)nseg * f.nx[1] * f.nx[2]);
    if (c->cfg.precision == RT_FP64) k_tr_adj<double><<<nblk, ADJ_NT, 0, c->stream>>>(A);
    else k_tr_adj<float><<<nblk, ADJ_NT, 0, c->stream>>>(A);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

// transport-only stage through the forward stage kernel (interaction off)
static rt_status transport_only(rt_ctx *c, const void *Isrc, const void *Ibase, void *Iout, const double *ug,
                                const double *alpha, double dtk, double *ug_scr, double *a_scr) {
    const int src = c->cfg.source;
    c->cfg.source = 0;
    rt_status st = rt_launch_stage(c, Isrc, Ibase, Iout, ug, ug_scr, alpha, alpha, a_scr, dtk, nullptr);
    c->cfg.source = src;
    return st;
}

extern "C" rt_status rt_step_adjoint(rt_ctx *c, const void *I_ckpt, const double *ug_ckpt, double dt, int nsteps,
                                     const double *dL_dI_out, const double *dL_dug_out, double *dL_dI_in,
                                     double *dL_dug_in, double *dL_dkappa, double *dL_deta) {
    if (!c) return RT_EINVAL;
    if (!I_ckpt || !ug_ckpt || !dL_dI_out || !dL_dI_in || !dL_dug_in || !dL_dkappa || !dL_deta || nsteps < 1)
        return adj_fail(c, RT_EINVAL, "rt_step_adjoint: null pointer or nsteps < 1");
    if (c->metric < 0 || !c->have_fluid) return adj_fail(c, RT_ESTATE, "rt_set_metric and rt_set_fluid must precede rt_step_adjoint");
    if (c->metric != RT_MINKOWSKI_CART || !c->static_fluid)
        return adj_fail(c, RT_EINVAL, "rt_step_adjoint: flat Cartesian geometry with the fluid at rest only");
    if (c->cfg.precision == RT_BF16) return adj_fail(c, RT_EINVAL, "rt_step_adjoint: FP64 or FP32 intensities only");
    if (c->nd > ADJ_NT) return adj_fail(c, RT_EINVAL, "rt_step_adjoint: at most 192 directions");
    if ((double)c->ncell * c->nd >= 2147483647.0)
        return adj_fail(c, RT_EINVAL, "rt_step_adjoint: n_cell * n_dir must be below 2^31");
    for (int a = 0; a < 3; ++a) {
        if (!c->active[a]) continue;
        int b0 = c->cfg.bc[a][0], b1 = c->cfg.bc[a][1];
        bool per = b0 == RT_BC_PERIODIC && b1 == RT_BC_PERIODIC, out = b0 == RT_BC_OUTFLOW && b1 == RT_BC_OUTFLOW;
        if (!per && !out) return adj_fail(c, RT_EINVAL, "rt_step_adjoint: periodic or outflow boundaries on both sides of an axis only");
        if (per && c->cfg.nx[a] < 4) return adj_fail(c, RT_EINVAL, "rt_step_adjoint: periodic axes need at least 4 cells");
    }
    if (!(dt > 0.0)) {
        if (c->dt_cfl <= 0.0) {
            rt_status st = rt_cfl_dt(c, 0.4, &c->dt_cfl);
            if (st != RT_OK) return st;
        }
        dt = c->dt_cfl;
    }
    const size_t nc = (size_t)c->ncell, ni = nc * c->nd;
    const int order = c->cfg.order;
    // arena: per step I^n, (order 2: I*_t, I*), I^{n+1}_t in the storage
    // type, u_g^n, (u_g*); reverse: intensity cotangents in the storage type
    // (two, plus the running one for FP32) and eight per-cell FP64 buffers
    const size_t es = c->esize, per_step_i = order == 2 ? 4 : 2, per_step_c = order == 2 ? 2 : 1;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const bool f64 = c->cfg.precision == RT_FP64;
    const size_t bI = up(ni * es), bX = bI, bC = up(nc * 8);
    const size_t need = per_step_i * nsteps * bI + (f64 ? 2 : 3) * bX + (per_step_c * nsteps + 8) * bC;
    if (c->adj_bytes < need) {
        if (c->adj) cudaFree(c->adj);
        c->adj = nullptr; c->adj_bytes = 0;
        RT_CUDA_TRY(c, cudaMalloc(&c->adj, need));
        c->adj_bytes = need;
    }
    char *p = (char *)c->adj;
    auto take = [&](size_t b) { char *r = p; p += b; return r; };
    std::vector<void *> In(nsteps), At(nsteps), Bs(nsteps), Ct(nsteps);
    std::vector<double *> un(nsteps), us(nsteps);
    for (int n = 0; n < nsteps; ++n) {
        In[n] = take(bI);
        if (order == 2) { At[n] = take(bI); Bs[n] = take(bI); }
        Ct[n] = take(bI);
    }
    for (int n = 0; n < nsteps; ++n) { un[n] = (double *)take(bC); if (order == 2) us[n] = (double *)take(bC); }
    void *X1 = take(bX), *X2 = take(bX);
    void *Ib = f64 ? (void *)dL_dI_in : (void *)take(bX);   // the running cotangent of I
    double *ub = (double *)take(bC), *ubn = (double *)take(bC), *ubs = (double *)take(bC), *an = (double *)take(bC);
    double *as_ = (double *)take(bC), *ug_scr = (double *)take(bC), *a_scr = (double *)take(bC);
    double *u_next = (double *)take(bC);
    void *I_last = X2;   // the recompute's final state is never read: any buffer of ni * es bytes

    // 1. forward recompute from the checkpoint
    RT_CUDA_TRY(c, cudaMemcpyAsync(In[0], I_ckpt, ni * es, cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(un[0], ug_ckpt, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    rt_status st;
    for (int n = 0; n < nsteps; ++n) {
        void *Inext = n + 1 < nsteps ? In[n + 1] : I_last;
        double *unext = n + 1 < nsteps ? un[n + 1] : u_next;
        if ((st = rt_launch_alpha(c, un[n], an)) != RT_OK) return st;
        if (order == 1) {
            if ((st = transport_only(c, In[n], In[n], Ct[n], un[n], an, dt, ug_scr, a_scr)) != RT_OK) return st;
            if ((st = launch_src(c, false, Ct[n], un[n], dt, Inext, unext, 0, 0, 0, 0, 0, 0, 0)) != RT_OK) return st;
        } else {
            if ((st = transport_only(c, In[n], In[n], At[n], un[n], an, 0.5 * dt, ug_scr, a_scr)) != RT_OK) return st;
            if ((st = launch_src(c, false, At[n], un[n], 0.5 * dt, Bs[n], us[n], 0, 0, 0, 0, 0, 0, 0)) != RT_OK) return st;
            if ((st = rt_launch_alpha(c, us[n], as_)) != RT_OK) return st;
            if ((st = transport_only(c, Bs[n], In[n], Ct[n], us[n], as_, dt, ug_scr, a_scr)) != RT_OK) return st;
            if ((st = launch_src(c, false, Ct[n], un[n], dt, Inext, unext, 0, 0, 0, 0, 0, 0, 0)) != RT_OK) return st;
        }
    }
    // 2. reverse sweep
    if (!f64) {
        k_cvt<double, float><<<(unsigned)((ni + 255) / 256), 256, 0, c->stream>>>(dL_dI_out, (float *)Ib, ni);
        RT_CUDA_TRY(c, cudaGetLastError());
    } else if (Ib != (void *)dL_dI_out) {
        RT_CUDA_TRY(c, cudaMemcpyAsync(Ib, dL_dI_out, ni * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    if (dL_dug_out) RT_CUDA_TRY(c, cudaMemcpyAsync(ub, dL_dug_out, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    else RT_CUDA_TRY(c, cudaMemsetAsync(ub, 0, nc * sizeof(double), c->stream));
    for (int n = nsteps - 1; n >= 0; --n) {
        if ((st = rt_launch_alpha(c, un[n], an)) != RT_OK) return st;
        if (order == 1) {
            // interaction over dt, then transport over dt from I^n
            if ((st = launch_src(c, true, Ct[n], un[n], dt, 0, 0, Ib, ub, X1, ubn, 0, dL_dkappa, dL_deta)) != RT_OK) return st;
            if ((st = launch_tr(c, In[n], un[n], an, dt, X1, Ib, 0, 1, nullptr, ubn, 1, dL_dkappa)) != RT_OK) return st;
        } else {
            if ((st = rt_launch_alpha(c, us[n], as_)) != RT_OK) return st;
            // corrector interaction (gas from u_g^n) and transport (fluxes of I*, opacity of u_g*)
            if ((st = launch_src(c, true, Ct[n], un[n], dt, 0, 0, Ib, ub, X1, ubn, 0, dL_dkappa, dL_deta)) != RT_OK) return st;
            // (Ib, read by the interaction above, now receives the corrector's base cotangent)
            if ((st = launch_tr(c, Bs[n], us[n], as_, dt, X1, X2, 0, 0, Ib, ubs, 0, dL_dkappa)) != RT_OK) return st;
            // predictor interaction and transport (both from I^n)
            if ((st = launch_src(c, true, At[n], un[n], 0.5 * dt, 0, 0, X2, ubs, X1, ubn, 1, dL_dkappa, dL_deta)) != RT_OK) return st;
            if ((st = launch_tr(c, In[n], un[n], an, 0.5 * dt, X1, Ib, 1, 1, nullptr, ubn, 1, dL_dkappa)) != RT_OK) return st;
        }
        std::swap(ub, ubn);
    }
    if (!f64) {
        k_cvt<float, double><<<(unsigned)((ni + 255) / 256), 256, 0, c->stream>>>((const float *)Ib, dL_dI_in, ni);
        RT_CUDA_TRY(c, cudaGetLastError());
    }
    RT_CUDA_TRY(c, cudaMemcpyAsync(dL_dug_in, ub, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return RT_OK;
}
