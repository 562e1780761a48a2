// stage.cu — one fused stage of the radiation step on sm_103a.
//
// A stage (section 3.6) is: explicit transport of the conserved n^0 n_0 I-hat
// over dtk with fluxes from I_src (eq. radiative_transfer_discrete: spatial
// flux eqs. spatial_fluxes_vacuum / rad_speeds / flux_Jiang on a piecewise-
// linear reconstruction, angular flux eq. angular_fluxes on a minimum-angle
// plane reconstruction), followed in the same kernel by the implicit
// radiation-gas interaction of section 3.5.2 on every cell of the tile.
//
// Work decomposition: one CTA = one run of TX consecutive cells along x1 with
// all directions; thread s owns direction s (the warp reads 32 consecutive
// directions of a cell: coalesced).  The direction-independent face
// coefficients (optical depth cut-offs, signal-speed factors, fluid advection)
// are computed once per face into shared memory.  The transported intensities
// of the tile stay in shared memory for the interaction, so each stage reads
// I_src (stencil, L2-resident neighbours), I_base, and writes I_out once.
// Interaction: per-cell angular sums by groups of 8 threads (shuffle
// reduction), one FP64 temperature solve per cell (one lane per cell), then
// the per-direction update and the exchange ledger.
#include "rt_internal.cuh"
#include <cmath>

namespace {

constexpr int TX = 16;       // cells per tile along x1
constexpr int GS = 8;        // threads per cell in the angular sums
constexpr double FOURPI = 12.566370614359172953850573533118;

struct StageArgs {
    int nx0, nx1, nx2, nd, ne;
    int act0, act1, act2;
    int bc[3][2];
    int beam_dir, beam_lo, beam_hi;
    double beam_I;
    int n_pole_zero;
    double dx0, dx1, dx2;
    double gam, arad, rho_exp, T_exp, rho_floor, abar;
    int tau_dt, limiter, ang_recon, transport, source;
    double dtk;
    const void *Isrc; const void *Ibase; void *Iout;
    const double *ug_in; double *ug_out; const double *alpha_in; double *alpha_out;
    const double *rho, *kap, *cs, *eta, *vel, *uhat;
    double *G;
    unsigned long long *fail;
    // grid
    const int *mirror, *nnb, *nbr, *ring_edge, *ring_back, *edge;
    const void *dirT, *wT, *mxT, *mgT, *mmT;   // math-type copies
    // geometry (curved)
    int gn0, ng0, ng1;
    const void *cenU, *fn, *fP, *ew;           // math-type tables
    const uint8_t *mask;
    const double *pt_V, *pt_n0, *pt_len, *pt_e;
};

template <typename T> __device__ __forceinline__ float tof(T v);
template <> __device__ __forceinline__ float tof<float>(float v) { return v; }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TS, typename TM> struct IO;
template <> struct IO<double, double> {
    __device__ static double ld(const void *p, size_t i) { return __ldg((const double *)p + i); }
    __device__ static double st(void *p, size_t i, double v) { ((double *)p)[i] = v; return v; }
};
template <> struct IO<float, float> {
    __device__ static float ld(const void *p, size_t i) { return __ldg((const float *)p + i); }
    __device__ static float st(void *p, size_t i, float v) { ((float *)p)[i] = v; return v; }
};
template <> struct IO<__nv_bfloat16, float> {
    __device__ static float ld(const void *p, size_t i) { return __bfloat162float(((const __nv_bfloat16 *)p)[i]); }
    __device__ static float st(void *p, size_t i, float v) {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        ((__nv_bfloat16 *)p)[i] = b;
        return __bfloat162float(b);
    }
};

template <typename TM> __device__ __forceinline__ TM ldT(const void *p, size_t i) { return __ldg((const TM *)p + i); }

template <typename TM> __device__ __forceinline__ TM limiter(int kind, TM dl, TM dr) {
    if (kind == RT_LIM_DONOR) return TM(0);
    if (dl * dr <= TM(0)) return TM(0);
    TM s = dl > TM(0) ? TM(1) : TM(-1);
    TM al = fabs(dl), ar = fabs(dr);
    if (kind == RT_LIM_MINMOD) return s * fmin(al, ar);
    TM m = fmin(TM(2) * al, TM(2) * ar);
    m = fmin(m, TM(0.5) * fabs(dl + dr));
    return s * m;
}

// comoving total opacity with the density floor (sections 3.5.2 and 3.7)
__device__ __forceinline__ double cell_alpha(const StageArgs &A, double rho, double ug, double kap, double cs) {
    if (!(rho >= A.rho_floor) || rho <= 0.0) return 0.0;
    double T = (A.gam - 1.0) * ug / rho;
    return kap * pow(rho, A.rho_exp) * pow(T, -A.T_exp) + cs * rho;
}

// Boundary mapping of a cell index that may lie up to two cells outside the
// domain along one axis.  Returns the interior cell; *mir toggles the pole
// direction mirror; *beam is set for the fixed-inflow face.
__device__ __forceinline__ int map_cell(const StageArgs &A, int i, int j, int k, bool *mir, bool *beam) {
    *mir = false; *beam = false;
    if (i < 0 || i >= A.nx0) {
        int side = i < 0 ? 0 : 1, bc = A.bc[0][side];
        if (bc == RT_BC_PERIODIC) i = (i + A.nx0) % A.nx0;
        else if (bc == RT_BC_POLE) { i = side ? 2 * A.nx0 - 1 - i : -1 - i; *mir = true; }
        else { if (bc == RT_BC_BEAM) *beam = true; i = side ? A.nx0 - 1 : 0; }
    }
    if (j < 0 || j >= A.nx1) {
        int side = j < 0 ? 0 : 1, bc = A.bc[1][side];
        if (bc == RT_BC_PERIODIC) j = (j + A.nx1) % A.nx1;
        else if (bc == RT_BC_POLE) {
            j = side ? 2 * A.nx1 - 1 - j : -1 - j; *mir = !*mir;
            if (A.nx2 > 1) k = (k + A.nx2 / 2) % A.nx2;
        } else { if (bc == RT_BC_BEAM) *beam = true; j = side ? A.nx1 - 1 : 0; }
    }
    if (k < 0 || k >= A.nx2) {
        int side = k < 0 ? 0 : 1, bc = A.bc[2][side];
        if (bc == RT_BC_PERIODIC) k = (k + A.nx2) % A.nx2;
        else if (bc == RT_BC_POLE) { k = side ? 2 * A.nx2 - 1 - k : -1 - k; *mir = !*mir; }
        else { if (bc == RT_BC_BEAM) *beam = true; k = side ? A.nx2 - 1 : 0; }
    }
    return (k * A.nx1 + j) * A.nx0 + i;
}

template <typename TS, typename TM>
__device__ __forceinline__ TM load_I(const StageArgs &A, const void *I, int i, int j, int k, int s) {
    bool mir, beam;
    int c = map_cell(A, i, j, k, &mir, &beam);
    if (beam) {
        // fixed inflow through the x1-lower face (only that face carries a beam)
        if (i < 0 && j >= A.beam_lo && j < A.beam_hi && s == A.beam_dir) return TM(A.beam_I);
        return TM(0);
    }
    int d = mir ? __ldg(A.mirror + s) : s;
    return IO<TS, TM>::ld(I, (size_t)c * A.nd + d);
}

struct FaceRec {
    double c1, c2, c3, kL, kR;
};

// direction-independent coefficients of the spatial flux across the face
// between cells l = (il, jl, kl) and r = l + e_ax (eqs. rad_speeds, flux_Jiang
// per unit n^a; the tau -> 0 limits f = 1, g = 0 give the vacuum flux)
__device__ FaceRec face_coeffs(const StageArgs &A, bool flat, int ax, int il, int jl, int kl) {
    int ir = il + (ax == 0), jr = jl + (ax == 1), kr = kl + (ax == 2);
    bool m1, b1;
    int cl = map_cell(A, il, jl, kl, &m1, &b1), cr = map_cell(A, ir, jr, kr, &m1, &b1);
    double al = A.alpha_in[cl], ar = A.alpha_in[cr];
    double len;
    if (A.tau_dt) len = A.dtk;
    else if (flat) len = ax == 0 ? A.dx0 : (ax == 1 ? A.dx1 : A.dx2);
    else {
        int gn1 = 0; (void)gn1;
        int p = (jr + A.ng1) * A.gn0 + (ir + A.ng0);
        if (ax == 2) p = (jl + A.ng1) * A.gn0 + (il + A.ng0);
        int npt_stride = A.gn0 * (A.nx1 + 2 * A.ng1);
        len = A.pt_len[(size_t)ax * npt_stride + p];
    }
    double tau = A.abar * 0.5 * (al + ar) * len;
    FaceRec R;
    if (tau > 0.0) {
        double f = sqrt(-expm1(-tau * tau)) / tau;
        double g = sqrt(-expm1(-tau * tau * tau * tau)) / tau;
        double e = exp(-tau), fg = f + g;
        R.c1 = f * e / fg; R.c2 = g * e / fg; R.c3 = f * g / fg;
        double cadv = -expm1(-tau);
        double vl = A.vel[3 * (size_t)cl + ax], vr = A.vel[3 * (size_t)cr + ax];
        R.kL = cadv * fmax(vl, 0.0); R.kR = cadv * fmin(vr, 0.0);
    } else {
        R.c1 = 1.0; R.c2 = 0.0; R.c3 = 0.0; R.kL = 0.0; R.kR = 0.0;
    }
    return R;
}

template <typename TM>
__device__ __forceinline__ TM face_phi(TM n, const TM *rec, TM IL, TM IR, TM Il, TM Ir) {
    TM cL = n > TM(0) ? rec[0] : rec[1];
    TM cR = n > TM(0) ? rec[1] : rec[0];
    return n * (cL * IL + cR * IR) - fabs(n) * rec[2] * (Ir - Il) + rec[3] * IL + rec[4] * IR;
}

// ------------------------------------------------------------ temperature
// h(T) of method 3 (eq. T_almost_fully_implicit divided by T^p), with the
// reading A'_1 = B1, A'_2 = B2 (no 1/(alpha_+ dt) prefactor); see the oracle.
struct TeqArgs { double B1, B2, W, Y, au, as, eta, arad, dt, p; };

__device__ __forceinline__ double tpow_neg(double T, double p) {
    if (p == 3.5) { double r = sqrt(T); return 1.0 / (T * T * T * r); }
    if (p == 0.0) return 1.0;
    return pow(T, -p);
}

__device__ __forceinline__ void teq_eval(const TeqArgs &q, double T, double *h, double *dh) {
    double tp = tpow_neg(T, q.p);            // T^-p
    double aa = q.au * tp;
    double T3 = T * T * T, T4 = T3 * T;
    double em = q.B2 * q.eta * q.arad * aa * T4;  // B2 eta au a T^(4-p)
    double lin = (aa + q.as) * q.dt - q.B2 * q.as;
    double gap = q.W - q.Y * T;
    *h = lin * gap - q.B1 - em;
    *dh = (-q.p * aa / T) * q.dt * gap - lin * q.Y - em * (4.0 - q.p) / T;
}

// safeguarded Newton on the bracket (lo, hi], h(lo) > 0 >= h(hi); h decreases
__device__ bool solve_T(const TeqArgs &q, double T0, double *Tout) {
    double hi = q.W / q.Y, lo;
    double h, dh;
    teq_eval(q, hi, &h, &dh);
    if (h >= 0.0) { *Tout = hi; return true; }
    double T = fmin(fmax(T0, 1e-300), hi);
    teq_eval(q, T, &h, &dh);
    if (h > 0.0) lo = T;
    else {
        hi = T; lo = T;
        int it = 0;
        do { lo *= 0.5; teq_eval(q, lo, &h, &dh); } while (!(h > 0.0) && ++it < 2200);
        if (!(h > 0.0)) { *Tout = lo; return false; }
        T = lo;
    }
    for (int it = 0; it < 200; ++it) {
        double Tn = T - h / dh;
        if (!(Tn > lo && Tn < hi)) Tn = (hi > 4.0 * lo) ? sqrt(lo * hi) : 0.5 * (lo + hi);
        double step = fabs(Tn - T);
        T = Tn;
        teq_eval(q, T, &h, &dh);
        if (h > 0.0) lo = T; else hi = T;
        if (h == 0.0 || step <= 4.0 * 2.220446049250313e-16 * T || hi - lo <= 4.0 * 2.220446049250313e-16 * hi) {
            *Tout = T;
            return true;
        }
    }
    *Tout = T;
    return false;
}

// ------------------------------------------------------------ the kernel
template <typename TS, typename TM, bool FLAT>
__global__ void __launch_bounds__(256) k_stage(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nd = A.nd;
    const int NT = blockDim.x;
    const int s = threadIdx.x;
    const bool act = s < nd;
    const int nseg = (A.nx0 + TX - 1) / TX;
    const int seg = blockIdx.x % nseg;
    const int row = blockIdx.x / nseg;
    const int j = row % A.nx1, k = row / A.nx1;
    const int i0 = seg * TX;
    const int nc = min(TX, A.nx0 - i0);
    const int nfx = nc + 1;
    const int nface = nfx + 4 * nc;

    // shared layout
    TM *It = (TM *)smem_raw;                       // [TX][nd] transported
    TM *Ip = It + TX * nd;                         // [TX][nd] after the interaction
    TM *Rec = Ip + TX * nd;                        // [(5 TX + 1)][5] face coefficients
    TM *Icell = Rec + (5 * TX + 1) * 5;            // [nd] (curved: angular stencil)
    TM *Arec = Icell + nd;                         // [nd][6] reconstructed edge values
    double *cs_ = (double *)(((uintptr_t)(Arec + 6 * nd) + 15) & ~(uintptr_t)15);   // per-cell scalars
    double *sEm = cs_, *sB1 = cs_ + TX, *sB2 = cs_ + 2 * TX, *sEp = cs_ + 3 * TX, *sR = cs_ + 4 * TX;  // sR [TX][4]
    TM *sN0 = (TM *)(cs_ + 8 * TX), *sEm2 = sN0 + TX, *sAd = sEm2 + TX;
    int *sFlag = (int *)(sAd + TX);

    // --- face coefficients
    if (A.transport) {
        for (int f = s; f < nface; f += NT) {
            FaceRec R;
            if (f < nfx) {
                if (!A.act0) continue;
                R = face_coeffs(A, FLAT, 0, i0 + f - 1, j, k);
            }
            else {
                int q = f - nfx, ii = q % nc, t = q / nc;   // t: 0 y-lower, 1 y-upper, 2 z-lower, 3 z-upper
                int ax = 1 + t / 2, up = t & 1;
                int jl = j, kl = k;
                if (ax == 1) { if (!A.act1) continue; jl = up ? j : j - 1; }
                else { if (!A.act2) continue; kl = up ? k : k - 1; }
                R = face_coeffs(A, FLAT, ax, i0 + ii, jl, kl);
            }
            TM *r = Rec + 5 * f;
            r[0] = (TM)R.c1; r[1] = (TM)R.c2; r[2] = (TM)R.c3; r[3] = (TM)R.kL; r[4] = (TM)R.kR;
        }
    }
    __syncthreads();

    const int npt_stride = A.gn0 * (A.nx1 + 2 * A.ng1);
    const size_t pd = (size_t)npt_stride * nd;

    // --- transport
    for (int ii = 0; ii < nc; ++ii) {
        const int i = i0 + ii;
        const size_t cidx = ((size_t)k * A.nx1 + j) * A.nx0 + i;
        const int pt = FLAT ? 0 : (j + A.ng1) * A.gn0 + (i + A.ng0);
        TM Ic = TM(0), Ib = TM(0);
        if (act) {
            Ic = IO<TS, TM>::ld(A.Isrc, cidx * nd + s);
            Ib = IO<TS, TM>::ld(A.Ibase, cidx * nd + s);
        }
        TM out = Ib;
        if (A.transport) {
            TM acc = TM(0);
            TM nh[3] = {TM(0), TM(0), TM(0)};
            if (act) for (int m = 0; m < 3; ++m) nh[m] = ldT<TM>(A.dirT, 3 * s + m);
            for (int ax = 0; ax < 3; ++ax) {
                int on = ax == 0 ? A.act0 : (ax == 1 ? A.act1 : A.act2);
                if (!on || !act) continue;
                int di = ax == 0, dj = ax == 1, dk = ax == 2;
                TM v0 = load_I<TS, TM>(A, A.Isrc, i - 2 * di, j - 2 * dj, k - 2 * dk, s);
                TM v1 = load_I<TS, TM>(A, A.Isrc, i - di, j - dj, k - dk, s);
                TM v3 = load_I<TS, TM>(A, A.Isrc, i + di, j + dj, k + dk, s);
                TM v4 = load_I<TS, TM>(A, A.Isrc, i + 2 * di, j + 2 * dj, k + 2 * dk, s);
                TM sm = limiter<TM>(A.limiter, Ic - v1, v1 - v0);
                TM s0 = limiter<TM>(A.limiter, v3 - Ic, Ic - v1);
                TM sp = limiter<TM>(A.limiter, v4 - v3, v3 - Ic);
                const TM *rlo, *rhi;
                if (ax == 0) { rlo = Rec + 5 * ii; rhi = Rec + 5 * (ii + 1); }
                else {
                    int base = nfx + (ax == 1 ? 0 : 2 * nc);
                    rlo = Rec + 5 * (base + ii); rhi = Rec + 5 * (base + nc + ii);
                }
                TM ILlo = v1 + TM(0.5) * sm, IRlo = Ic - TM(0.5) * s0;
                TM ILhi = Ic + TM(0.5) * s0, IRhi = v3 - TM(0.5) * sp;
                if (FLAT) {
                    TM n = nh[ax];
                    TM Flo = face_phi<TM>(n, rlo, ILlo, IRlo, v1, Ic);
                    TM Fhi = face_phi<TM>(n, rhi, ILhi, IRhi, Ic, v3);
                    TM dxa = TM(ax == 0 ? A.dx0 : (ax == 1 ? A.dx1 : A.dx2));
                    acc += (Fhi - Flo) / dxa;
                } else {
                    // face points: lower face of this cell and of the next cell along ax
                    int ptn = ax == 0 ? pt + 1 : (ax == 1 ? pt + A.gn0 : pt);
                    int ptp = ax == 0 ? pt - 1 : (ax == 1 ? pt - A.gn0 : pt);
                    size_t o = (size_t)ax * pd;
                    uint8_t mc = A.mask[(size_t)pt * nd + s];
                    uint8_t mlo = A.mask[(size_t)ptp * nd + s], mhi = A.mask[(size_t)ptn * nd + s];
                    TM Flo = TM(0), Fhi = TM(0);
                    if (((mlo ^ mc) & 2) == 0) {
                        TM n = ldT<TM>(A.fn, o + (size_t)pt * nd + s), P = ldT<TM>(A.fP, o + (size_t)pt * nd + s);
                        if (P != TM(0)) Flo = P * face_phi<TM>(n, rlo, ILlo, IRlo, v1, Ic);
                    }
                    if (((mhi ^ mc) & 2) == 0) {
                        TM n = ldT<TM>(A.fn, o + (size_t)ptn * nd + s), P = ldT<TM>(A.fP, o + (size_t)ptn * nd + s);
                        if (P != TM(0)) Fhi = P * face_phi<TM>(n, rhi, ILhi, IRhi, Ic, v3);
                    }
                    acc += Fhi - Flo;
                }
            }
            if (FLAT) {
                out = Ib - TM(A.dtk) * acc;
            } else {
                TM ang = TM(0);
                // angular flux across the Voronoi edges of direction s
                if (act) Icell[s] = Ic;
                __syncthreads();
                int kk = act ? __ldg(A.nnb + s) : 0;
                if (act) {
                    TM rec[RT_MAXNB];
                    if (A.ang_recon == 1) {
                        for (int q = 0; q < kk; ++q) rec[q] = Ic;
                    } else {
                        TM dI[RT_MAXNB];
                        for (int q = 0; q < kk; ++q) dI[q] = Icell[__ldg(A.nbr + 6 * s + q)] - Ic;
                        int best = -1; TM bn = TM(0), ba = TM(0), bb = TM(0);
                        for (int q = 0; q < kk; ++q) {
                            int q1 = q + 1 == kk ? 0 : q + 1;
                            const size_t o = (size_t)(6 * s + q) * 3;
                            TM ga = ldT<TM>(A.mgT, o), gb = ldT<TM>(A.mgT, o + 1), gc = ldT<TM>(A.mgT, o + 2);
                            TM al = ga * dI[q] + gb * dI[q1];
                            TM be = gb * dI[q] + gc * dI[q1];
                            TM nr = al * dI[q] + be * dI[q1];
                            if (best < 0 || nr < bn) { best = q; bn = nr; ba = al; bb = be; }
                        }
                        int b1 = best + 1 == kk ? 0 : best + 1;
                        const size_t ox0 = (size_t)(6 * s + best) * 3, ox1 = (size_t)(6 * s + b1) * 3;
                        TM x0[3], x1[3];
                        for (int m = 0; m < 3; ++m) { x0[m] = ldT<TM>(A.mxT, ox0 + m); x1[m] = ldT<TM>(A.mxT, ox1 + m); }
                        for (int q = 0; q < kk; ++q) {
                            const size_t om = (size_t)(6 * s + q) * 3;
                            TM xm0 = ldT<TM>(A.mmT, om), xm1 = ldT<TM>(A.mmT, om + 1), xm2 = ldT<TM>(A.mmT, om + 2);
                            TM p0 = x0[0] * xm0 + x0[1] * xm1 + x0[2] * xm2;
                            TM p1 = x1[0] * xm0 + x1[1] * xm1 + x1[2] * xm2;
                            rec[q] = Ic + ba * p0 + bb * p1;
                        }
                    }
                    for (int q = 0; q < kk; ++q) Arec[6 * s + q] = rec[q];
                }
                __syncthreads();
                if (act) {
                    for (int q = 0; q < kk; ++q) {
                        int e = __ldg(A.ring_edge + 6 * s + q), t = __ldg(A.nbr + 6 * s + q);
                        int back = __ldg(A.ring_back + 6 * s + q);
                        bool own = __ldg(A.edge + 2 * e) == s;
                        TM w = ldT<TM>(A.ew, (size_t)pt * A.ne + e);
                        TM Io = Arec[6 * s + q], It2 = Arec[6 * t + back];
                        TM IL = own ? Io : It2, IR = own ? It2 : Io;
                        TM F = w * (w > TM(0) ? IL : IR);
                        ang += own ? F : -F;
                    }
                    ang /= ldT<TM>(A.wT, s);
                }
                __syncthreads();
                if (act) {
                    TM U = ldT<TM>(A.cenU, (size_t)pt * nd + s);
                    TM V = TM(A.pt_V[pt]);
                    TM Un = U * Ib - TM(A.dtk) * (acc / V + ang);
                    out = Un / U;
                }
            }
        }
        if (act) {
            bool zero = false;
            if (A.transport) {
                if (!FLAT) zero = (A.mask[(size_t)pt * nd + s] & 1) != 0;
                if (A.n_pole_zero > 0 && (j < A.n_pole_zero || j >= A.nx1 - A.n_pole_zero)) zero = true;
            }
            It[ii * nd + s] = zero ? TM(0) : out;
        }
    }
    __syncthreads();

    // --- interaction (section 3.5.2)
    const int lane8 = threadIdx.x & (GS - 1);
    const int cpp = NT / GS;      // cells per pass
    for (int c0 = 0; c0 < nc; c0 += cpp) {
        int ci = c0 + threadIdx.x / GS;
        TM Em = 0, B1 = 0, B2 = 0, cEm = 0;
        bool on = false;
        if (ci < nc) {
            const int i = i0 + ci;
            const size_t cidx = ((size_t)k * A.nx1 + j) * A.nx0 + i;
            const int pt = FLAT ? 0 : (j + A.ng1) * A.gn0 + (i + A.ng0);
            double rho = A.rho[cidx], ug = A.ug_in[cidx];
            double Y = rho / (A.gam - 1.0), Tm = ug / Y;
            double au = A.kap[cidx] * pow(rho, A.rho_exp), as = A.cs[cidx] * rho;
            double atm = (Tm > 0.0) ? au * tpow_neg(Tm, A.T_exp) + as : 0.0;
            on = A.source && rho >= A.rho_floor && rho > 0.0 && atm > 0.0;
            TM u0 = TM(A.uhat[4 * cidx]), u1 = TM(A.uhat[4 * cidx + 1]), u2 = TM(A.uhat[4 * cidx + 2]),
               u3 = TM(A.uhat[4 * cidx + 3]);
            TM n0 = FLAT ? TM(1) : TM(A.pt_n0[pt]);
            TM adt = TM(atm * A.dtk);
            if (on) {
                for (int d = lane8; d < nd; d += GS) {
                    TM x = ldT<TM>(A.dirT, 3 * d), y = ldT<TM>(A.dirT, 3 * d + 1), z = ldT<TM>(A.dirT, 3 * d + 2);
                    TM D = u0 - (u1 * x + u2 * y + u3 * z);
                    TM w = ldT<TM>(A.wT, d);
                    TM t = D * D * It[ci * nd + d] * w;
                    // compensated sum of the comoving energy
                    TM yk = t - cEm, tk = Em + yk;
                    cEm = (tk - Em) - yk; Em = tk;
                    TM K = adt / (n0 + D * adt);
                    B1 += n0 * K * t;
                    B2 += K * w / D;
                }
            }
        }
        // every lane of the warp takes part in the shuffles (idle groups add zeros)
        double dEm = (double)Em - (double)cEm, dB1 = B1, dB2 = B2;
        for (int o = 1; o < GS; o <<= 1) {
            dEm += __shfl_xor_sync(0xffffffffu, dEm, o);
            dB1 += __shfl_xor_sync(0xffffffffu, dB1, o);
            dB2 += __shfl_xor_sync(0xffffffffu, dB2, o);
        }
        if (ci < nc && lane8 == 0) { sEm[ci] = dEm; sB1[ci] = dB1; sB2[ci] = dB2; sFlag[ci] = on; }
    }
    __syncthreads();
    // one lane per cell: FP64 temperature solve and per-cell update constants
    for (int ci = threadIdx.x; ci < nc; ci += NT) {
        const int i = i0 + ci;
        const size_t cidx = ((size_t)k * A.nx1 + j) * A.nx0 + i;
        const int pt = FLAT ? 0 : (j + A.ng1) * A.gn0 + (i + A.ng0);
        double n0 = FLAT ? 1.0 : A.pt_n0[pt];
        sN0[ci] = (TM)n0;
        if (!sFlag[ci]) { sEm2[ci] = TM(0); sAd[ci] = TM(0); continue; }
        double rho = A.rho[cidx], ug = A.ug_in[cidx];
        double Y = rho / (A.gam - 1.0), Tm = ug / Y;
        double au = A.kap[cidx] * pow(rho, A.rho_exp), as = A.cs[cidx] * rho;
        TeqArgs q{sB1[ci], sB2[ci] * A.dtk / FOURPI, sEm[ci] + Y * Tm, Y, au, as, A.eta[cidx], A.arad, A.dtk, A.T_exp};
        double Tp;
        if (!solve_T(q, Tm, &Tp)) atomicAdd(A.fail, 1ull);
        double Est = q.W - Y * Tp;
        double aap = au * tpow_neg(Tp, A.T_exp), atp = aap + as;
        double em = q.eta * aap * A.arad * Tp * Tp * Tp * Tp + as * Est;
        sEm2[ci] = (TM)(A.dtk * em / FOURPI);
        sAd[ci] = (TM)(atp * A.dtk);
    }
    __syncthreads();
    // per-direction update, store
    for (int ci = 0; ci < nc; ++ci) {
        const int i = i0 + ci;
        const size_t cidx = ((size_t)k * A.nx1 + j) * A.nx0 + i;
        if (!act) continue;
        TM It0 = It[ci * nd + s];
        TM v = It0;
        if (sFlag[ci]) {
            const int pt = FLAT ? 0 : (j + A.ng1) * A.gn0 + (i + A.ng0);
            TM x = ldT<TM>(A.dirT, 3 * s), y = ldT<TM>(A.dirT, 3 * s + 1), z = ldT<TM>(A.dirT, 3 * s + 2);
            TM D = TM(A.uhat[4 * cidx]) - (TM(A.uhat[4 * cidx + 1]) * x + TM(A.uhat[4 * cidx + 2]) * y +
                                           TM(A.uhat[4 * cidx + 3]) * z);
            v = (sN0[ci] * It0 + sEm2[ci] / (D * D * D)) / (sN0[ci] + D * sAd[ci]);
            bool zero = false;
            if (!FLAT) zero = (A.mask[(size_t)pt * nd + s] & 1) != 0;
            if (A.n_pole_zero > 0 && (j < A.n_pole_zero || j >= A.nx1 - A.n_pole_zero)) zero = true;
            if (zero) v = TM(0);
        }
        Ip[ci * nd + s] = IO<TS, TM>::st(A.Iout, cidx * nd + s, v);
    }
    __syncthreads();
    // exchange ledger and force on the gas
    for (int c0 = 0; c0 < nc; c0 += cpp) {
        int ci = c0 + threadIdx.x / GS;
        bool valid = ci < nc;
        int cc = valid ? ci : 0;
        const int i = i0 + cc;
        const size_t cidx = ((size_t)k * A.nx1 + j) * A.nx0 + i;
        bool on = valid && sFlag[cc];
        TM Ep = 0, cEp = 0, r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        if (on) {
            TM u0 = TM(A.uhat[4 * cidx]), u1 = TM(A.uhat[4 * cidx + 1]), u2 = TM(A.uhat[4 * cidx + 2]),
               u3 = TM(A.uhat[4 * cidx + 3]);
            for (int d = lane8; d < nd; d += GS) {
                TM x = ldT<TM>(A.dirT, 3 * d), y = ldT<TM>(A.dirT, 3 * d + 1), z = ldT<TM>(A.dirT, 3 * d + 2);
                TM w = ldT<TM>(A.wT, d);
                TM D = u0 - (u1 * x + u2 * y + u3 * z);
                TM ip = Ip[cc * nd + d];
                TM t = D * D * ip * w;
                TM yk = t - cEp, tk = Ep + yk;
                cEp = (tk - Ep) - yk; Ep = tk;
                TM dI = (ip - It[cc * nd + d]) * w;
                r0 += dI; r1 += x * dI; r2 += y * dI; r3 += z * dI;
            }
        }
        double dEp = (double)Ep - (double)cEp, d0 = r0, d1 = r1, d2 = r2, d3 = r3;
        for (int o = 1; o < GS; o <<= 1) {
            dEp += __shfl_xor_sync(0xffffffffu, dEp, o);
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            d3 += __shfl_xor_sync(0xffffffffu, d3, o);
        }
        if (valid && lane8 == 0) {
            double ugm = A.ug_in[cidx];
            double ugp = on ? ugm - (dEp - sEm[cc]) : ugm;
            A.ug_out[cidx] = ugp;
            A.alpha_out[cidx] = cell_alpha(A, A.rho[cidx], ugp, A.kap[cidx], A.cs[cidx]);
            if (A.G) {
                double dR[4] = {d0, d1, d2, d3};
                if (!on) dR[0] = dR[1] = dR[2] = dR[3] = 0.0;
                for (int m = 0; m < 4; ++m) {
                    double g;
                    if (FLAT) g = dR[m];
                    else {
                        const int pt = (j + A.ng1) * A.gn0 + (i + A.ng0);
                        const double *E = A.pt_e + 16 * (size_t)pt;
                        g = E[m] * dR[0] + E[4 + m] * dR[1] + E[8 + m] * dR[2] + E[12 + m] * dR[3];
                    }
                    A.G[4 * cidx + m] = -g / A.dtk;
                }
            }
        }
    }
}

__global__ void k_alpha(int ncell, double gam, double rho_floor, double rho_exp, double T_exp,
                        const double *__restrict__ rho, const double *__restrict__ ug, const double *__restrict__ kap,
                        const double *__restrict__ cs, double *__restrict__ alpha) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double r = rho[c];
    if (!(r >= rho_floor) || r <= 0.0) { alpha[c] = 0.0; return; }
    double T = (gam - 1.0) * ug[c] / r;
    alpha[c] = kap[c] * pow(r, rho_exp) * pow(T, -T_exp) + cs[c] * r;
}

template <typename TS, typename TM, bool FLAT>
rt_status launch(rt_ctx *c, const StageArgs &A, int NT) {
    size_t smem = sizeof(TM) * (2 * TX * A.nd + (5 * TX + 1) * 5 + A.nd + 6 * A.nd) + 16 + sizeof(double) * 8 * TX +
                  sizeof(TM) * 3 * TX + sizeof(int) * TX;
    auto kern = k_stage<TS, TM, FLAT>;
    if (smem > 48 * 1024) RT_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nseg = (A.nx0 + TX - 1) / TX;
    size_t nblk = (size_t)nseg * A.nx1 * A.nx2;
    kern<<<(unsigned)nblk, NT, smem, c->stream>>>(A);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

}  // namespace

rt_status rt_launch_alpha(rt_ctx *c, const double *ug, double *alpha) {
    const rt_config &f = c->cfg;
    k_alpha<<<(c->ncell + 255) / 256, 256, 0, c->stream>>>(c->ncell, f.gam, f.rho_floor, f.rho_exp, f.T_exp, c->rho, ug,
                                                          c->kap, c->cs, alpha);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

rt_status rt_launch_stage(rt_ctx *c, const void *Isrc, const void *Ibase, void *Iout, const double *ug_in,
                          double *ug_out, const double *alpha_in, double *alpha_out, double dtk, double *G) {
    const rt_config &f = c->cfg;
    const rt_grid *g = c->g;
    StageArgs A{};
    A.nx0 = f.nx[0]; A.nx1 = f.nx[1]; A.nx2 = f.nx[2]; A.nd = c->nd; A.ne = c->ne;
    A.act0 = c->active[0]; A.act1 = c->active[1]; A.act2 = c->active[2];
    for (int a = 0; a < 3; ++a) for (int s = 0; s < 2; ++s) A.bc[a][s] = f.bc[a][s];
    A.beam_dir = f.beam_dir; A.beam_lo = f.beam_lo; A.beam_hi = f.beam_hi; A.beam_I = f.beam_I;
    A.n_pole_zero = f.n_pole_zero;
    A.dx0 = f.dx[0]; A.dx1 = f.dx[1]; A.dx2 = f.dx[2];
    A.gam = f.gam; A.arad = f.arad; A.rho_exp = f.rho_exp; A.T_exp = f.T_exp; A.rho_floor = f.rho_floor;
    A.abar = f.abar; A.tau_dt = f.tau_dt; A.limiter = f.limiter; A.ang_recon = f.ang_recon;
    A.transport = f.transport; A.source = f.source; A.dtk = dtk;
    A.Isrc = Isrc; A.Ibase = Ibase; A.Iout = Iout; A.ug_in = ug_in; A.ug_out = ug_out;
    A.alpha_in = alpha_in; A.alpha_out = alpha_out;
    A.rho = c->rho; A.kap = c->kap; A.cs = c->cs; A.eta = c->eta; A.vel = c->vel; A.uhat = c->uhat; A.G = G;
    A.fail = c->fail;
    A.mirror = g->mirror; A.nnb = g->nnb; A.nbr = g->nbr; A.ring_edge = g->ring_edge; A.ring_back = g->ring_back;
    A.edge = g->edge;
    bool dbl = f.precision == RT_FP64;
    A.dirT = dbl ? (const void *)g->dir : (const void *)g->dirf;
    A.wT = dbl ? (const void *)g->w : (const void *)g->wf;
    A.mxT = dbl ? (const void *)g->mx : (const void *)g->mxf;
    A.mgT = dbl ? (const void *)g->mg : (const void *)g->mgf;
    A.mmT = dbl ? (const void *)g->mm : (const void *)g->mmf;
    bool flat = c->metric == RT_MINKOWSKI_CART;
    A.ng0 = c->active[0] ? 2 : 0; A.ng1 = c->active[1] ? 2 : 0; A.gn0 = c->gn[0];
    if (!flat) {
        A.cenU = dbl ? (const void *)c->cenU_d : (const void *)c->cenU_f;
        A.fn = dbl ? (const void *)c->fn_d : (const void *)c->fn_f;
        A.fP = dbl ? (const void *)c->fP_d : (const void *)c->fP_f;
        A.ew = dbl ? (const void *)c->ew_d : (const void *)c->ew_f;
        A.mask = c->mask; A.pt_V = c->pt_V; A.pt_n0 = c->pt_n0; A.pt_len = c->pt_len; A.pt_e = c->pt_e;
    }
    int NT = ((c->nd + 31) / 32) * 32;
    if (NT < 64) NT = 64;
    if (NT > 256) { c->err = "more than 256 directions per cell are not supported by the stage kernel"; return RT_EINVAL; }
    if (f.precision == RT_FP64) return flat ? launch<double, double, true>(c, A, NT) : launch<double, double, false>(c, A, NT);
    if (f.precision == RT_FP32) return flat ? launch<float, float, true>(c, A, NT) : launch<float, float, false>(c, A, NT);
    return flat ? launch<__nv_bfloat16, float, true>(c, A, NT) : launch<__nv_bfloat16, float, false>(c, A, NT);
}
