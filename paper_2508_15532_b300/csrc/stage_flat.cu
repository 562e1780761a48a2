// stage_flat.cu — fast path of the stage kernel for flat Cartesian geometry
// with the fluid at rest in every cell (the periodic opacity/coupling box).
//
// Same scheme as stage.cu (section 3.6: transport over dtk, then the implicit
// interaction of section 3.5.2), specialised where the general kernel spends
// its instructions:
//  - the 32 transported intensities of the brick (one per cell, for this
//    thread's direction) stay in registers; no shared-memory tile;
//  - angular sums are warp transpose-reductions (31 shuffles per 32 cells)
//    followed by one shared-memory pass over the warps;
//  - at rest (D = 1, n^0 = 1) the coupling coefficients K, B1, B2 are per
//    cell, so a single sum (E-bar) feeds the temperature solve, and the
//    ledger and the force on the gas follow in closed form:
//      I_+ = (I + c) / (1 + a),  E-bar_+ = (E-bar_- + c sum w) / (1 + a),
//      Delta R^{0 i} = (c sum n^i w - a sum n^i I w) / (1 + a),
//    with a = alpha(T_+) dt, c = dt j(T_+) / (4 pi) (eq. fluid_interaction_discrete);
//  - MC limiter and face records of three coefficients (no fluid advection).
#include "stage_common.cuh"
#include "f32x2.cuh"

namespace {
using namespace rtk;

template <typename TM> struct __align__(4 * sizeof(TM)) Rec4 { TM c1, c2, c3, pad; };

// asynchronous 8-byte global -> shared copy, and waiting for this thread's copies
__device__ __forceinline__ void cp_async8(double *smem, const double *gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// half of the monotonised central slope, sign(dl) min(|dl|, |dr|, |dl + dr|/4),
// 0 where the one-sided differences differ in sign (halving is exact, so this
// is bit-identical to half of the MC slope)
template <typename TM> __device__ __forceinline__ TM mc_half(TM dl, TM dr) {
    TM m = fmin(fmin(fabs(dl), fabs(dr)), TM(0.25) * fabs(dl + dr));
    return (dl * dr > TM(0)) ? copysign(m, dl) : TM(0);
}

// per-unit-n_0 spatial flux of one direction through one face (see stage.cu):
// n (cL I_L + cR I_R) - |n| c3 (I_r - I_l) with (cL, cR) = (c1, c2) for n > 0
// and (c2, c1) for n < 0 (two selects; measured faster than the branch-free
// max(n,0)/min(n,0) form, which needs more registers)
template <typename TM>
__device__ __forceinline__ TM phi_s(TM n, TM an, const Rec4<TM> &r, TM IL, TM IR, TM Il, TM Ir) {
    TM cL = n > TM(0) ? r.c1 : r.c2, cR = n > TM(0) ? r.c2 : r.c1;
    return n * (cL * IL + cR * IR) - an * r.c3 * (Ir - Il);
}

// 32 values per lane -> lane l holds the sum over the warp of value l
template <typename TM> __device__ __forceinline__ TM transpose_sum(TM (&v)[NCELL], int lane) {
#pragma unroll
    for (int n = 16; n >= 1; n >>= 1) {
        const bool hi = (lane & n) != 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            TM keep = hi ? v[i + n] : v[i];
            TM send = hi ? v[i] : v[i + n];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, n);
        }
    }
    return v[0];
}

// FP32 math: four CTAs of 192 threads per SM.  Each SM sub-partition holds
// 16K registers and a CTA's six warps spread over the four, so four CTAs
// (six warps on each sub-partition) leave 80 registers a thread; this fits
// because the transported brick lives in shared memory (24 KB per CTA).
// Measured: 4 CTAs beat 3 (96 registers, brick in registers) and 5 (64
// registers, heavy spills).  FP64 math: two CTAs, brick in registers.
template <typename TM> struct MinBlocks { static constexpr int v = 4; };
template <> struct MinBlocks<double> { static constexpr int v = 2; };
constexpr int FS_NT = 192;

template <typename TS, typename TM, int BY, int BZ, bool WANTG, bool SIMPLE>
__global__ void __launch_bounds__(FS_NT, MinBlocks<TM>::v) k_stage_fs(const StageArgs A) {
    constexpr int TXC = NCELL / (BY * BZ), NOWN = BY * BZ;
    __shared__ int xmap[TXC + 4];
    __shared__ int rowY[BZ * (BY + 4)], rowZ[BY * (BZ + 4)];
    __shared__ Rec4<TM> recX[NOWN * (TXC + 1)], recY[BZ * (BY + 1) * TXC], recZ[BY * (BZ + 1) * TXC];
    __shared__ TM part[FS_NT / 32][4][NCELL];
    __shared__ TM cEm[NCELL], cInv[NCELL];
    __shared__ int cOn[NCELL];
    // per-cell inputs of the interaction (Y, u_g, alpha, kappa rho^m,
    // alpha^s, eta), copied asynchronously at the start so that their
    // latency hides behind the transport
    __shared__ double cIn[6][NCELL];

    const int nd = A.nd, NT = blockDim.x, s = threadIdx.x, lane = s & 31, warp = s >> 5;
    const bool act = s < nd;
    const int nseg = (A.nx0 + TXC - 1) / TXC;
    const int seg = blockIdx.x % nseg, rest = blockIdx.x / nseg, nyb = A.nx1 / BY;
    const int j0 = (rest % nyb) * BY, k0 = (rest / nyb) * BZ, i0 = seg * TXC;
    const int nc = min(TXC, A.nx0 - i0);

    for (int t = s; t < TXC + 4; t += NT) {
        int fl = 0;
        xmap[t] = map_axis(A, 0, i0 - 2 + t, &fl, nullptr) | fl;
    }
    for (int t = s; t < BZ * (BY + 4); t += NT) rowY[t] = row_desc(A, j0 - 2 + t % (BY + 4), k0 + t / (BY + 4));
    for (int t = s; t < BY * (BZ + 4); t += NT) rowZ[t] = row_desc(A, j0 + t / (BZ + 4), k0 - 2 + t % (BZ + 4));
    // local cell lc = o TXC + ii with own row o = r BY + q (lane lc of warp 0)
    const int lc_ii = lane % TXC, lc_o = lane / TXC;
    const size_t lc_cell = ((size_t)(k0 + lc_o / BY) * A.nx1 + j0 + lc_o % BY) * A.nx0 + i0 + lc_ii;
    const bool lc_valid = lc_ii < nc;
    if (warp == 0 && lc_valid) {
        const double *srcs[6] = {A.cc_Y, A.ug_in, A.alpha_int, A.cc_au, A.cc_as, A.eta};
#pragma unroll
        for (int q = 0; q < 6; ++q) cp_async8(&cIn[q][lane], srcs[q] + lc_cell);
    }
    cp_commit_all();
    __syncthreads();

    // face coefficients c1 = f e/(f+g), c2 = g e/(f+g), c3 = f g/(f+g) of the
    // optical depth tau = abar (alpha_l + alpha_r)/2 dx (eq. rad_speeds)
    auto coeffs = [&](int cl, int cr, double len, Rec4<TM> &r) {
        double tau = A.abar * 0.5 * (A.alpha_in[cl] + A.alpha_in[cr]) * (A.tau_dt ? A.dtk : len);
        if (tau > 0.0) {
            TM t = (TM)tau;
            TM f = sqrt(-expm1(-t * t)) / t, g = sqrt(-expm1(-t * t * t * t)) / t, e = exp(-t), fg = f + g;
            r.c1 = f * e / fg; r.c2 = g * e / fg; r.c3 = f * g / fg;
        } else {
            r.c1 = TM(1); r.c2 = TM(0); r.c3 = TM(0);
        }
        r.pad = TM(0);
    };
    if (A.transport) {
        const int nX = A.act0 ? NOWN * (nc + 1) : 0, nY = A.act1 ? BZ * (BY + 1) * nc : 0;
        const int nZ = A.act2 ? BY * (BZ + 1) * nc : 0;
        for (int t = s; t < nX + nY + nZ; t += NT) {
            if (t < nX) {
                int o = t / (nc + 1), f = t % (nc + 1);
                int rb = rowY[(o / BY) * (BY + 4) + o % BY + 2] & F_MASK;
                coeffs(rb + (xmap[f + 1] & F_MASK), rb + (xmap[f + 2] & F_MASK), A.dx0, recX[o * (TXC + 1) + f]);
            } else if (t < nX + nY) {
                int u = t - nX, ii = u % nc, v = u / nc, f = v % (BY + 1), r = v / (BY + 1);
                coeffs((rowY[r * (BY + 4) + f + 1] & F_MASK) + i0 + ii, (rowY[r * (BY + 4) + f + 2] & F_MASK) + i0 + ii,
                       A.dx1, recY[(r * (BY + 1) + f) * TXC + ii]);
            } else {
                int u = t - nX - nY, ii = u % nc, v = u / nc, f = v % (BZ + 1), q = v / (BZ + 1);
                coeffs((rowZ[q * (BZ + 4) + f + 1] & F_MASK) + i0 + ii, (rowZ[q * (BZ + 4) + f + 2] & F_MASK) + i0 + ii,
                       A.dx2, recZ[(q * (BZ + 1) + f) * TXC + ii]);
            }
        }
    }
    __syncthreads();

    const TS *Isrc = (const TS *)A.Isrc;
    const int smir = act ? __ldg(A.mirror + s) : 0;
    TM nh[3] = {TM(0), TM(0), TM(0)}, w = TM(0);
    if (act) {
        for (int m = 0; m < 3; ++m) nh[m] = ldT<TM>(A.dirT, 3 * s + m);
        w = ldT<TM>(A.wT, s);
    }
    const TM an[3] = {fabs(nh[0]), fabs(nh[1]), fabs(nh[2])};
    const TM dtk = (TM)A.dtk;
    const TM cdx[3] = {dtk / (TM)A.dx0, dtk / (TM)A.dx1, dtk / (TM)A.dx2};

    // per-thread element offsets of the stencil rows (-1: fixed zero row)
    // (SIMPLE: periodic/outflow boundaries only, no fixed or mirrored rows)
    auto roff = [&](int desc) -> int {
        if (!SIMPLE && (desc & F_FIX)) return -1;
        return (desc & F_MASK) * nd + ((!SIMPLE && (desc & F_MIR)) ? smir : s);
    };
    auto ldo = [&](int off, int i) -> TM {
        if (!SIMPLE && off < 0) return TM(0);
        return IO<TS, TM>::ld(Isrc, (unsigned)(off + i * nd));
    };
    auto ldx = [&](int ownoff, int xd, int jrow) -> TM {   // own row, x1 position from the descriptor
        if (!SIMPLE && (xd & F_FIX)) return (s == A.beam_dir && jrow >= A.beam_lo && jrow < A.beam_hi) ? TM(A.beam_I) : TM(0);
        int off = ownoff + (xd & F_MASK) * nd;
        if (!SIMPLE && (xd & F_MIR)) off += smir - s;
        return IO<TS, TM>::ld(Isrc, (unsigned)off);
    };

    // transported intensities of the brick: shared memory for FP32 math (it
    // frees 32 registers, so four CTAs fit per SM), registers for FP64 math
    constexpr bool SIT = sizeof(TM) == 4;
    __shared__ float sIt[SIT ? NCELL : 1][SIT ? FS_NT : 1];
    TM It[SIT ? 1 : NCELL];
#pragma unroll
    for (int c = 0; c < (SIT ? 1 : NCELL); ++c) It[c] = TM(0);
    auto putIt = [&](int c, TM v) { if constexpr (SIT) sIt[c][s] = (float)v; else It[c] = v; };
    auto getIt = [&](int c) -> TM { if constexpr (SIT) return (TM)sIt[c][s]; else return It[c]; };

    if (act) {
        int oy[BZ][BY + 4], oz[BY][BZ + 4];
#pragma unroll
        for (int r = 0; r < BZ; ++r)
#pragma unroll
            for (int q = 0; q < BY + 4; ++q) oy[r][q] = roff(rowY[r * (BY + 4) + q]);
#pragma unroll
        for (int q = 0; q < BY; ++q)
#pragma unroll
            for (int r = 0; r < BZ + 4; ++r) oz[q][r] = roff(rowZ[q * (BZ + 4) + r]);
        const bool same_base = A.Isrc == A.Ibase;
        // own-row offsets count from the first ghost plane of an x3 slab
        // (StageArgs::kb); the base array starts at the owned origin
        const int kbo = A.kb * A.nx1 * A.nx0 * nd;
        if (A.transport) {
            TM W0[NOWN], W1[NOWN], S0[NOWN], Flo[NOWN];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                W0[o] = W1[o] = S0[o] = Flo[o] = TM(0);
                if (A.act0) {
                    const int q = o % BY, r = o / BY, own = oy[r][q + 2];
                    TM Im2 = ldx(own, xmap[0], j0 + q), Im1 = ldx(own, xmap[1], j0 + q);
                    TM I0 = ldx(own, xmap[2], j0 + q), I1 = ldx(own, xmap[3], j0 + q);
                    TM sm1 = mc_half(I0 - Im1, Im1 - Im2), s0 = mc_half(I1 - I0, I0 - Im1);
                    Flo[o] = phi_s(nh[0], an[0], recX[o * (TXC + 1)], Im1 + sm1, I0 - s0, Im1, I0);
                    W0[o] = I0; W1[o] = I1; S0[o] = s0;
                }
            }
#pragma unroll
            for (int ii = 0; ii < TXC; ++ii) {
                if (ii < nc) {
                    const int i = i0 + ii;
                    TM acc[NOWN], Ic[NOWN];
#pragma unroll
                    for (int o = 0; o < NOWN; ++o) {
                        acc[o] = TM(0);
                        Ic[o] = A.act0 ? W0[o] : ldo(oy[o / BY][o % BY + 2], i);
                    }
                    if (A.act0) {
#pragma unroll
                        for (int o = 0; o < NOWN; ++o) {
                            const int q = o % BY, r = o / BY;
                            TM I2 = ldx(oy[r][q + 2], xmap[ii + 4], j0 + q);
                            TM s1 = mc_half(I2 - W1[o], W1[o] - W0[o]);
                            TM phi = phi_s(nh[0], an[0], recX[o * (TXC + 1) + ii + 1], W0[o] + S0[o],
                                           W1[o] - s1, W0[o], W1[o]);
                            acc[o] += cdx[0] * (phi - Flo[o]);
                            Flo[o] = phi; W0[o] = W1[o]; W1[o] = I2; S0[o] = s1;
                        }
                    }
                    if (A.act1) {
#pragma unroll
                        for (int r = 0; r < BZ; ++r) {
                            TM Y[BY + 4], sy[BY + 4], F[BY + 1];
#pragma unroll
                            for (int q = 0; q < BY + 4; ++q) Y[q] = (q >= 2 && q < BY + 2) ? Ic[r * BY + q - 2] : ldo(oy[r][q], i);
#pragma unroll
                            for (int q = 1; q < BY + 3; ++q) sy[q] = mc_half(Y[q + 1] - Y[q], Y[q] - Y[q - 1]);
#pragma unroll
                            for (int f = 0; f <= BY; ++f)
                                F[f] = phi_s(nh[1], an[1], recY[(r * (BY + 1) + f) * TXC + ii], Y[f + 1] + sy[f + 1],
                                             Y[f + 2] - sy[f + 2], Y[f + 1], Y[f + 2]);
#pragma unroll
                            for (int q = 0; q < BY; ++q) acc[r * BY + q] += cdx[1] * (F[q + 1] - F[q]);
                        }
                    }
                    if (A.act2) {
#pragma unroll
                        for (int q = 0; q < BY; ++q) {
                            TM Z[BZ + 4], sz[BZ + 4], F[BZ + 1];
#pragma unroll
                            for (int r = 0; r < BZ + 4; ++r) Z[r] = (r >= 2 && r < BZ + 2) ? Ic[(r - 2) * BY + q] : ldo(oz[q][r], i);
#pragma unroll
                            for (int r = 1; r < BZ + 3; ++r) sz[r] = mc_half(Z[r + 1] - Z[r], Z[r] - Z[r - 1]);
#pragma unroll
                            for (int f = 0; f <= BZ; ++f)
                                F[f] = phi_s(nh[2], an[2], recZ[(q * (BZ + 1) + f) * TXC + ii], Z[f + 1] + sz[f + 1],
                                             Z[f + 2] - sz[f + 2], Z[f + 1], Z[f + 2]);
#pragma unroll
                            for (int r = 0; r < BZ; ++r) acc[r * BY + q] += cdx[2] * (F[r + 1] - F[r]);
                        }
                    }
#pragma unroll
                    for (int o = 0; o < NOWN; ++o) {
                        TM Ib = same_base ? Ic[o]
                                          : IO<TS, TM>::ld(A.Ibase, (size_t)(oy[o / BY][o % BY + 2] - kbo + i * nd));
                        putIt(o * TXC + ii, Ib - acc[o]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int o = 0; o < NOWN; ++o)
#pragma unroll
                for (int ii = 0; ii < TXC; ++ii)
                    if (ii < nc) putIt(o * TXC + ii, IO<TS, TM>::ld(A.Ibase, (size_t)(oy[o / BY][o % BY + 2] - kbo + (i0 + ii) * nd)));
        }
    }

    // ---- interaction (section 3.5.2), fluid at rest
    if (warp == 0) {
        cp_wait_all();
        int on = 0;
        if (lc_valid) {
            double Y = cIn[0][lane], ug = cIn[1][lane], am = cIn[2][lane];
            on = A.source && A.cc_on[lc_cell] && am > 0.0 && Y > 0.0 && ug > 0.0;
        }
        cOn[lane] = on;
    }
    {
        TM v[NCELL];
#pragma unroll
        for (int c = 0; c < NCELL; ++c) v[c] = (act && c % TXC < nc) ? getIt(c) * w : TM(0);
        part[warp][0][lane] = transpose_sum(v, lane);
        if (WANTG) {
#pragma unroll
            for (int m = 0; m < 3; ++m) {
#pragma unroll
                for (int c = 0; c < NCELL; ++c) v[c] = (act && c % TXC < nc) ? getIt(c) * w * nh[m] : TM(0);
                part[warp][1 + m][lane] = transpose_sum(v, lane);
            }
        }
    }
    __syncthreads();
    if (warp == 0 && lc_valid) {
        const size_t cidx = lc_cell;
        const int nw = NT / 32;
        TM ce = TM(0), ci = TM(1);
        const double ugm = cIn[1][lane];
        if (cOn[lane]) {
            // warp partials summed in the math type (FP32 for the mixed path:
            // FP64 adds and conversions are costly here), then widened once
            TM Emt = TM(0), Ft[3] = {TM(0), TM(0), TM(0)};
            for (int g = 0; g < nw; ++g) Emt += part[g][0][lane];
            if (WANTG)
                for (int m = 0; m < 3; ++m)
                    for (int g = 0; g < nw; ++g) Ft[m] += part[g][1 + m][lane];
            double Em = (double)Emt, F[3] = {(double)Ft[0], (double)Ft[1], (double)Ft[2]};
            const double dt = A.dtk, adt = cIn[2][lane] * dt;
            const double K = adt / (1.0 + adt);
            const double Y = cIn[0][lane], au = cIn[3][lane], as = cIn[4][lane];
            // FP64 divisions are costly on this part: one reciprocal of Y per cell
            const double iY = 1.0 / Y, Tm = ugm * iY;
            Teq<double> q{K * Em, K * A.sumw * dt * (1.0 / FOURPI), Em + ugm, Y, Tm, Em, au, as,
                          cIn[5][lane], A.arad, dt, A.T_exp, iY};
            double X, a, c, inv, alpha_new;
            bool ok;
            if (sizeof(TM) == 4) {
                ok = solve_mixed(q, &X);
                // update constants in the storage math precision; the ledger uses
                // exactly the constants the stored intensities are built from
                const float Tp = (float)(Tm + (Em - X) * iY);
                const float aap = (float)au * tpow_neg<float>(Tp, (float)A.T_exp);
                const float af = (aap + (float)as) * (float)dt;
                const float cf = (float)dt * ((float)q.eta * aap * (float)A.arad * Tp * Tp * Tp * Tp + (float)as * (float)X) /
                                 (float)FOURPI;
                const float invf = 1.0f / (1.0f + af);
                a = af; c = cf; inv = invf;
            } else {
                double lo = 0.0, hi = q.W;
                ok = newton_E<double>(q, Em, lo, hi, 200, 4.0 * 2.220446049250313e-16, &X);
                const double Tp = Tm + (Em - X) * iY;
                const double aap = au * tpow_neg<double>(Tp, A.T_exp);
                a = (aap + as) * dt;
                c = dt * (q.eta * aap * A.arad * Tp * Tp * Tp * Tp + as * X) * (1.0 / FOURPI);
                inv = 1.0 / (1.0 + a);
            }
            if (!ok) atomicAdd(A.fail, 1ull);
            if (A.sv_X) { A.sv_Em[cidx] = Em; A.sv_X[cidx] = X; }
            ce = (TM)c; ci = (TM)inv;
            // exchange ledger in closed form (I_+ = (I + c)/(1 + a) in every direction)
            const double Ep = (Em + c * A.sumw) * inv;
            const double ugp = ugm - (Ep - Em);
            A.ug_out[cidx] = ugp;
            const double T = ugp * iY;
            if (sizeof(TM) == 4) alpha_new = T > 0.0 ? (double)((float)au * tpow_neg<float>((float)T, (float)A.T_exp) + (float)as) : 0.0;
            else alpha_new = T > 0.0 ? au * tpow_neg<double>(T, A.T_exp) + as : 0.0;
            A.alpha_out[cidx] = alpha_new;
            if (WANTG && A.G) {
                const double idt = 1.0 / dt;
                A.G[4 * cidx] = -(Ep - Em) * idt;
                for (int m = 0; m < 3; ++m) A.G[4 * cidx + 1 + m] = -((c * A.sumnw[m] - a * F[m]) * inv) * idt;
            }
        } else {
            A.ug_out[cidx] = ugm;
            A.alpha_out[cidx] = cIn[2][lane];
            if (WANTG && A.G) for (int m = 0; m < 4; ++m) A.G[4 * cidx + m] = 0.0;
        }
        cEm[lane] = ce; cInv[lane] = ci;
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int o = 0; o < NOWN; ++o) {
            const int q = o % BY, r = o / BY;
            const size_t base = ((size_t)(k0 + r) * A.nx1 + j0 + q) * A.nx0 + i0;
#pragma unroll
            for (int ii = 0; ii < TXC; ++ii) {
                if (ii < nc) {
                    const int lc = o * TXC + ii;
                    TM v = getIt(lc);
                    if (cOn[lc]) v = (v + cEm[lc]) * cInv[lc];
                    IO<TS, TM>::st(A.Iout, (base + ii) * nd + s, v);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Packed FP32 variant of k_stage_fs: each thread owns a pair of adjacent
// directions (2p, 2p+1) (n_dir = 10 n^2 + 2 is even) and works on both with
// f32x2 arithmetic (add/sub/mul/fma.rn.f32x2) and 8-byte loads and stores,
// which halves the arithmetic, load and address instructions per cell-angle.
// FP32 or BF16 storage, periodic/outflow boundaries, 162 directions (the
// count is a template argument).  Five CTAs of 96 threads per SM.
__device__ __forceinline__ F2 ld2(const float *p) { float2 v = __ldg(reinterpret_cast<const float2 *>(p)); return F2{v.x, v.y}; }
__device__ __forceinline__ F2 ld2(const __nv_bfloat16 *p) {
    float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    return F2{v.x, v.y};
}
__device__ __forceinline__ void st2(float *p, F2 v) { __stcs(reinterpret_cast<float2 *>(p), make_float2(v.x, v.y)); }
__device__ __forceinline__ void st2(__nv_bfloat16 *p, F2 v) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
}

// the face flux per component, n (cL I_L + cR I_R) - |n| c3 (I_r - I_l) with
// (cL, cR) = (c1, c2) for n > 0 and (c2, c1) for n < 0, written without
// selects: n cL = n P + |n| D, n cR = n P - |n| D (P = (c1 + c2)/2,
// D = (c1 - c2)/2), so the flux is n P (I_L + I_R) + |n| (D (I_L - I_R) - c3 (I_r - I_l));
// the record holds (P, D, -c3)
// the record is stored with each coefficient duplicated (P, P, D, D) and
// (-c3, -c3), so that the packed instructions take it without register moves
struct __align__(16) RecP { float P0, P1, D0, D1; };
__device__ __forceinline__ F2 phi2(F2 n, F2 an, const RecP &r, const float2 &c3, F2 IL, F2 IR, F2 Il, F2 Ir) {
    const F2 u = fma2(u2(c3), Ir - Il, F2{r.D0, r.D1} * (IL - IR));
    return fma2(n * F2{r.P0, r.P1}, IL + IR, an * u);
}

// Threads per CTA of the packed kernel for ND directions: one thread per
// direction pair, rounded up to whole warps.
template <int ND> struct Fp2Shape {
    static constexpr int NT = ((ND / 2 + 31) / 32) * 32;
    static constexpr int MINB = NT <= 32 ? 16 : (NT <= 64 ? 8 : 5);
};

// cell index along one periodic or outflow axis for any q (set-up only)
// (RT_BC_HALO: the caller's ghost planes, addressed by signed offsets from the
// owned origin)
__device__ __forceinline__ int wrap_po(int q, int n, int bclo, int bchi) {
    if (q < 0) return bclo == RT_BC_PERIODIC ? ((q % n) + n) % n : (bclo == RT_BC_HALO ? q : 0);
    if (q >= n) return bchi == RT_BC_PERIODIC ? q % n : (bchi == RT_BC_HALO ? q : n - 1);
    return q;
}

// SB: the stage's base intensities are its input (the predictor), fixed at
// compile time so that that instance carries no base-prefetch code.
// ND: the number of directions, fixed at compile time, so that the offsets of
// consecutive cells along x1 are immediates of the loads and stores.
// Row and x1 offsets are resolved once per CTA into shared memory; a thread
// adds them to its own direction-pair pointer.
template <typename TS, int ND, int BY, int BZ, bool WANTG, bool SB>
__global__ void __launch_bounds__(Fp2Shape<ND>::NT, Fp2Shape<ND>::MINB) k_stage_fp2(const StageArgs A) {
    constexpr int NT = Fp2Shape<ND>::NT;
    constexpr int TXC = NCELL / (BY * BZ), NOWN = BY * BZ, NW = NT / 32;
    constexpr int NRX = NOWN * (TXC + 1), NRY = BZ * (BY + 1) * TXC, NRZ = BY * (BZ + 1) * TXC;
    __shared__ RecP rec[NRX + NRY + NRZ];
    __shared__ float2 rc3[NRX + NRY + NRZ];
    // element offsets (x ND) of the own rows, the two halo rows on each side along
    // x2 (per own x3 row) and x3 (per own x2 row) at x1 = 0, and of the x1
    // positions i0 - 2 .. i0 + TXC + 1 with the x1 boundaries applied
    __shared__ int sRow[NOWN + 4 * BZ + 4 * BY], sX[TXC + 4], sXo[TXC];
    __shared__ float part[NW][NCELL];
    __shared__ float cEm[NCELL], cInv[NCELL];
    __shared__ int cOn[NCELL];
    __shared__ double cIn[6][NCELL];
    __shared__ __align__(8) float sIt[NCELL][2 * NT];
    // one x1 position ahead: the own rows' next values and, for the corrector,
    // the base intensities (both first reads from HBM), copied asynchronously
    constexpr bool PFX = sizeof(TS) == 4;
    // unrolling of the x1 loop; measured at 128^3 x 162: FP32 storage runs
    // 13% faster unrolled by 4 than fully and 5% faster again rolled (its
    // instruction-fetch stalls fall with the code size), BF16 storage 10%
    // slower unrolled by 4 than fully
    constexpr int XUNROLL = PFX ? 1 : TXC;
    __shared__ __align__(8) float pfb[2][2 * NOWN][PFX ? 2 * NT : 2];

    const int p = threadIdx.x, lane = p & 31, warp = p >> 5;
    const int d0 = 2 * p;
    const bool act = d0 < ND;   // n_dir is even: both directions of the pair exist
    const int nx0 = A.nx0, nx1 = A.nx1, nx2 = A.nx2;
    const int nseg = (nx0 + TXC - 1) / TXC;
    const int seg = blockIdx.x % nseg, rest = blockIdx.x / nseg, nyb = nx1 / BY;
    const int j0 = (rest % nyb) * BY, k0 = (rest / nyb) * BZ, i0 = seg * TXC;
    const int nc = min(TXC, nx0 - i0);
    // cell index of (0, j, k) and offset of (i, ...) along x1, boundaries applied
    auto crow = [&](int j, int k) -> int {
        return (wrap_po(k, nx2, A.bc[2][0], A.bc[2][1]) * nx1 + wrap_po(j, nx1, A.bc[1][0], A.bc[1][1])) * nx0;
    };
    auto cx = [&](int i) -> int { return wrap_po(i, nx0, A.bc[0][0], A.bc[0][1]); };

    const int lc_ii = lane % TXC, lc_o = lane / TXC;
    const size_t lc_cell = (size_t)crow(j0 + lc_o % BY, k0 + lc_o / BY) + i0 + lc_ii;
    const bool lc_valid = lc_ii < nc;
    if (warp == 0 && lc_valid) {
        const double *srcs[6] = {A.cc_Y, A.ug_in, A.alpha_int, A.cc_au, A.cc_as, A.eta};
#pragma unroll
        for (int q = 0; q < 6; ++q) cp_async8(&cIn[q][lane], srcs[q] + lc_cell);
    }
    cp_commit_all();

    // face records: the two cell opacities of every record are fetched with
    // cp.async first, so that their latency overlaps the row set-up and the
    // x1-window loads below; record t takes them from sAl[2t], sAl[2t + 1]
    // (staged in sIt, which the transport fills only later)
    double *sAl = reinterpret_cast<double *>(&sIt[0][0]);
    static_assert(2 * (NRX + NRY + NRZ) * sizeof(double) <= sizeof(float) * NCELL * 2 * NT, "staging fits in sIt");
    const int nX = A.transport && A.act0 ? NRX : 0, nY = A.transport && A.act1 ? NRY : 0;
    const int nZ = A.transport && A.act2 ? NRZ : 0;
    // cells and length of record t (positions beyond a ragged x1 tail use
    // clamped cells: computed but never stored)
    auto rec_cells = [&](int t, int &cl, int &cr, double &len, int &slot) {
        if (t < nX) {
            int o = t / (TXC + 1), f = t % (TXC + 1);
            int rb = crow(j0 + o % BY, k0 + o / BY);
            cl = rb + cx(min(i0 + f, nx0) - 1); cr = rb + cx(min(i0 + f, nx0)); len = A.dx0; slot = t;
        } else if (t < nX + nY) {
            int u = t - nX, ii = u % TXC, v = u / TXC, f = v % (BY + 1), r = v / (BY + 1);
            const int ic = min(i0 + ii, nx0 - 1);
            cl = crow(j0 + f - 1, k0 + r) + ic; cr = crow(j0 + f, k0 + r) + ic; len = A.dx1;
            slot = NRX + (r * (BY + 1) + f) * TXC + ii;
        } else {
            int u = t - nX - nY, ii = u % TXC, v = u / TXC, f = v % (BZ + 1), q = v / (BZ + 1);
            const int ic = min(i0 + ii, nx0 - 1);
            cl = crow(j0 + q, k0 + f - 1) + ic; cr = crow(j0 + q, k0 + f) + ic; len = A.dx2;
            slot = NRX + NRY + (q * (BZ + 1) + f) * TXC + ii;
        }
    };
    for (int t = p; t < nX + nY + nZ; t += NT) {
        int cl, cr, slot; double len;
        rec_cells(t, cl, cr, len, slot);
        cp_async8(&sAl[2 * t], A.alpha_in + cl);
        cp_async8(&sAl[2 * t + 1], A.alpha_in + cr);
    }
    cp_commit_all();
    auto hrow = [&](int h, int nb) -> int { return h < 2 ? h - 2 : nb + h - 2; };   // halo slot h = 0..3
    for (int t = p; t < NOWN + 4 * BZ + 4 * BY; t += NT) {
        int v = 0;
        if (t < NOWN) v = crow(j0 + t % BY, k0 + t / BY);
        else if (t < NOWN + 4 * BZ) { const int u = t - NOWN; if (A.act1) v = crow(j0 + hrow(u % 4, BY), k0 + u / 4); }
        else { const int u = t - NOWN - 4 * BZ; if (A.act2) v = crow(j0 + u / 4, k0 + hrow(u % 4, BZ)); }
        sRow[t] = v * ND;
    }
    for (int t = p; t < TXC + 4; t += NT) sX[t] = (A.act0 ? cx(i0 - 2 + t) : min(max(i0 - 2 + t, 0), nx0 - 1)) * ND;
    for (int t = p; t < TXC; t += NT) sXo[t] = min(i0 + t, nx0 - 1) * ND;
    __syncthreads();

    const TS *Ib = (const TS *)A.Isrc + d0;     // this thread's direction pair
    F2 nh[3] = {f2(0.0f), f2(0.0f), f2(0.0f)}, w = f2(0.0f);
    if (act) {
        for (int m = 0; m < 3; ++m) nh[m] = F2{((const float *)A.dirT)[3 * d0 + m], ((const float *)A.dirT)[3 * d0 + 3 + m]};
        w = ld2((const float *)A.wT + d0);
    }
    const F2 an[3] = {F2{fabsf(nh[0].x), fabsf(nh[0].y)}, F2{fabsf(nh[1].x), fabsf(nh[1].y)}, F2{fabsf(nh[2].x), fabsf(nh[2].y)}};
    const float dtk = (float)A.dtk;
    const F2 cdx[3] = {f2(dtk / (float)A.dx0), f2(dtk / (float)A.dx1), f2(dtk / (float)A.dx2)};
    auto ldI = [&](int off) -> F2 { return ld2(Ib + off); };
    auto putIt = [&](int c, F2 v) { *reinterpret_cast<float2 *>(&sIt[c][d0]) = make_float2(v.x, v.y); };
    auto getIt = [&](int c) -> F2 { float2 v = *reinterpret_cast<const float2 *>(&sIt[c][d0]); return F2{v.x, v.y}; };
    int own[NOWN];
#pragma unroll
    for (int o = 0; o < NOWN; ++o) own[o] = sRow[o];
    // the x1 window's first four values of every own row, in flight while the
    // face records are formed
    F2 Xw[NOWN][4];
#pragma unroll
    for (int o = 0; o < NOWN; ++o)
#pragma unroll
        for (int q = 0; q < 4; ++q) Xw[o][q] = (act && A.transport && A.act0) ? ldI(own[o] + sX[q]) : f2(0.0f);
    cp_wait_all();
    for (int t = p; t < nX + nY + nZ; t += NT) {
        int cl, cr, slot; double len;
        rec_cells(t, cl, cr, len, slot);
        double tau = A.abar * 0.5 * (sAl[2 * t] + sAl[2 * t + 1]) * (A.tau_dt ? A.dtk : len);
        float P = 0.5f, D = 0.5f, C = 0.0f;
        if (tau > 0.0) {
            float tt = (float)tau;
            float f = sqrtf(-expm1f(-tt * tt)) / tt, g = sqrtf(-expm1f(-tt * tt * tt * tt)) / tt, e = expf(-tt), fg = f + g;
            const float c1 = f * e / fg, c2 = g * e / fg;
            P = 0.5f * (c1 + c2); D = 0.5f * (c1 - c2); C = -(f * g / fg);
        }
        rec[slot] = RecP{P, P, D, D};
        rc3[slot] = make_float2(C, C);
    }
    __syncthreads();

    if (act) {
        constexpr bool same_base = SB;
        auto cp8 = [&](float *dst, const TS *src) {
            unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
        };
        auto pf_issue = [&](int ii) {
            if constexpr (PFX) {
                const int st = ii & 1, xo = sX[ii + 4], io = sXo[ii];
#pragma unroll
                for (int o = 0; o < NOWN; ++o) {
                    if (A.act0) cp8(&pfb[st][o][d0], Ib + (own[o] + xo));
                    if (!same_base) cp8(&pfb[st][NOWN + o][d0], (const TS *)A.Ibase + d0 + (own[o] + io));
                }
            }
        };
        auto pf_get = [&](int st, int k) -> F2 { return F2{pfb[st][k][d0], pfb[st][k][d0 + 1]}; };
        if (A.transport) {
            F2 W0[NOWN], W1[NOWN], S0[NOWN], Flo[NOWN];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                W0[o] = W1[o] = S0[o] = Flo[o] = f2(0.0f);
                if (A.act0) {
                    const F2 Im2 = Xw[o][0], Im1 = Xw[o][1], I0 = Xw[o][2], I1 = Xw[o][3];
                    F2 sm1 = mc_half2(I0 - Im1, Im1 - Im2), s0 = mc_half2(I1 - I0, I0 - Im1);
                    const int rs = o * (TXC + 1);
                    Flo[o] = phi2(nh[0], an[0], rec[rs], rc3[rs], Im1 + sm1, I0 - s0, Im1, I0);
                    W0[o] = I0; W1[o] = I1; S0[o] = s0;
                }
            }
            if (PFX) { pf_issue(0); cp_commit_all(); }
            // positions beyond a ragged x1 tail (ii >= nc) are computed from
            // clamped (in-bounds) neighbours and never stored: the loop needs no
            // per-position test
#pragma unroll XUNROLL
            for (int ii = 0; ii < TXC; ++ii) {
                {
                    const int io = sXo[ii];
                    const int pst = ii & 1;
                    if (PFX) {
                        if (ii + 1 < TXC) pf_issue(ii + 1);
                        cp_commit_all();
                        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                    }
                    F2 acc[NOWN], Ic[NOWN];
#pragma unroll
                    for (int o = 0; o < NOWN; ++o) {
                        acc[o] = f2(0.0f);
                        Ic[o] = A.act0 ? W0[o] : ldI(own[o] + io);
                    }
                    if (A.act0) {
                        const int x2 = sX[ii + 4];
#pragma unroll
                        for (int o = 0; o < NOWN; ++o) {
                            F2 I2 = PFX ? pf_get(pst, o) : ldI(own[o] + x2);
                            F2 s1 = mc_half2(I2 - W1[o], W1[o] - W0[o]);
                            const int rs = o * (TXC + 1) + ii + 1;
                            F2 phi = phi2(nh[0], an[0], rec[rs], rc3[rs], W0[o] + S0[o], W1[o] - s1, W0[o], W1[o]);
                            acc[o] = fma2(cdx[0], phi - Flo[o], acc[o]);
                            Flo[o] = phi; W0[o] = W1[o]; W1[o] = I2; S0[o] = s1;
                        }
                    }
                    if (A.act1) {
#pragma unroll
                        for (int r = 0; r < BZ; ++r) {
                            F2 Y[BY + 4], sy[BY + 4], F[BY + 1];
#pragma unroll
                            for (int q = 0; q < BY + 4; ++q) {
                                if (q >= 2 && q < BY + 2) Y[q] = Ic[r * BY + q - 2];
                                else Y[q] = ldI(sRow[NOWN + 4 * r + (q < 2 ? q : q - BY)] + io);
                            }
#pragma unroll
                            for (int q = 1; q < BY + 3; ++q) sy[q] = mc_half2(Y[q + 1] - Y[q], Y[q] - Y[q - 1]);
#pragma unroll
                            for (int f = 0; f <= BY; ++f)
                            {
                                const int rs = NRX + (r * (BY + 1) + f) * TXC + ii;
                                F[f] = phi2(nh[1], an[1], rec[rs], rc3[rs], Y[f + 1] + sy[f + 1],
                                            Y[f + 2] - sy[f + 2], Y[f + 1], Y[f + 2]);
                            }
#pragma unroll
                            for (int q = 0; q < BY; ++q) acc[r * BY + q] = fma2(cdx[1], F[q + 1] - F[q], acc[r * BY + q]);
                        }
                    }
                    if (A.act2) {
#pragma unroll
                        for (int q = 0; q < BY; ++q) {
                            F2 Z[BZ + 4], sz[BZ + 4], F[BZ + 1];
#pragma unroll
                            for (int r = 0; r < BZ + 4; ++r) {
                                if (r >= 2 && r < BZ + 2) Z[r] = Ic[(r - 2) * BY + q];
                                else Z[r] = ldI(sRow[NOWN + 4 * BZ + 4 * q + (r < 2 ? r : r - BZ)] + io);
                            }
#pragma unroll
                            for (int r = 1; r < BZ + 3; ++r) sz[r] = mc_half2(Z[r + 1] - Z[r], Z[r] - Z[r - 1]);
#pragma unroll
                            for (int f = 0; f <= BZ; ++f)
                            {
                                const int rs = NRX + NRY + (q * (BZ + 1) + f) * TXC + ii;
                                F[f] = phi2(nh[2], an[2], rec[rs], rc3[rs], Z[f + 1] + sz[f + 1],
                                            Z[f + 2] - sz[f + 2], Z[f + 1], Z[f + 2]);
                            }
#pragma unroll
                            for (int r = 0; r < BZ; ++r) acc[r * BY + q] = fma2(cdx[2], F[r + 1] - F[r], acc[r * BY + q]);
                        }
                    }
#pragma unroll
                    for (int o = 0; o < NOWN; ++o) {
                        F2 Ib0 = same_base ? Ic[o]
                                 : (PFX ? pf_get(pst, NOWN + o) : ld2((const TS *)A.Ibase + d0 + (own[o] + io)));
                        putIt(o * TXC + ii, Ib0 - acc[o]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int o = 0; o < NOWN; ++o)
#pragma unroll
                for (int ii = 0; ii < TXC; ++ii)
                    if (ii < nc) putIt(o * TXC + ii, ld2((const TS *)A.Ibase + d0 + (own[o] + (i0 + ii) * ND)));
        }
    }

    // ---- interaction (section 3.5.2), fluid at rest (as k_stage_fs, FP32 storage)
    if (warp == 0) {
        cp_wait_all();
        int on = 0;
        if (lc_valid) {
            double Y = cIn[0][lane], ug = cIn[1][lane], am = cIn[2][lane];
            on = A.source && A.cc_on[lc_cell] && am > 0.0 && Y > 0.0 && ug > 0.0;
        }
        cOn[lane] = on;
    }
    {
        float v[NCELL];
#pragma unroll
        for (int c = 0; c < NCELL; ++c) {
            F2 t = (act && c % TXC < nc) ? getIt(c) * w : f2(0.0f);
            v[c] = t.x + t.y;
        }
        part[warp][lane] = transpose_sum(v, lane);
    }
    __syncthreads();
    if (warp == 0 && lc_valid) {
        const size_t cidx = lc_cell;
        float ce = 0.0f, ci = 1.0f;
        const double ugm = cIn[1][lane];
        if (cOn[lane]) {
            float Emt = 0.0f;
            for (int g = 0; g < NW; ++g) Emt += part[g][lane];
            double Em = (double)Emt;
            const double dt = A.dtk, adt = cIn[2][lane] * dt;
            const double K = adt * rcp64(1.0 + adt);
            const double Y = cIn[0][lane], au = cIn[3][lane], as = cIn[4][lane];
            const double iY = rcp64(Y), Tm = ugm * iY;
            Teq<double> q{K * Em, K * A.sumw * dt * (1.0 / FOURPI), Em + ugm, Y, Tm, Em, au, as,
                          cIn[5][lane], A.arad, dt, A.T_exp, iY};
            double X;
            bool ok = solve_mixed(q, &X);
            const float Tp = (float)(Tm + (Em - X) * iY);
            const float aap = (float)au * tpow_neg<float>(Tp, (float)A.T_exp);
            const float af = (aap + (float)as) * (float)dt;
            const float cf = (float)dt * ((float)q.eta * aap * (float)A.arad * Tp * Tp * Tp * Tp + (float)as * (float)X) /
                             (float)FOURPI;
            const float invf = 1.0f / (1.0f + af);
            if (!ok) atomicAdd(A.fail, 1ull);
            if (A.sv_X) { A.sv_Em[cidx] = Em; A.sv_X[cidx] = X; }
            ce = cf; ci = invf;
            const double c = cf, inv = invf;
            const double Ep = (Em + c * A.sumw) * inv;
            const double ugp = ugm - (Ep - Em);
            A.ug_out[cidx] = ugp;
            const double T = ugp * iY;
            A.alpha_out[cidx] = T > 0.0 ? (double)((float)au * tpow_neg<float>((float)T, (float)A.T_exp) + (float)as) : 0.0;
            // the force on the gas (section 3.5.3) follows from (a, c) and the
            // moments of the stored I_+ = (I + c) / (1 + a) when it is asked for
            // (rt_moments): Delta R^{0 mu} = c sum n^mu dOmega - a sum n^mu I_+ dOmega
            if (WANTG) A.gac[cidx] = make_float2(af, cf);
        } else {
            A.ug_out[cidx] = ugm;
            A.alpha_out[cidx] = cIn[2][lane];
            if (WANTG) A.gac[cidx] = make_float2(0.0f, 0.0f);
        }
        cEm[lane] = ce; cInv[lane] = ci;
    }
    __syncthreads();
    if (act) {
        TS *Ob = (TS *)A.Iout + d0;
#pragma unroll
        for (int o = 0; o < NOWN; ++o) {
#pragma unroll
            for (int ii = 0; ii < TXC; ++ii) {
                if (ii < nc) {
                    const int lc = o * TXC + ii;
                    F2 v = getIt(lc);
                    if (cOn[lc]) v = (v + f2(cEm[lc])) * f2(cInv[lc]);
                    st2(Ob + (own[o] + (i0 + ii) * ND), v);
                }
            }
        }
    }
}

template <typename TS, typename TM, int BY, int BZ>
rt_status launch_fs(rt_ctx *c, const StageArgs &A0, int NT) {
    const StageArgs &A = A0;
    constexpr int TXC = NCELL / (BY * BZ);
    size_t nblk = (size_t)((A.nx0 + TXC - 1) / TXC) * (A.nx1 / BY) * (A.nx2 / BZ);
    bool simple = true;
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd)
            simple = simple && (A.bc[a][sd] == RT_BC_PERIODIC || A.bc[a][sd] == RT_BC_OUTFLOW || A.bc[a][sd] == RT_BC_HALO);
    if constexpr (sizeof(TM) == 4) {
        if (simple && A.nd == 162) {
            constexpr int ND = 162, PNT = Fp2Shape<ND>::NT;
            StageArgs A = A0;
            if (A.kb) {     // signed offsets from the owned origin (see StageArgs::kb)
                A.Isrc = (const char *)A.Isrc + c->hcells * c->nd * c->esize;
                A.alpha_in += c->hcells;
                A.vel += 3 * c->hcells;
                A.kb = 0;
            }
            const bool sb = A.Isrc == A.Ibase;
            auto kern = A.G ? (sb ? k_stage_fp2<TS, ND, BY, BZ, true, true> : k_stage_fp2<TS, ND, BY, BZ, true, false>)
                            : (sb ? k_stage_fp2<TS, ND, BY, BZ, false, true> : k_stage_fp2<TS, ND, BY, BZ, false, false>);
            kern<<<(unsigned)nblk, PNT, 0, c->stream>>>(A);
            RT_CUDA_TRY(c, cudaGetLastError());
            if (A.G) { c->g_lazy = true; c->g_dt = A.dtk; }
            return RT_OK;
        }
    }
    if (simple) {
        if (A.G) k_stage_fs<TS, TM, BY, BZ, true, true><<<(unsigned)nblk, NT, 0, c->stream>>>(A);
        else k_stage_fs<TS, TM, BY, BZ, false, true><<<(unsigned)nblk, NT, 0, c->stream>>>(A);
    } else {
        if (A.G) k_stage_fs<TS, TM, BY, BZ, true, false><<<(unsigned)nblk, NT, 0, c->stream>>>(A);
        else k_stage_fs<TS, TM, BY, BZ, false, false><<<(unsigned)nblk, NT, 0, c->stream>>>(A);
    }
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

template <typename TS, typename TM>
rt_status launch_fs_blk(rt_ctx *c, const StageArgs &A, int NT) {
    bool by = A.act1 && A.nx1 % 2 == 0, bz = A.act2 && A.nx2 % 2 == 0;
    if (by && bz) return launch_fs<TS, TM, 2, 2>(c, A, NT);
    if (by) return launch_fs<TS, TM, 2, 1>(c, A, NT);
    return launch_fs<TS, TM, 1, 1>(c, A, NT);
}

}  // namespace

bool rt_stage_fast_ok(const rt_ctx *c) {
    return c->metric == RT_MINKOWSKI_CART && c->static_fluid && c->cfg.limiter == RT_LIM_MC && rt_coupling3(c) &&
           c->cfg.n_pole_zero == 0 && c->nd <= FS_NT && (double)(c->ncell + 2 * c->hcells) * c->nd < 2147483647.0;
}

rt_status rt_launch_stage_fs(rt_ctx *c, const StageArgs &A, int NT) {
    if (c->cfg.precision == RT_FP64) return launch_fs_blk<double, double>(c, A, NT);
    if (c->cfg.precision == RT_FP32) return launch_fs_blk<float, float>(c, A, NT);
    return launch_fs_blk<__nv_bfloat16, float>(c, A, NT);
}
