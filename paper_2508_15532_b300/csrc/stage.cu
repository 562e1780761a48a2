// stage.cu — one fused stage of the radiation step on sm_103a.
//
// A stage (section 3.6) is the explicit transport of the conserved n^0 n_0 I
// over dtk with fluxes from I_src (eq. radiative_transfer_discrete: spatial
// flux eqs. spatial_fluxes_vacuum / rad_speeds / flux_Jiang on a piecewise-
// linear reconstruction, angular flux eq. angular_fluxes on a minimum-angle
// plane reconstruction), followed in the same kernel by the implicit
// radiation-gas interaction of section 3.5.2 on every cell of the tile.
//
// Work decomposition (HBM-bound design):
//  - one CTA owns a brick of 32 cells: TXC consecutive cells along x1 times
//    BY x BZ rows (x2, x3), with all directions; thread s owns direction s, so
//    every warp-wide load or store touches 32 consecutive directions of one
//    cell (coalesced, cell-major layout);
//  - each thread marches along x1 with a sliding register window (one new
//    value, one slope and one face flux per cell); the x2/x3 stencils of the
//    BY x BZ rows are register columns, so every slope and face flux of the
//    brick is evaluated once; boundary conditions are resolved per CTA into
//    row/column descriptors in shared memory (no ghost arrays);
//  - the direction-independent face coefficients (optical-depth cut-offs,
//    signal-speed factors, fluid advection) are computed once per face;
//  - the transported brick stays in shared memory for the interaction: each
//    stage reads I_src (neighbours mostly from L2), I_base, and writes I_out
//    exactly once;
//  - interaction: per-cell angular sums in direction chunks (lane = cell, no
//    shuffles), one warp (lane = cell) solves the 32 temperature equations —
//    FP32 Newton iterations finished by an FP64 Newton step in the mixed
//    path, FP64 throughout in the FP64 path — then the per-direction update
//    and the FP64 energy ledger.
#include "stage_common.cuh"

namespace {
using namespace rtk;

// LK: the limiter kind fixed at compile time (RT_LIM_MC), or -1 to read it
// from the arguments.  NC: cells per CTA (32; 16 or 8 where the directions'
// shared-memory rows of 32 cells would not fit).  MAXT: the launch bound, 256
// threads (up to 256 directions, one per thread), 192 (curved geometry: up
// to 192 directions) or 1024 (finer grids, at most 64 registers per thread).
// MINB: CTAs per SM the registers must allow
template <typename TS, typename TM, bool FLAT, int BY, int BZ, int LK, int NC, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_stage(const StageArgs A) {
    constexpr int TXC = NC / (BY * BZ);
    constexpr int NOWN = BY * BZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nd = A.nd, ndp = nd + 1;
    const int NT = blockDim.x;
    const int s = threadIdx.x;
    const bool act = s < nd;
    const int nseg = (A.nx0 + TXC - 1) / TXC;
    const int seg = blockIdx.x % nseg;
    const int rest = blockIdx.x / nseg;
    const int nyb = A.nx1 / BY;
    const int j0 = (rest % nyb) * BY, k0 = (rest / nyb) * BZ;
    const int i0 = seg * TXC;
    const int nc = min(TXC, A.nx0 - i0);

    // ---- shared layout
    TM *It = (TM *)smem_raw;                                  // [NC][ndp]
    // It holds the transported intensities I*, then (after the update) the
    // interaction's change I_+ - I* of every element, which is all the
    // exchange ledger needs
    TM *recX = It + NC * ndp;                                 // [NOWN][TXC+1][5]
    TM *recY = recX + NOWN * (TXC + 1) * 5;                   // [BZ][BY+1][TXC][5]
    TM *recZ = recY + BZ * (BY + 1) * TXC * 5;                // [BY][BZ+1][TXC][5]
    TM *scU = recZ + BY * (BZ + 1) * TXC * 5;                 // [NC][4] tetrad-frame fluid velocity
    TM *scN0 = scU + 4 * NC, *scK = scN0 + NC, *scEm = scK + NC, *scA = scEm + NC;
    TM *Icell = scA + NC;                                     // [NOWN][nd]   (curved only)
    TM *Arec = Icell + (FLAT ? 0 : NOWN * nd);                // [NOWN][6][nd] (curved only; slot-major: own slots conflict-free)
    // the interaction's chunk sums, used only after the transport, share the
    // angular rows' space (less shared memory leaves more L1 to the tables)
    double *part = (double *)(((uintptr_t)Icell + 15) & ~(uintptr_t)15);   // [NT / NC][NC][6]
    const uintptr_t end_ang = (uintptr_t)(Arec + (FLAT ? 0 : 6 * NOWN * nd)), end_part = (uintptr_t)(part + NT * 6);
    int *xmap = (int *)(end_ang > end_part ? end_ang : end_part);   // [TXC+4]
    int *rowY = xmap + TXC + 4;                               // [BZ][BY+4]
    int *rowZ = rowY + BZ * (BY + 4);                         // [BY][BZ+4]
    int *scOn = rowZ + BY * (BZ + 4);                         // [NC]

    // ---- boundary descriptors
    for (int t = s; t < TXC + 4; t += NT) {
        int fl = 0;
        int im = map_axis(A, 0, i0 - 2 + t, &fl, nullptr);
        xmap[t] = im | fl;
    }
    for (int t = s; t < BZ * (BY + 4); t += NT) {
        int r = t / (BY + 4), q = t % (BY + 4);
        rowY[t] = row_desc(A, j0 - 2 + q, k0 + r);
    }
    for (int t = s; t < BY * (BZ + 4); t += NT) {
        int q = t / (BZ + 4), r = t % (BZ + 4);
        rowZ[t] = row_desc(A, j0 + q, k0 - 2 + r);
    }
    __syncthreads();

    // ---- face coefficients (direction independent)
    auto coeffs = [&](int ax, int cl, int cr, double len, TM *rec) {
        double al = A.alpha_in[cl], ar = A.alpha_in[cr];
        double tau = A.abar * 0.5 * (al + ar) * (A.tau_dt ? A.dtk : len);
        if (tau > 0.0) {
            TM t = (TM)tau;
            TM f = sqrt(-expm1(-t * t)) / t;
            TM g = sqrt(-expm1(-t * t * t * t)) / t;
            TM e = exp(-t), fg = f + g;
            TM cadv = -expm1(-t);
            rec[0] = f * e / fg; rec[1] = g * e / fg; rec[2] = f * g / fg;
            rec[3] = cadv * (TM)fmax(A.vel[3 * (size_t)cl + ax], 0.0);
            rec[4] = cadv * (TM)fmin(A.vel[3 * (size_t)cr + ax], 0.0);
        } else {
            rec[0] = TM(1); rec[1] = TM(0); rec[2] = TM(0); rec[3] = TM(0); rec[4] = TM(0);
        }
    };
    auto plen = [&](int ax, int i, int j) -> double {
        if (FLAT) return ax == 0 ? A.dx0 : (ax == 1 ? A.dx1 : A.dx2);
        int npt = A.gn0 * (A.nx1 + 2 * A.ng1);
        return A.pt_len[(size_t)ax * npt + (j + A.ng1) * A.gn0 + (i + A.ng0)];
    };
    if (A.transport) {
        const int nX = A.act0 ? NOWN * (nc + 1) : 0, nY = A.act1 ? BZ * (BY + 1) * nc : 0;
        const int nZ = A.act2 ? BY * (BZ + 1) * nc : 0;
        for (int t = s; t < nX + nY + nZ; t += NT) {
            if (t < nX) {
                int o = t / (nc + 1), f = t % (nc + 1);
                int q = o % BY, r = o / BY;
                int rb = rowY[r * (BY + 4) + q + 2] & F_MASK;
                coeffs(0, rb + (xmap[f + 1] & F_MASK), rb + (xmap[f + 2] & F_MASK), plen(0, i0 + f, j0 + q),
                       recX + (o * (TXC + 1) + f) * 5);
            } else if (t < nX + nY) {
                int u = t - nX, ii = u % nc, v = u / nc, f = v % (BY + 1), r = v / (BY + 1);
                int rl = rowY[r * (BY + 4) + f + 1] & F_MASK, rr = rowY[r * (BY + 4) + f + 2] & F_MASK;
                coeffs(1, rl + i0 + ii, rr + i0 + ii, plen(1, i0 + ii, j0 + f), recY + ((r * (BY + 1) + f) * TXC + ii) * 5);
            } else {
                int u = t - nX - nY, ii = u % nc, v = u / nc, f = v % (BZ + 1), q = v / (BZ + 1);
                int rl = rowZ[q * (BZ + 4) + f + 1] & F_MASK, rr = rowZ[q * (BZ + 4) + f + 2] & F_MASK;
                coeffs(2, rl + i0 + ii, rr + i0 + ii, plen(2, i0 + ii, j0 + q), recZ + ((q * (BZ + 1) + f) * TXC + ii) * 5);
            }
        }
    }
    __syncthreads();

    // ---- transport
    const int npt = FLAT ? 1 : A.gn0 * (A.nx1 + 2 * A.ng1);
    const size_t pd = (size_t)npt * nd;
    const int smir = act ? __ldg(A.mirror + s) : 0;
    TM nh[3] = {TM(0), TM(0), TM(0)};
    if (act) for (int m = 0; m < 3; ++m) nh[m] = ldT<TM>(A.dirT, 3 * s + m);
    const TM dtk = (TM)A.dtk;
    const TM cdx[3] = {dtk / (TM)A.dx0, dtk / (TM)A.dx1, dtk / (TM)A.dx2};
    const bool same_base = A.Isrc == A.Ibase;

    auto ld_row = [&](int desc, int i) -> TM {      // direction s in row desc at interior x1 index i
        if (desc & F_FIX) return TM(0);
        int d = (desc & F_MIR) ? smir : s;
        return IO<TS, TM>::ld(A.Isrc, (size_t)((desc & F_MASK) + i) * nd + d);
    };
    auto ld_x = [&](int rowbase, int xd, int jrow) -> TM {   // own row, x1 index from the descriptor
        if (xd & F_FIX) return (s == A.beam_dir && jrow >= A.beam_lo && jrow < A.beam_hi) ? TM(A.beam_I) : TM(0);
        int d = (xd & F_MIR) ? smir : s;
        return IO<TS, TM>::ld(A.Isrc, (size_t)(rowbase + (xd & F_MASK)) * nd + d);
    };
    // curved-geometry face: flux = P phi with n^a and dA n_0 from the tables;
    // no flux across a sign change of n_0 between the two cells (mask bit 1)
    auto geo_face = [&](int ax, int pt_face, int pt_l, int pt_r, TM &n, TM &P) {
        uint8_t ml = A.mask[(size_t)pt_l * nd + s], mr = A.mask[(size_t)pt_r * nd + s];
        size_t o = (size_t)ax * pd + (size_t)pt_face * nd + s;
        n = ldT<TM>(A.fn, o);
        P = ((ml ^ mr) & 2) ? TM(0) : ldT<TM>(A.fP, o);
    };

    if (A.transport) {
        // x1 sliding window per own row: value at i, i+1, slope at i, flux at i - 1/2
        TM W0[NOWN], W1[NOWN], S0[NOWN], Flo[NOWN];
#pragma unroll
        for (int o = 0; o < NOWN; ++o) { W0[o] = W1[o] = S0[o] = Flo[o] = TM(0); }
        if (act && A.act0) {
#pragma unroll
            for (int o = 0; o < NOWN; ++o) {
                const int q = o % BY, r = o / BY, jr = j0 + q;
                const int rb = rowY[r * (BY + 4) + q + 2] & F_MASK;
                TM Im2 = ld_x(rb, xmap[0], jr), Im1 = ld_x(rb, xmap[1], jr);
                TM I0 = ld_x(rb, xmap[2], jr), I1 = ld_x(rb, xmap[3], jr);
                TM sm1 = limiter<TM>(LK >= 0 ? LK : A.limiter, I0 - Im1, Im1 - Im2);
                TM s0 = limiter<TM>(LK >= 0 ? LK : A.limiter, I1 - I0, I0 - Im1);
                const TM *rc = recX + (o * (TXC + 1)) * 5;
                TM IL = fma(TM(0.5), sm1, Im1), IR = fma(TM(-0.5), s0, I0);
                TM phi;
                if (FLAT) phi = face_phi<TM>(nh[0], rc, IL, IR, Im1, I0);
                else {
                    TM n, P;
                    int p0 = (jr + A.ng1) * A.gn0 + (i0 + A.ng0);
                    geo_face(0, p0, p0 - 1, p0, n, P);
                    phi = P * face_phi<TM>(n, rc, IL, IR, Im1, I0);
                }
                W0[o] = I0; W1[o] = I1; S0[o] = s0; Flo[o] = phi;
            }
        }
        // ring of direction s: neighbours, edges, back slots, which side of
        // each edge s is, the MAPR Gram inverses, 1/dOmega (curved geometry)
        int rg_kk = 0, rg_nb[RT_MAXNB], rg_e[RT_MAXNB], rg_bk[RT_MAXNB];
        unsigned rg_own = 0u;
        TM rg_g[3 * RT_MAXNB], rg_winv = TM(0);
#pragma unroll
        for (int q = 0; q < RT_MAXNB; ++q) { rg_nb[q] = s; rg_e[q] = 0; rg_bk[q] = 0; }
#pragma unroll
        for (int q = 0; q < 3 * RT_MAXNB; ++q) rg_g[q] = TM(0);
        if (!FLAT && act) {
            rg_kk = __ldg(A.nnb + s);
            rg_winv = TM(1) / ldT<TM>(A.wT, s);
#pragma unroll
            for (int q = 0; q < RT_MAXNB; ++q) {
                if (q < rg_kk) {
                    rg_nb[q] = __ldg(A.nbr + 6 * s + q);
                    rg_e[q] = __ldg(A.ring_edge + 6 * s + q);
                    rg_bk[q] = __ldg(A.ring_back + 6 * s + q);
                    rg_own |= (unsigned)(__ldg(A.edge + 2 * rg_e[q]) == s) << q;
#pragma unroll
                    for (int m = 0; m < 3; ++m) rg_g[3 * q + m] = ldT<TM>(A.mgT, (size_t)(6 * s + q) * 3 + m);
                }
            }
            if (rg_kk == 5) {
                // a pentagon's ring is padded to six: neighbour 5 repeats
                // neighbour 0 (so plane 4 pairs neighbours 4 and 0 like the
                // others pair q and q + 1), and plane 5, which would pair 0 with
                // itself, gets a NaN Gram inverse: its norm is NaN, never below
                // the threshold, and drops out of the minimum (fmin ignores NaN)
                rg_nb[5] = rg_nb[0];
#pragma unroll
                for (int m = 0; m < 3; ++m) rg_g[15 + m] = qnan<TM>();
            }
        }
        for (int ii = 0; ii < nc; ++ii) {
            const int i = i0 + ii;
            TM acc[NOWN], Ic[NOWN];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) { acc[o] = TM(0); Ic[o] = TM(0); }
            if (act) {
#pragma unroll
                for (int o = 0; o < NOWN; ++o) {
                    const int q = o % BY, r = o / BY;
                    Ic[o] = A.act0 ? W0[o] : ld_row(rowY[r * (BY + 4) + q + 2], i);
                }
                if (A.act0) {
#pragma unroll
                    for (int o = 0; o < NOWN; ++o) {
                        const int q = o % BY, r = o / BY, jr = j0 + q;
                        const int rb = rowY[r * (BY + 4) + q + 2] & F_MASK;
                        TM I2 = ld_x(rb, xmap[ii + 4], jr);
                        TM s1 = limiter<TM>(LK >= 0 ? LK : A.limiter, I2 - W1[o], W1[o] - W0[o]);
                        const TM *rc = recX + (o * (TXC + 1) + ii + 1) * 5;
                        TM IL = fma(TM(0.5), S0[o], W0[o]), IR = fma(TM(-0.5), s1, W1[o]);
                        TM phi;
                        if (FLAT) phi = face_phi<TM>(nh[0], rc, IL, IR, W0[o], W1[o]);
                        else {
                            TM n, P;
                            int p1 = (jr + A.ng1) * A.gn0 + (i + 1 + A.ng0);
                            geo_face(0, p1, p1 - 1, p1, n, P);
                            phi = P * face_phi<TM>(n, rc, IL, IR, W0[o], W1[o]);
                        }
                        acc[o] = FLAT ? fma(cdx[0], phi - Flo[o], acc[o]) : acc[o] + (phi - Flo[o]);
                        Flo[o] = phi; W0[o] = W1[o]; W1[o] = I2; S0[o] = s1;
                    }
                }
                if (A.act1) {
#pragma unroll
                    for (int r = 0; r < BZ; ++r) {
                        TM Y[BY + 4], sy[BY + 4], F[BY + 1];
#pragma unroll
                        for (int q = 0; q < BY + 4; ++q)
                            Y[q] = (q >= 2 && q < BY + 2) ? Ic[r * BY + q - 2] : ld_row(rowY[r * (BY + 4) + q], i);
                        sy[0] = sy[BY + 3] = TM(0);
#pragma unroll
                        for (int q = 1; q < BY + 3; ++q) sy[q] = limiter<TM>(LK >= 0 ? LK : A.limiter, Y[q + 1] - Y[q], Y[q] - Y[q - 1]);
#pragma unroll
                        for (int f = 0; f <= BY; ++f) {
                            const TM *rc = recY + ((r * (BY + 1) + f) * TXC + ii) * 5;
                            TM IL = fma(TM(0.5), sy[f + 1], Y[f + 1]), IR = fma(TM(-0.5), sy[f + 2], Y[f + 2]);
                            if (FLAT) F[f] = face_phi<TM>(nh[1], rc, IL, IR, Y[f + 1], Y[f + 2]);
                            else {
                                TM n, P;
                                int pu = (j0 + f + A.ng1) * A.gn0 + (i + A.ng0);
                                geo_face(1, pu, pu - A.gn0, pu, n, P);
                                F[f] = P * face_phi<TM>(n, rc, IL, IR, Y[f + 1], Y[f + 2]);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < BY; ++q) acc[r * BY + q] = FLAT ? fma(cdx[1], F[q + 1] - F[q], acc[r * BY + q]) : acc[r * BY + q] + (F[q + 1] - F[q]);
                    }
                }
                if (A.act2) {
#pragma unroll
                    for (int q = 0; q < BY; ++q) {
                        TM Z[BZ + 4], sz[BZ + 4], F[BZ + 1];
#pragma unroll
                        for (int r = 0; r < BZ + 4; ++r)
                            Z[r] = (r >= 2 && r < BZ + 2) ? Ic[(r - 2) * BY + q] : ld_row(rowZ[q * (BZ + 4) + r], i);
                        sz[0] = sz[BZ + 3] = TM(0);
#pragma unroll
                        for (int r = 1; r < BZ + 3; ++r) sz[r] = limiter<TM>(LK >= 0 ? LK : A.limiter, Z[r + 1] - Z[r], Z[r] - Z[r - 1]);
#pragma unroll
                        for (int f = 0; f <= BZ; ++f) {
                            const TM *rc = recZ + ((q * (BZ + 1) + f) * TXC + ii) * 5;
                            TM IL = fma(TM(0.5), sz[f + 1], Z[f + 1]), IR = fma(TM(-0.5), sz[f + 2], Z[f + 2]);
                            if (FLAT) F[f] = face_phi<TM>(nh[2], rc, IL, IR, Z[f + 1], Z[f + 2]);
                            else {
                                TM n, P;
                                int pc = (j0 + q + A.ng1) * A.gn0 + (i + A.ng0);
                                geo_face(2, pc, pc, pc, n, P);
                                F[f] = P * face_phi<TM>(n, rc, IL, IR, Z[f + 1], Z[f + 2]);
                            }
                        }
#pragma unroll
                        for (int r = 0; r < BZ; ++r) acc[r * BY + q] = FLAT ? fma(cdx[2], F[r + 1] - F[r], acc[r * BY + q]) : acc[r * BY + q] + (F[r + 1] - F[r]);
                    }
                }
            }
            // angular flux (curved geometry): minimum-angle plane reconstruction
            // of every direction at the edge midpoints, edge fluxes with the
            // upwind side of n_0(m) v(m).u_e (eq. angular_fluxes); ring data of
            // direction s in registers (rg_*), loops over the ring unrolled
            TM ang[NOWN];
#pragma unroll
            for (int o = 0; o < NOWN; ++o) ang[o] = TM(0);
            if (!FLAT) {
                if (act)
                    for (int o = 0; o < NOWN; ++o) Icell[o * nd + s] = Ic[o];
                __syncthreads();
                // the own-row loops of the angular part stay rolled: unrolled they
                // quadruple the code of the x1 loop and stall on instruction fetch
                // (measured 8% slower at 256 x 128 x 128; 168 against 128 registers)
                if (act) {
#pragma unroll 1
                    for (int o = 0; o < NOWN; ++o) {
                        TM rec[RT_MAXNB];
                        const TM Io0 = Icell[o * nd + s];
                        if (A.ang_recon == 1) {
#pragma unroll
                            for (int q = 0; q < RT_MAXNB; ++q) rec[q] = Io0;
                        } else {
                            TM dI[RT_MAXNB], al[RT_MAXNB], be[RT_MAXNB], nr[RT_MAXNB];
#pragma unroll
                            for (int q = 0; q < RT_MAXNB; ++q) dI[q] = Icell[o * nd + rg_nb[q]] - Io0;
#pragma unroll
                            for (int q = 0; q < RT_MAXNB; ++q) {
                                const TM d1 = dI[q + 1 < RT_MAXNB ? q + 1 : 0];
                                al[q] = fma(rg_g[3 * q], dI[q], rg_g[3 * q + 1] * d1);
                                be[q] = fma(rg_g[3 * q + 1], dI[q], rg_g[3 * q + 2] * d1);
                                nr[q] = fma(al[q], dI[q], be[q] * d1);
                            }
                            TM mn = nr[0];
#pragma unroll
                            for (int q = 1; q < RT_MAXNB; ++q) mn = fmin(mn, nr[q]);
                            // near-equal norms tie (mirror-symmetric neighbourhoods); first in ring order wins
                            const TM thr = mn + TM(1e-6) * fabs(mn);
                            int best = 0;
                            TM ab = TM(0), bb = TM(0);
#pragma unroll
                            for (int q = RT_MAXNB - 1; q >= 0; --q)
                                if (nr[q] <= thr) { best = q; ab = al[q]; bb = be[q]; }
                            // precomputed dot products of the plane's dual basis with the
                            // edge midpoints (plane-major, direction-fastest: coalesced;
                            // measured 82.6 -> 76.2 ms per 256 x 128 x 128 torus step)
                            const size_t od = (size_t)(6 * best) * nd + s;
#pragma unroll
                            for (int q = 0; q < RT_MAXNB; ++q) {
                                TM m0, m1;
                                ldT2(A.mdT, od + (size_t)q * nd, m0, m1);
                                rec[q] = fma(bb, m1, fma(ab, m0, Io0));
                            }
                        }
#pragma unroll
                        for (int q = 0; q < RT_MAXNB; ++q) Arec[(o * 6 + q) * nd + s] = rec[q];
                    }
                }
                __syncthreads();
                if (act) {
                    // eq. angular_fluxes: the flux through edge q is w_q times the
                    // upwind reconstruction, the side given by the sign of v.u_e
                    // (w = dlam n_0 v.u_e, eneg: u_e reversed).  With BY = 1 every
                    // own row lies on the same (x1, x2) point, whose edge weights
                    // and upwind sides are loaded once for all rows
                    TM ewq[RT_MAXNB];
                    unsigned upq = 0u;
#pragma unroll
                    for (int q = 0; q < RT_MAXNB; ++q) ewq[q] = TM(0);
                    if constexpr (BY == 1) {
                        // folded per ring slot: the signed weight (+w on the edge's
                        // own side) and whether the upwind value is s's own; a
                        // pentagon's padding slot keeps weight 0
                        const size_t pe0 = (size_t)((j0 + A.ng1) * A.gn0 + (i + A.ng0)) * A.ne;
#pragma unroll
                        for (int q = 0; q < RT_MAXNB; ++q)
                            if (q < rg_kk) {
                                const TM w = ldT<TM>(A.ew, pe0 + rg_e[q]);
                                const bool own = (rg_own >> q) & 1u;
                                const bool up = (w > TM(0)) != (__ldg(A.eneg + pe0 + rg_e[q]) != 0);
                                ewq[q] = own ? w : -w;
                                upq |= (unsigned)(own == up) << q;
                            }
                    }
#pragma unroll 1
                    for (int o = 0; o < NOWN; ++o) {
                        const int pc = (j0 + o % BY + A.ng1) * A.gn0 + (i + A.ng0);
                        TM a = TM(0);
#pragma unroll
                        for (int q = 0; q < RT_MAXNB; ++q) {
                            // with BY = 1 a pentagon's padding slot has weight 0 and
                            // reads valid slots (neighbour 0's slot 0)
                            if (BY == 1 || q < rg_kk) {
                                const TM Io = Arec[(o * 6 + q) * nd + s], It2 = Arec[(o * 6 + rg_bk[q]) * nd + rg_nb[q]];
                                if constexpr (BY == 1) {
                                    a = fma(ewq[q], ((upq >> q) & 1u) ? Io : It2, a);
                                } else {
                                    const bool own = (rg_own >> q) & 1u;
                                    const size_t pe = (size_t)pc * A.ne + rg_e[q];
                                    const TM w = ldT<TM>(A.ew, pe);
                                    const bool up = (w > TM(0)) != (__ldg(A.eneg + pe) != 0);
                                    TM IL = own ? Io : It2, IR = own ? It2 : Io;
                                    a = fma(own ? w : -w, up ? IL : IR, a);
                                }
                            }
                        }
#pragma unroll
                        for (int u = 0; u < NOWN; ++u)
                            if (u == o) ang[u] = a * rg_winv;
                    }
                }
                __syncthreads();
            }
            if (act) {
#pragma unroll
                for (int o = 0; o < NOWN; ++o) {
                    const int q = o % BY, r = o / BY, j = j0 + q, k = k0 + r;
                    const size_t cidx = ((size_t)k * A.nx1 + j) * A.nx0 + i;
                    TM Ib = same_base ? Ic[o] : IO<TS, TM>::ld(A.Ibase, cidx * nd + s);
                    TM out;
                    bool zero = A.n_pole_zero > 0 && (j < A.n_pole_zero || j >= A.nx1 - A.n_pole_zero);
                    if (FLAT) out = Ib - acc[o];
                    else {
                        const int pc = (j + A.ng1) * A.gn0 + (i + A.ng0);
                        // (U Ib - dt (acc / V + ang)) / U with the reciprocals of the
                        // point's U = n^0 n_0 and volume V, which the own rows on one
                        // (x1, x2) point share (evaluated once per point)
                        const TM iU = TM(1) / ldT<TM>(A.cenU, (size_t)pc * nd + s);
                        const TM iV = TM(1) / (TM)A.pt_V[pc];
                        out = Ib - dtk * fma(acc[o], iV, ang[o]) * iU;
                        zero = zero || (A.mask[(size_t)pc * nd + s] & 1);
                    }
                    It[((r * BY + q) * TXC + ii) * ndp + s] = zero ? TM(0) : out;
                }
            }
        }
    } else if (act) {
        for (int o = 0; o < NOWN; ++o)
            for (int ii = 0; ii < nc; ++ii) {
                const int q = o % BY, r = o / BY;
                const size_t cidx = ((size_t)(k0 + r) * A.nx1 + j0 + q) * A.nx0 + i0 + ii;
                It[(o * TXC + ii) * ndp + s] = IO<TS, TM>::ld(A.Ibase, cidx * nd + s);
            }
    }

    // ---- interaction (section 3.5.2); local cell lc = (r BY + q) TXC + ii
    auto gcell = [&](int lc, int &ii, int &j) -> size_t {
        ii = lc % TXC;
        int o = lc / TXC;
        j = j0 + o % BY;
        int k = k0 + o / BY;
        return ((size_t)k * A.nx1 + j) * A.nx0 + i0 + ii;
    };
    int all_static = 1;
    if (s < NC) {
        int ii, j;
        size_t cidx = gcell(s, ii, j);
        int on = 0;
        if (ii < nc) {
            double Y = A.cc_Y[cidx], ug = A.ug_in[cidx], am = A.alpha_int[cidx];
            double Tm = Y > 0.0 ? ug / Y : 0.0;
            on = A.source && A.cc_on[cidx] && am > 0.0 && Tm > 0.0;
            const int pc = FLAT ? 0 : (j + A.ng1) * A.gn0 + (i0 + ii + A.ng0);
            double n0 = FLAT ? 1.0 : A.pt_n0[pc];
            // u-hat^0 is kept as u-hat^0 - 1 (exact in FP64 for u^0 in [1, 2]):
            // D = 1 + ((u^0 - 1) - u.n) then carries no FP32 rounding of u^0,
            // which would shift every direction's D the same way
            scU[4 * s] = (TM)(A.uhat[4 * cidx] - 1.0);
            for (int m = 1; m < 4; ++m) scU[4 * s + m] = (TM)A.uhat[4 * cidx + m];
            scN0[s] = (TM)n0;
            scK[s] = (TM)(am * A.dtk);
            if (on && !(A.uhat[4 * cidx + 1] == 0.0 && A.uhat[4 * cidx + 2] == 0.0 && A.uhat[4 * cidx + 3] == 0.0 &&
                        A.uhat[4 * cidx] == 1.0 && n0 == 1.0))
                all_static = 0;
        }
        scOn[s] = on;
    }
    all_static = __syncthreads_and(all_static);

    // angular sums in direction chunks: E-bar_- (compensated), B1, B2 (eqs.
    // A1, A2 in the reading of method 3); K = alpha_- dt / (n^0 + D alpha_- dt).
    // B1 and B2 are compensated too in FP32: with alpha^s dt >> 1 the solve's
    // coefficient alpha dt - B2 alpha^s cancels to ~1/(alpha dt) of its terms
    // and magnifies B2's rounding by as much
    const int nchunk = NT / NC;
    {
        const int c = s % NC, g = s / NC;
        TM Em = 0, cEm = 0, B1 = 0, B2 = 0, cB1 = 0, cB2 = 0;
        auto kadd = [](TM &sum, TM &comp, TM v) {
            if constexpr (sizeof(TM) == 4) {
                const TM y = v - comp, t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            } else {
                sum += v;
            }
        };
        if ((c % TXC) < nc && scOn[c]) {
            const TM u0m = scU[4 * c], u1 = scU[4 * c + 1], u2 = scU[4 * c + 2], u3 = scU[4 * c + 3];
            const TM n0 = scN0[c], adt = scK[c], kn = dv<TM>(adt, n0);
            const TM *row = It + c * ndp;
            for (int d = g; d < nd; d += nchunk) {
                TM w = ldT<TM>(A.wT, d);
                TM t;
                if (all_static) t = row[d] * w;
                else {
                    TM D = TM(1) + (u0m - fma(u1, ldT<TM>(A.dirT, 3 * d),
                                              fma(u2, ldT<TM>(A.dirT, 3 * d + 1), u3 * ldT<TM>(A.dirT, 3 * d + 2))));
                    t = D * D * row[d] * w;
                    if constexpr (sizeof(TM) == 4) {
                        // rq = n^0 / (n^0 + D alpha dt), K = (alpha dt / n^0) rq; the
                        // sum gathers the small remainder w-bar rq of
                        // B2 = dt/(4 pi) (sum w-bar - sum w-bar rq) (w-bar = w / D^2),
                        // whose leading sum is per-cell FP64 (wbar): B2 then
                        // carries no FP32 rounding that the solve's cancellation
                        // alpha dt - B2 alpha^s would magnify
                        const TM iD = dv<TM>(TM(1), D), rq = dv<TM>(n0, fma(D, adt, n0));
                        kadd(B1, cB1, n0 * (kn * rq) * t);
                        kadd(B2, cB2, w * iD * iD * rq);
                    } else {
                        TM K = dv<TM>(adt, fma(D, adt, n0));
                        kadd(B1, cB1, n0 * K * t);
                        kadd(B2, cB2, dv<TM>(K * w, D));
                    }
                }
                TM yk = t - cEm, tk = Em + yk;
                cEm = (tk - Em) - yk; Em = tk;
            }
        }
        double *pp = part + (g * NC + c) * 6;
        pp[0] = (double)Em - (double)cEm; pp[1] = (double)B1 - (double)cB1; pp[2] = (double)B2 - (double)cB2;
    }
    __syncthreads();
    // one lane per cell: temperature solve and per-cell update constants
    if (s < NC) {
        int ii, j;
        size_t cidx = gcell(s, ii, j);
        if (ii < nc && scOn[s]) {
            double Em = 0, B1 = 0, B2 = 0;
            for (int g = 0; g < nchunk; ++g) {
                const double *pp = part + (g * NC + s) * 6;
                Em += pp[0]; B1 += pp[1]; B2 += pp[2];
            }
            const double dt = A.dtk, adt = A.alpha_int[cidx] * dt;
            // the isotropic source is spread with the solid angles the sums
            // use: in FP32 their sum differs from 4 pi by ~1e-7, which the
            // solve's cancellation at alpha^s dt >> 1 would magnify into a
            // bias of the scattered energy repeated every stage
            const double qw = sizeof(TM) == 4 ? A.sumwf : FOURPI;
            if (all_static) {        // D = 1, n^0 = 1: K is per cell
                double K = adt / (1.0 + adt);
                B1 = K * Em;
                B2 = K * (sizeof(TM) == 4 ? A.sumwf : A.sumw);
            } else if (sizeof(TM) == 4) {
                B2 = A.wbar[cidx] - B2;
            }
            B2 *= dt / qw;
            const double Y = A.cc_Y[cidx], ug = A.ug_in[cidx], Tm = ug / Y;
            if (A.coupling != 3) {
                // methods 1 and 2: A1 = B1 / (alpha_- dt), A2 = B2 / (alpha_- dt); the
                // intensity update keeps the explicit alpha_-
                const double iY = 1.0 / Y, au = A.cc_au[cidx], as = A.cc_as[cidx];
                const M12 q{B1 / adt, B2 / adt, Em + ug, Y, iY, Tm, Em, au, as, A.eta[cidx], A.arad, A.T_exp,
                            au * tpow_neg<double>(Tm, A.T_exp), A.coupling};
                double X;
                if (!solve_m12(q, &X)) {       // no positive temperature: the cell is left as it was
                    atomicAdd(A.fail, 1ull);
                    scOn[s] = 0;
                } else {
                    const double Tp = Tm + (Em - X) * iY;
                    const double aap = A.coupling == 1 ? q.aam : au * tpow_neg<double>(Tp, A.T_exp);
                    const double em = q.eta * aap * A.arad * Tp * Tp * Tp * Tp + as * X;
                    if (A.sv_X) { A.sv_Em[cidx] = Em; A.sv_X[cidx] = X; }
                    scEm[s] = (TM)(dt * em / qw);
                    scA[s] = (TM)adt;
                }
            } else {
            Teq<double> q = make_teq<double>(B1, B2, Em + ug, Y, Tm, Em, A.cc_au[cidx], A.cc_as[cidx], A.eta[cidx], A.arad,
                                             dt, A.T_exp);
            double lo = 0.0, hi = q.W, X;
            bool ok;
            if (sizeof(TM) == 4) {
                // FP32 Newton iterations, then one FP64 Newton step
                Teq<float> qf{(float)q.B1, (float)q.B2, (float)q.W, (float)q.Y, (float)q.Tm, (float)q.Em, (float)q.au,
                              (float)q.as, (float)q.eta, (float)q.arad, (float)q.dt, (float)q.p, (float)q.iY};
                float flo = 0.0f, fhi = (float)q.W, fx;
                newton_E<float>(qf, (float)Em, flo, fhi, 60, 1e-7f, &fx);
                // FP64 Newton from the FP32 root (one or two steps in practice)
                ok = newton_E<double>(q, (double)fx, lo, hi, 200, 4.0 * 2.220446049250313e-16, &X);
            } else {
                ok = newton_E<double>(q, Em, lo, hi, 200, 4.0 * 2.220446049250313e-16, &X);
            }
            if (!ok) atomicAdd(A.fail, 1ull);
            if (A.sv_X) { A.sv_Em[cidx] = Em; A.sv_X[cidx] = X; }
            const double Tp = Tm + (Em - X) / Y;
            const double aap = A.cc_au[cidx] * tpow_neg<double>(Tp, A.T_exp), atp = aap + A.cc_as[cidx];
            const double em = A.eta[cidx] * aap * A.arad * Tp * Tp * Tp * Tp + A.cc_as[cidx] * X;
            scEm[s] = (TM)(dt * em / qw);
            scA[s] = (TM)(atp * dt);
            }
        }
    }
    __syncthreads();
    // per-direction update (eq. fluid_interaction_discrete with alpha(T_+) and
    // emission at T_+), masks, store
    if (act) {
        for (int lc = 0; lc < NC; ++lc) {
            int ii, j;
            size_t cidx = gcell(lc, ii, j);
            if (ii >= nc) continue;
            TM v = It[lc * ndp + s];
            const TM v0 = v;
            if (scOn[lc]) {
                if (all_static) v = (v + scEm[lc]) / (TM(1) + scA[lc]);
                else {
                    TM D = TM(1) + (scU[4 * lc] - fma(scU[4 * lc + 1], nh[0], fma(scU[4 * lc + 2], nh[1], scU[4 * lc + 3] * nh[2])));
                    TM n0 = scN0[lc];
                    v = dv<TM>(fma(n0, v, dv<TM>(scEm[lc], D * D * D)), fma(D, scA[lc], n0));
                }
                bool zero = A.n_pole_zero > 0 && (j < A.n_pole_zero || j >= A.nx1 - A.n_pole_zero);
                if (!FLAT) zero = zero || (A.mask[(size_t)((j + A.ng1) * A.gn0 + (i0 + ii + A.ng0)) * nd + s] & 1);
                if (zero) v = TM(0);
            }
            It[lc * ndp + s] = IO<TS, TM>::st(A.Iout, cidx * nd + s, v) - v0;   // the stored I_+ minus I*
        }
    }
    __syncthreads();
    // exchange ledger: E-bar(I_+) - E-bar(I*) and Delta R^{0 a} in direction
    // chunks, summed from the per-element changes (no cancellation)
    {
        const int c = s % NC, g = s / NC;
        TM Ep = 0, cEp = 0, r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        if ((c % TXC) < nc && scOn[c]) {
            const TM u0m = scU[4 * c], u1 = scU[4 * c + 1], u2 = scU[4 * c + 2], u3 = scU[4 * c + 3];
            const TM *rd = It + c * ndp;
            for (int d = g; d < nd; d += nchunk) {
                TM w = ldT<TM>(A.wT, d);
                TM x = ldT<TM>(A.dirT, 3 * d), y = ldT<TM>(A.dirT, 3 * d + 1), z = ldT<TM>(A.dirT, 3 * d + 2);
                TM D = all_static ? TM(1) : TM(1) + (u0m - fma(u1, x, fma(u2, y, u3 * z)));
                TM t = D * D * rd[d] * w;
                TM yk = t - cEp, tk = Ep + yk;
                cEp = (tk - Ep) - yk; Ep = tk;
                TM dI = rd[d] * w;
                r0 += dI; r1 = fma(x, dI, r1); r2 = fma(y, dI, r2); r3 = fma(z, dI, r3);
            }
        }
        double *pp = part + (g * NC + c) * 6;
        pp[0] = (double)Ep - (double)cEp; pp[1] = r0; pp[2] = r1; pp[3] = r2; pp[4] = r3;
    }
    __syncthreads();
    if (s < NC) {
        int ii, j;
        size_t cidx = gcell(s, ii, j);
        if (ii < nc) {
            double ugm = A.ug_in[cidx];
            if (scOn[s]) {
                double Ep = 0, dR[4] = {0, 0, 0, 0};
                for (int g = 0; g < nchunk; ++g) {
                    const double *pp = part + (g * NC + s) * 6;
                    Ep += pp[0]; dR[0] += pp[1]; dR[1] += pp[2]; dR[2] += pp[3]; dR[3] += pp[4];
                }
                double ugp = ugm - Ep;          // Ep: E-bar(I_+) - E-bar(I*)
                A.ug_out[cidx] = ugp;
                double T = ugp / A.cc_Y[cidx];
                A.alpha_out[cidx] = T > 0.0 ? A.cc_au[cidx] * tpow_neg<double>(T, A.T_exp) + A.cc_as[cidx] : 0.0;
                if (A.G) {
                    for (int m = 0; m < 4; ++m) {
                        double gm;
                        if (FLAT) gm = dR[m];
                        else {
                            const double *E = A.pt_e + 16 * (size_t)((j + A.ng1) * A.gn0 + (i0 + ii + A.ng0));
                            gm = E[m] * dR[0] + E[4 + m] * dR[1] + E[8 + m] * dR[2] + E[12 + m] * dR[3];
                        }
                        A.G[4 * cidx + m] = -gm / A.dtk;
                    }
                }
            } else {
                A.ug_out[cidx] = ugm;
                A.alpha_out[cidx] = A.alpha_int[cidx];
                if (A.G) for (int m = 0; m < 4; ++m) A.G[4 * cidx + m] = 0.0;
            }
        }
    }
}

__global__ void k_alpha(int ncell, double T_exp, const double *__restrict__ cc_au, const double *__restrict__ cc_as,
                        const double *__restrict__ cc_Y, const uint8_t *__restrict__ cc_on,
                        const double *__restrict__ ug, double *__restrict__ alpha) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double T = cc_Y[c] > 0.0 ? ug[c] / cc_Y[c] : 0.0;
    alpha[c] = (cc_on[c] && T > 0.0) ? cc_au[c] * tpow_neg<double>(T, T_exp) + cc_as[c] : 0.0;
}

// per-cell constants of the fluid: alpha^a prefactor kappa rho^m, alpha^s,
// Y = rho/(Gamma - 1), and the density-floor switch (section 3.7)
__global__ void k_cellconst(int ncell, double gam, double rho_exp, double rho_floor, const double *__restrict__ rho,
                            const double *__restrict__ kap, const double *__restrict__ cs, double *__restrict__ au,
                            double *__restrict__ as, double *__restrict__ Y, uint8_t *__restrict__ on) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double r = rho[c];
    bool ok = r >= rho_floor && r > 0.0;
    on[c] = ok;
    au[c] = ok ? kap[c] * pow(r, rho_exp) : 0.0;
    as[c] = ok ? cs[c] * r : 0.0;
    Y[c] = r / (gam - 1.0);
}

// shared memory of one CTA of k_stage: the brick's intensities (I*, then the
// interaction's changes), face records, per-cell constants, the curved
// geometry's angular rows and (in the same space) the chunk partial sums,
// boundary descriptors
template <typename TM, bool FLAT, int BY, int BZ, int NC>
size_t stage_smem(int nd, int NT) {
    constexpr int TXC = NC / (BY * BZ), NOWN = BY * BZ;
    const size_t ndp = nd + 1;
    const size_t tm = NC * ndp + NOWN * (TXC + 1) * 5 + BZ * (BY + 1) * TXC * 5 + BY * (BZ + 1) * TXC * 5 + 8 * NC;
    const size_t ang = FLAT ? 0 : sizeof(TM) * 7 * (size_t)NOWN * nd;   // angular rows
    const size_t prt = 16 + sizeof(double) * (size_t)NT * 6;           // chunk sums (same space)
    return sizeof(TM) * tm + (ang > prt ? ang : prt) + sizeof(int) * (TXC + 4 + BZ * (BY + 4) + BY * (BZ + 4) + NC);
}

template <typename TS, typename TM, bool FLAT, int BY, int BZ, int NC, int MAXT, int MINB = 1>
rt_status launch(rt_ctx *c, const StageArgs &A, int NT) {
    constexpr int TXC = NC / (BY * BZ);
    const size_t smem = stage_smem<TM, FLAT, BY, BZ, NC>(A.nd, NT);
    auto kern = k_stage<TS, TM, FLAT, BY, BZ, -1, NC, MAXT, MINB>;
    if constexpr (MAXT <= MAXNT)
        if (A.limiter == RT_LIM_MC) kern = k_stage<TS, TM, FLAT, BY, BZ, RT_LIM_MC, NC, MAXT, MINB>;
    RT_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nseg = (A.nx0 + TXC - 1) / TXC;
    size_t nblk = (size_t)nseg * (A.nx1 / BY) * (A.nx2 / BZ);
    kern<<<(unsigned)nblk, NT, smem, c->stream>>>(A);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

template <typename TS, typename TM, bool FLAT>
rt_status launch_blk(rt_ctx *c, const StageArgs &A, int NT) {
    if (NT > MAXNT) {
        // finer grids (more than 256 directions): one direction per thread,
        // up to 1024 threads, 1 x 1 bricks of 32, 16 or 8 cells as shared
        // memory allows
        if (stage_smem<TM, FLAT, 1, 1, 32>(A.nd, NT) <= SMEM_MAX) return launch<TS, TM, FLAT, 1, 1, 32, MAXNT_BIG>(c, A, NT);
        if (stage_smem<TM, FLAT, 1, 1, 16>(A.nd, NT) <= SMEM_MAX) return launch<TS, TM, FLAT, 1, 1, 16, MAXNT_BIG>(c, A, NT);
        if (stage_smem<TM, FLAT, 1, 1, 8>(A.nd, NT) <= SMEM_MAX) return launch<TS, TM, FLAT, 1, 1, 8, MAXNT_BIG>(c, A, NT);
        c->err = "the stage kernel's shared memory cannot hold this many directions";
        return RT_EINVAL;
    }
    bool by = A.act1 && A.nx1 % 2 == 0, bz = A.act2 && A.nx2 % 2 == 0;
    if constexpr (!FLAT) {
        // curved geometry: the tables do not depend on x3 (phi), so 8 x 1 x 4
        // bricks, whose four rows share every table entry, beat 8 x 2 x 2
        // bricks (measured 96.0 against 110.9 ms per 256 x 128 x 128 torus
        // step); the kernel is latency-bound: three CTAs of 192 threads per
        // SM (96 registers) took it to 83.8 ms, and with the brick's single
        // intensity tile four (80 registers) run it in 63.2 ms
        constexpr int MB = sizeof(TM) == 4 ? CURV_MINB : 1;   // FP64: shared memory allows one CTA
        if (NT <= CURV_NT) {
            if (A.act2 && A.nx2 % 4 == 0) return launch<TS, TM, FLAT, 1, 4, NCELL, CURV_NT, MB>(c, A, NT);
            if (by && bz) return launch<TS, TM, FLAT, 2, 2, NCELL, CURV_NT, MB>(c, A, NT);
            if (by) return launch<TS, TM, FLAT, 2, 1, NCELL, CURV_NT, MB>(c, A, NT);
            return launch<TS, TM, FLAT, 1, 1, NCELL, CURV_NT, MB>(c, A, NT);
        }
    }
    if (by && bz) return launch<TS, TM, FLAT, 2, 2, NCELL, MAXNT>(c, A, NT);
    if (by) return launch<TS, TM, FLAT, 2, 1, NCELL, MAXNT>(c, A, NT);
    return launch<TS, TM, FLAT, 1, 1, NCELL, MAXNT>(c, A, NT);
}

}  // namespace

rt_status rt_launch_cellconst(rt_ctx *c) {
    const rt_config &f = c->cfg;
    k_cellconst<<<(c->ncell + 255) / 256, 256, 0, c->stream>>>(c->ncell, f.gam, f.rho_exp, f.rho_floor, c->rho, c->kap,
                                                              c->cs, c->cc_au, c->cc_as, c->cc_Y, c->cc_on);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

rt_status rt_launch_alpha(rt_ctx *c, const double *ug, double *alpha) {
    k_alpha<<<(c->ncell + 255) / 256, 256, 0, c->stream>>>(c->ncell, c->cfg.T_exp, c->cc_au, c->cc_as, c->cc_Y,
                                                          c->cc_on, ug, alpha);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

rt_status rt_launch_stage(rt_ctx *c, const void *Isrc, const void *Ibase, void *Iout, const double *ug_in,
                          double *ug_out, const double *alpha_in, const double *alpha_int, double *alpha_out,
                          double dtk, double *G) {
    const rt_config &f = c->cfg;
    const rt_grid *g = c->g;
    StageArgs A{};
    A.nx0 = f.nx[0]; A.nx1 = f.nx[1]; A.nx2 = f.nx[2]; A.nd = c->nd; A.ne = c->ne;
    A.act0 = c->active[0]; A.act1 = c->active[1]; A.act2 = c->active[2];
    for (int a = 0; a < 3; ++a) for (int s = 0; s < 2; ++s) A.bc[a][s] = f.bc[a][s];
    A.beam_dir = f.beam_dir; A.beam_lo = f.beam_lo; A.beam_hi = f.beam_hi; A.beam_I = f.beam_I;
    A.n_pole_zero = f.n_pole_zero;
    A.dx0 = f.dx[0]; A.dx1 = f.dx[1]; A.dx2 = f.dx[2];
    A.gam = f.gam; A.arad = f.arad; A.T_exp = f.T_exp; A.abar = f.abar; A.sumw = c->sumw; A.sumwf = c->sumwf;
    A.tau_dt = f.tau_dt; A.limiter = f.limiter; A.ang_recon = f.ang_recon;
    A.transport = f.transport; A.source = f.source; A.dtk = dtk;
    A.coupling = rt_coupling3(c) ? 3 : f.coupling;
    A.Isrc = Isrc; A.Ibase = Ibase; A.Iout = Iout; A.ug_in = ug_in; A.ug_out = ug_out;
    A.alpha_in = alpha_in; A.alpha_int = alpha_int; A.alpha_out = alpha_out;
    A.cc_au = c->cc_au; A.cc_as = c->cc_as; A.cc_Y = c->cc_Y; A.cc_on = c->cc_on;
    A.eta = c->eta; A.vel = c->vel; A.uhat = c->uhat; A.wbar = c->wbar; A.G = G; A.gac = c->gac; A.fail = c->fail;
    if (G) c->g_lazy = false;   // set again below if the packed kernel defers G
    A.sv_Em = c->sv_Em; A.sv_X = c->sv_X;
    A.mirror = g->mirror; A.nnb = g->nnb; A.nbr = g->nbr; A.ring_edge = g->ring_edge; A.ring_back = g->ring_back;
    A.edge = g->edge;
    bool dbl = f.precision == RT_FP64;
    A.dirT = dbl ? (const void *)g->dir : (const void *)g->dirf;
    A.wT = dbl ? (const void *)g->w : (const void *)g->wf;
    A.mxT = dbl ? (const void *)g->mx : (const void *)g->mxf;
    A.mgT = dbl ? (const void *)g->mg : (const void *)g->mgf;
    A.mmT = dbl ? (const void *)g->mm : (const void *)g->mmf;
    A.mdT = dbl ? (const void *)g->md : (const void *)g->mdf;
    bool flat = c->metric == RT_MINKOWSKI_CART;
    A.ng0 = c->active[0] ? 2 : 0; A.ng1 = c->active[1] ? 2 : 0; A.gn0 = c->gn[0];
    if (!flat) {
        A.cenU = dbl ? (const void *)c->cenU_d : (const void *)c->cenU_f;
        A.fn = dbl ? (const void *)c->fn_d : (const void *)c->fn_f;
        A.fP = dbl ? (const void *)c->fP_d : (const void *)c->fP_f;
        A.ew = dbl ? (const void *)c->ew_d : (const void *)c->ew_f;
        A.eneg = c->eneg;
        A.mask = c->mask; A.pt_V = c->pt_V; A.pt_n0 = c->pt_n0; A.pt_len = c->pt_len; A.pt_e = c->pt_e;
    }
    for (int m = 0; m < 3; ++m) A.sumnw[m] = c->sumnw[m];
    if (c->halo) {
        // neighbour-read arrays from the first ghost plane (see StageArgs::kb)
        A.kb = 2;
        A.Isrc = (const char *)Isrc - c->hcells * c->nd * c->esize;
        A.alpha_in = alpha_in - c->hcells;
        A.vel = c->vel - 3 * c->hcells;
    }
    int NT = ((c->nd + 31) / 32) * 32;
    if (NT < 64) NT = 64;
    if (NT > MAXNT_BIG) { c->err = "more than 1024 directions per cell are not supported by the stage kernel"; return RT_EINVAL; }
    if (rt_stage_fast_ok(c)) return rt_launch_stage_fs(c, A, NT);
    if (f.precision == RT_FP64)
        return flat ? launch_blk<double, double, true>(c, A, NT) : launch_blk<double, double, false>(c, A, NT);
    if (f.precision == RT_FP32)
        return flat ? launch_blk<float, float, true>(c, A, NT) : launch_blk<float, float, false>(c, A, NT);
    return flat ? launch_blk<__nv_bfloat16, float, true>(c, A, NT) : launch_blk<__nv_bfloat16, float, false>(c, A, NT);
}
