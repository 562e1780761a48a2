// rt_internal.cuh — private structures of librt_b300 (the CUDA radiation step).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/rt.h"

#define RT_MAXNB 6

// Geodesic grid: host topology + device geometry (all FP64 on the device,
// FP32 copies for the mixed path).
struct rt_grid {
    int n = 0, nd = 0, ne = 0;
    std::vector<double> h_dir, h_w;        // host copies for rt_grid_query
    std::vector<int> h_nnb, h_nbr, h_mirror, h_ring_edge, h_ring_back, h_edge;
    // device, per direction s
    double *dir = nullptr;       // [nd*3]
    double *w = nullptr;         // [nd] solid angle
    int *nnb = nullptr;          // [nd]
    int *nbr = nullptr;          // [nd*6] ccw ring, smallest index first
    int *ring_edge = nullptr;    // [nd*6]
    int *ring_back = nullptr;    // [nd*6] slot of s in nbr's ring
    int *mirror = nullptr;       // [nd] (n1,-n2,-n3)
    int *edge = nullptr;         // [ne*2] s < s'
    double *emid = nullptr;      // [ne*3]
    double *eu = nullptr;        // [ne*3] unit normal from s to s'
    double *dlam = nullptr;      // [ne]
    // minimum-angle plane reconstruction tables, per (s, ring slot q)
    double *mx = nullptr;        // [nd*6*3] gnomonic image of neighbour q in the tangent plane of s
    double *mg = nullptr;        // [nd*6*3] inverse Gram matrix (a, b, c) of the pair (q, q+1)
    double *mm = nullptr;        // [nd*6*3] gnomonic image of the midpoint of edge q
    // md[((b*6 + q)*nd + s)*2 + {0,1}] = mx(s, b).mm(s, q), mx(s, b+1).mm(s, q):
    // the reconstruction weights of edge midpoint q for the plane of pair b;
    // direction-fastest, so that a warp's lookups for one plane coalesce
    double *md = nullptr;        // [6*6*nd*2]
    float *dirf = nullptr, *wf = nullptr, *mxf = nullptr, *mgf = nullptr, *mmf = nullptr, *mdf = nullptr;
};

// Per-context device state.
struct rt_ctx {
    rt_config cfg{};
    const rt_grid *g = nullptr;
    cudaStream_t stream = nullptr;
    int device = -1;             // CUDA device current at rt_create: every buffer lives there
    int ncell = 0, nd = 0, ne = 0;
    int active[3] = {0, 0, 0};
    int gn[2] = {0, 0};          // ghosted extents of the (x1, x2) geometry table
    int metric = -1;             // rt_metric_kind once set
    double M = 1.0, a = 0.0;
    bool have_fluid = false, have_I = false;
    size_t esize = 8;            // bytes per stored intensity
    std::string err;

    // x3 slab of a decomposed box (RT_BC_HALO on an x3 face): the intensity
    // arrays, the flux opacities and the coordinate velocity carry two ghost
    // planes below and above the owned cells; the pointers below point at the
    // owned cell 0 and the allocations start 2 planes earlier
    bool halo = false;
    bool halo_fluid = false;      // rt_set_fluid_halo called since rt_set_fluid
    int next_stage = 0;           // rt_step_stage: the stage the step in progress expects
    size_t hcells = 0;            // cells in two planes (2 nx0 nx1) when halo, else 0
    // intensity state: current, predictor, next (rotated after each step)
    void *I[3] = {nullptr, nullptr, nullptr};
    double *ug[3] = {nullptr, nullptr, nullptr};
    double *alpha[2] = {nullptr, nullptr};   // comoving opacity of the flux stage
    // fluid
    double *rho = nullptr, *kap = nullptr, *cs = nullptr, *eta = nullptr, *ucon = nullptr;
    double *vel = nullptr;       // [ncell*3] coordinate velocity u^a/u^0
    double *uhat = nullptr;      // [ncell*4] tetrad-frame fluid velocity
    // [ncell] sum_s w_s / D_s^2 in FP64, D_s = u-hat^0 - u-hat.n_s, with the
    // solid angles the context's stage kernels use (FP32-rounded for FP32 and
    // BF16 storage): the leading part of the interaction's sum B2
    double *wbar = nullptr;
    double *G = nullptr;         // [ncell*4]
    // the packed FP32 stage kernel leaves the force on the gas of its
    // interaction as per-cell (a, c) (I_+ = (I + c)/(1 + a)); rt_moments then
    // forms G from them and the moments of the current state (g_lazy)
    float2 *gac = nullptr;       // [ncell]
    bool g_lazy = false;
    double g_dt = 0.0;
    // per-cell constants of the fluid: kappa rho^m, alpha_s rho, rho/(Gamma-1), floor switch
    double *cc_au = nullptr, *cc_as = nullptr, *cc_Y = nullptr;
    uint8_t *cc_on = nullptr;
    double sumw = 0.0;           // sum of the solid angles (4 pi to rounding)
    double sumwf = 0.0;          // sum of the FP32-rounded solid angles (the FP32 paths' quadrature)
    double sumnw[3] = {0, 0, 0}; // sum of n-hat dOmega (0 to rounding)
    bool static_fluid = false;   // u-hat = (1, 0, 0, 0) in every cell (set by rt_set_fluid)
    unsigned long long *fail = nullptr;   // device counter of unconverged solves

    // geometry tables over ghosted (i, j) points (Kerr-Schild); flat: unused
    double *pt_e = nullptr;      // [npt*16] e^mu_(a) at cell centres
    double *pt_ei = nullptr;     // [npt*16] e^(a)_mu
    double *pt_V = nullptr;      // [npt] sqrt(-g) dx1 dx2 dx3
    double *pt_n0 = nullptr;     // [npt] n^0 (direction independent for normal observers)
    double *pt_len = nullptr;    // [3*npt] proper length sqrt(g_aa) dx_a at the lower face
    double *pt_om = nullptr;     // [npt*64] Ricci rotation coefficients
    double *cenU_d = nullptr; float *cenU_f = nullptr;     // [npt*nd] n^0 n_0
    uint8_t *mask = nullptr;     // [npt*nd] bit0: |n_0| < cut, bit1: n_0 > 0
    double *fn_d = nullptr; float *fn_f = nullptr;         // [3*npt*nd] n^a at the lower face
    double *fP_d = nullptr; float *fP_f = nullptr;         // [3*npt*nd] dA_a n_0 at the lower face
    double *ew_d = nullptr; float *ew_f = nullptr;         // [npt*ne] dlam_e n_0(m) v(m).u_e
    uint8_t *eneg = nullptr;     // [npt*ne] 1 where n_0(m) < 0: the upwind side follows v.u, i.e. the opposite sign of ew
    double dt_cfl = 0.0;
    // arena of the reverse pass (rt_step_adjoint), grown on demand
    double *adj = nullptr;
    size_t adj_bytes = 0;
    // the forward recording held in the arena (rt_step_record): its id (0 =
    // none), steps and step size
    long long rec_id = 0;
    int rec_N = 0;
    double rec_dt = 0.0;
    // set during the reverse pass's recompute: the stage kernels save each
    // cell's E-bar_- and temperature-solve root X there (null otherwise)
    double *sv_Em = nullptr, *sv_X = nullptr;
    // optional per-launch timing of the stage kernel
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t ev_used = 0;
};

// start of the allocation behind an array whose pointer sits hcells cells of
// `per` bytes after it (x3 halo planes), for cudaFree
inline void *rt_halo_base(const rt_ctx *c, void *p, size_t per) {
    return p ? (void *)((char *)p - c->hcells * per) : nullptr;
}

#define RT_CUDA_TRY(c, call)                                                          \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            if (c) (c)->err = std::string(#call) + ": " + cudaGetErrorString(e_);   \
            return e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;           \
        }                                                                             \
    } while (0)

// RT_EINVAL unless the calling thread's current device is the context's (its
// buffers and stream belong to that device; a launch elsewhere would read
// another GPU's pointers)
rt_status rt_check_device(rt_ctx *c);

// geometry (geometry.cu)
rt_status rt_build_geometry(rt_ctx *c);
rt_status rt_compute_uhat(rt_ctx *c);
// grid device geometry (grid.cu)
rt_status rt_grid_device_geometry(rt_grid *g, std::string &err);
// stage launcher (stage.cu)
rt_status rt_launch_stage(rt_ctx *c, const void *Isrc, const void *Ibase, void *Iout,
                          const double *ug_in, double *ug_out, const double *alpha_in, const double *alpha_int,
                          double *alpha_out, double dtk, double *G);
rt_status rt_launch_alpha(rt_ctx *c, const double *ug, double *alpha);
rt_status rt_launch_cellconst(rt_ctx *c);

// moments (moments.cu)
rt_status rt_launch_moments(rt_ctx *c, double *R, double *Ebar);
// G of a deferred interaction (g_lazy) into c->G from the current state; clears g_lazy
rt_status rt_resolve_g(rt_ctx *c);
rt_status rt_launch_cfl(rt_ctx *c, double *dt_min_host);
