// api.cu — the C ABI of librt_b300 (see include/rt.h for the contract).
#include "rt_internal.cuh"
#include <cstring>
#include <utility>

static std::string g_create_err;

// any cell whose tetrad-frame fluid velocity is not (1, 0, 0, 0)
__global__ void k_moving(int ncell, const double *__restrict__ uhat, int *__restrict__ flag) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double *u = uhat + 4 * (size_t)c;
    if (!(u[0] == 1.0 && u[1] == 0.0 && u[2] == 0.0 && u[3] == 0.0)) atomicOr(flag, 1);
}

static rt_status fail(rt_ctx *c, rt_status st, const char *msg) {
    if (c) c->err = msg;
    return st;
}

rt_status rt_check_device(rt_ctx *c) {
    int dev = -1;
    RT_CUDA_TRY(c, cudaGetDevice(&dev));
    if (dev != c->device) {
        c->err = "the current CUDA device (" + std::to_string(dev) + ") is not the context's (" +
                 std::to_string(c->device) + ")";
        return RT_EINVAL;
    }
    return RT_OK;
}

static void free_ctx(rt_ctx *c) {
    if (!c) return;
    for (auto &pr : c->ev) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    const size_t ie = c->nd * c->esize;
    void *ptrs[] = {rt_halo_base(c, c->I[0], ie), rt_halo_base(c, c->I[1], ie), rt_halo_base(c, c->I[2], ie),
                    c->ug[0], c->ug[1], c->ug[2], rt_halo_base(c, c->alpha[0], 8), rt_halo_base(c, c->alpha[1], 8),
                    c->rho, c->kap, c->cs, c->eta, c->ucon, rt_halo_base(c, c->vel, 24), c->uhat, c->wbar, c->G, c->fail, c->pt_e, c->pt_ei, c->pt_V,
                    c->pt_n0, c->pt_len, c->pt_om, c->cenU_d, c->cenU_f, c->mask, c->fn_d, c->fn_f, c->fP_d,
                    c->fP_f, c->ew_d, c->ew_f, c->eneg, c->cc_au, c->cc_as, c->cc_Y, c->cc_on, c->adj, c->gac};
    for (void *p : ptrs) if (p) cudaFree(p);
    delete c;
}

extern "C" rt_status rt_create(const rt_grid *g, const rt_config *cfg, void *cuda_stream, rt_ctx **out) {
    if (!g || !cfg || !out) return RT_EINVAL;
    *out = nullptr;
    const rt_config &f = *cfg;
    for (int a = 0; a < 3; ++a) {
        if (f.nx[a] < 1 || !(f.dx[a] > 0.0)) { g_create_err = "nx must be >= 1 and dx > 0"; return RT_EINVAL; }
        for (int s = 0; s < 2; ++s)
            if (f.bc[a][s] < 0 || f.bc[a][s] > 4) { g_create_err = "unknown boundary kind"; return RT_EINVAL; }
        if (f.nx[a] > 1 && f.nx[a] < 2) { g_create_err = "active axes need at least 2 cells"; return RT_EINVAL; }
    }
    if (f.precision < 0 || f.precision > 2 || f.order < 1 || f.order > 2 || !(f.gam > 1.0) ||
        f.T_exp < 0.0 || f.T_exp >= 4.0 || f.limiter < 0 || f.limiter > 2 || f.coupling < 0 || f.coupling > 3) {
        g_create_err = "invalid precision, order, gamma, T_exp, limiter or coupling method";
        return RT_EINVAL;
    }
    const bool halo = f.bc[2][0] == RT_BC_HALO || f.bc[2][1] == RT_BC_HALO;
    if (f.bc[0][0] == RT_BC_HALO || f.bc[0][1] == RT_BC_HALO || f.bc[1][0] == RT_BC_HALO || f.bc[1][1] == RT_BC_HALO ||
        (halo && (f.nx[2] < 2 || f.bc[1][0] == RT_BC_POLE || f.bc[1][1] == RT_BC_POLE || f.bc[0][0] == RT_BC_BEAM))) {
        g_create_err = "halo boundaries: x3 faces only, at least 2 x3 cells, no pole boundary on x2, no beam";
        return RT_EINVAL;
    }
    if (f.bc[1][0] == RT_BC_POLE && f.nx[2] > 1 && (f.nx[2] % 2)) {
        g_create_err = "the pole boundary needs an even number of x3 cells";
        return RT_EINVAL;
    }
    rt_ctx *c = new rt_ctx();
    c->cfg = f;
    c->g = g;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        g_create_err = "no current CUDA device";
        delete c;
        return RT_ECUDA;
    }
    c->nd = g->nd; c->ne = g->ne;
    c->ncell = f.nx[0] * f.nx[1] * f.nx[2];
    for (int a = 0; a < 3; ++a) c->active[a] = f.nx[a] > 1;
    c->esize = f.precision == RT_FP64 ? 8 : (f.precision == RT_FP32 ? 4 : 2);
    size_t nc = (size_t)c->ncell;
    c->halo = halo;
    c->hcells = halo ? 2 * (size_t)f.nx[0] * f.nx[1] : 0;
    const size_t ie = c->nd * c->esize, nh = nc + 2 * c->hcells;
    cudaError_t e = cudaSuccess;
    // halo arrays: two ghost planes on each side, zeroed, pointer at the owned origin
    auto halo_alloc = [&](void **p, size_t per) {
        if (e != cudaSuccess) return;
        void *raw = nullptr;
        e = cudaMalloc(&raw, nh * per);
        if (e == cudaSuccess && c->hcells) e = cudaMemset(raw, 0, nh * per);
        if (e == cudaSuccess) *p = (char *)raw + c->hcells * per;
    };
    for (int q = 0; q < 3; ++q) halo_alloc(&c->I[q], ie);
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaMalloc(&c->ug[q], nc * 8);
    for (int q = 0; q < 2; ++q) halo_alloc((void **)&c->alpha[q], 8);
    double **fl[] = {&c->rho, &c->kap, &c->cs, &c->eta};
    for (auto p : fl) if (e == cudaSuccess) e = cudaMalloc(p, nc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->ucon, nc * 32);
    halo_alloc((void **)&c->vel, 24);
    if (e == cudaSuccess) e = cudaMalloc(&c->uhat, nc * 32);
    if (e == cudaSuccess) e = cudaMalloc(&c->wbar, nc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->G, nc * 32);
    if (e == cudaSuccess) e = cudaMalloc(&c->fail, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->cc_au, nc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->cc_as, nc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->cc_Y, nc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->cc_on, nc);
    if (e == cudaSuccess) e = cudaMalloc(&c->gac, nc * sizeof(float2));
    for (int d = 0; d < g->nd; ++d) {
        c->sumw += g->h_w[d];
        c->sumwf += (double)(float)g->h_w[d];
        for (int m = 0; m < 3; ++m) c->sumnw[m] += g->h_dir[3 * d + m] * g->h_w[d];
    }
    if (e == cudaSuccess) e = cudaMemset(c->G, 0, nc * 32);
    if (e != cudaSuccess) {
        g_create_err = std::string("allocation: ") + cudaGetErrorString(e);
        free_ctx(c);
        return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
    }
    *out = c;
    return RT_OK;
}

extern "C" void rt_destroy(rt_ctx *c) {
    if (c && c->stream) cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

extern "C" const char *rt_last_error(const rt_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

extern "C" rt_status rt_set_metric(rt_ctx *c, int kind, const double *params) {
    if (!c) return RT_EINVAL;
    if (kind < RT_MINKOWSKI_CART || kind > RT_CART_CYLTETRAD) return fail(c, RT_EINVAL, "unknown metric kind");
    if (c->metric >= 0) return fail(c, RT_ESTATE, "the metric is already set");
    if (rt_status d = rt_check_device(c)) return d;
    if (kind == RT_KERR_SCHILD) {
        if (!params) return fail(c, RT_EINVAL, "Kerr-Schild needs {M, a}");
        c->M = params[0]; c->a = params[1];
        if (!(c->M >= 0.0) || !(std::fabs(c->a) <= c->M || c->M == 0.0)) return fail(c, RT_EINVAL, "need M >= 0, |a| <= M");
        c->metric = kind;
        return rt_build_geometry(c);
    }
    if (kind == RT_SNAKE) {
        if (!params) return fail(c, RT_EINVAL, "snake coordinates need {A, k}");
        c->M = params[0]; c->a = params[1];     // the geometry kernels take (A, k) in (M, a)
        c->metric = kind;
        return rt_build_geometry(c);
    }
    if (kind == RT_CART_CYLTETRAD) {
        const rt_config &f = c->cfg;
        // the cylindrical frame is undefined on the axis: no cell, ghost cell
        // or face of the geometry table may reach it
        auto spans0 = [&](int a) { return f.x0[a] - 2.0 * f.dx[a] <= 0.0 && f.x0[a] + (f.nx[a] + 2) * f.dx[a] >= 0.0; };
        if (spans0(0) && spans0(1))
            return fail(c, RT_EINVAL, "the cylindrical tetrad needs a box away from the axis x = y = 0");
        c->metric = kind;
        return rt_build_geometry(c);
    }
    c->metric = kind;
    c->gn[0] = c->cfg.nx[0] + (c->active[0] ? 4 : 0);
    c->gn[1] = c->cfg.nx[1] + (c->active[1] ? 4 : 0);
    return RT_OK;
}

extern "C" rt_status rt_set_fluid(rt_ctx *c, const double *rho, const double *u_gas, const double *ucon,
                                  const double *kappa, const double *alpha_s_coef, const double *eta) {
    if (!c) return RT_EINVAL;
    if (c->metric < 0) return fail(c, RT_ESTATE, "rt_set_metric must precede rt_set_fluid");
    if (!rho || !u_gas || !ucon || !kappa || !alpha_s_coef) return fail(c, RT_EINVAL, "null fluid array");
    if (rt_status d = rt_check_device(c)) return d;
    c->rec_id = 0;   // a forward recording belongs to the fluid it ran with
    c->halo_fluid = false;
    size_t n = (size_t)c->ncell * 8;
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->rho, rho, n, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->ug[0], u_gas, n, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->ucon, ucon, 4 * n, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->kap, kappa, n, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->cs, alpha_s_coef, n, cudaMemcpyDefault, c->stream));
    if (eta) RT_CUDA_TRY(c, cudaMemcpyAsync(c->eta, eta, n, cudaMemcpyDefault, c->stream));
    else {
        std::vector<double> ones(c->ncell, 1.0);
        RT_CUDA_TRY(c, cudaMemcpyAsync(c->eta, ones.data(), n, cudaMemcpyHostToDevice, c->stream));
        RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    rt_status st = rt_compute_uhat(c);
    if (st != RT_OK) return st;
    st = rt_launch_cellconst(c);
    if (st != RT_OK) return st;
    {
        int *d = nullptr, h = 0;
        RT_CUDA_TRY(c, cudaMalloc(&d, sizeof(int)));
        cudaMemsetAsync(d, 0, sizeof(int), c->stream);
        k_moving<<<(c->ncell + 255) / 256, 256, 0, c->stream>>>(c->ncell, c->uhat, d);
        cudaError_t e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(d);
        if (e != cudaSuccess) { c->err = std::string("rt_set_fluid: ") + cudaGetErrorString(e); return RT_ECUDA; }
        c->static_fluid = (h == 0) && c->metric == RT_MINKOWSKI_CART;
    }
    st = rt_launch_alpha(c, c->ug[0], c->alpha[0]);
    if (st != RT_OK) return st;
    c->have_fluid = true;
    return RT_OK;
}

extern "C" rt_status rt_set_intensity(rt_ctx *c, const void *I) {
    if (!c || !I) return RT_EINVAL;
    if (rt_status d = rt_check_device(c)) return d;
    // no interaction has acted on the new state yet: its force on the gas is
    // zero (a deferred G of the replaced state is dropped, not computed)
    c->g_lazy = false;
    RT_CUDA_TRY(c, cudaMemsetAsync(c->G, 0, (size_t)c->ncell * 32, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->I[0], I, (size_t)c->ncell * c->nd * c->esize, cudaMemcpyDefault, c->stream));
    c->have_I = true;
    return RT_OK;
}

static bool is_host(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return true; }
    return at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged;
}

extern "C" rt_status rt_get_intensity(rt_ctx *c, void *I) {
    if (!c || !I) return RT_EINVAL;
    if (!c->have_I) return fail(c, RT_ESTATE, "no intensity set");
    if (rt_status d = rt_check_device(c)) return d;
    RT_CUDA_TRY(c, cudaMemcpyAsync(I, c->I[0], (size_t)c->ncell * c->nd * c->esize, cudaMemcpyDefault, c->stream));
    if (is_host(I)) RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RT_OK;
}

extern "C" rt_status rt_set_ugas(rt_ctx *c, const double *u_gas) {
    if (!c || !u_gas) return RT_EINVAL;
    if (!c->have_fluid) return fail(c, RT_ESTATE, "rt_set_fluid must precede rt_set_ugas");
    if (rt_status d = rt_check_device(c)) return d;
    RT_CUDA_TRY(c, cudaMemcpyAsync(c->ug[0], u_gas, (size_t)c->ncell * 8, cudaMemcpyDefault, c->stream));
    return rt_launch_alpha(c, c->ug[0], c->alpha[0]);
}

extern "C" rt_status rt_get_ugas(rt_ctx *c, double *u_gas) {
    if (!c || !u_gas) return RT_EINVAL;
    if (!c->have_fluid) return fail(c, RT_ESTATE, "no fluid set");
    if (rt_status d = rt_check_device(c)) return d;
    RT_CUDA_TRY(c, cudaMemcpyAsync(u_gas, c->ug[0], (size_t)c->ncell * 8, cudaMemcpyDefault, c->stream));
    if (is_host(u_gas)) RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RT_OK;
}

extern "C" rt_status rt_cfl_dt(rt_ctx *c, double cfl, double *dt) {
    if (!c || !dt || !(cfl > 0.0)) return RT_EINVAL;
    if (c->metric < 0) return fail(c, RT_ESTATE, "rt_set_metric must precede rt_cfl_dt");
    if (rt_status d = rt_check_device(c)) return d;
    double m;
    rt_status st = rt_launch_cfl(c, &m);
    if (st != RT_OK) return st;
    *dt = cfl * m;
    return RT_OK;
}

// stage launch, bracketed by an event pair when timing is on
static rt_status timed_stage(rt_ctx *c, const void *Isrc, const void *Ibase, void *Iout, const double *ug_in,
                             double *ug_out, const double *a_in, const double *a_int, double *a_out, double dtk,
                             double *G) {
    if (!c->timing) return rt_launch_stage(c, Isrc, Ibase, Iout, ug_in, ug_out, a_in, a_int, a_out, dtk, G);
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t a, b;
        RT_CUDA_TRY(c, cudaEventCreate(&a));
        RT_CUDA_TRY(c, cudaEventCreate(&b));
        c->ev.push_back({a, b});
    }
    auto &pr = c->ev[c->ev_used++];
    RT_CUDA_TRY(c, cudaEventRecord(pr.first, c->stream));
    rt_status st = rt_launch_stage(c, Isrc, Ibase, Iout, ug_in, ug_out, a_in, a_int, a_out, dtk, G);
    RT_CUDA_TRY(c, cudaEventRecord(pr.second, c->stream));
    return st;
}

extern "C" rt_status rt_set_timing(rt_ctx *c, int on) {
    if (!c) return RT_EINVAL;
    c->timing = on != 0;
    c->ev_used = 0;
    return RT_OK;
}

extern "C" rt_status rt_get_timing(rt_ctx *c, double *ms, long long *launches) {
    if (!c) return RT_EINVAL;
    RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    for (size_t q = 0; q < c->ev_used; ++q) {
        float m = 0.0f;
        RT_CUDA_TRY(c, cudaEventElapsedTime(&m, c->ev[q].first, c->ev[q].second));
        tot += m;
    }
    if (ms) *ms = tot;
    if (launches) *launches = (long long)c->ev_used;
    c->ev_used = 0;
    return RT_OK;
}

extern "C" rt_status rt_step(rt_ctx *c, double dt, int nsteps, double *dt_used, long long *n_fail) {
    if (!c || nsteps < 0) return RT_EINVAL;
    if (c->metric < 0 || !c->have_fluid || !c->have_I) return fail(c, RT_ESTATE, "metric, fluid and intensity must be set");
    if (c->halo) return fail(c, RT_EINVAL, "a context with x3 halo faces steps by rt_step_stage, exchanging halos between stages");
    if (c->next_stage != 0) return fail(c, RT_ESTATE, "rt_step: a step begun by rt_step_stage is not finished");
    if (rt_status d = rt_check_device(c)) return d;
    if (!(dt > 0.0)) {
        if (c->dt_cfl <= 0.0) {
            rt_status st = rt_cfl_dt(c, 0.4, &c->dt_cfl);
            if (st != RT_OK) return st;
        }
        dt = c->dt_cfl;
    }
    if (dt_used) *dt_used = dt;
    if (n_fail) RT_CUDA_TRY(c, cudaMemsetAsync(c->fail, 0, sizeof(unsigned long long), c->stream));
    for (int n = 0; n < nsteps; ++n) {
        rt_status st;
        if (c->cfg.order == 1) {
            st = timed_stage(c, c->I[0], c->I[0], c->I[2], c->ug[0], c->ug[2], c->alpha[0], c->alpha[0], c->alpha[1],
                             dt, c->G);
            if (st != RT_OK) return st;
            std::swap(c->alpha[0], c->alpha[1]);
        } else {
            // predictor: fluxes and interaction from (I^n, u_g^n)
            st = timed_stage(c, c->I[0], c->I[0], c->I[1], c->ug[0], c->ug[1], c->alpha[0], c->alpha[0], c->alpha[1],
                             0.5 * dt, nullptr);
            if (st != RT_OK) return st;
            // corrector: fluxes from (I*, u_g*), base I^n, interaction from u_g^n;
            // alpha(u_g^n) is read and overwritten cell by cell by the same CTA
            st = timed_stage(c, c->I[1], c->I[0], c->I[2], c->ug[0], c->ug[2], c->alpha[1], c->alpha[0], c->alpha[0],
                             dt, c->G);
            if (st != RT_OK) return st;
        }
        std::swap(c->I[0], c->I[2]);
        std::swap(c->ug[0], c->ug[2]);
    }
    if (n_fail) {
        unsigned long long h = 0;
        RT_CUDA_TRY(c, cudaMemcpyAsync(&h, c->fail, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        *n_fail = (long long)h;
        if (h) return fail(c, RT_ENOCONV, "temperature solve did not converge in some cells");
    }
    return RT_OK;
}

extern "C" rt_status rt_moments(rt_ctx *c, double *R, double *Ebar, double *G) {
    if (!c) return RT_EINVAL;
    if (!c->have_fluid || !c->have_I) return fail(c, RT_ESTATE, "fluid and intensity must be set");
    if (rt_status d = rt_check_device(c)) return d;
    size_t nc = (size_t)c->ncell;
    bool hostR = R && is_host(R), hostE = Ebar && is_host(Ebar);
    double *dR = R, *dE = Ebar;
    if (hostR) RT_CUDA_TRY(c, cudaMalloc(&dR, nc * 80));
    if (hostE) RT_CUDA_TRY(c, cudaMalloc(&dE, nc * 8));
    rt_status st = G && c->g_lazy ? rt_resolve_g(c) : RT_OK;
    if (st == RT_OK) st = rt_launch_moments(c, dR, dE);
    if (st == RT_OK && hostR) RT_CUDA_TRY(c, cudaMemcpyAsync(R, dR, nc * 80, cudaMemcpyDeviceToHost, c->stream));
    if (st == RT_OK && hostE) RT_CUDA_TRY(c, cudaMemcpyAsync(Ebar, dE, nc * 8, cudaMemcpyDeviceToHost, c->stream));
    if (G) RT_CUDA_TRY(c, cudaMemcpyAsync(G, c->G, nc * 32, cudaMemcpyDefault, c->stream));
    if (hostR || hostE || (G && is_host(G))) RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (hostR) cudaFree(dR);
    if (hostE) cudaFree(dE);
    return st;
}

// ---------------------------------------------------------------- x3 slabs
// (spatial domain decomposition: the caller exchanges two ghost planes per
// side between the stages of rt_step_stage; see include/rt.h)

// the stage source of `stage`: intensities and flux opacity
static void stage_source(rt_ctx *c, int stage, void **I, double **alpha) {
    const int q = (c->cfg.order == 2 && stage == 1) ? 1 : 0;
    *I = c->I[q];
    *alpha = c->alpha[q];
}

extern "C" rt_status rt_halo_bytes(const rt_ctx *c, size_t *bytes) {
    if (!c || !bytes) return RT_EINVAL;
    const size_t P = (size_t)c->cfg.nx[0] * c->cfg.nx[1];
    *bytes = c->halo ? 2 * P * c->nd * c->esize + P * 8 : 0;
    return RT_OK;
}

extern "C" rt_status rt_halo_pack(rt_ctx *c, int stage, void *lo, void *hi) {
    if (!c || !lo || !hi) return RT_EINVAL;
    if (!c->halo) return fail(c, RT_EINVAL, "rt_halo_pack: the context has no x3 halo face");
    if (stage < 0 || stage > (c->cfg.order == 2 ? 1 : 0)) return fail(c, RT_EINVAL, "rt_halo_pack: no such stage");
    if (stage != c->next_stage) return fail(c, RT_ESTATE, "rt_halo_pack: the halo of the next stage only");
    if (rt_status d = rt_check_device(c)) return d;
    void *I; double *al;
    stage_source(c, stage, &I, &al);
    const size_t P = (size_t)c->cfg.nx[0] * c->cfg.nx[1], bI = 2 * P * c->nd * c->esize;
    const size_t last = (size_t)c->ncell - 2 * P;
    char *dl = (char *)lo, *dh = (char *)hi;
    RT_CUDA_TRY(c, cudaMemcpyAsync(dl, I, bI, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(dl + bI, al, P * 8, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(dh, (char *)I + last * c->nd * c->esize, bI, cudaMemcpyDefault, c->stream));
    RT_CUDA_TRY(c, cudaMemcpyAsync(dh + bI, al + (size_t)c->ncell - P, P * 8, cudaMemcpyDefault, c->stream));
    return RT_OK;
}

extern "C" rt_status rt_halo_unpack(rt_ctx *c, int stage, const void *lo, const void *hi) {
    if (!c) return RT_EINVAL;
    if (!c->halo) return fail(c, RT_EINVAL, "rt_halo_unpack: the context has no x3 halo face");
    if (stage < 0 || stage > (c->cfg.order == 2 ? 1 : 0)) return fail(c, RT_EINVAL, "rt_halo_unpack: no such stage");
    if (stage != c->next_stage) return fail(c, RT_ESTATE, "rt_halo_unpack: the halo of the next stage only");
    if (rt_status d = rt_check_device(c)) return d;
    void *I; double *al;
    stage_source(c, stage, &I, &al);
    const size_t P = (size_t)c->cfg.nx[0] * c->cfg.nx[1], bI = 2 * P * c->nd * c->esize;
    const char *sl = (const char *)lo, *sh = (const char *)hi;
    // a side whose x3 face is the box's own boundary takes no ghost planes
    if (c->cfg.bc[2][0] == RT_BC_HALO) {
        if (!lo) return fail(c, RT_EINVAL, "rt_halo_unpack: null lower halo");
        RT_CUDA_TRY(c, cudaMemcpyAsync((char *)I - bI, sl, bI, cudaMemcpyDefault, c->stream));
        RT_CUDA_TRY(c, cudaMemcpyAsync(al - P, sl + bI, P * 8, cudaMemcpyDefault, c->stream));
    }
    if (c->cfg.bc[2][1] == RT_BC_HALO) {
        if (!hi) return fail(c, RT_EINVAL, "rt_halo_unpack: null upper halo");
        RT_CUDA_TRY(c, cudaMemcpyAsync((char *)I + (size_t)c->ncell * c->nd * c->esize, sh, bI, cudaMemcpyDefault,
                                       c->stream));
        RT_CUDA_TRY(c, cudaMemcpyAsync(al + c->ncell, sh + bI, P * 8, cudaMemcpyDefault, c->stream));
    }
    return RT_OK;
}

extern "C" rt_status rt_set_fluid_halo(rt_ctx *c, const double *lo, const double *hi) {
    if (!c) return RT_EINVAL;
    if (!c->halo) return fail(c, RT_EINVAL, "rt_set_fluid_halo: the context has no x3 halo face");
    if (!c->have_fluid) return fail(c, RT_ESTATE, "rt_set_fluid must precede rt_set_fluid_halo");
    if (rt_status d = rt_check_device(c)) return d;
    const size_t P2 = c->hcells;
    const double *src[2] = {lo, hi};
    std::vector<double> h(7 * P2), v(3 * P2);
    for (int sd = 0; sd < 2; ++sd) {
        if (c->cfg.bc[2][sd] != RT_BC_HALO) continue;
        if (!src[sd]) return fail(c, RT_EINVAL, "rt_set_fluid_halo: null halo fluid");
        RT_CUDA_TRY(c, cudaMemcpyAsync(h.data(), src[sd], 7 * P2 * 8, cudaMemcpyDefault, c->stream));
        RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (size_t q = 0; q < P2; ++q)
            for (int a = 0; a < 3; ++a) v[3 * q + a] = h[7 * q + 4 + a] / h[7 * q + 3];
        double *dst = sd == 0 ? c->vel - 3 * P2 : c->vel + 3 * (size_t)c->ncell;
        RT_CUDA_TRY(c, cudaMemcpyAsync(dst, v.data(), 3 * P2 * 8, cudaMemcpyHostToDevice, c->stream));
        RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    c->halo_fluid = true;
    return RT_OK;
}

extern "C" rt_status rt_step_stage(rt_ctx *c, double dt, int stage, long long *n_fail) {
    if (!c) return RT_EINVAL;
    if (c->metric < 0 || !c->have_fluid || !c->have_I) return fail(c, RT_ESTATE, "metric, fluid and intensity must be set");
    if (rt_status d = rt_check_device(c)) return d;
    const int last = c->cfg.order == 2 ? 1 : 0;
    if (stage < 0 || stage > last || stage != c->next_stage) return fail(c, RT_ESTATE, "rt_step_stage: stage out of order");
    if (c->halo && !c->static_fluid && !c->halo_fluid)
        return fail(c, RT_ESTATE, "a moving fluid needs rt_set_fluid_halo before rt_step_stage");
    if (!(dt > 0.0)) {
        if (c->dt_cfl <= 0.0) {
            rt_status st = rt_cfl_dt(c, 0.4, &c->dt_cfl);
            if (st != RT_OK) return st;
        }
        dt = c->dt_cfl;
    }
    if (n_fail) RT_CUDA_TRY(c, cudaMemsetAsync(c->fail, 0, sizeof(unsigned long long), c->stream));
    rt_status st;
    if (last == 0) {
        st = timed_stage(c, c->I[0], c->I[0], c->I[2], c->ug[0], c->ug[2], c->alpha[0], c->alpha[0], c->alpha[1], dt, c->G);
        if (st != RT_OK) return st;
        std::swap(c->alpha[0], c->alpha[1]);
    } else if (stage == 0) {
        st = timed_stage(c, c->I[0], c->I[0], c->I[1], c->ug[0], c->ug[1], c->alpha[0], c->alpha[0], c->alpha[1],
                         0.5 * dt, nullptr);
        if (st != RT_OK) return st;
    } else {
        st = timed_stage(c, c->I[1], c->I[0], c->I[2], c->ug[0], c->ug[2], c->alpha[1], c->alpha[0], c->alpha[0], dt, c->G);
        if (st != RT_OK) return st;
    }
    if (stage == last) {
        std::swap(c->I[0], c->I[2]);
        std::swap(c->ug[0], c->ug[2]);
        c->next_stage = 0;
    } else {
        c->next_stage = stage + 1;
    }
    if (n_fail) {
        unsigned long long h = 0;
        RT_CUDA_TRY(c, cudaMemcpyAsync(&h, c->fail, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        RT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        *n_fail = (long long)h;
        if (h) return fail(c, RT_ENOCONV, "temperature solve did not converge in some cells");
    }
    return RT_OK;
}
