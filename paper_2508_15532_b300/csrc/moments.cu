// moments.cu — radiation moments (eq. R) and the light-crossing time-step bound.
#include "rt_internal.cuh"
#include <cstring>
#include <mutex>

namespace {

template <typename TS> __device__ __forceinline__ double ldd(const void *p, size_t i);
template <> __device__ __forceinline__ double ldd<double>(const void *p, size_t i) { return ((const double *)p)[i]; }
template <> __device__ __forceinline__ double ldd<float>(const void *p, size_t i) { return ((const float *)p)[i]; }
template <> __device__ __forceinline__ double ldd<__nv_bfloat16>(const void *p, size_t i) {
    return __bfloat162float(((const __nv_bfloat16 *)p)[i]);
}

// one warp per cell: R^{mu nu} = sum_s n^mu n^nu I_s dOmega_s (coordinate
// components, n^mu = e^mu_(a) nhat^(a)) and E-bar = sum_s D_s^2 I_s dOmega_s
template <typename TS>
__global__ void k_moments(int ncell, int nd, int nx0, int nx1, int gn0, int ng0, int ng1, int flat,
                          const void *__restrict__ I, const double *__restrict__ dir, const double *__restrict__ w,
                          const double *__restrict__ pe, const double *__restrict__ uhat, double *__restrict__ R,
                          double *__restrict__ Ebar) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= ncell) return;
    const int c = warp;
    double E[16];
    if (flat) {
        for (int q = 0; q < 16; ++q) E[q] = (q % 5 == 0) ? 1.0 : 0.0;
    } else {
        int i = c % nx0, j = (c / nx0) % nx1;
        const double *p = pe + 16 * (size_t)((j + ng1) * gn0 + (i + ng0));
        for (int q = 0; q < 16; ++q) E[q] = p[q];
    }
    const double *u = uhat + 4 * (size_t)c;
    double acc[11] = {0};
    for (int s = lane; s < nd; s += 32) {
        double nh[4] = {1.0, dir[3 * s], dir[3 * s + 1], dir[3 * s + 2]};
        double n[4];
        for (int m = 0; m < 4; ++m) n[m] = E[m] * nh[0] + E[4 + m] * nh[1] + E[8 + m] * nh[2] + E[12 + m] * nh[3];
        double Iw = ldd<TS>(I, (size_t)c * nd + s) * w[s];
        int q = 0;
        for (int m = 0; m < 4; ++m)
            for (int k = m; k < 4; ++k) acc[q++] += n[m] * n[k] * Iw;
        double D = u[0] - (u[1] * nh[1] + u[2] * nh[2] + u[3] * nh[3]);
        acc[10] += D * D * Iw;
    }
    for (int q = 0; q < 11; ++q)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0) {
        if (R) for (int q = 0; q < 10; ++q) R[10 * (size_t)c + q] = acc[q];
        if (Ebar) Ebar[c] = acc[10];
    }
}

// Force on the gas of an interaction of the packed FP32 stage kernel (flat
// geometry, fluid at rest), formed from its per-cell (a, c) and the state it
// left, I_+ = (I + c)/(1 + a): Delta R^{0 mu} = c sum_s n^mu dOmega_s
// - a sum_s n^mu I_+ dOmega_s, G = -Delta R^{0 mu} / dt (section 3.5.3).  One
// warp per cell, FP64 sums.
template <typename TS>
__global__ void k_gdefer(int ncell, int nd, const void *__restrict__ I, const double *__restrict__ dir,
                         const double *__restrict__ w, const float2 *__restrict__ gac, double sumw, double sn0,
                         double sn1, double sn2, double idt, double *__restrict__ G) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= ncell) return;
    const int c = warp;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = lane; s < nd; s += 32) {
        const double Iw = ldd<TS>(I, (size_t)c * nd + s) * w[s];
        acc[0] += Iw;
        for (int m = 0; m < 3; ++m) acc[1 + m] += dir[3 * s + m] * Iw;
    }
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0) {
        const double a = gac[c].x, cc = gac[c].y;
        const double sn[4] = {sumw, sn0, sn1, sn2};
        for (int m = 0; m < 4; ++m) G[4 * (size_t)c + m] = -(cc * sn[m] - a * acc[m]) * idt;
    }
}

// minimum over cells (pole-zeroed rows excluded), active axes and directions
// of dx^a n^0 / |n^a|; positive doubles order like their bit patterns
__global__ void k_cfl(int nx0, int nx1, int nd, int gn0, int ng0, int ng1, int flat, int npole, int a0, int a1,
                      int a2, double dx0, double dx1, double dx2, const double *__restrict__ dir,
                      const double *__restrict__ pe, unsigned long long *__restrict__ out) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t npts = flat ? 1 : (size_t)nx0 * nx1;
    if (idx >= npts * nd) return;
    int s = (int)(idx % nd);
    int p = (int)(idx / nd);
    int i = p % nx0, j = p / nx0;
    if (!flat && npole > 0 && (j < npole || j >= nx1 - npole)) return;
    double E[16];
    if (flat) for (int q = 0; q < 16; ++q) E[q] = (q % 5 == 0) ? 1.0 : 0.0;
    else {
        const double *pp = pe + 16 * (size_t)((j + ng1) * gn0 + (i + ng0));
        for (int q = 0; q < 16; ++q) E[q] = pp[q];
    }
    double nh[4] = {1.0, dir[3 * s], dir[3 * s + 1], dir[3 * s + 2]};
    double n[4];
    for (int m = 0; m < 4; ++m) n[m] = E[m] * nh[0] + E[4 + m] * nh[1] + E[8 + m] * nh[2] + E[12 + m] * nh[3];
    double best = 1e300;
    double dxs[3] = {dx0, dx1, dx2};
    int act[3] = {a0, a1, a2};
    for (int a = 0; a < 3; ++a) {
        if (!act[a] || n[a + 1] == 0.0) continue;
        double t = dxs[a] * n[0] / fabs(n[a + 1]);
        best = fmin(best, t);
    }
    atomicMin(out, (unsigned long long)__double_as_longlong(best));
}

}  // namespace

rt_status rt_launch_moments(rt_ctx *c, double *R, double *Ebar) {
    int ng0 = c->active[0] ? 2 : 0, ng1 = c->active[1] ? 2 : 0;
    int flat = c->metric == RT_MINKOWSKI_CART;
    unsigned blocks = (unsigned)(((size_t)c->ncell * 32 + 255) / 256);
    auto P = c->cfg.precision;
    if (P == RT_FP64)
        k_moments<double><<<blocks, 256, 0, c->stream>>>(c->ncell, c->nd, c->cfg.nx[0], c->cfg.nx[1], c->gn[0], ng0, ng1,
                                                         flat, c->I[0], c->g->dir, c->g->w, c->pt_e, c->uhat, R, Ebar);
    else if (P == RT_FP32)
        k_moments<float><<<blocks, 256, 0, c->stream>>>(c->ncell, c->nd, c->cfg.nx[0], c->cfg.nx[1], c->gn[0], ng0, ng1,
                                                        flat, c->I[0], c->g->dir, c->g->w, c->pt_e, c->uhat, R, Ebar);
    else
        k_moments<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>(c->ncell, c->nd, c->cfg.nx[0], c->cfg.nx[1], c->gn[0],
                                                                ng0, ng1, flat, c->I[0], c->g->dir, c->g->w, c->pt_e,
                                                                c->uhat, R, Ebar);
    RT_CUDA_TRY(c, cudaGetLastError());
    return RT_OK;
}

rt_status rt_resolve_g(rt_ctx *c) {
    if (!c->g_lazy) return RT_OK;
    unsigned blocks = (unsigned)(((size_t)c->ncell * 32 + 255) / 256);
    const double idt = 1.0 / c->g_dt;
    if (c->cfg.precision == RT_FP32)
        k_gdefer<float><<<blocks, 256, 0, c->stream>>>(c->ncell, c->nd, c->I[0], c->g->dir, c->g->w, c->gac, c->sumw,
                                                       c->sumnw[0], c->sumnw[1], c->sumnw[2], idt, c->G);
    else
        k_gdefer<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>(c->ncell, c->nd, c->I[0], c->g->dir, c->g->w, c->gac,
                                                               c->sumw, c->sumnw[0], c->sumnw[1], c->sumnw[2], idt, c->G);
    RT_CUDA_TRY(c, cudaGetLastError());
    c->g_lazy = false;
    return RT_OK;
}

rt_status rt_launch_cfl(rt_ctx *c, double *dt_min_host) {
    unsigned long long *d = nullptr;
    RT_CUDA_TRY(c, cudaMalloc(&d, sizeof(unsigned long long)));
    double big = 1e300;
    unsigned long long bits;
    memcpy(&bits, &big, sizeof(bits));
    cudaMemcpyAsync(d, &bits, sizeof(bits), cudaMemcpyHostToDevice, c->stream);
    int flat = c->metric == RT_MINKOWSKI_CART;
    size_t n = (flat ? 1 : (size_t)c->cfg.nx[0] * c->cfg.nx[1]) * c->nd;
    int ng0 = c->active[0] ? 2 : 0, ng1 = c->active[1] ? 2 : 0;
    k_cfl<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->cfg.nx[0], c->cfg.nx[1], c->nd, c->gn[0], ng0, ng1, flat,
                                                              c->cfg.n_pole_zero, c->active[0], c->active[1],
                                                              c->active[2], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2],
                                                              c->g->dir, c->pt_e, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) { c->err = std::string("cfl: ") + cudaGetErrorString(e); return RT_ECUDA; }
    memcpy(dt_min_host, &bits, sizeof(bits));
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free time-step bound.
//
// rt_cfl_dt obtains its 8-byte reduction word with cudaMalloc on every call.
// Some callers cannot allocate device memory between steps: a host code whose
// memory manager owns the whole device (a caching allocator or a fixed pool,
// where a raw cudaMalloc can fail or fragment it), or a time loop that must
// not stall other streams (cudaFree synchronises the device).  For them the
// same minimum is taken in two passes over a file-scope scratch array: each
// block of CFL_NA_THREADS threads reduces CFL_NA_ITEMS (point, direction)
// items to one partial minimum, and one block reduces the partials.  Every
// slot that is read was written earlier in the same call, so nothing has to
// be cleared between calls.
namespace {

constexpr int CFL_NA_THREADS = 256;
constexpr int CFL_NA_ITEMS = CFL_NA_THREADS * 8;
constexpr int CFL_NA_MAX_BLOCKS = 8192;   // 64 KB of partials + the result

// partial minima [0, CFL_NA_MAX_BLOCKS) and the result at CFL_NA_MAX_BLOCKS;
// every GPU that loads this library holds it until the process exits
static __device__ __align__(256) double cfl_na_scratch[CFL_NA_MAX_BLOCKS + 1];

// dx^a n^0 / |n^a| minimised over active axes for one (point, direction)
// item; the pole-zeroed rows give +1e300 (the same quantity as k_cfl)
__device__ double cfl_na_item(size_t idx, int nx0, int nx1, int nd, int gn0, int ng0, int ng1, int flat, int npole,
                              const int act[3], const double dxs[3], const double *__restrict__ dir,
                              const double *__restrict__ pe) {
    int s = (int)(idx % nd);
    int p = (int)(idx / nd);
    int i = p % nx0, j = p / nx0;
    if (!flat && npole > 0 && (j < npole || j >= nx1 - npole)) return 1e300;
    double E[16];
    if (flat) for (int q = 0; q < 16; ++q) E[q] = (q % 5 == 0) ? 1.0 : 0.0;
    else {
        const double *pp = pe + 16 * (size_t)((j + ng1) * gn0 + (i + ng0));
        for (int q = 0; q < 16; ++q) E[q] = pp[q];
    }
    double nh[4] = {1.0, dir[3 * s], dir[3 * s + 1], dir[3 * s + 2]};
    double n[4];
    for (int m = 0; m < 4; ++m) n[m] = E[m] * nh[0] + E[4 + m] * nh[1] + E[8 + m] * nh[2] + E[12 + m] * nh[3];
    double best = 1e300;
    for (int a = 0; a < 3; ++a) {
        if (!act[a] || n[a + 1] == 0.0) continue;
        best = fmin(best, dxs[a] * n[0] / fabs(n[a + 1]));
    }
    return best;
}

__device__ double cfl_na_block_min(double v) {
    __shared__ double wmin[CFL_NA_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < CFL_NA_THREADS / 32 ? wmin[threadIdx.x] : 1e300;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(CFL_NA_THREADS)
k_cfl_na_part(size_t nitem, int nx0, int nx1, int nd, int gn0, int ng0, int ng1, int flat, int npole, int a0, int a1,
              int a2, double dx0, double dx1, double dx2, const double *__restrict__ dir,
              const double *__restrict__ pe, double *__restrict__ scratch) {
    const int act[3] = {a0, a1, a2};
    const double dxs[3] = {dx0, dx1, dx2};
    double v = 1e300;
    size_t base = (size_t)blockIdx.x * CFL_NA_ITEMS;
    for (int k = threadIdx.x; k < CFL_NA_ITEMS; k += CFL_NA_THREADS) {
        size_t idx = base + k;
        if (idx < nitem) v = fmin(v, cfl_na_item(idx, nx0, nx1, nd, gn0, ng0, ng1, flat, npole, act, dxs, dir, pe));
    }
    v = cfl_na_block_min(v);
    if (threadIdx.x == 0) scratch[blockIdx.x] = v;
}

__global__ void __launch_bounds__(CFL_NA_THREADS) k_cfl_na_final(int nblk, double *__restrict__ scratch) {
    double v = 1e300;
    for (int b = threadIdx.x; b < nblk; b += CFL_NA_THREADS) v = fmin(v, scratch[b]);
    v = cfl_na_block_min(v);
    if (threadIdx.x == 0) scratch[CFL_NA_MAX_BLOCKS] = v;
}

// device address of cfl_na_scratch, looked up once per device
constexpr int CFL_NA_MAX_DEVICES = 64;
std::mutex cfl_na_mutex;
double *cfl_na_ptr[CFL_NA_MAX_DEVICES] = {};

}  // namespace

extern "C" rt_status rt_cfl_dt_noalloc(rt_ctx *c, double cfl, double *dt) {
    if (!c || !dt || !(cfl > 0.0)) return RT_EINVAL;
    if (c->metric < 0) {
        c->err = "rt_set_metric must precede rt_cfl_dt_noalloc";
        return RT_ESTATE;
    }
    int flat = c->metric == RT_MINKOWSKI_CART;
    size_t nitem = (flat ? 1 : (size_t)c->cfg.nx[0] * c->cfg.nx[1]) * c->nd;
    size_t nblk = (nitem + CFL_NA_ITEMS - 1) / CFL_NA_ITEMS;
    if (nblk > (size_t)CFL_NA_MAX_BLOCKS) {
        c->err = "rt_cfl_dt_noalloc: " + std::to_string(nitem) + " (point, direction) items exceed the static scratch "
                 "limit of " + std::to_string((size_t)CFL_NA_MAX_BLOCKS * CFL_NA_ITEMS) + "; use rt_cfl_dt";
        return RT_EINVAL;
    }
    if (rt_status d = rt_check_device(c)) return d;
    const int dev = c->device;
    if (dev < 0 || dev >= CFL_NA_MAX_DEVICES) {
        c->err = "rt_cfl_dt_noalloc: device ordinal beyond " + std::to_string(CFL_NA_MAX_DEVICES);
        return RT_EINVAL;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(cfl_na_mutex);
        if (!cfl_na_ptr[dev]) {
            // first call on this device (with it current): resolve the array's
            // device address; the host-side name is only a stand-in
            cudaError_t e = cudaGetSymbolAddress((void **)&cfl_na_ptr[dev], cfl_na_scratch);
            if (e != cudaSuccess) {
                cfl_na_ptr[dev] = nullptr;
                c->err = std::string("rt_cfl_dt_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return RT_ECUDA;
            }
        }
        scratch = cfl_na_ptr[dev];
    }
    int ng0 = c->active[0] ? 2 : 0, ng1 = c->active[1] ? 2 : 0;
    k_cfl_na_part<<<(unsigned)nblk, CFL_NA_THREADS, 0, c->stream>>>(
        nitem, c->cfg.nx[0], c->cfg.nx[1], c->nd, c->gn[0], ng0, ng1, flat, c->cfg.n_pole_zero, c->active[0],
        c->active[1], c->active[2], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2], c->g->dir, c->pt_e, scratch);
    k_cfl_na_final<<<1, CFL_NA_THREADS, 0, c->stream>>>((int)nblk, scratch);
    double m = 0.0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, scratch + CFL_NA_MAX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("rt_cfl_dt_noalloc: ") + cudaGetErrorString(e);
        return RT_ECUDA;
    }
    *dt = cfl * m;
    return RT_OK;
}
