// grid.cu — geodesic angular grid (section 3.3): host topology, device geometry.
//
// Host: the icosahedron (vertices at the cyclic permutations of (0, +-1, +-phi)),
// log2(n) rounds of edge bisection with projection to the unit sphere, the
// canonical direction order, and neighbour rings ordered counter-clockwise by
// their angle in the tangent plane (first slot: smallest neighbour index).
// Device (one thread per direction, FP64): Voronoi vertices (circumcentres of
// the Delaunay triangles), cell solid angles, Voronoi edge lengths, midpoints
// and normals, and the tables of the minimum-angle plane reconstruction.
#include "rt_internal.cuh"
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <set>

namespace {

using V3 = std::array<double, 3>;

V3 unit(const V3 &a) {
    double r = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    return {a[0] / r, a[1] / r, a[2] / r};
}

double sq(const V3 &a, const V3 &b) {
    double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
    return x * x + y * y + z * z;
}

// order key of the canonical direction order
struct DirKey {
    long long zkey;
    double phi;
    bool operator<(const DirKey &o) const { return zkey != o.zkey ? zkey < o.zkey : phi < o.phi; }
};
DirKey key_of(const V3 &p) {
    auto snap = [](double v) { return std::fabs(v) < 1e-12 ? 0.0 : v; };
    return {std::llround(-p[2] * 1e9), std::atan2(snap(p[1]), snap(p[0]))};
}

}  // namespace

// ---------------------------------------------------------------- device part
__device__ inline void d_cross(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ inline double d_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ inline void d_unit(double *a) {
    double r = sqrt(d_dot(a, a));
    a[0] /= r; a[1] /= r; a[2] /= r;
}

// solid angle of the spherical triangle (a, b, c), counter-clockwise positive
__device__ inline double d_tri_area(const double *a, const double *b, const double *c) {
    double bc[3];
    d_cross(b, c, bc);
    return 2.0 * atan2(d_dot(a, bc), 1.0 + d_dot(a, b) + d_dot(b, c) + d_dot(c, a));
}

__global__ void k_grid_geometry(int nd, const double *__restrict__ dir, const int *__restrict__ nnb,
                                const int *__restrict__ nbr, const int *__restrict__ ring_edge,
                                double *__restrict__ w, double *__restrict__ emid, double *__restrict__ eu,
                                double *__restrict__ dlam, double *__restrict__ mx, double *__restrict__ mg,
                                double *__restrict__ mm) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nd) return;
    const double *ns = dir + 3 * s;
    int k = nnb[s];
    double V[RT_MAXNB][3];
    // Voronoi vertex between ring slots q and q+1: circumcentre of (s, q, q+1)
    for (int q = 0; q < k; ++q) {
        const double *p = dir + 3 * nbr[6 * s + q];
        const double *r = dir + 3 * nbr[6 * s + (q + 1) % k];
        double a[3] = {p[0] - ns[0], p[1] - ns[1], p[2] - ns[2]};
        double b[3] = {r[0] - ns[0], r[1] - ns[1], r[2] - ns[2]};
        d_cross(a, b, V[q]);
        d_unit(V[q]);
    }
    // polygon area as a fan from its first vertex
    double area = 0.0;
    for (int q = 1; q + 1 < k; ++q) area += d_tri_area(V[0], V[q], V[q + 1]);
    w[s] = area;
    for (int q = 0; q < k; ++q) {
        const double *a = V[(q + k - 1) % k], *b = V[q];
        double mid[3] = {a[0] + b[0], a[1] + b[1], a[2] + b[2]};
        d_unit(mid);
        int t = nbr[6 * s + q];
        if (t > s) {   // the lower index owns the edge record
            int e = ring_edge[6 * s + q];
            double ab[3];
            d_cross(a, b, ab);
            dlam[e] = atan2(sqrt(d_dot(ab, ab)), d_dot(a, b));
            const double *nt = dir + 3 * t;
            double u[3] = {nt[0] - ns[0], nt[1] - ns[1], nt[2] - ns[2]};
            d_unit(u);
            for (int m = 0; m < 3; ++m) { emid[3 * e + m] = mid[m]; eu[3 * e + m] = u[m]; }
        }
        // gnomonic images in the tangent plane of s
        const double *nt = dir + 3 * t;
        double dt_ = d_dot(nt, ns), dm = d_dot(mid, ns);
        for (int m = 0; m < 3; ++m) {
            mx[(6 * s + q) * 3 + m] = nt[m] / dt_ - ns[m];
            mm[(6 * s + q) * 3 + m] = mid[m] / dm - ns[m];
        }
    }
    for (int q = 0; q < k; ++q) {
        const double *x0 = mx + (6 * s + q) * 3, *x1 = mx + (6 * s + (q + 1) % k) * 3;
        double g00 = d_dot(x0, x0), g01 = d_dot(x0, x1), g11 = d_dot(x1, x1);
        double det = g00 * g11 - g01 * g01;
        mg[(6 * s + q) * 3 + 0] = g11 / det;
        mg[(6 * s + q) * 3 + 1] = -g01 / det;
        mg[(6 * s + q) * 3 + 2] = g00 / det;
    }
}

// reconstruction weights of the minimum-angle planes: for direction s, pair
// (b, b+1) of its ring and edge midpoint q, the dot products of the pair's
// gnomonic neighbour images with the midpoint's image (zero outside the ring)
__global__ void k_mapr_dots(int nd, const int *__restrict__ nnb, const double *__restrict__ mx,
                            const double *__restrict__ mm, double *__restrict__ md) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 36 * nd) return;
    int s = t / 36, b = (t / 6) % 6, q = t % 6, kk = nnb[s];
    double d0 = 0.0, d1 = 0.0;
    if (b < kk && q < kk) {
        int b1 = b + 1 == kk ? 0 : b + 1;
        const double *x0 = mx + (size_t)(6 * s + b) * 3, *x1 = mx + (size_t)(6 * s + b1) * 3;
        const double *xm = mm + (size_t)(6 * s + q) * 3;
        d0 = x0[0] * xm[0] + x0[1] * xm[1] + x0[2] * xm[2];
        d1 = x1[0] * xm[0] + x1[1] * xm[1] + x1[2] * xm[2];
    }
    const size_t o = ((size_t)(b * 6 + q) * nd + s) * 2;
    md[o] = d0;
    md[o + 1] = d1;
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

static cudaError_t dalloc_copy(void **dst, const void *src, size_t bytes) {
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (src) return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return cudaMemset(*dst, 0, bytes);
}

rt_status rt_grid_device_geometry(rt_grid *g, std::string &err) {
    int nd = g->nd, ne = g->ne;
    cudaError_t e = cudaSuccess;
#define GA(p, src, bytes) if (e == cudaSuccess) e = dalloc_copy((void **)&(p), (src), (bytes))
    GA(g->dir, g->h_dir.data(), sizeof(double) * 3 * nd);
    GA(g->nnb, g->h_nnb.data(), sizeof(int) * nd);
    GA(g->nbr, g->h_nbr.data(), sizeof(int) * 6 * nd);
    GA(g->ring_edge, g->h_ring_edge.data(), sizeof(int) * 6 * nd);
    GA(g->ring_back, g->h_ring_back.data(), sizeof(int) * 6 * nd);
    GA(g->mirror, g->h_mirror.data(), sizeof(int) * nd);
    GA(g->edge, g->h_edge.data(), sizeof(int) * 2 * ne);
    GA(g->w, nullptr, sizeof(double) * nd);
    GA(g->emid, nullptr, sizeof(double) * 3 * ne);
    GA(g->eu, nullptr, sizeof(double) * 3 * ne);
    GA(g->dlam, nullptr, sizeof(double) * ne);
    GA(g->mx, nullptr, sizeof(double) * 18 * nd);
    GA(g->mg, nullptr, sizeof(double) * 18 * nd);
    GA(g->mm, nullptr, sizeof(double) * 18 * nd);
    GA(g->dirf, nullptr, sizeof(float) * 3 * nd);
    GA(g->wf, nullptr, sizeof(float) * nd);
    GA(g->mxf, nullptr, sizeof(float) * 18 * nd);
    GA(g->mgf, nullptr, sizeof(float) * 18 * nd);
    GA(g->mmf, nullptr, sizeof(float) * 18 * nd);
    GA(g->md, nullptr, sizeof(double) * 72 * nd);
    GA(g->mdf, nullptr, sizeof(float) * 72 * nd);
#undef GA
    if (e != cudaSuccess) { err = std::string("grid allocation: ") + cudaGetErrorString(e); return RT_ENOMEM; }
    k_grid_geometry<<<(nd + 127) / 128, 128>>>(nd, g->dir, g->nnb, g->nbr, g->ring_edge, g->w, g->emid, g->eu,
                                               g->dlam, g->mx, g->mg, g->mm);
    auto tof = [&](const double *a, float *b, size_t n) { k_to_float<<<(unsigned)((n + 255) / 256), 256>>>(a, b, n); };
    tof(g->dir, g->dirf, 3 * (size_t)nd); tof(g->w, g->wf, nd);
    k_mapr_dots<<<(36 * nd + 255) / 256, 256>>>(nd, g->nnb, g->mx, g->mm, g->md);
    tof(g->mx, g->mxf, 18 * (size_t)nd); tof(g->mg, g->mgf, 18 * (size_t)nd); tof(g->mm, g->mmf, 18 * (size_t)nd);
    tof(g->md, g->mdf, 72 * (size_t)nd);
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        g->h_w.resize(nd);
        e = cudaMemcpy(g->h_w.data(), g->w, sizeof(double) * nd, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) { err = std::string("grid geometry: ") + cudaGetErrorString(e); return RT_ECUDA; }
    return RT_OK;
}

static void free_grid(rt_grid *g) {
    if (!g) return;
    void *ptrs[] = {g->dir, g->w, g->nnb, g->nbr, g->ring_edge, g->ring_back, g->mirror, g->edge, g->emid,
                    g->eu, g->dlam, g->mx, g->mg, g->mm, g->dirf, g->wf, g->mxf, g->mgf, g->mmf, g->md, g->mdf};
    for (void *p : ptrs) if (p) cudaFree(p);
    delete g;
}

static thread_local std::string g_grid_err;

extern "C" rt_status rt_create_geodesic_grid(int n, rt_grid **out) {
    if (!out) return RT_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 32 || (n & (n - 1))) { g_grid_err = "n must be a power of two in [1, 32]"; return RT_EINVAL; }
    // icosahedron
    const double phi = 0.5 * (1.0 + std::sqrt(5.0));
    std::vector<V3> P;
    for (int c = 0; c < 3; ++c)
        for (double u : {-1.0, 1.0})
            for (double v : {-phi, phi}) {
                V3 p{0.0, 0.0, 0.0};
                p[(c + 1) % 3] = u; p[(c + 2) % 3] = v;
                P.push_back(p);
            }
    std::vector<std::array<int, 3>> T;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j)
            for (int k = j + 1; k < 12; ++k) {
                if (std::fabs(sq(P[i], P[j]) - 4.0) > 1e-9 || std::fabs(sq(P[j], P[k]) - 4.0) > 1e-9 ||
                    std::fabs(sq(P[i], P[k]) - 4.0) > 1e-9) continue;
                V3 a{P[j][0] - P[i][0], P[j][1] - P[i][1], P[j][2] - P[i][2]};
                V3 b{P[k][0] - P[i][0], P[k][1] - P[i][1], P[k][2] - P[i][2]};
                V3 cr{a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
                double out_ = cr[0] * P[i][0] + cr[1] * P[i][1] + cr[2] * P[i][2];
                if (out_ > 0) T.push_back({i, j, k}); else T.push_back({i, k, j});
            }
    for (auto &p : P) p = unit(p);
    for (int m = n; m > 1; m /= 2) {
        std::map<std::pair<int, int>, int> mid;
        auto midpoint = [&](int a, int b) {
            auto key = std::make_pair(std::min(a, b), std::max(a, b));
            auto it = mid.find(key);
            if (it != mid.end()) return it->second;
            V3 q{P[a][0] + P[b][0], P[a][1] + P[b][1], P[a][2] + P[b][2]};
            P.push_back(unit(q));
            int id = (int)P.size() - 1;
            mid[key] = id;
            return id;
        };
        std::vector<std::array<int, 3>> T2;
        T2.reserve(T.size() * 4);
        for (auto &t : T) {
            int ab = midpoint(t[0], t[1]), bc = midpoint(t[1], t[2]), ca = midpoint(t[2], t[0]);
            T2.push_back({t[0], ab, ca}); T2.push_back({ab, t[1], bc});
            T2.push_back({ca, bc, t[2]}); T2.push_back({ab, bc, ca});
        }
        T.swap(T2);
    }
    int nd = (int)P.size();
    if (nd != 10 * n * n + 2) { g_grid_err = "grid construction failed"; return RT_EINVAL; }
    // canonical order
    std::vector<int> order(nd), rank(nd);
    for (int i = 0; i < nd; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return key_of(P[a]) < key_of(P[b]); });
    for (int i = 0; i < nd; ++i) rank[order[i]] = i;
    std::vector<V3> D(nd);
    for (int i = 0; i < nd; ++i) D[i] = P[order[i]];
    // adjacency from triangle edges, then rings sorted by tangent-plane angle
    std::vector<std::set<int>> adj(nd);
    for (auto &t : T)
        for (int q = 0; q < 3; ++q) {
            int a = rank[t[q]], b = rank[t[(q + 1) % 3]];
            adj[a].insert(b); adj[b].insert(a);
        }
    rt_grid *g = new rt_grid();
    g->n = n; g->nd = nd; g->ne = 30 * n * n;
    g->h_dir.resize(3 * nd); g->h_nnb.resize(nd); g->h_nbr.assign(6 * nd, -1);
    g->h_ring_edge.assign(6 * nd, -1); g->h_ring_back.assign(6 * nd, -1); g->h_mirror.assign(nd, -1);
    for (int s = 0; s < nd; ++s) {
        for (int m = 0; m < 3; ++m) g->h_dir[3 * s + m] = D[s][m];
        std::vector<int> ring(adj[s].begin(), adj[s].end());
        const V3 &c = D[s];
        const V3 &f = D[ring[0]];
        double fc = f[0] * c[0] + f[1] * c[1] + f[2] * c[2];
        V3 t1 = unit({f[0] - fc * c[0], f[1] - fc * c[1], f[2] - fc * c[2]});
        V3 t2{c[1] * t1[2] - c[2] * t1[1], c[2] * t1[0] - c[0] * t1[2], c[0] * t1[1] - c[1] * t1[0]};
        std::vector<std::pair<double, int>> ang;
        for (int t : ring) {
            const V3 &p = D[t];
            ang.push_back({std::atan2(p[0] * t2[0] + p[1] * t2[1] + p[2] * t2[2], p[0] * t1[0] + p[1] * t1[1] + p[2] * t1[2]), t});
        }
        std::sort(ang.begin(), ang.end());
        int k = (int)ang.size();
        int start = 0;
        for (int q = 1; q < k; ++q) if (ang[q].second < ang[start].second) start = q;
        g->h_nnb[s] = k;
        for (int q = 0; q < k; ++q) g->h_nbr[6 * s + q] = ang[(start + q) % k].second;
    }
    // edges: owned by the lower index, in ring order
    for (int s = 0; s < nd; ++s)
        for (int q = 0; q < g->h_nnb[s]; ++q) {
            int t = g->h_nbr[6 * s + q];
            if (t < s) continue;
            int e = (int)g->h_edge.size() / 2;
            g->h_edge.push_back(s); g->h_edge.push_back(t);
            g->h_ring_edge[6 * s + q] = e;
        }
    for (int s = 0; s < nd; ++s)
        for (int q = 0; q < g->h_nnb[s]; ++q) {
            int t = g->h_nbr[6 * s + q];
            for (int r = 0; r < g->h_nnb[t]; ++r)
                if (g->h_nbr[6 * t + r] == s) {
                    g->h_ring_back[6 * s + q] = r;
                    if (t < s) g->h_ring_edge[6 * s + q] = g->h_ring_edge[6 * t + r];
                }
        }
    // pole mirror (n1, -n2, -n3)
    for (int s = 0; s < nd; ++s) {
        V3 p{D[s][0], -D[s][1], -D[s][2]};
        for (int t = 0; t < nd; ++t)
            if (sq(D[t], p) < 1e-20) { g->h_mirror[s] = t; break; }
    }
    if ((int)g->h_edge.size() != 2 * g->ne) { free_grid(g); g_grid_err = "edge count mismatch"; return RT_EINVAL; }
    rt_status st = rt_grid_device_geometry(g, g_grid_err);
    if (st != RT_OK) { free_grid(g); return st; }
    *out = g;
    return RT_OK;
}

extern "C" rt_status rt_grid_query(const rt_grid *g, int *n_dir, int *n_edge, double *dirs, double *weights) {
    if (!g) return RT_EINVAL;
    if (n_dir) *n_dir = g->nd;
    if (n_edge) *n_edge = g->ne;
    if (dirs) std::copy(g->h_dir.begin(), g->h_dir.end(), dirs);
    if (weights) std::copy(g->h_w.begin(), g->h_w.end(), weights);
    return RT_OK;
}

extern "C" void rt_destroy_grid(rt_grid *g) { free_grid(g); }

extern "C" const char *rt_grid_last_error(void) { return g_grid_err.c_str(); }
