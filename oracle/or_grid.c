/*
 * or_grid.c — geodesic angular grid of the oracle (section 3.3, "Geodesic Grid").
 * TEST INFRASTRUCTURE ONLY (see rt_oracle.h).
 *
 * Construction as the paper describes it: the 12 icosahedron vertices on the
 * unit sphere, repeated bisection of every triangle edge with projection of the
 * new vertex onto the sphere (each triangle -> 4), and the Voronoi diagram of
 * the final Delaunay triangulation.  The Voronoi cell of direction s is its
 * angular cell; its solid angle is the quadrature weight, its 5 or 6 edges are
 * the angular cell boundaries across which the angular flux of eq.
 * (angular_fluxes) is taken.
 *
 * Canonical direction order (a convention shared with the CUDA library, which
 * implements it separately): ascending key1 = llround(-n_z * 1e9), then
 * ascending atan2(y, x) with |x|,|y| < 1e-12 snapped to +0.
 * Ring order: counter-clockwise about the outward normal, starting at the
 * neighbour with the smallest index.
 */
#include "or_internal.h"

typedef struct { double x, y, z; } vec;

static vec vnorm(vec a) { double r = sqrt(a.x*a.x + a.y*a.y + a.z*a.z); vec o = {a.x/r, a.y/r, a.z/r}; return o; }
static vec vsub(vec a, vec b) { vec o = {a.x-b.x, a.y-b.y, a.z-b.z}; return o; }
static vec vadd(vec a, vec b) { vec o = {a.x+b.x, a.y+b.y, a.z+b.z}; return o; }
static double vdot(vec a, vec b) { return a.x*b.x + a.y*b.y + a.z*b.z; }
static vec vcross(vec a, vec b) { vec o = {a.y*b.z - a.z*b.y, a.z*b.x - a.x*b.z, a.x*b.y - a.y*b.x}; return o; }

typedef struct { int nv; vec *v; } mesh;

static int add_vertex(mesh *m, vec p) { m->v[m->nv] = p; return m->nv++; }

/* midpoint lookup: each vertex keeps up to 6 (neighbour, midpoint) pairs */
typedef struct { int cnt; int nb[8]; int mid[8]; } midtab;

static int midpoint(mesh *m, midtab *t, int a, int b) {
    for (int q = 0; q < t[a].cnt; ++q) if (t[a].nb[q] == b) return t[a].mid[q];
    vec p = vnorm(vadd(m->v[a], m->v[b]));          /* bisect, project to sphere */
    int id = add_vertex(m, p);
    t[a].nb[t[a].cnt] = b; t[a].mid[t[a].cnt++] = id;
    t[b].nb[t[b].cnt] = a; t[b].mid[t[b].cnt++] = id;
    return id;
}

static double snap(double v) { return fabs(v) < 1e-12 ? 0.0 : v; }
static long long key1(vec p) { return llround(-p.z * 1e9); }
static double key2(vec p) { return atan2(snap(p.y), snap(p.x)); }

static const vec *g_sortv;
static int cmp_dir(const void *A, const void *B) {
    vec p = g_sortv[*(const int *)A], q = g_sortv[*(const int *)B];
    long long a1 = key1(p), b1 = key1(q);
    if (a1 != b1) return a1 < b1 ? -1 : 1;
    double a2 = key2(p), b2 = key2(q);
    return a2 < b2 ? -1 : (a2 > b2 ? 1 : 0);
}

/* Van Oosterom & Strackee solid angle of the spherical triangle (a, b, c) */
static double tri_solid_angle(vec a, vec b, vec c) {
    double num = vdot(a, vcross(b, c));
    double den = 1.0 + vdot(a, b) + vdot(b, c) + vdot(c, a);
    return 2.0 * atan2(num, den);
}

int or_build_grid(or_grid *G, int n) {
    if (n < 1 || (n & (n - 1))) return -1;
    int levels = 0; while ((1 << levels) < n) ++levels;
    int nd = 10 * n * n + 2, nf = 20 * n * n;
    mesh m; m.nv = 0;
    m.v = (vec *)malloc(sizeof(vec) * nd);
    int (*faces)[3] = malloc(sizeof(int[3]) * nf);
    int (*nfaces)[3] = malloc(sizeof(int[3]) * nf);
    midtab *mt = calloc(nd, sizeof(midtab));

    /* icosahedron: cyclic permutations of (0, +-1, +-phi) */
    const double ph = 0.5 * (1.0 + sqrt(5.0));
    for (int s1 = -1; s1 <= 1; s1 += 2)
        for (int s2 = -1; s2 <= 1; s2 += 2) {
            vec a = {0.0, (double)s1, s2 * ph}, b = {(double)s1, s2 * ph, 0.0}, c = {s2 * ph, 0.0, (double)s1};
            add_vertex(&m, a); add_vertex(&m, b); add_vertex(&m, c);
        }
    /* faces: triples of mutually adjacent vertices (edge length 2 before projection) */
    int nf0 = 0;
    for (int i = 0; i < 12; ++i) for (int j = i + 1; j < 12; ++j) for (int k = j + 1; k < 12; ++k) {
        double dij = vdot(vsub(m.v[i], m.v[j]), vsub(m.v[i], m.v[j]));
        double djk = vdot(vsub(m.v[j], m.v[k]), vsub(m.v[j], m.v[k]));
        double dki = vdot(vsub(m.v[k], m.v[i]), vsub(m.v[k], m.v[i]));
        if (fabs(dij - 4) < 1e-9 && fabs(djk - 4) < 1e-9 && fabs(dki - 4) < 1e-9) {
            vec nrm = vcross(vsub(m.v[j], m.v[i]), vsub(m.v[k], m.v[i]));
            if (vdot(nrm, m.v[i]) > 0) { faces[nf0][0] = i; faces[nf0][1] = j; faces[nf0][2] = k; }
            else { faces[nf0][0] = i; faces[nf0][1] = k; faces[nf0][2] = j; }
            ++nf0;
        }
    }
    for (int i = 0; i < 12; ++i) m.v[i] = vnorm(m.v[i]);
    int cur = nf0;
    /* repeated bisection */
    for (int L = 0; L < levels; ++L) {
        for (int i = 0; i < m.nv; ++i) mt[i].cnt = 0;
        int nn = 0;
        for (int f = 0; f < cur; ++f) {
            int a = faces[f][0], b = faces[f][1], c = faces[f][2];
            int ab = midpoint(&m, mt, a, b), bc = midpoint(&m, mt, b, c), ca = midpoint(&m, mt, c, a);
            int q[4][3] = {{a, ab, ca}, {b, bc, ab}, {c, ca, bc}, {ab, bc, ca}};
            for (int t = 0; t < 4; ++t) { nfaces[nn][0] = q[t][0]; nfaces[nn][1] = q[t][1]; nfaces[nn][2] = q[t][2]; ++nn; }
        }
        cur = nn;
        memcpy(faces, nfaces, sizeof(int[3]) * nn);
    }
    if (m.nv != nd || cur != nf) { free(m.v); free(faces); free(nfaces); free(mt); return -2; }

    /* canonical order */
    int *perm = malloc(sizeof(int) * nd), *inv = malloc(sizeof(int) * nd);
    for (int i = 0; i < nd; ++i) perm[i] = i;
    g_sortv = m.v; qsort(perm, nd, sizeof(int), cmp_dir);
    for (int i = 0; i < nd; ++i) inv[perm[i]] = i;
    vec *dir = malloc(sizeof(vec) * nd);
    for (int i = 0; i < nd; ++i) dir[i] = m.v[perm[i]];
    for (int f = 0; f < nf; ++f) for (int t = 0; t < 3; ++t) faces[f][t] = inv[faces[f][t]];

    /* Voronoi vertex of each Delaunay triangle: its circumcentre on the sphere */
    vec *cc = malloc(sizeof(vec) * nf);
    for (int f = 0; f < nf; ++f) {
        vec a = dir[faces[f][0]], b = dir[faces[f][1]], c = dir[faces[f][2]];
        cc[f] = vnorm(vcross(vsub(b, a), vsub(c, a)));  /* counter-clockwise faces: outward */
    }
    G->nd = nd; G->ne = 30 * n * n;
    G->dir = malloc(sizeof(double) * 3 * nd); G->w = malloc(sizeof(double) * nd);
    G->nnb = malloc(sizeof(int) * nd); G->nbr = malloc(sizeof(int) * 6 * nd);
    G->ring_edge = malloc(sizeof(int) * 6 * nd); G->ring_back = malloc(sizeof(int) * 6 * nd);
    G->edge = malloc(sizeof(int) * 2 * G->ne); G->dlam = malloc(sizeof(double) * G->ne);
    G->emid = malloc(sizeof(double) * 3 * G->ne); G->eu = malloc(sizeof(double) * 3 * G->ne);
    G->vor = malloc(sizeof(double) * 3 * 6 * nd);
    for (int s = 0; s < nd; ++s) { G->dir[3*s] = dir[s].x; G->dir[3*s+1] = dir[s].y; G->dir[3*s+2] = dir[s].z; }

    /* ring of every direction: faces around s chained counter-clockwise */
    int *inc = malloc(sizeof(int) * 6 * nd), *ninc = calloc(nd, sizeof(int));
    for (int f = 0; f < nf; ++f) for (int t = 0; t < 3; ++t) { int s = faces[f][t]; inc[6*s + ninc[s]++] = f; }
    for (int s = 0; s < nd; ++s) {
        int k = ninc[s];
        int bnext[6], cnext[6], fid[6];
        for (int q = 0; q < k; ++q) {
            int f = inc[6*s + q], t = 0;
            while (faces[f][t] != s) ++t;
            bnext[q] = faces[f][(t + 1) % 3]; cnext[q] = faces[f][(t + 2) % 3]; fid[q] = f;
        }
        int order[6], used[6] = {0};
        order[0] = 0; used[0] = 1;
        for (int q = 1; q < k; ++q) {
            int prev = order[q - 1], found = -1;
            for (int r = 0; r < k; ++r) if (!used[r] && bnext[r] == cnext[prev]) { found = r; break; }
            order[q] = found; used[found] = 1;
        }
        /* neighbour ring: b of each chained face; Voronoi vertex q lies between nbr q and q+1 */
        int nb[6]; vec vv[6];
        for (int q = 0; q < k; ++q) { nb[q] = bnext[order[q]]; vv[q] = cc[fid[order[q]]]; }
        int start = 0;
        for (int q = 1; q < k; ++q) if (nb[q] < nb[start]) start = q;
        G->nnb[s] = k;
        for (int q = 0; q < 6; ++q) { G->nbr[6*s + q] = -1; G->ring_edge[6*s + q] = -1; G->ring_back[6*s + q] = -1; }
        for (int q = 0; q < k; ++q) {
            int src = (start + q) % k;
            G->nbr[6*s + q] = nb[src];
            G->vor[3*(6*s + q)] = vv[src].x; G->vor[3*(6*s + q) + 1] = vv[src].y; G->vor[3*(6*s + q) + 2] = vv[src].z;
        }
        /* solid angle: fan of spherical triangles (s, V_q, V_q+1) */
        double area = 0.0;
        for (int q = 0; q < k; ++q) {
            vec a = {G->vor[3*(6*s+q)], G->vor[3*(6*s+q)+1], G->vor[3*(6*s+q)+2]};
            int q1 = (q + 1) % k;
            vec b = {G->vor[3*(6*s+q1)], G->vor[3*(6*s+q1)+1], G->vor[3*(6*s+q1)+2]};
            area += tri_solid_angle(dir[s], a, b);
        }
        G->w[s] = area;
    }
    /* edges (s < s'): the Voronoi edge between s and nbr q runs from V_{q-1} to V_q */
    int ne = 0;
    for (int s = 0; s < nd; ++s) {
        int k = G->nnb[s];
        for (int q = 0; q < k; ++q) {
            int t = G->nbr[6*s + q];
            if (t < s) continue;
            int qm = (q + k - 1) % k;
            vec a = {G->vor[3*(6*s+qm)], G->vor[3*(6*s+qm)+1], G->vor[3*(6*s+qm)+2]};
            vec b = {G->vor[3*(6*s+q)], G->vor[3*(6*s+q)+1], G->vor[3*(6*s+q)+2]};
            G->edge[2*ne] = s; G->edge[2*ne + 1] = t;
            G->dlam[ne] = atan2(sqrt(vdot(vcross(a, b), vcross(a, b))), vdot(a, b));
            vec mm = vnorm(vadd(a, b));
            vec uu = vnorm(vsub(dir[t], dir[s]));
            G->emid[3*ne] = mm.x; G->emid[3*ne+1] = mm.y; G->emid[3*ne+2] = mm.z;
            G->eu[3*ne] = uu.x; G->eu[3*ne+1] = uu.y; G->eu[3*ne+2] = uu.z;
            ++ne;
        }
    }
    /* ring slot -> edge, and the slot of s in the neighbour's ring */
    for (int e = 0; e < ne; ++e) {
        int s = G->edge[2*e], t = G->edge[2*e+1];
        for (int q = 0; q < G->nnb[s]; ++q) if (G->nbr[6*s+q] == t) G->ring_edge[6*s+q] = e;
        for (int q = 0; q < G->nnb[t]; ++q) if (G->nbr[6*t+q] == s) G->ring_edge[6*t+q] = e;
    }
    for (int s = 0; s < nd; ++s) for (int q = 0; q < G->nnb[s]; ++q) {
        int t = G->nbr[6*s+q];
        for (int r = 0; r < G->nnb[t]; ++r) if (G->nbr[6*t+r] == s) G->ring_back[6*s+q] = r;
    }
    /* mirror map of the pole boundary: (n1, n2, n3) -> (n1, -n2, -n3) */
    G->mirror = malloc(sizeof(int) * nd);
    for (int s = 0; s < nd; ++s) {
        vec p = {dir[s].x, -dir[s].y, -dir[s].z};
        int best = -1; double bd = 1e300;
        for (int t = 0; t < nd; ++t) { vec d = vsub(dir[t], p); double q = vdot(d, d); if (q < bd) { bd = q; best = t; } }
        G->mirror[s] = (bd < 1e-20) ? best : -1;
    }
    free(inc); free(ninc); free(cc); free(dir); free(perm); free(inv);
    free(m.v); free(faces); free(nfaces); free(mt);
    return ne == G->ne ? 0 : -3;
}

void or_free_grid(or_grid *G) {
    free(G->dir); free(G->w); free(G->nnb); free(G->nbr); free(G->ring_edge); free(G->ring_back);
    free(G->edge); free(G->dlam); free(G->emid); free(G->eu); free(G->vor); free(G->mirror);
}
