/*
 * tof_oracle.c -- plain, slow FP64 CPU oracle of the ToF ReSTIR hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this library.  It shares no code, header, table or
 * helper with the CUDA path; the two agree only through the seeded input arrays and the
 * published definitions both restate (Philox4x32-10, Moller-Trumbore, the paper's equations).
 *
 * What it computes (Kim, Jarosz, Pediredla, "ToF ReSTIR", ACM TOG 45(4) 2026):
 *   Sec. 3.1  time-of-flight path integral I(tau) = int W_tau(L(x)) f(x) dmu(x), with c = 1
 *   Sec. 3.2  RIS (basic, MIS) and generalized RIS with shift maps and the generalized balance
 *             heuristic (eq. GRIS_resampling_weight, eq. GRIS_MIS_weight)
 *   Sec. 4.1  offset-path perturbation at the reconnection vertex of a hybrid shift
 *   Sec. 4.2  2-D surface parameterisation xi of the reconnection vertex
 *   Sec. 4.3  average-gradient gauge, Newton iteration with backtracking, shift Jacobian by
 *             implicit differentiation, frame factor, gradient and Hessian of L
 *   Sec. 4.5  transient histograms as independent per-bin gates; candidates deposited into
 *             their own bin ("path reuse" of Jarabo 2014)
 *   Sec. 5    reservoir stores the vertex after the reconnection vertex; delta light sources
 *             (point light with NEE, collimated laser spot)
 *
 * Readings where the paper is silent, garbled or inconsistent are stated at the function that
 * applies them.
 *
 * Everything is double precision.  Random numbers come from Philox4x32-10 (Salmon et al. 2011)
 * keyed by (seed) and counted by (pixel, frame, stream, purpose), so the CUDA path and this
 * oracle draw identical numbers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OPI 3.14159265358979323846

/* ============================================================================================
 * small vector algebra
 * ==========================================================================================*/
typedef struct { double x, y, z; } v3;
static v3 V(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 vadd(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 vsub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 vmul(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static double vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 vcross(v3 a, v3 b) { return V(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double vlen(v3 a) { return sqrt(vdot(a, a)); }
static v3 vnorm(v3 a) { double l = vlen(a); return l > 0 ? vmul(a, 1.0 / l) : V(0, 0, 0); }
static v3 vload(const double* p) { return V(p[0], p[1], p[2]); }

/* ============================================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3",
 * SC 2011): 10 rounds of the 4x32 Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and
 * Weyl key increments 0x9E3779B9 / 0xBB67AE85.
 * ==========================================================================================*/
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* purposes (low byte of the 4th counter word) */
enum { P_JITTER = 1, P_BSDF = 2, P_RIS = 3, P_NEIGHBOR = 4, P_MERGE = 5,
       P_ELL_RIS = 6,   /* selection of an ellipsoidal candidate */
       P_ELL = 7 };     /* P_ELL + q, q = 0..5: the ellipsoidal connection's draws */

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void rng4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, out);
}

/* ============================================================================================
 * materials and BSDFs (the paper uses diffuse, glossy and specular materials, Sec. 6; the
 * microfacet model is Walter et al. 2007 GGX with the separable Smith shadowing term and a
 * constant Fresnel equal to the albedo)
 * ==========================================================================================*/
enum { M_LAMBERT = 0, M_GGX = 1, M_MIRROR = 2 };
enum { C_ROUGH = 0, C_GLOSSY = 1, C_DELTA = 2 };
typedef struct { int type; double albedo, alpha; } omat;

static int mat_class(const omat* m) {
    if (m->type == M_MIRROR) return C_DELTA;
    if (m->type == M_GGX && m->alpha < 0.2) return C_GLOSSY;
    return C_ROUGH;
}

static double ggx_D(double nh, double a) {
    double a2 = a * a, t = nh * nh * (a2 - 1.0) + 1.0;
    return a2 / (OPI * t * t);
}
static double ggx_G1(double nv, double a) {
    double a2 = a * a;
    return 2.0 * nv / (nv + sqrt(a2 + (1.0 - a2) * nv * nv));
}

/* BSDF value f_s(wi, wo) for unit directions wi (toward the previous vertex) and wo (toward the
 * next); n is the geometric normal of either orientation.  Reflection only; delta lobes give 0. */
double or_bsdf_eval(int type, double albedo, double alpha, const double* nn, const double* wii, const double* woo) {
    v3 n = vload(nn), wi = vload(wii), wo = vload(woo);
    double ci = vdot(n, wi), co = vdot(n, wo);
    if (ci * co <= 0.0) return 0.0;
    if (ci < 0) { ci = -ci; co = -co; n = vmul(n, -1.0); }
    if (type == M_LAMBERT) return albedo / OPI;
    if (type == M_GGX) {
        v3 h = vnorm(vadd(wi, wo));
        double nh = vdot(n, h);
        if (nh <= 0) return 0.0;
        return albedo * ggx_D(nh, alpha) * ggx_G1(ci, alpha) * ggx_G1(co, alpha) / (4.0 * ci * co);
    }
    return 0.0;
}
static double bsdf_f(const omat* m, v3 n, v3 wi, v3 wo) {
    double a[3] = {n.x, n.y, n.z}, b[3] = {wi.x, wi.y, wi.z}, c[3] = {wo.x, wo.y, wo.z};
    return or_bsdf_eval(m->type, m->albedo, m->alpha, a, b, c);
}

/* solid-angle pdf of sampling wo at a surface with normal n, given wi */
static double bsdf_pdf(const omat* m, v3 n, v3 wi, v3 wo) {
    double ci = vdot(n, wi), co = vdot(n, wo);
    if (ci * co <= 0.0) return 0.0;
    if (ci < 0) { ci = -ci; co = -co; n = vmul(n, -1.0); }
    if (m->type == M_LAMBERT) return co / OPI;
    if (m->type == M_GGX) {
        v3 h = vnorm(vadd(wi, wo));
        double nh = vdot(n, h), oh = vdot(wo, h);
        if (nh <= 0 || oh <= 0) return 0.0;
        return ggx_D(nh, m->alpha) * nh / (4.0 * oh);
    }
    return 0.0;
}

/* orthonormal tangent frame (t, b, n) around a unit normal: t = normalize(a x n), b = n x t, with
 * the reference axis a one of two fixed generic unit vectors (a1, and a2 perpendicular to it,
 * used when |n.a1| >= 0.6).  The frame must be a deterministic function of n, and any such frame
 * is discontinuous somewhere on the sphere; this one puts the switch on a cone around a generic
 * direction that mesh normals (axis-aligned walls, symmetric tessellations) do not meet exactly,
 * so float and double evaluations of the same normal pick the same branch. */
static void onb(v3 n, v3* t, v3* b) {
    const v3 a1 = {0.4140355211239282, 0.731736150464251, 0.5414210869105452};
    const v3 a2 = {0.0, 0.5947978113475719, -0.8038753408434284};
    v3 a = fabs(vdot(n, a1)) < 0.6 ? a1 : a2;
    *t = vnorm(vcross(a, n));
    *b = vcross(n, *t);
}

/* sample wo given wi; returns 0 on failure.  *thr = f_s |cos_o| / pdf (albedo for delta). */
static int bsdf_sample(const omat* m, v3 n, v3 wi, double u0, double u1, v3* wo, double* pdf, double* thr, int* delta) {
    if (vdot(n, wi) < 0) n = vmul(n, -1.0);
    *delta = 0;
    if (m->type == M_MIRROR) {
        *wo = vsub(vmul(n, 2.0 * vdot(wi, n)), wi);
        *pdf = 1.0; *thr = m->albedo; *delta = 1;
        return 1;
    }
    v3 t, b;
    onb(n, &t, &b);
    if (m->type == M_LAMBERT) {
        double r = sqrt(u0), ph = 2.0 * OPI * u1;
        double lz = sqrt(fmax(0.0, 1.0 - u0));
        *wo = vadd(vadd(vmul(t, r * cos(ph)), vmul(b, r * sin(ph))), vmul(n, lz));
    } else {
        double a = m->alpha;
        double tan2 = a * a * u0 / (1.0 - u0);
        double ct = 1.0 / sqrt(1.0 + tan2), st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * OPI * u1;
        v3 h = vadd(vadd(vmul(t, st * cos(ph)), vmul(b, st * sin(ph))), vmul(n, ct));
        *wo = vsub(vmul(h, 2.0 * vdot(wi, h)), wi);
    }
    double co = vdot(n, *wo);
    if (co <= 0.0) return 0;
    *pdf = bsdf_pdf(m, n, wi, *wo);
    double f = bsdf_f(m, n, wi, *wo);
    if (!(*pdf > 0.0) || !(f > 0.0)) return 0;
    *thr = f * co / *pdf;
    return 1;
}

/* ============================================================================================
 * scene geometry: world-space triangles (rigidly transformed per object), median-split BVH
 * ==========================================================================================*/
typedef struct { double lo[3], hi[3]; int left, right, start, count; } onode;
typedef struct {
    int nt, nobj, nmat;
    double* tv;     /* nt*9 world corners */
    int* tmat;      /* material per triangle */
    omat* mats;
    double* xf;     /* nobj*12, kept to decide whether two frames have identical geometry */
    int nnodes;
    onode* nodes;
    int* prim;
    int eP;         /* leaves of the triangle-index hierarchy of the ellipsoidal connection */
    double* enode;  /* 2*eP nodes in heap order, 8 doubles each: lo[3], hi[3], area, unused */
    int* adj;       /* nt*3: across the edge opposite vertex i of t, 4 * neighbour + the neighbour's
                       vertex opposite that edge, or -1 (boundary, non-manifold or another object) */
} ogeom;

static const double* tri_v(const ogeom* g, int t) { return g->tv + 9 * (size_t)t; }

static double* g_cent;    /* build-time scratch for the comparator (single-threaded build) */
static int g_axis;
static int cmp_prim(const void* a, const void* b) {
    double ca = g_cent[3 * *(const int*)a + g_axis], cb = g_cent[3 * *(const int*)b + g_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (*(const int*)a) - (*(const int*)b);
}

static int bvh_build_rec(ogeom* g, double* cent, int start, int count) {
    int id = g->nnodes++;
    onode* nd = &g->nodes[id];
    for (int k = 0; k < 3; ++k) { nd->lo[k] = 1e300; nd->hi[k] = -1e300; }
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int i = start; i < start + count; ++i) {
        const double* v = tri_v(g, g->prim[i]);
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) {
                if (v[3 * c + k] < nd->lo[k]) nd->lo[k] = v[3 * c + k];
                if (v[3 * c + k] > nd->hi[k]) nd->hi[k] = v[3 * c + k];
            }
        for (int k = 0; k < 3; ++k) {
            double c = cent[3 * g->prim[i] + k];
            if (c < clo[k]) clo[k] = c;
            if (c > chi[k]) chi[k] = c;
        }
    }
    if (count <= 4) { nd->left = nd->right = -1; nd->start = start; nd->count = count; return id; }
    int axis = 0;
    for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    g_cent = cent; g_axis = axis;
    qsort(g->prim + start, (size_t)count, sizeof(int), cmp_prim);
    int half = count / 2;
    int l = bvh_build_rec(g, cent, start, half);
    int r = bvh_build_rec(g, cent, start + half, count - half);
    nd = &g->nodes[id];
    nd->left = l; nd->right = r; nd->start = start; nd->count = 0;
    return id;
}

/* edge adjacency from the index buffer: an edge (its two vertex indices) shared by exactly two
 * triangles of one object links them */
typedef struct { uint32_t a, b; int tri, opp; } oedge;
static int cmp_edge(const void* x, const void* y) {
    const oedge* e = (const oedge*)x;
    const oedge* f = (const oedge*)y;
    if (e->a != f->a) return e->a < f->a ? -1 : 1;
    if (e->b != f->b) return e->b < f->b ? -1 : 1;
    return e->tri - f->tri;
}
static void build_adjacency(ogeom* g, const uint32_t* tris, const uint32_t* tri_obj, int nt) {
    g->adj = (int*)malloc(sizeof(int) * 3 * (size_t)(nt > 0 ? nt : 1));
    oedge* E = (oedge*)malloc(sizeof(oedge) * 3 * (size_t)(nt > 0 ? nt : 1));
    for (int t = 0; t < nt; ++t)
        for (int i = 0; i < 3; ++i) {
            uint32_t u = tris[3 * t + (i + 1) % 3], w = tris[3 * t + (i + 2) % 3];
            oedge* e = &E[3 * t + i];
            e->a = u < w ? u : w; e->b = u < w ? w : u; e->tri = t; e->opp = i;
            g->adj[3 * t + i] = -1;
        }
    qsort(E, 3 * (size_t)nt, sizeof(oedge), cmp_edge);
    for (int k = 0; k < 3 * nt;) {
        int m = k + 1;
        while (m < 3 * nt && E[m].a == E[k].a && E[m].b == E[k].b) ++m;
        if (m - k == 2 && tri_obj[E[k].tri] == tri_obj[E[k + 1].tri] && E[k].tri != E[k + 1].tri) {
            g->adj[3 * E[k].tri + E[k].opp] = 4 * E[k + 1].tri + E[k + 1].opp;
            g->adj[3 * E[k + 1].tri + E[k + 1].opp] = 4 * E[k].tri + E[k].opp;
        }
        k = m;
    }
    free(E);
}

/* The hierarchy the ellipsoidal connection walks (Sec. 5 "Ellipsoidal Path Connection": BVH
 * nodes weighted by the area of the triangles below them).  It is the implicit binary tree over
 * triangle index ranges: eP = the smallest power of two >= nt leaves, node n (1 <= n < 2 eP) has
 * children 2n and 2n + 1, triangle t is leaf eP + t, padding leaves are empty.  Its shape depends
 * on the scene alone, not on how a ray-tracing hierarchy was built. */
#define ELL_MAX_LEVELS 22
static void etree_build(ogeom* g) {
    int P = 1;
    while (P < g->nt) P <<= 1;
    g->eP = P;
    g->enode = (double*)malloc(sizeof(double) * 8 * 2 * (size_t)P);
    for (int i = 0; i < P; ++i) {
        double* e = g->enode + 8 * (size_t)(P + i);
        for (int k = 0; k < 3; ++k) { e[k] = 1e300; e[3 + k] = -1e300; }
        e[6] = e[7] = 0.0;
        if (i < g->nt) {
            const double* v = tri_v(g, i);
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) {
                    if (v[3 * c + k] < e[k]) e[k] = v[3 * c + k];
                    if (v[3 * c + k] > e[3 + k]) e[3 + k] = v[3 * c + k];
                }
            v3 v0 = vload(v);
            e[6] = 0.5 * vlen(vcross(vsub(vload(v + 3), v0), vsub(vload(v + 6), v0)));
        }
    }
    for (int n = P - 1; n >= 1; --n) {
        double* e = g->enode + 8 * (size_t)n;
        const double* a = g->enode + 8 * (size_t)(2 * n);
        const double* b = g->enode + 8 * (size_t)(2 * n + 1);
        for (int k = 0; k < 3; ++k) { e[k] = fmin(a[k], b[k]); e[3 + k] = fmax(a[3 + k], b[3 + k]); }
        e[6] = a[6] + b[6];
        e[7] = 0.0;
    }
}

/* verts: object-local vertices; xforms: nobj row-major 3x4 object-to-world matrices */
ogeom* or_geom_create(const double* verts, int nv, const uint32_t* tris, int nt, const uint32_t* tri_obj,
                      const uint32_t* obj_mat, int nobj, const double* mats, int nmat, const double* xforms) {
    (void)nv;
    ogeom* g = (ogeom*)calloc(1, sizeof(ogeom));
    g->nt = nt; g->nobj = nobj; g->nmat = nmat;
    g->tv = (double*)malloc(sizeof(double) * 9 * (size_t)(nt > 0 ? nt : 1));
    g->tmat = (int*)malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
    g->mats = (omat*)malloc(sizeof(omat) * (size_t)(nmat > 0 ? nmat : 1));
    g->xf = (double*)malloc(sizeof(double) * 12 * (size_t)(nobj > 0 ? nobj : 1));
    memcpy(g->xf, xforms, sizeof(double) * 12 * (size_t)nobj);
    for (int m = 0; m < nmat; ++m) { g->mats[m].type = (int)mats[3 * m]; g->mats[m].albedo = mats[3 * m + 1]; g->mats[m].alpha = mats[3 * m + 2]; }
    for (int t = 0; t < nt; ++t) {
        const double* M = xforms + 12 * (size_t)tri_obj[t];
        for (int c = 0; c < 3; ++c) {
            const double* p = verts + 3 * (size_t)tris[3 * t + c];
            for (int r = 0; r < 3; ++r)
                g->tv[9 * (size_t)t + 3 * c + r] = M[4 * r] * p[0] + M[4 * r + 1] * p[1] + M[4 * r + 2] * p[2] + M[4 * r + 3];
        }
        g->tmat[t] = (int)obj_mat[tri_obj[t]];
    }
    g->nodes = (onode*)malloc(sizeof(onode) * (size_t)(2 * (nt > 0 ? nt : 1)));
    g->prim = (int*)malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
    double* cent = (double*)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    for (int t = 0; t < nt; ++t) {
        g->prim[t] = t;
        const double* v = tri_v(g, t);
        for (int k = 0; k < 3; ++k) cent[3 * t + k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
    }
    g->nnodes = 0;
    if (nt > 0) bvh_build_rec(g, cent, 0, nt);
    free(cent);
    build_adjacency(g, tris, tri_obj, nt);
    etree_build(g);
    return g;
}

void or_geom_destroy(ogeom* g) {
    if (!g) return;
    free(g->tv); free(g->tmat); free(g->mats); free(g->xf); free(g->nodes); free(g->prim); free(g->adj); free(g->enode); free(g);
}

/* Moller-Trumbore ray/triangle test (Moller, Trumbore 1997); t in (tmin, tmax).  The barycentric
 * tests accept BARY_EPS outside the triangle so that a ray through an edge shared by two triangles
 * hits at least one of them whatever the rounding (no cracks on tessellated surfaces). */
#define BARY_EPS 1e-6
static int tri_hit(const double* v, v3 o, v3 d, double tmin, double tmax, double* t, double* b1, double* b2) {
    v3 v0 = vload(v), e1 = vsub(vload(v + 3), v0), e2 = vsub(vload(v + 6), v0);
    v3 pv = vcross(d, e2);
    double det = vdot(e1, pv);
    if (fabs(det) < 1e-14) return 0;
    double inv = 1.0 / det;
    v3 tv = vsub(o, v0);
    double u = vdot(tv, pv) * inv;
    if (u < -BARY_EPS || u > 1.0 + BARY_EPS) return 0;
    v3 qv = vcross(tv, e1);
    double w = vdot(d, qv) * inv;
    if (w < -BARY_EPS || u + w > 1.0 + BARY_EPS) return 0;
    double tt = vdot(e2, qv) * inv;
    if (!(tt > tmin && tt < tmax)) return 0;
    *t = tt; *b1 = u; *b2 = w;
    return 1;
}

static int box_hit(const onode* nd, v3 o, v3 invd, double tmax) {
    double t0 = 0.0, t1 = tmax;
    double oo[3] = {o.x, o.y, o.z}, id[3] = {invd.x, invd.y, invd.z};
    for (int k = 0; k < 3; ++k) {
        double a = (nd->lo[k] - oo[k]) * id[k], b = (nd->hi[k] - oo[k]) * id[k];
        if (a > b) { double s = a; a = b; b = s; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* closest hit along o + t d, t in (0, tmax); any_hit = 1 returns on the first hit */
static int trace(const ogeom* g, v3 o, v3 d, double tmax, int any_hit, int* tri, double* b1, double* b2, double* tout) {
    if (g->nnodes == 0) return 0;
    v3 invd = V(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
    int stack[128], sp = 0, found = 0;
    double best = tmax;
    stack[sp++] = 0;
    while (sp) {
        const onode* nd = &g->nodes[stack[--sp]];
        if (!box_hit(nd, o, invd, best)) continue;
        if (nd->left < 0) {
            for (int i = nd->start; i < nd->start + nd->count; ++i) {
                double t, u, w;
                /* closest hit; at equal distance the lower triangle index wins (order-independent) */
                if (tri_hit(tri_v(g, g->prim[i]), o, d, 0.0, found ? best * (1.0 + 1e-12) + 1e-300 : best, &t, &u, &w) &&
                    (!found || t < best || (t == best && g->prim[i] < *tri))) {
                    best = t; *tri = g->prim[i]; *b1 = u; *b2 = w; found = 1;
                    if (any_hit) { *tout = t; return 1; }
                }
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    if (found) *tout = best;
    return found;
}

int or_geom_intersect(const ogeom* g, const double* o, const double* d, double tmax, int brute,
                      double* t, int* tri, double* b1, double* b2) {
    v3 oo = vload(o), dd = vload(d);
    if (!brute) return trace(g, oo, dd, tmax, 0, tri, b1, b2, t);
    int found = 0;
    double best = tmax;
    for (int i = 0; i < g->nt; ++i) {
        double tt, u, w;
        if (tri_hit(tri_v(g, i), oo, dd, 0.0, found ? best * (1.0 + 1e-12) + 1e-300 : best, &tt, &u, &w) &&
            (!found || tt < best || (tt == best && i < *tri))) { best = tt; *tri = i; *b1 = u; *b2 = w; found = 1; }
    }
    if (found) *t = best;
    return found;
}

/* ============================================================================================
 * surface points, ray offsets, visibility
 * ==========================================================================================*/
typedef struct { int tri; double b1, b2; v3 p, n; int mat; } osurf;

static osurf surf_at(const ogeom* g, int tri, double b1, double b2) {
    osurf s;
    const double* v = tri_v(g, tri);
    v3 v0 = vload(v), e1 = vsub(vload(v + 3), v0), e2 = vsub(vload(v + 6), v0);
    s.tri = tri; s.b1 = b1; s.b2 = b2;
    s.p = vadd(v0, vadd(vmul(e1, b1), vmul(e2, b2)));
    s.n = vnorm(vcross(e1, e2));
    s.mat = g->tmat[tri];
    return s;
}

/* offset a surface point along its normal toward the side of direction dir */
static v3 offset_point(v3 p, v3 n, v3 dir, double eps) {
    return vdot(n, dir) >= 0.0 ? vadd(p, vmul(n, eps)) : vsub(p, vmul(n, eps));
}

/* closest hit of a ray leaving surface point s in unit direction d */
static int trace_from(const ogeom* g, const osurf* s, v3 d, double eps, osurf* hit, double* t) {
    v3 o = offset_point(s->p, s->n, d, eps);
    int tri; double b1, b2;
    if (!trace(g, o, d, 1e30, 0, &tri, &b1, &b2, t)) return 0;
    *hit = surf_at(g, tri, b1, b2);
    return 1;
}

/* mutual visibility of surface point a and either surface point b (bn != NULL) or point b */
static int visible(const ogeom* g, v3 a, v3 an, v3 b, const v3* bn, double eps) {
    v3 ao = offset_point(a, an, vsub(b, a), eps);
    v3 bo = bn ? offset_point(b, *bn, vsub(a, b), eps) : b;
    v3 d = vsub(bo, ao);
    double dist = vlen(d);
    if (!(dist > 0)) return 1;
    d = vmul(d, 1.0 / dist);
    int tri; double b1, b2, t;
    return !trace(g, ao, d, dist, 1, &tri, &b1, &b2, &t);
}

/* ============================================================================================
 * sensors, emitters, domains
 * ==========================================================================================*/
typedef struct {
    int mode, W, H;
    double pos[3], fwd[3], up[3], fov_y;
    double wall_o[3], wall_u[3], wall_v[3];
} osensor;
typedef struct { int type; double pos[3], dir[3], power; } oemitter;
typedef struct {
    int depth, n_cand, n_spatial, radius, n_spatial_iters, temporal;
    double m_cap;
    int newton_max_iter;
    double newton_tol_frac, jac_max, d_min, ray_eps;
    uint32_t flags;
    double shrink_k;     /* Sec. 4.4 shrink mapping: gate widened K times for initial sampling (<= 1: off) */
    int shrink_fine;     /* trees kept in the gate itself (canonical samples); 0 = all trees widened */
} oparams;
enum { F_DIRECT = 1, F_NAIVE = 2, F_PAIRWISE = 4, F_GAUGE_AXIS_T = 8, F_GAUGE_AXIS_B = 16, F_GAUGE_START = 32,
       F_WALK = 64, F_BIN_REUSE = 128, F_ELLIPSOID = 256 };
/* gauge of the Newton system (Sec. 4.3 "Selecting a Good Gauge Condition") */
enum { G_AVERAGE = 0, G_AXIS_T = 1, G_AXIS_B = 2, G_START = 3 };
static int gauge_of(uint32_t flags) {
    if (flags & F_GAUGE_AXIS_T) return G_AXIS_T;
    if (flags & F_GAUGE_AXIS_B) return G_AXIS_B;
    if (flags & F_GAUGE_START) return G_START;
    return G_AVERAGE;
}

/* Sec. 5 "Light Source": a point light (direct NEE) or a collimated laser whose spot acts as a
 * secondary emitter I(w) = P f_s(spot; to laser, w) |cos| (a light ray is traced first). */
typedef struct {
    int kind;        /* 0 none, 1 point, 2 spot */
    v3 pos;
    double I;        /* point intensity or laser power */
    osurf s;         /* spot surface */
    v3 to_origin;    /* unit direction from the spot toward the laser */
    double emit_len; /* laser origin -> spot length, part of the optical path */
} olight;

static int light_same(const olight* a, const olight* b) {
    if (a->kind != b->kind) return 0;
    if (a->kind == 0) return 1;
    if (a->pos.x != b->pos.x || a->pos.y != b->pos.y || a->pos.z != b->pos.z || a->I != b->I) return 0;
    if (a->kind == 2) {
        if (a->s.tri != b->s.tri || a->s.b1 != b->s.b1 || a->s.b2 != b->s.b2) return 0;
        if (a->to_origin.x != b->to_origin.x || a->to_origin.y != b->to_origin.y || a->to_origin.z != b->to_origin.z) return 0;
        if (a->emit_len != b->emit_len) return 0;
    }
    return 1;
}

/* intensity leaving the light toward point x, the light position and the extra path length */
static double light_I(const ogeom* g, const olight* L, v3 x, v3* lpos) {
    *lpos = L->kind == 2 ? L->s.p : L->pos;
    if (L->kind == 1) return L->I;
    if (L->kind == 2) {
        v3 w = vnorm(vsub(x, L->s.p));
        double f = bsdf_f(&g->mats[L->s.mat], L->s.n, L->to_origin, w);
        return L->I * f * fabs(vdot(L->s.n, w));
    }
    return 0.0;
}

/* light factor of a path ending at vertex x: I_e(x) |cos_x| / d^2 (no BSDF, no visibility) */
static double light_term(const ogeom* g, const olight* L, const osurf* x, v3* wl, double* seg) {
    v3 lp;
    double I = light_I(g, L, x->p, &lp);
    v3 d = vsub(lp, x->p);
    double dist = vlen(d);
    if (!(dist > 0) || !(I > 0)) return 0.0;
    *wl = vmul(d, 1.0 / dist);
    *seg = dist + (L->kind == 2 ? L->emit_len : 0.0);
    return I * fabs(vdot(x->n, *wl)) / (dist * dist);
}

static int light_visible(const ogeom* g, const olight* L, const osurf* x, double eps) {
    if (L->kind == 2) return visible(g, x->p, x->n, L->s.p, &L->s.n, eps);
    return visible(g, x->p, x->n, L->pos, NULL, eps);
}

/* G-buffer entry of one pixel */
typedef struct { int valid; osurf s; double t; } ogb;

/* A reservoir's domain: one pixel of one frame (Sec. 3.2: each pixel/time step is its own
 * integration domain Omega_i with its own target function). */
typedef struct {
    const ogeom* g;
    int valid;
    v3 x0;          /* camera / device position */
    osurf y1;       /* primary hit */
    double o;       /* offset subtracted from L before gating (confocal convention) */
    double L0, dL;  /* gate [L0, L0 + dL) of the gated variable tau = L - o */
    olight light;
} odomain;

/* ============================================================================================
 * path records (the reservoir sample, Sec. 5 "Reservoir Implementation": the reservoir follows
 * ReSTIR PT and additionally stores the vertex after the reconnection vertex, with the
 * reconnection radiance attached to that next vertex)
 * ==========================================================================================*/
#define MAXD 8
typedef struct {
    int valid;
    double W, M, phat, tau;
    uint32_t key_px, key_frame;
    int tree, k, r;
    int cls[MAXD];       /* classes of x_1..x_{r-1} (index 1..) */
    v3 xprev;            /* x_{r-1}, world position in this record's own frame */
    double pdf_pre;      /* product of area pdfs of x_2..x_{r-1} */
    int p_tri; double p_b1, p_b2;
    int ns;              /* number of suffix vertices x_{r+1}..x_k (k - r) */
    int s_tri[4]; double s_b1[4], s_b2[4];
    double Lsuf;         /* cached radiance factor of the suffix beyond x_{r+1} */
} orec;

static const orec EMPTY_REC = {0};

/* ============================================================================================
 * path-length derivatives (Sec. 4.3 "Gradient and Hessian Evaluation")
 *   L(p) = |p1 - p| + |p2 - p|
 *   grad_p L = -(d1 + d2) = -s,  hess_p L = A = (I - d1 d1^T)/|p1 - p| + (I - d2 d2^T)/|p2 - p|
 *   grad_xi L = J^T(-s),  hess_xi L = J^T A J + Q with Q = 0 (exact on planar triangles)
 * ==========================================================================================*/
typedef struct { v3 o, t, b; } oframe2;     /* p(xi) = o + xi1 t + xi2 b, orthonormal t, b */

static oframe2 tri_frame(const ogeom* g, int tri) {
    const double* v = tri_v(g, tri);
    v3 v0 = vload(v), e1 = vsub(vload(v + 3), v0), e2 = vsub(vload(v + 6), v0);
    oframe2 f;
    f.o = v0;
    f.t = vnorm(e1);
    v3 n = vnorm(vcross(e1, e2));
    f.b = vcross(n, f.t);
    return f;
}
static v3 frame_point(const oframe2* f, const double xi[2]) {
    return vadd(f->o, vadd(vmul(f->t, xi[0]), vmul(f->b, xi[1])));
}

/* L, grad (2) and symmetric Hessian (h11, h12, h22) of L(xi) for neighbours p1, p2 */
void or_length_derivs(const double* p1d, const double* p2d, const double* od, const double* td, const double* bd,
                      const double xi[2], double* Lout, double g[2], double h[3]) {
    oframe2 f = {vload(od), vload(td), vload(bd)};
    v3 p1 = vload(p1d), p2 = vload(p2d), p = frame_point(&f, xi);
    v3 a1 = vsub(p1, p), a2 = vsub(p2, p);
    double l1 = vlen(a1), l2 = vlen(a2);
    v3 d1 = vmul(a1, 1.0 / l1), d2 = vmul(a2, 1.0 / l2);
    v3 s = vadd(d1, d2);
    *Lout = l1 + l2;
    g[0] = -vdot(f.t, s);
    g[1] = -vdot(f.b, s);
    /* J^T A J with A u = (u - d1 (d1.u))/l1 + (u - d2 (d2.u))/l2 */
    double tt = (1.0 - vdot(d1, f.t) * vdot(d1, f.t)) / l1 + (1.0 - vdot(d2, f.t) * vdot(d2, f.t)) / l2;
    double tb = (0.0 - vdot(d1, f.t) * vdot(d1, f.b)) / l1 + (0.0 - vdot(d2, f.t) * vdot(d2, f.b)) / l2;
    double bb = (1.0 - vdot(d1, f.b) * vdot(d1, f.b)) / l1 + (1.0 - vdot(d2, f.b) * vdot(d2, f.b)) / l2;
    h[0] = tt; h[1] = tb; h[2] = bb;
}

typedef struct {
    v3 p1x, p2x; oframe2 fx;   /* base path: neighbours and frame of the reconnection vertex */
    v3 p1y, p2y; oframe2 fy;   /* offset path: neighbours and frame (same triangle, its frame) */
    int gauge;                 /* G_AVERAGE (the paper's choice) or a comparison gauge */
} onewton;

static void derivs(v3 p1, v3 p2, const oframe2* f, const double xi[2], double* L, double g[2], double h[3]) {
    double a[3] = {p1.x, p1.y, p1.z}, b[3] = {p2.x, p2.y, p2.z};
    double o[3] = {f->o.x, f->o.y, f->o.z}, t[3] = {f->t.x, f->t.y, f->t.z}, bb[3] = {f->b.x, f->b.y, f->b.z};
    or_length_derivs(a, b, o, t, bb, xi, L, g, h);
}

/* Sec. 4.3: F(xi, xi') = [ L_y(xi') - L_x(xi) - delta ; (R m)^T (xi' - xi) ],
 * m = (grad L_x(xi) + grad L_y(xi')) / 2, R the 90-degree rotation (x, y) -> (-y, x).
 * Each gradient is taken on its own path (base path x for xi, offset path y for xi'), which
 * is what makes the gauge symmetric under swapping the two paths (the reversibility argument
 * of the average-gradient gauge).  The comparison gauges of the same section replace the second
 * row: a fixed axis G(xi) = a^T xi (G_AXIS_T keeps the b coordinate, moving along t; G_AXIS_B
 * keeps the t coordinate) or the gradient at the start point alone, m = grad L_x(xi) (G_START,
 * not reversible: the paper's counterexample). */
static void eval_F(const onewton* N, const double xi[2], double delta, const double xp[2],
                   double gx[2], double hx[3], double Lx, double F[2], double gy[2], double hy[3], double m[2]) {
    double Ly;
    derivs(N->p1y, N->p2y, &N->fy, xp, &Ly, gy, hy);
    m[0] = 0.5 * (gx[0] + gy[0]);
    m[1] = 0.5 * (gx[1] + gy[1]);
    double Rm[2] = {-m[1], m[0]};
    F[0] = Ly - Lx - delta;
    if (N->gauge == G_AXIS_T) F[1] = xp[1] - xi[1];
    else if (N->gauge == G_AXIS_B) F[1] = xp[0] - xi[0];
    else if (N->gauge == G_START) F[1] = -gx[1] * (xp[0] - xi[0]) + gx[0] * (xp[1] - xi[1]);
    else F[1] = Rm[0] * (xp[0] - xi[0]) + Rm[1] * (xp[1] - xi[1]);
}

/* rows of dF/dxi' (A) and dF/dxi (Bm), by differentiating F directly:
 *   dF1/dxi' = grad L_y(xi'),  dF2/dxi' = R m - 0.5 H_y(xi') R (xi' - xi)
 *   dF1/dxi  = -grad L_x(xi),  dF2/dxi  = -(R m + 0.5 H_x(xi) R (xi' - xi))
 * (the printed dF/dxi' second row carries +0.5; the derivative of the stated F, using
 *  R^T = -R, carries -0.5 -- the sign used here, pinned by finite differences in the tests) */
static void jac_F(int gauge, const double xi[2], const double xp[2], const double gx[2], const double hx[3],
                  const double gy[2], const double hy[3], const double m[2], double A[4], double Bm[4]) {
    double Rm[2] = {-m[1], m[0]};
    double dd[2] = {xp[0] - xi[0], xp[1] - xi[1]};
    double Rd[2] = {-dd[1], dd[0]};
    double HyRd[2] = {hy[0] * Rd[0] + hy[1] * Rd[1], hy[1] * Rd[0] + hy[2] * Rd[1]};
    double HxRd[2] = {hx[0] * Rd[0] + hx[1] * Rd[1], hx[1] * Rd[0] + hx[2] * Rd[1]};
    A[0] = gy[0]; A[1] = gy[1];
    Bm[0] = -gx[0]; Bm[1] = -gx[1];
    if (gauge == G_AXIS_T) { A[2] = 0.0; A[3] = 1.0; Bm[2] = 0.0; Bm[3] = -1.0; return; }
    if (gauge == G_AXIS_B) { A[2] = 1.0; A[3] = 0.0; Bm[2] = -1.0; Bm[3] = 0.0; return; }
    if (gauge == G_START) {
        /* F2 = (R g_x)^T d: dF2/dxi' = R g_x, dF2/dxi = -(R g_x + H_x R d) */
        A[2] = -gx[1]; A[3] = gx[0];
        Bm[2] = -(-gx[1] + HxRd[0]); Bm[3] = -(gx[0] + HxRd[1]);
        return;
    }
    A[2] = Rm[0] - 0.5 * HyRd[0]; A[3] = Rm[1] - 0.5 * HyRd[1];
    Bm[2] = -(Rm[0] + 0.5 * HxRd[0]); Bm[3] = -(Rm[1] + 0.5 * HxRd[1]);
}

/* Newton iteration of Sec. 4.3 with backtracking (step halved up to 4 times when |F|_inf does
 * not decrease).  Stops when |F|_inf <= tol_stop -- after one more full step at that point, kept
 * if |F|_inf does not grow -- or after max_iter iterations, extended by up to max_iter more while
 * |F|_inf is already within tol_succ (the paper's success band, 1 % of the gate width).
 * Success: converged, |F|_inf <= tol_stop.  Returns 1 on success; xp = xi', *jdet = |det(dxi'/dxi)| =
 * |det(dF/dxi)| / |det(dF/dxi')| (implicit differentiation), *iters = iterations used. */
static int newton_solve(const onewton* N, const double xi[2], double delta, int max_iter, double tol_stop,
                        double tol_succ, double xp[2], double* jdet, int* iters) {
    double Lx, gx[2], hx[3];
    derivs(N->p1x, N->p2x, &N->fx, xi, &Lx, gx, hx);
    xp[0] = xi[0]; xp[1] = xi[1];
    double F[2], gy[2], hy[3], m[2];
    eval_F(N, xi, delta, xp, gx, hx, Lx, F, gy, hy, m);
    int it = 0, polished = 0;
    /* the paper's budget is max_iter iterations; a solve that spends it inside the success band
     * (|F| <= tol_succ) short of convergence continues toward the root, at most max_iter more, so
     * that an accepted shift is the root F = 0 and not a point of the band */
    while (it < 2 * max_iter) {
        double nF = fmax(fabs(F[0]), fabs(F[1]));
        if (it >= max_iter && !(nF <= tol_succ)) break;
        int polish = 0;
        if (nF <= tol_stop) {
            /* converged: one more full Newton step at the root, kept if |F| does not grow, so that
             * the result is the root itself and not the first iterate under the tolerance (not
             * counted as an iteration) */
            if (polished || !(nF > 0)) break;
            polish = polished = 1;
        }
        double A[4], Bm[4];
        jac_F(N->gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
        double det = A[0] * A[3] - A[1] * A[2];
        if (!(fabs(det) > 1e-300)) break;
        double step[2] = {-(A[3] * F[0] - A[1] * F[1]) / det, -(-A[2] * F[0] + A[0] * F[1]) / det};
        double lam = 1.0;
        int accepted = 0;
        for (int ls = 0; ls < (polish ? 1 : 5); ++ls) {
            double cand[2] = {xp[0] + lam * step[0], xp[1] + lam * step[1]};
            double Fc[2], gyc[2], hyc[3], mc[2];
            eval_F(N, xi, delta, cand, gx, hx, Lx, Fc, gyc, hyc, mc);
            if (polish ? fmax(fabs(Fc[0]), fabs(Fc[1])) <= nF : fmax(fabs(Fc[0]), fabs(Fc[1])) < nF) {
                xp[0] = cand[0]; xp[1] = cand[1];
                F[0] = Fc[0]; F[1] = Fc[1];
                gy[0] = gyc[0]; gy[1] = gyc[1]; hy[0] = hyc[0]; hy[1] = hyc[1]; hy[2] = hyc[2];
                m[0] = mc[0]; m[1] = mc[1];
                accepted = 1;
                break;
            }
            lam *= 0.5;
        }
        if (!accepted) break;
        if (!polish) ++it;
    }
    *iters = it;
    /* success: converged (|F| <= tol_stop), so that the shift satisfies its constraint and stays
     * invertible; a solve stalled inside the band is rejected */
    if (!(fmax(fabs(F[0]), fabs(F[1])) <= tol_stop)) return 0;
    double A[4], Bm[4];
    jac_F(N->gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
    double dA = A[0] * A[3] - A[1] * A[2], dB = Bm[0] * Bm[3] - Bm[1] * Bm[2];
    if (!(fabs(dA) > 0)) return 0;
    *jdet = fabs(dB / dA);
    return isfinite(*jdet);
}

/* exported for the pins: solve on explicit geometry (both frames given) with a gauge */
int or_newton_g(const double* p1x, const double* p2x, const double* fxo, const double* fxt, const double* fxb,
                const double* p1y, const double* p2y, const double* fyo, const double* fyt, const double* fyb,
                const double xi[2], double delta, int max_iter, double tol_stop, double tol_succ,
                double xp[2], double* jdet, int* iters, double F_out[2], int gauge) {
    onewton N;
    N.gauge = gauge;
    N.p1x = vload(p1x); N.p2x = vload(p2x); N.fx.o = vload(fxo); N.fx.t = vload(fxt); N.fx.b = vload(fxb);
    N.p1y = vload(p1y); N.p2y = vload(p2y); N.fy.o = vload(fyo); N.fy.t = vload(fyt); N.fy.b = vload(fyb);
    *jdet = 0; *iters = 0;
    int ok = newton_solve(&N, xi, delta, max_iter, tol_stop, tol_succ, xp, jdet, iters);
    double Lx, gx[2], hx[3], gy[2], hy[3], m[2];
    derivs(N.p1x, N.p2x, &N.fx, xi, &Lx, gx, hx);
    eval_F(&N, xi, delta, xp, gx, hx, Lx, F_out, gy, hy, m);
    return ok;
}
int or_newton(const double* p1x, const double* p2x, const double* fxo, const double* fxt, const double* fxb,
              const double* p1y, const double* p2y, const double* fyo, const double* fyt, const double* fyb,
              const double xi[2], double delta, int max_iter, double tol_stop, double tol_succ,
              double xp[2], double* jdet, int* iters, double F_out[2]) {
    return or_newton_g(p1x, p2x, fxo, fxt, fxb, p1y, p2y, fyo, fyt, fyb, xi, delta, max_iter, tol_stop, tol_succ, xp, jdet,
                       iters, F_out, G_AVERAGE);
}

/* barycentrics (b1, b2) of in-plane coordinates xi on triangle tri */
static void xi_to_bary(const ogeom* g, int tri, const oframe2* f, const double xi[2], double* b1, double* b2) {
    const double* v = tri_v(g, tri);
    v3 v0 = vload(v), e1 = vsub(vload(v + 3), v0), e2 = vsub(vload(v + 6), v0);
    double e1t = vdot(e1, f->t), e2t = vdot(e2, f->t), e2b = vdot(e2, f->b);
    *b2 = xi[1] / e2b;
    *b1 = (xi[0] - *b2 * e2t) / e1t;
}
static void point_to_xi(const oframe2* f, v3 p, double xi[2]) {
    v3 d = vsub(p, f->o);
    xi[0] = vdot(d, f->t);
    xi[1] = vdot(d, f->b);
}

/* ============================================================================================
 * cross-triangle walk of the reconnection vertex (opt-in; the paper parameterises p on the
 * surface, Sec. 4.2, without saying what happens at a triangle's edge, and this walk is one answer:
 * the vertex continues on the neighbouring triangle instead of failing the shift).  The Newton unknown xi'
 * lives in a 2-D chart: the plane of p's triangle, into which each neighbour entered is unfolded
 * about the shared edge (an isometry, so lengths, gradients and |det| carry over).  A candidate
 * that leaves the current triangle crosses its exit edge into the neighbour; the walk fails at a
 * boundary or after MAX_CROSS crossings.  Two developments of one triangle strip differ by a rigid
 * motion, under which the average-gradient gauge is invariant, so the walk keeps the shift
 * reversible.
 * ==========================================================================================*/
#define MAX_CROSS 3
typedef struct { int tri; oframe2 f; double q[3][2]; } owalk;   /* f: chart -> 3-D on tri; q: its corners */

static void walk_init(const ogeom* g, int tri, owalk* W) {
    W->tri = tri;
    W->f = tri_frame(g, tri);
    const double* v = tri_v(g, tri);
    for (int j = 0; j < 3; ++j) {
        v3 d = vsub(vload(v + 3 * j), W->f.o);
        W->q[j][0] = vdot(d, W->f.t);
        W->q[j][1] = vdot(d, W->f.b);
    }
}
static void walk_bary(const owalk* W, const double c[2], double lam[3]) {
    double a0 = W->q[1][0] - W->q[0][0], a1 = W->q[1][1] - W->q[0][1];
    double b0 = W->q[2][0] - W->q[0][0], b1 = W->q[2][1] - W->q[0][1];
    double d0 = c[0] - W->q[0][0], d1 = c[1] - W->q[0][1];
    double det = a0 * b1 - a1 * b0;
    lam[1] = (d0 * b1 - d1 * b0) / det;
    lam[2] = (a0 * d1 - a1 * d0) / det;
    lam[0] = 1.0 - lam[1] - lam[2];
}
/* move W along the chart segment from -> to (from inside W) until the triangle holding `to` */
static int walk_locate(const ogeom* g, owalk* W, const double from_in[2], const double to[2]) {
    double from[2] = {from_in[0], from_in[1]};
    for (int k = 0; k <= MAX_CROSS; ++k) {
        double lt[3], lf[3];
        walk_bary(W, to, lt);
        if (lt[0] >= -BARY_EPS && lt[1] >= -BARY_EPS && lt[2] >= -BARY_EPS) return 1;
        if (k == MAX_CROSS) break;
        walk_bary(W, from, lf);
        int ex = -1;
        double sbest = 1e300;
        for (int i = 0; i < 3; ++i) {
            if (!(lt[i] < -BARY_EPS)) continue;
            double den = lf[i] - lt[i];
            double sx = den > 0 ? lf[i] / den : 0.0;
            if (sx < 0) sx = 0;
            if (sx < sbest) { sbest = sx; ex = i; }
        }
        if (ex < 0) return 0;
        int n = g->adj[3 * W->tri + ex];
        if (n < 0) return 0;
        int nb = n >> 2, opp = n & 3;
        int ia = (ex + 1) % 3, ib = (ex + 2) % 3;
        const double* v = tri_v(g, W->tri);
        v3 A = vload(v + 3 * ia), B = vload(v + 3 * ib), C = vload(tri_v(g, nb) + 3 * opp);
        double a[2] = {W->q[ia][0], W->q[ia][1]}, b[2] = {W->q[ib][0], W->q[ib][1]};
        /* 3-D: edge direction U and in-plane normal N toward the neighbour's third corner;
         * chart: edge direction u and normal n away from the current triangle's third corner */
        v3 U = vnorm(vsub(B, A));
        v3 CA = vsub(C, A);
        v3 Nv = vnorm(vsub(CA, vmul(U, vdot(CA, U))));
        double ul = hypot(b[0] - a[0], b[1] - a[1]);
        double u[2] = {(b[0] - a[0]) / ul, (b[1] - a[1]) / ul};
        double nn[2] = {-u[1], u[0]};
        if ((W->q[ex][0] - a[0]) * nn[0] + (W->q[ex][1] - a[1]) * nn[1] > 0) { nn[0] = -nn[0]; nn[1] = -nn[1]; }
        /* p(c) = A + ((c - a).u) U + ((c - a).n) N = o + c0 t + c1 b */
        owalk Nw;
        Nw.tri = nb;
        Nw.f.t = vadd(vmul(U, u[0]), vmul(Nv, nn[0]));
        Nw.f.b = vadd(vmul(U, u[1]), vmul(Nv, nn[1]));
        Nw.f.o = vsub(A, vadd(vmul(U, a[0] * u[0] + a[1] * u[1]), vmul(Nv, a[0] * nn[0] + a[1] * nn[1])));
        const double* vn = tri_v(g, nb);
        for (int j = 0; j < 3; ++j) {
            v3 d = vsub(vload(vn + 3 * j), Nw.f.o);
            Nw.q[j][0] = vdot(d, Nw.f.t);
            Nw.q[j][1] = vdot(d, Nw.f.b);
        }
        from[0] += sbest * (to[0] - from[0]);
        from[1] += sbest * (to[1] - from[1]);
        *W = Nw;
    }
    return 0;
}

/* Newton with the offset vertex walking across triangles (W: its triangle and chart).  Newton runs
 * on the plane of W's triangle exactly as without the walk; when the converged point lies outside
 * the triangle, W walks along the chart segment from the solve's start to it (unfolding each
 * neighbour it crosses) and Newton continues from that point on the new triangle's plane, with a
 * fresh iteration budget, for at most MAX_CROSS re-solves. */
static int newton_solve_walk(const ogeom* gi, const onewton* N0, owalk* W, const double xi[2], double delta, int max_iter,
                             double tol_stop, double tol_succ, double xp[2], double* jdet, int* iters) {
    onewton N = *N0;
    N.fy = W->f;
    double Lx, gx[2], hx[3];
    derivs(N.p1x, N.p2x, &N.fx, xi, &Lx, gx, hx);
    xp[0] = xi[0]; xp[1] = xi[1];
    double start[2] = {xi[0], xi[1]};
    double F[2], gy[2], hy[3], m[2];
    int total = 0;
    for (int cross = 0;; ++cross) {
        eval_F(&N, xi, delta, xp, gx, hx, Lx, F, gy, hy, m);
        int it = 0, polished = 0;
        while (it < 2 * max_iter) {   /* budget as in newton_solve */
            double nF = fmax(fabs(F[0]), fabs(F[1]));
            if (it >= max_iter && !(nF <= tol_succ)) break;
            int polish = 0;
            if (nF <= tol_stop) {
                /* converged: one more full Newton step at the root, kept if |F| does not grow, so that
                 * the result is the root itself and not the first iterate under the tolerance (not
                 * counted as an iteration) */
                if (polished || !(nF > 0)) break;
                polish = polished = 1;
            }
            double A[4], Bm[4];
            jac_F(N.gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
            double det = A[0] * A[3] - A[1] * A[2];
            if (!(fabs(det) > 1e-300)) break;
            double step[2] = {-(A[3] * F[0] - A[1] * F[1]) / det, -(-A[2] * F[0] + A[0] * F[1]) / det};
            double lam = 1.0;
            int accepted = 0;
            for (int ls = 0; ls < (polish ? 1 : 5); ++ls) {
                double cand[2] = {xp[0] + lam * step[0], xp[1] + lam * step[1]};
                double Fc[2], gyc[2], hyc[3], mc[2];
                eval_F(&N, xi, delta, cand, gx, hx, Lx, Fc, gyc, hyc, mc);
                if (polish ? fmax(fabs(Fc[0]), fabs(Fc[1])) <= nF : fmax(fabs(Fc[0]), fabs(Fc[1])) < nF) {
                    xp[0] = cand[0]; xp[1] = cand[1];
                    F[0] = Fc[0]; F[1] = Fc[1];
                    gy[0] = gyc[0]; gy[1] = gyc[1]; hy[0] = hyc[0]; hy[1] = hyc[1]; hy[2] = hyc[2];
                    m[0] = mc[0]; m[1] = mc[1];
                    accepted = 1;
                    break;
                }
                lam *= 0.5;
            }
            if (!accepted) break;
            if (!polish) ++it;
        }
        total += it;
        if (!(fmax(fabs(F[0]), fabs(F[1])) <= tol_stop)) break;   /* converged, as in newton_solve */
        double lm[3];
        walk_bary(W, xp, lm);
        if (lm[0] >= -BARY_EPS && lm[1] >= -BARY_EPS && lm[2] >= -BARY_EPS) {
            *iters = total;
            double A[4], Bm[4];
            jac_F(N.gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
            double dA = A[0] * A[3] - A[1] * A[2], dB = Bm[0] * Bm[3] - Bm[1] * Bm[2];
            if (!(fabs(dA) > 0)) return 0;
            *jdet = fabs(dB / dA);
            return isfinite(*jdet);
        }
        if (cross == MAX_CROSS) break;
        /* the plane's solution lies outside the triangle: walk there and solve again */
        if (!walk_locate(gi, W, start, xp)) break;
        N.fy = W->f;
        start[0] = xp[0]; start[1] = xp[1];
    }
    *iters = total;
    return 0;
}

/* ============================================================================================
 * path evaluation helpers
 * ==========================================================================================*/
/* geometry term between two surface points (no visibility) */
static double Gterm(const osurf* a, const osurf* b) {
    v3 d = vsub(b->p, a->p);
    double d2 = vdot(d, d);
    if (!(d2 > 0)) return 0.0;
    v3 w = vmul(d, 1.0 / sqrt(d2));
    return fabs(vdot(a->n, w)) * fabs(vdot(b->n, w)) / d2;
}
static v3 dir_to(v3 from, v3 to) { return vnorm(vsub(to, from)); }

/* reconnectability of vertex i on a path x_1..x_k (Sec. 4.1: reconnect at the first
 * consecutive diffuse vertex; the path-length perturbation also re-evaluates the BSDF of the
 * vertex after it, so that vertex must be rough as well, or be the light) */
static int connectable(const int* cls, const v3* pos, int k, int i, double dmin) {
    if (cls[i - 1] != C_ROUGH || cls[i] != C_ROUGH) return 0;
    if (vlen(vsub(pos[i - 1], pos[i])) <= dmin) return 0;
    if (i < k) {
        if (cls[i + 1] != C_ROUGH) return 0;
        if (vlen(vsub(pos[i], pos[i + 1])) <= dmin) return 0;
    }
    return 1;
}
static int find_r(const int* cls, const v3* pos, int k, double dmin) {
    for (int i = 2; i <= k; ++i) if (connectable(cls, pos, k, i, dmin)) return i;
    return 0;
}

/* ============================================================================================
 * stats
 * ==========================================================================================*/
typedef struct { double newton_calls, newton_iters, newton_ok, shift_calls, shift_ok; } ostats;
static void stat_add(double* a, double v) {
#ifdef _OPENMP
#pragma omp atomic
#endif
    *a += v;
}

/* ============================================================================================
 * the shift map (Sec. 4.1-4.3): hybrid shift (random replay up to x_{r-1}, reconnection at
 * p = x_r) followed by the path-length-aware perturbation of p, from domain Dj (the record's
 * own) to domain Di.  Returns 1 on success with the offset path record, its target p_hat in Di
 * and the Jacobian |dS/dx|.
 *
 * gm (optional) replaces the translation of the path length by the scaling of Sec. 4.4 (the
 * path-length shrink mapping): the offset path's gated length is tau' = c + s (tau - c), accepted
 * in [lo, hi), instead of keeping its position inside Di's gate.  s = 1/K shrinks a sample drawn
 * in a gate K times wider about its centre c into the gate; s = K expands it back.  Newton is the
 * same with delta = tau' - tau; only the constraint row of dF/dxi scales by s, so the Jacobian
 * gains the factor s.
 * ==========================================================================================*/
typedef struct { double scale, centre, lo, hi; } ogatemap;

static int shift_rec_g(const orec* x, const odomain* Dj, const odomain* Di, const oparams* P, uint64_t seed,
                       int geom_static, orec* y, double* phat_out, double* jac_out, ostats* st, const ogatemap* gm) {
    if (!x->valid || x->r < 2 || !Di->valid || !Dj->valid) return 0;
    const ogeom* gi = Di->g;
    const ogeom* gj = Dj->g;
    const int k = x->k, r = x->r;
    const double eps = P->ray_eps;
    if (st) stat_add(&st->shift_calls, 1);

    /* (1) random replay of x_2..x_{r-1} from y_1 with the base path's random numbers */
    osurf yv[MAXD + 1];
    v3 ypos[MAXD + 2];
    int ycls[MAXD + 2];
    yv[1] = Di->y1;
    double plen = vlen(vsub(Di->x0, yv[1].p));
    double fpre = 1.0, pdf_pre_y = 1.0;
    for (int j = 1; j <= r - 2; ++j) {
        uint32_t u[4];
        rng4(seed, x->key_px, x->key_frame, ((uint32_t)x->tree << 8) | (uint32_t)j, P_BSDF, u);
        v3 wi = dir_to(yv[j].p, j == 1 ? Di->x0 : yv[j - 1].p);
        const omat* m = &gi->mats[yv[j].mat];
        if (mat_class(m) != x->cls[j]) return 0;
        v3 wo; double pdf, thr; int delta;
        if (!bsdf_sample(m, yv[j].n, wi, u01(u[0]), u01(u[1]), &wo, &pdf, &thr, &delta)) return 0;
        double t;
        if (!trace_from(gi, &yv[j], wo, eps, &yv[j + 1], &t)) return 0;
        double seg = vlen(vsub(yv[j + 1].p, yv[j].p));
        plen += seg;
        if (delta) {
            fpre *= m->albedo;
        } else {
            fpre *= bsdf_f(m, yv[j].n, wi, wo) * Gterm(&yv[j], &yv[j + 1]);
            pdf_pre_y *= pdf * fabs(vdot(yv[j + 1].n, wo)) / (seg * seg);
        }
    }
    if (mat_class(&gi->mats[yv[r - 1].mat]) != x->cls[r - 1]) return 0;

    /* (2) suffix x_{r+1}..x_k and the light, evaluated in the target domain */
    osurf sv[5];
    for (int q = 0; q < x->ns; ++q) sv[q] = surf_at(gi, x->s_tri[q], x->s_b1[q], x->s_b2[q]);
    const olight* Li = &Di->light;
    if (Li->kind == 0) return 0;
    v3 lpos_i = Li->kind == 2 ? Li->s.p : Li->pos;
    double emit_i = Li->kind == 2 ? Li->emit_len : 0.0;
    double slen = 0.0;
    for (int q = 0; q + 1 < x->ns; ++q) slen += vlen(vsub(sv[q].p, sv[q + 1].p));
    if (x->ns > 0) slen += vlen(vsub(sv[x->ns - 1].p, lpos_i)) + emit_i;
    else slen += emit_i;
    v3 p2y = x->ns > 0 ? sv[0].p : lpos_i;

    /* (3) base-path quantities in the record's own frame */
    oframe2 fx = tri_frame(gj, x->p_tri);
    osurf pbase = surf_at(gj, x->p_tri, x->p_b1, x->p_b2);
    v3 p2x;
    if (x->ns > 0) p2x = surf_at(gj, x->s_tri[0], x->s_b1[0], x->s_b2[0]).p;
    else p2x = Dj->light.kind == 2 ? Dj->light.s.p : Dj->light.pos;
    double xi[2];
    point_to_xi(&fx, pbase.p, xi);

    /* (4) Newton solve for xi' (eq. path_length_constraint: L(y') = L(x) + delta, with delta
     * chosen so the sample keeps its position inside the gate of the target domain) */
    onewton N;
    N.p1x = x->xprev; N.p2x = p2x; N.fx = fx; N.gauge = gauge_of(P->flags);
    N.p1y = yv[r - 1].p; N.p2y = p2y; N.fy = tri_frame(gi, x->p_tri);
    double Lx_seg = vlen(vsub(x->xprev, pbase.p)) + vlen(vsub(p2x, pbase.p));
    /* target gated length tau' of the offset path, and the matching target for L_y(xi') */
    double tau_t = gm ? gm->centre + gm->scale * (x->tau - gm->centre) : x->tau - Dj->L0 + Di->L0;
    double ell = tau_t + Di->o - plen - slen;
    double delta = ell - Lx_seg;
    double xp[2], jnewton = 1.0;
    int iters = 0;
    const int walk = (P->flags & F_WALK) && !(P->flags & F_NAIVE);
    owalk W;
    if (walk) walk_init(gi, x->p_tri, &W);
    if (P->flags & F_NAIVE) {
        xp[0] = xi[0]; xp[1] = xi[1];
    } else {
        double tol_stop = 1e-6 * fabs(gm ? tau_t + Di->o : x->tau + Di->o + Di->L0 - Dj->L0);
        double tol_succ = P->newton_tol_frac * (gm ? gm->hi - gm->lo : Di->dL);
        int ok = walk ? newton_solve_walk(gi, &N, &W, xi, delta, P->newton_max_iter, tol_stop, tol_succ, xp, &jnewton, &iters)
                      : newton_solve(&N, xi, delta, P->newton_max_iter, tol_stop, tol_succ, xp, &jnewton, &iters);
        if (st) { stat_add(&st->newton_calls, 1); stat_add(&st->newton_iters, iters); if (ok) stat_add(&st->newton_ok, 1); }
        if (!ok) return 0;
        if (!(jnewton >= 1.0 / P->jac_max && jnewton <= P->jac_max)) return 0;
    }
    double nb1, nb2;
    int ptri = x->p_tri;
    if (walk) {
        double lam[3];
        walk_bary(&W, xp, lam);
        ptri = W.tri; nb1 = lam[1]; nb2 = lam[2];
    } else {
        xi_to_bary(gi, x->p_tri, &N.fy, xp, &nb1, &nb2);
    }
    if (!(nb1 >= -BARY_EPS && nb2 >= -BARY_EPS && nb1 + nb2 <= 1.0 + BARY_EPS)) return 0;
    osurf pp = surf_at(gi, ptri, nb1, nb2);

    /* (5) the offset path must reconnect at the same index (bijectivity of the hybrid shift) */
    {
        int cls[MAXD + 2];
        v3 pos[MAXD + 2];
        for (int j = 1; j <= r - 1; ++j) { cls[j] = mat_class(&gi->mats[yv[j].mat]); pos[j] = yv[j].p; }
        cls[r] = mat_class(&gi->mats[pp.mat]); pos[r] = pp.p;
        for (int q = 0; q < x->ns; ++q) { cls[r + 1 + q] = mat_class(&gi->mats[sv[q].mat]); pos[r + 1 + q] = sv[q].p; }
        if (find_r(cls, pos, k, P->d_min) != r) return 0;
        (void)ycls; (void)ypos;
    }

    /* (6) visibility of the two reconnection segments */
    if (!visible(gi, yv[r - 1].p, yv[r - 1].n, pp.p, &pp.n, eps)) return 0;
    if (x->ns > 0) { if (!visible(gi, pp.p, pp.n, sv[0].p, &sv[0].n, eps)) return 0; }
    else if (!light_visible(gi, Li, &pp, eps)) return 0;

    /* (7) target function of the offset path in domain Di */
    v3 wprev = dir_to(yv[r - 1].p, r - 1 == 1 ? Di->x0 : yv[r - 2].p);
    double f = fpre;
    f *= bsdf_f(&gi->mats[yv[r - 1].mat], yv[r - 1].n, wprev, dir_to(yv[r - 1].p, pp.p));
    f *= Gterm(&yv[r - 1], &pp);
    double Lsuf_i = x->Lsuf;
    if (x->ns == 0) {
        v3 wl; double seg;
        double lt = light_term(gi, Li, &pp, &wl, &seg);
        f *= bsdf_f(&gi->mats[pp.mat], pp.n, dir_to(pp.p, yv[r - 1].p), wl) * lt;
    } else {
        f *= bsdf_f(&gi->mats[pp.mat], pp.n, dir_to(pp.p, yv[r - 1].p), dir_to(pp.p, sv[0].p));
        f *= Gterm(&pp, &sv[0]);
        v3 wnext;
        if (x->ns > 1) wnext = dir_to(sv[0].p, sv[1].p);
        else wnext = dir_to(sv[0].p, lpos_i);
        f *= bsdf_f(&gi->mats[sv[0].mat], sv[0].n, dir_to(sv[0].p, pp.p), wnext);
        int cache_ok = geom_static && light_same(&Dj->light, Li);
        if (!cache_ok) {
            /* Sec. 5: the reconnection information is re-evaluated when the scene or the light
             * differs between the two domains */
            double Ls = 1.0;
            for (int q = 1; q < x->ns; ++q) {
                const omat* mq = &gi->mats[sv[q].mat];
                double gg = mat_class(&gi->mats[sv[q - 1].mat]) == C_DELTA ? 1.0 : Gterm(&sv[q - 1], &sv[q]);
                if (mat_class(mq) == C_DELTA) {
                    if (!geom_static) return 0;
                    Ls *= gg * mq->albedo;
                } else {
                    v3 wn = q + 1 < x->ns ? dir_to(sv[q].p, sv[q + 1].p) : dir_to(sv[q].p, lpos_i);
                    Ls *= gg * bsdf_f(mq, sv[q].n, dir_to(sv[q].p, sv[q - 1].p), wn);
                }
                if (!visible(gi, sv[q - 1].p, sv[q - 1].n, sv[q].p, &sv[q].n, eps)) return 0;
            }
            v3 wl; double seg;
            Ls *= light_term(gi, Li, &sv[x->ns - 1], &wl, &seg);
            if (!light_visible(gi, Li, &sv[x->ns - 1], eps)) return 0;
            Lsuf_i = Ls;
        }
        f *= Lsuf_i;
    }
    double Lnew = plen + vlen(vsub(yv[r - 1].p, pp.p)) + vlen(vsub(pp.p, p2y)) + slen;
    double tau = Lnew - Di->o;
    if (gm) { if (!(tau >= gm->lo && tau < gm->hi)) return 0; }
    else if (!(tau >= Di->L0 && tau < Di->L0 + Di->dL)) return 0;
    if (!(f > 0) || !isfinite(f)) return 0;

    /* (8) Jacobian: replay pdf ratios (area measure) times the Newton determinant; the frame
     * factor sqrt(det J'^T J') / sqrt(det J^T J) is 1 for the orthonormal in-plane frames; a
     * scaling gate map contributes its factor s */
    double jac = (x->pdf_pre / pdf_pre_y) * jnewton * (gm ? gm->scale : 1.0);
    if (!(jac > 0) || !isfinite(jac)) return 0;

    *y = *x;
    y->tau = tau;
    y->xprev = yv[r - 1].p;
    y->pdf_pre = pdf_pre_y;
    y->p_tri = ptri; y->p_b1 = nb1; y->p_b2 = nb2;
    y->Lsuf = Lsuf_i;
    y->phat = f;
    *phat_out = f;
    *jac_out = jac;
    if (st) stat_add(&st->shift_ok, 1);
    return 1;
}

static int shift_rec(const orec* x, const odomain* Dj, const odomain* Di, const oparams* P, uint64_t seed,
                     int geom_static, orec* y, double* phat_out, double* jac_out, ostats* st) {
    return shift_rec_g(x, Dj, Di, P, seed, geom_static, y, phat_out, jac_out, st, NULL);
}

/* ============================================================================================
 * frame state
 * ==========================================================================================*/
typedef struct {
    const ogeom* g;
    osensor s; oemitter e;
    double L0, dL; int B;
    uint32_t frame;
    olight laser;          /* resolved laser spot (emitter type 1) */
    ogb* gb;               /* W*H */
    orec* res;             /* W*H*Bn */
    double* M;             /* W*H confidence per pixel, shared by all bins */
    uint8_t* ok;           /* W*H : computed and untainted */
} oframe;

typedef struct {
    int W, H, Bn;
    int has_prev;
    int cur;
    oframe fr[2];
    ostats st;
} oview;

oview* or_view_create(int W, int H, int B) {
    oview* v = (oview*)calloc(1, sizeof(oview));
    v->W = W; v->H = H; v->Bn = B > 0 ? B : 1;
    for (int i = 0; i < 2; ++i) {
        v->fr[i].gb = (ogb*)calloc((size_t)W * H, sizeof(ogb));
        v->fr[i].res = (orec*)calloc((size_t)W * H * v->Bn, sizeof(orec));
        v->fr[i].ok = (uint8_t*)calloc((size_t)W * H, 1);
        v->fr[i].M = (double*)calloc((size_t)W * H, sizeof(double));
    }
    return v;
}
void or_view_destroy(oview* v) {
    if (!v) return;
    for (int i = 0; i < 2; ++i) { free(v->fr[i].gb); free(v->fr[i].res); free(v->fr[i].ok); free(v->fr[i].M); }
    free(v);
}
void or_view_reset(oview* v) { v->has_prev = 0; }
void or_view_stats(const oview* v, double out[5]) {
    out[0] = v->st.newton_calls; out[1] = v->st.newton_iters; out[2] = v->st.newton_ok;
    out[3] = v->st.shift_calls; out[4] = v->st.shift_ok;
}

/* pinhole / confocal primary ray of pixel (ix, iy) with sub-pixel jitter (u0, u1) */
static void primary_ray(const osensor* s, int ix, int iy, double u0, double u1, v3* o, v3* d) {
    *o = vload(s->pos);
    if (s->mode == 1) {
        v3 w = vadd(vload(s->wall_o), vadd(vmul(vload(s->wall_u), (ix + 0.5) / s->W), vmul(vload(s->wall_v), (iy + 0.5) / s->H)));
        *d = vnorm(vsub(w, *o));
        return;
    }
    v3 f = vnorm(vload(s->fwd));
    v3 rt = vnorm(vcross(f, vload(s->up)));
    v3 up = vcross(rt, f);
    double th = tan(0.5 * s->fov_y), asp = (double)s->W / (double)s->H;
    double sx = (2.0 * (ix + u0) / s->W - 1.0) * th * asp;
    double sy = (1.0 - 2.0 * (iy + u1) / s->H) * th;
    *d = vnorm(vadd(f, vadd(vmul(rt, sx), vmul(up, sy))));
}

/* pixel of a world point in a pinhole sensor (back-projection for temporal reuse) */
static int project(const osensor* s, v3 p, int* ix, int* iy) {
    v3 f = vnorm(vload(s->fwd));
    v3 rt = vnorm(vcross(f, vload(s->up)));
    v3 up = vcross(rt, f);
    v3 d = vsub(p, vload(s->pos));
    double z = vdot(d, f);
    if (!(z > 0)) return 0;
    double th = tan(0.5 * s->fov_y), asp = (double)s->W / (double)s->H;
    double sx = vdot(d, rt) / z / (th * asp), sy = vdot(d, up) / z / th;
    double fx = (sx + 1.0) * 0.5 * s->W, fy = (1.0 - sy) * 0.5 * s->H;
    if (!(fx >= 0 && fy >= 0)) return 0;
    int x = (int)floor(fx), y = (int)floor(fy);
    if (x >= s->W || y >= s->H) return 0;
    *ix = x; *iy = y;
    return 1;
}

static odomain make_domain(const oframe* F, int pix, const oparams* P, double L0, double dL) {
    odomain D;
    memset(&D, 0, sizeof(D));
    D.g = F->g;
    D.x0 = vload(F->s.pos);
    const ogb* gb = &F->gb[pix];
    D.valid = gb->valid;
    D.L0 = L0; D.dL = dL;
    if (!gb->valid) return D;
    D.y1 = gb->s;
    D.o = F->s.mode == 1 ? 2.0 * gb->t : 0.0;
    if (F->e.type == 0) { D.light.kind = 1; D.light.pos = vload(F->e.pos); D.light.I = F->e.power; }
    else if (F->e.type == 1) D.light = F->laser;
    else {
        D.light.kind = 2; D.light.s = gb->s; D.light.I = F->e.power;
        D.light.to_origin = vnorm(vsub(vload(F->e.pos), gb->s.p));
        D.light.emit_len = vlen(vsub(vload(F->e.pos), gb->s.p));
        D.light.pos = gb->s.p;
    }
    (void)P;
    return D;
}


/* ============================================================================================
 * ellipsoidal path connection for NEE (Sec. 4.4 "Initialization with Ellipsoidal Path
 * Connection", Sec. 5 "Ellipsoidal Path Connection"; Pediredla et al. 2019).  From a rough
 * vertex x whose prefix has length len, a vertex z is placed so that the path x -> z -> light
 * lands in the gate:
 *   (1) l = |x - z| + |z - q| (q the light position) uniform on [l_a, l_b), the interval the gate
 *       leaves (l_a raised to |x - q|);
 *   (2) a triangle by a top-down walk of the index hierarchy above: at each node the child is
 *       taken with probability proportional to its weight, the area below it, or zero where the
 *       node's box cannot meet the ellipsoid with foci x, q and major axis l (the paper's
 *       heuristic weights; the test is conservative: the distances of x and of q to the box bound
 *       l from below, their distances to the box's farthest points bound it from above);
 *   (3) on the triangle's plane the ellipsoid cuts an ellipse; z is uniform in the ellipse's
 *       parametric angle phi over the arcs inside the triangle (total angle Phi).
 * Area density of z (coarea formula: dA = dl ds / |grad_plane l|, ds = |dz/dphi| dphi):
 *   p_ell(z) = P(tri | l) / (l_b - l_a) / Phi * |grad_plane l(z)| / |dz/dphi|.
 * Ellipsoids thinner than b = 0.05 a (a the semi-major axis: l within about 1.25e-3 l of |x - q|)
 * place no vertex, in the sampler and in the density alike; the MIS with the path tree covers them.
 * (There z depends on l - |x - q|, a difference of path lengths that single precision resolves to
 * ~1e-6 m; the cut keeps the GPU's FP32 placement within ~5e-5 of this FP64 one.)
 * ==========================================================================================*/
static double enode_w(const double* e, v3 x, v3 q, double ell) {
    if (!(e[6] > 0)) return 0.0;
    double px[3] = {x.x, x.y, x.z}, pq[3] = {q.x, q.y, q.z};
    double dx2 = 0.0, dq2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double cx = fmin(fmax(px[k], e[k]), e[3 + k]), cq = fmin(fmax(pq[k], e[k]), e[3 + k]);
        dx2 += (px[k] - cx) * (px[k] - cx);
        dq2 += (pq[k] - cq) * (pq[k] - cq);
    }
    double lb = sqrt(dx2) + sqrt(dq2);
    if (lb > ell) return 0.0;
    double fx2 = 0.0, fq2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double a = fmax(fabs(px[k] - e[k]), fabs(px[k] - e[3 + k])), b = fmax(fabs(pq[k] - e[k]), fabs(pq[k] - e[3 + k]));
        fx2 += a * a; fq2 += b * b;
    }
    double ub = sqrt(fx2) + sqrt(fq2);
    return ell <= ub ? e[6] : 0.0;
}

static int elog2(int P) { int L = 0; while ((1 << L) < P) ++L; return L; }

/* step (2): the triangle (or -1) and its probability; u: one uniform per level */
static int etree_pick(const ogeom* g, v3 x, v3 q, double ell, const double* u, double* prob) {
    int n = 1, lvl = 0;
    double p = 1.0;
    while (n < g->eP) {
        double w0 = enode_w(g->enode + 8 * (size_t)(2 * n), x, q, ell);
        double w1 = enode_w(g->enode + 8 * (size_t)(2 * n + 1), x, q, ell);
        double s = w0 + w1;
        if (!(s > 0)) return -1;
        if (u[lvl] * s < w0) { n = 2 * n; p *= w0 / s; }
        else { n = 2 * n + 1; p *= w1 / s; }
        ++lvl;
    }
    *prob = p;
    return n - g->eP;
}
/* P(tri | l) of step (2), walking the root-to-leaf path of tri */
static double etree_prob(const ogeom* g, int tri, v3 x, v3 q, double ell) {
    const int L = elog2(g->eP), leaf = g->eP + tri;
    double p = 1.0;
    for (int i = 0; i < L; ++i) {
        int n = leaf >> (L - i), next = leaf >> (L - i - 1);
        double w0 = enode_w(g->enode + 8 * (size_t)(2 * n), x, q, ell);
        double w1 = enode_w(g->enode + 8 * (size_t)(2 * n + 1), x, q, ell);
        double s = w0 + w1, w = next == 2 * n ? w0 : w1;
        if (!(s > 0) || !(w > 0)) return 0.0;
        p *= w / s;
    }
    return p;
}

/* step (3): the ellipse the ellipsoid (foci x, q; major axis l) cuts from the plane of tri, in the
 * triangle's frame (o = v0, t, b):  xi = xo + w0 + R1 cos(phi) g1 + R2 sin(phi) g2, and the arcs
 * of phi inside the triangle.  With m the centre, a = l/2, c = |q - x|/2, b^2 = a^2 - c^2,
 * d = (q - x)/|q - x|, n the normal, h = (m - v0).n, the plane's points m - h n + w1 t + w2 b
 * satisfy |r|^2 + beta (r.d)^2 = b^2 (beta = -c^2/a^2), i.e. w^T (I + beta g g^T) w
 * - 2 beta h (d.n) g.w + h^2 (1 + beta (d.n)^2) - b^2 = 0 with g = (d.t, d.b): centre
 * w0 = beta h (d.n) g / gamma, gamma = 1 + beta |g|^2, and (w - w0)^T A (w - w0) = kappa =
 * b^2 (1 - h^2 / (a^2 gamma)); radii sqrt(kappa / gamma) along g, sqrt(kappa) across it. */
typedef struct {
    double xo[2], w0[2], g1[2], g2[2], R1, R2;
    int narc;
    double a0[6], alen[6];
    double Phi;
} oellip;

static int ellip_inside(const double c[3][2], double orient, double px, double py) {
    for (int i = 0; i < 3; ++i) {
        const double* a = c[i];
        const double* b = c[(i + 1) % 3];
        double cr = (b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0]);
        if (cr * orient < 0) return 0;
    }
    return 1;
}

/* zp: a point known to lie on the ellipse (the density evaluated at a vertex placed by other
 * means), or NULL.  With a point, kappa is the ellipse's quadratic form at it, which equals the
 * expression above without its cancellation where the plane nearly touches the ellipsoid (the point
 * near the plane's mirror point of x and q, where l is minimal). */
static int ellip_on_tri(const ogeom* g, int tri, v3 x, v3 q, double ell, oellip* E, const v3* zp) {
    oframe2 f = tri_frame(g, tri);
    v3 n = vcross(f.t, f.b);
    v3 m = vmul(vadd(x, q), 0.5);
    double a = 0.5 * ell, c = 0.5 * vlen(vsub(q, x));
    double b2 = a * a - c * c;
    if (!(b2 >= 2.5e-3 * a * a)) return 0;
    v3 d = c > 0 ? vmul(vsub(q, x), 0.5 / c) : V(0, 0, 0);
    double beta = -(c * c) / (a * a);
    double dt = vdot(d, f.t), db = vdot(d, f.b), dn = vdot(d, n);
    double h = vdot(vsub(m, f.o), n);
    double gamma = 1.0 + beta * (dt * dt + db * db);
    E->xo[0] = vdot(vsub(m, f.o), f.t);
    E->xo[1] = vdot(vsub(m, f.o), f.b);
    E->w0[0] = beta * h * dn * dt / gamma;
    E->w0[1] = beta * h * dn * db / gamma;
    double kappa;
    if (zp) {
        double d0 = vdot(vsub(*zp, f.o), f.t) - E->xo[0] - E->w0[0], d1 = vdot(vsub(*zp, f.o), f.b) - E->xo[1] - E->w0[1];
        double gd = dt * d0 + db * d1;
        kappa = d0 * d0 + d1 * d1 + beta * gd * gd;
    } else {
        kappa = b2 * (1.0 - h * h / (a * a * gamma));
    }
    if (!(kappa > 0)) return 0;
    double gl = sqrt(dt * dt + db * db);
    if (gl > 1e-12) { E->g1[0] = dt / gl; E->g1[1] = db / gl; }
    else { E->g1[0] = 1.0; E->g1[1] = 0.0; }
    E->g2[0] = -E->g1[1]; E->g2[1] = E->g1[0];
    E->R1 = sqrt(kappa / gamma);
    E->R2 = sqrt(kappa);
    /* corners in the unit-circle coordinates of the ellipse */
    const double* v = tri_v(g, tri);
    v3 v0 = vload(v);
    double cc[3][2];
    for (int i = 0; i < 3; ++i) {
        v3 dv = vsub(vload(v + 3 * i), v0);
        double w[2] = {vdot(dv, f.t) - E->xo[0] - E->w0[0], vdot(dv, f.b) - E->xo[1] - E->w0[1]};
        cc[i][0] = (w[0] * E->g1[0] + w[1] * E->g1[1]) / E->R1;
        cc[i][1] = (w[0] * E->g2[0] + w[1] * E->g2[1]) / E->R2;
    }
    double orient = (cc[1][0] - cc[0][0]) * (cc[2][1] - cc[0][1]) - (cc[1][1] - cc[0][1]) * (cc[2][0] - cc[0][0]);
    if (orient == 0.0) return 0;
    /* crossings of the unit circle with the edges */
    double ph[6];
    int np = 0;
    for (int i = 0; i < 3; ++i) {
        const double* P0 = cc[i];
        const double* P1 = cc[(i + 1) % 3];
        double e0 = P1[0] - P0[0], e1 = P1[1] - P0[1];
        double A2 = e0 * e0 + e1 * e1, B2 = P0[0] * e0 + P0[1] * e1, C2 = P0[0] * P0[0] + P0[1] * P0[1] - 1.0;
        double disc = B2 * B2 - A2 * C2;
        if (!(disc > 0) || !(A2 > 0)) continue;
        double sq = sqrt(disc);
        double sr[2] = {(-B2 - sq) / A2, (-B2 + sq) / A2};
        for (int k = 0; k < 2; ++k)
            if (sr[k] >= 0.0 && sr[k] <= 1.0) ph[np++] = atan2(P0[1] + sr[k] * e1, P0[0] + sr[k] * e0);
    }
    for (int i = 1; i < np; ++i)
        for (int j = i; j > 0 && ph[j - 1] > ph[j]; --j) { double t = ph[j]; ph[j] = ph[j - 1]; ph[j - 1] = t; }
    E->narc = 0;
    E->Phi = 0.0;
    if (np == 0) {
        if (ellip_inside(cc, orient, 1.0, 0.0)) { E->narc = 1; E->a0[0] = 0.0; E->alen[0] = 2.0 * OPI; E->Phi = 2.0 * OPI; }
    } else {
        for (int i = 0; i < np; ++i) {
            double s0 = ph[i], s1 = i + 1 < np ? ph[i + 1] : ph[0] + 2.0 * OPI;
            if (!(s1 > s0)) continue;
            double mid = 0.5 * (s0 + s1);
            if (!ellip_inside(cc, orient, cos(mid), sin(mid))) continue;
            E->a0[E->narc] = s0; E->alen[E->narc] = s1 - s0; E->narc++;
            E->Phi += s1 - s0;
        }
    }
    return E->Phi > 0;
}

/* interval [l_a, l_b) of l = |x - z| + |z - q| that puts the path in [glo, ghi); 0 if empty */
static int ell_range(const odomain* D, v3 x, double len, double glo, double ghi, v3* q, double* la, double* lb) {
    if (D->light.kind == 0) return 0;
    *q = D->light.kind == 2 ? D->light.s.p : D->light.pos;
    double e = D->light.kind == 2 ? D->light.emit_len : 0.0;
    *la = fmax(glo + D->o - len - e, vlen(vsub(x, *q)));
    *lb = ghi + D->o - len - e;
    return *lb > *la;
}

/* density factor |grad_plane l(z)| / |dz/dphi| and P(tri | l) (1/(l_b - l_a) and 1/Phi apart) */
static double ell_point_factor(const oellip* E, const oframe2* f, v3 z, v3 x, v3 q) {
    v3 gr = vadd(dir_to(x, z), dir_to(q, z));
    double gt = vdot(gr, f->t), gb = vdot(gr, f->b);
    double gp = sqrt(gt * gt + gb * gb);
    double w[2] = {vdot(vsub(z, f->o), f->t) - E->xo[0] - E->w0[0], vdot(vsub(z, f->o), f->b) - E->xo[1] - E->w0[1]};
    double c0 = (w[0] * E->g1[0] + w[1] * E->g1[1]) / E->R1, c1 = (w[0] * E->g2[0] + w[1] * E->g2[1]) / E->R2;
    double cl = sqrt(c0 * c0 + c1 * c1);
    if (!(cl > 0)) return 0.0;
    c0 /= cl; c1 /= cl;
    double dz = sqrt(E->R1 * E->R1 * c1 * c1 + E->R2 * E->R2 * c0 * c0);
    return dz > 0 ? gp / dz : 0.0;
}

/* steps (2)-(3) for l_a <= l < l_b given the draws u (u[0] -> l, u[1] -> phi, u[2..] -> the levels) */
static int ell_sample_core(const ogeom* g, v3 x, v3 q, double la, double lb, const uint32_t u[24], osurf* z, double* pdf) {
    if (g->nt < 1 || elog2(g->eP) > ELL_MAX_LEVELS || !(lb > la)) return 0;
    double ell = la + u01(u[0]) * (lb - la);
    double ul[ELL_MAX_LEVELS];
    for (int k = 0; k < ELL_MAX_LEVELS; ++k) ul[k] = u01(u[2 + k]);
    double ptri;
    int tri = etree_pick(g, x, q, ell, ul, &ptri);
    if (tri < 0) return 0;
    oellip E;
    if (!ellip_on_tri(g, tri, x, q, ell, &E, NULL)) return 0;
    double t = u01(u[1]) * E.Phi, cum = 0.0, phi = 0.0;
    for (int i = 0; i < E.narc; ++i) {
        if (t < cum + E.alen[i] || i == E.narc - 1) { phi = E.a0[i] + fmin(t - cum, E.alen[i]); break; }
        cum += E.alen[i];
    }
    double cp = cos(phi), sp = sin(phi);
    double xi[2] = {E.xo[0] + E.w0[0] + E.R1 * cp * E.g1[0] + E.R2 * sp * E.g2[0],
                    E.xo[1] + E.w0[1] + E.R1 * cp * E.g1[1] + E.R2 * sp * E.g2[1]};
    oframe2 f = tri_frame(g, tri);
    double b1, b2;
    xi_to_bary(g, tri, &f, xi, &b1, &b2);
    *z = surf_at(g, tri, b1, b2);
    *pdf = ptri / (lb - la) / E.Phi * ell_point_factor(&E, &f, z->p, x, q);
    return *pdf > 0;
}
static double ell_pdf_core(const ogeom* g, v3 x, v3 q, double la, double lb, const osurf* z) {
    if (g->nt < 1 || elog2(g->eP) > ELL_MAX_LEVELS || !(lb > la)) return 0.0;
    double ell = vlen(vsub(z->p, x)) + vlen(vsub(q, z->p));
    if (!(ell >= la && ell < lb)) return 0.0;
    double ptri = etree_prob(g, z->tri, x, q, ell);
    if (!(ptri > 0)) return 0.0;
    oellip E;
    if (!ellip_on_tri(g, z->tri, x, q, ell, &E, &z->p)) return 0.0;
    oframe2 f = tri_frame(g, z->tri);
    return ptri / (lb - la) / E.Phi * ell_point_factor(&E, &f, z->p, x, q);
}

/* sample z from vertex x (prefix length len, path tree `tree`, vertex index d); 1 if placed */
static int ell_sample(const ogeom* g, const odomain* D, uint64_t seed, uint32_t px, uint32_t frame, int tree, int d,
                      const osurf* x, double len, double glo, double ghi, osurf* z, double* pdf) {
    v3 q;
    double la, lb;
    if (!ell_range(D, x->p, len, glo, ghi, &q, &la, &lb)) return 0;
    uint32_t u[24];
    for (int k = 0; k < 6; ++k) rng4(seed, px, frame, ((uint32_t)tree << 8) | (uint32_t)d, P_ELL + k, u + 4 * k);
    return ell_sample_core(g, x->p, q, la, lb, u, z, pdf);
}

/* p_ell(z) of a vertex z reached from x by other means (0 where the sampler cannot place it) */
static double ell_pdf(const ogeom* g, const odomain* D, const osurf* x, double len, double glo, double ghi, const osurf* z) {
    v3 q;
    double la, lb;
    if (!ell_range(D, x->p, len, glo, ghi, &q, &la, &lb)) return 0.0;
    return ell_pdf_core(g, x->p, q, la, lb, z);
}

/* test access: one ellipsoidal placement from x toward light position q on [la, lb) with the draws
 * u[24]; out = (tri, b1, b2, pdf, z.xyz); returns 1 if placed.  And the density at (tri, b1, b2). */
int or_ell_sample(const ogeom* g, const double* x, const double* q, double la, double lb, const uint32_t* u, double out[7]) {
    osurf z;
    double pdf = 0.0;
    if (!ell_sample_core(g, vload(x), vload(q), la, lb, u, &z, &pdf)) return 0;
    out[0] = z.tri; out[1] = z.b1; out[2] = z.b2; out[3] = pdf; out[4] = z.p.x; out[5] = z.p.y; out[6] = z.p.z;
    return 1;
}
double or_ell_pdf(const ogeom* g, const double* x, const double* q, double la, double lb, int tri, double b1, double b2) {
    osurf z = surf_at(g, tri, b1, b2);
    return ell_pdf_core(g, vload(x), vload(q), la, lb, &z);
}
/* P(tri | l) of the hierarchy walk, for every triangle (out[nt]) */
void or_ell_tri_probs(const ogeom* g, const double* x, const double* q, double ell, double* out) {
    for (int t = 0; t < g->nt; ++t) out[t] = etree_prob(g, t, vload(x), vload(q), ell);
}

/* ============================================================================================
 * resampling primitives shared by every RIS / GRIS step of the pipeline (Sec. 3.2)
 * ==========================================================================================*/
/* One step of streaming resampling: the running weight sum S grows by the candidate's resampling
 * weight w > 0, and the candidate replaces the current selection when u S < w (u uniform in
 * [0, 1)).  Over a stream of candidates the last replacement is the selection, which picks
 * candidate i with probability w_i / sum_j w_j (basic RIS and the GRIS merge alike). */
static int ris_accept(double* S, double w, double u) {
    *S += w;
    return u * *S < w;
}
/* unbiased contribution weight of the selected sample y: the sum of the resampling weights over
 * the target at y, W_y = (sum_j w_j) / p_hat(y) (Sec. 3.2, RIS and GRIS estimators) */
static double ris_W(double S, double phat) { return S / phat; }
/* MIS weight of candidate s in a GRIS merge of n domains with confidences M, given
 * T_j = p_hat_{<-j}(y_s), the target of domain j at y_s carried back by the inverse shift with its
 * Jacobian (0 where that shift fails), T_0 = p_hat_0(y_s) of the canonical domain, T_s the
 * candidate's own domain term.  Generalized balance heuristic (eq. GRIS_MIS_weight, every term
 * evaluated at the same y_s): m_s = M_s T_s / sum_j M_j T_j.  Pairwise (an opt-in from the
 * ReSTIR literature): the canonical domain pairs with each reused domain i as a two-technique
 * balance heuristic with confidences M_0/k and M_i, weighted by a_i = (M_i + M_0/k) / sum_j M_j;
 * m_0 = sum_i a_i (M_0/k) T_0 / ((M_0/k) T_0 + M_i T_i), m_s = a_s M_s T_s / (M_s T_s + (M_0/k) T_0).
 * Either way the weights of one y over the domains that can produce it sum to 1. */
static double gris_mis(const double* M, const double* T, int n, int s, int pairwise) {
    if (pairwise && n > 1) {
        const int k = n - 1;
        double Msum = 0.0;
        for (int j = 0; j < n; ++j) Msum += M[j];
        const double Mck = M[0] / k;
        if (s == 0) {
            double m = 0.0;
            for (int i = 1; i < n; ++i) {
                double pc = Mck * T[0], ti = M[i] * T[i];
                m += (M[i] + Mck) / Msum * (pc / (pc + ti));
            }
            return m;
        }
        double pi = M[s] * T[s], pc = Mck * T[0];
        return (M[s] + Mck) / Msum * (pi / (pi + pc));
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += M[j] * T[j];
    return den > 0 ? M[s] * T[s] / den : 0.0;
}

/* ============================================================================================
 * initial candidates (Sec. 3.2 RIS, stage (1); Sec. 4.5 per-bin deposit for transients)
 * Path trees: BSDF-sampled paths with NEE to the delta light at every vertex; the candidate of
 * length k is the NEE path ending at x_k.  w = (1/N) p_hat / p with p_hat = f 1[tau in gate].
 * ==========================================================================================*/
typedef struct { osurf v[MAXD + 2]; double pdfA[MAXD + 2]; int cls[MAXD + 2]; } opathbuf;

/* f(x) in area measure of the path x_1..x_k with NEE to the light (no visibility) */
static double path_f(const ogeom* g, const odomain* D, const opathbuf* pb, int k) {
    double f = 1.0;
    for (int j = 1; j <= k; ++j) {
        const omat* m = &g->mats[pb->v[j].mat];
        v3 wi = dir_to(pb->v[j].p, j == 1 ? D->x0 : pb->v[j - 1].p);
        if (j < k) {
            if (mat_class(m) == C_DELTA) f *= m->albedo;
            else f *= bsdf_f(m, pb->v[j].n, wi, dir_to(pb->v[j].p, pb->v[j + 1].p)) * Gterm(&pb->v[j], &pb->v[j + 1]);
        } else {
            v3 wl; double seg;
            double lt = light_term(g, &D->light, &pb->v[k], &wl, &seg);
            f *= bsdf_f(m, pb->v[k].n, wi, wl) * lt;
        }
    }
    return f;
}

static void build_rec(const ogeom* g, const odomain* D, const opathbuf* pb, int k, int tree, uint32_t px,
                      uint32_t frame, double tau, const oparams* P, orec* R) {
    memset(R, 0, sizeof(*R));
    R->valid = 1;
    R->tau = tau;
    R->key_px = px; R->key_frame = frame; R->tree = tree; R->k = k;
    R->phat = path_f(g, D, pb, k);
    v3 pos[MAXD + 2];
    for (int j = 1; j <= k; ++j) pos[j] = pb->v[j].p;
    int r = find_r(pb->cls, pos, k, P->d_min);
    R->r = r;
    if (r == 0) return;
    for (int j = 1; j < r; ++j) R->cls[j] = pb->cls[j];
    R->xprev = pb->v[r - 1].p;
    R->pdf_pre = 1.0;
    for (int j = 2; j <= r - 1; ++j) R->pdf_pre *= pb->pdfA[j];
    R->p_tri = pb->v[r].tri; R->p_b1 = pb->v[r].b1; R->p_b2 = pb->v[r].b2;
    R->ns = k - r;
    for (int q = 0; q < R->ns; ++q) { R->s_tri[q] = pb->v[r + 1 + q].tri; R->s_b1[q] = pb->v[r + 1 + q].b1; R->s_b2[q] = pb->v[r + 1 + q].b2; }
    /* suffix factor beyond x_{r+1}: prod_{j=r+2..k} G(x_{j-1}, x_j) f_s(x_j) * light term */
    if (R->ns > 0) {
        double Ls = 1.0;
        for (int j = r + 2; j <= k; ++j) {
            const omat* m = &g->mats[pb->v[j].mat];
            const omat* mprev = &g->mats[pb->v[j - 1].mat];
            double gg = mat_class(mprev) == C_DELTA ? 1.0 : Gterm(&pb->v[j - 1], &pb->v[j]);
            if (mat_class(m) == C_DELTA) { Ls *= gg * m->albedo; continue; }
            v3 wi = dir_to(pb->v[j].p, pb->v[j - 1].p);
            v3 wo;
            if (j < k) wo = dir_to(pb->v[j].p, pb->v[j + 1].p);
            else { double seg; light_term(g, &D->light, &pb->v[k], &wo, &seg); }
            Ls *= gg * bsdf_f(m, pb->v[j].n, wi, wo);
        }
        v3 wl; double seg;
        Ls *= light_term(g, &D->light, &pb->v[k], &wl, &seg);
        R->Lsuf = Ls;
    }
}

/* One path tree; calls the candidate sink for every NEE path of length k in [kmin, depth].
 * The sink receives (k, c = f/p without the gate, tau, the strategy: 0 the tree's own NEE, 1 the
 * ellipsoidal connection).  With `ell`, every rough vertex x_d (d < depth) also places a vertex z
 * by the ellipsoidal connection, a candidate of length d + 1; it and the tree's NEE candidate of
 * the same length (whose last vertex x_{d+1} the tree sampled from x_d) are combined by the
 * balance heuristic over the two densities of that vertex (Sec. 5: MIS between the direct and the
 * ellipsoidal connection):  c_tree *= p_tree / (p_tree + p_ell),  c_ell = f / (p_tree + p_ell). */
typedef void (*cand_sink)(void* ctx, int k, double c, double tau, const opathbuf* pb, int strategy);

static void trace_tree(const ogeom* g, const odomain* D, const oparams* P, uint64_t seed, uint32_t px, uint32_t frame,
                       int tree, int gated_lo_hi, double glo, double ghi, int ell, cand_sink sink, void* ctx) {
    opathbuf pb;
    pb.v[1] = D->y1;
    pb.cls[1] = mat_class(&g->mats[D->y1.mat]);
    pb.pdfA[1] = 1.0;
    double len = vlen(vsub(D->x0, D->y1.p));
    double beta = 1.0;
    int kmin = (P->flags & F_DIRECT) ? 1 : 2;
    int ell_prev = 0;        /* the ellipsoidal connection was available at x_{d-1} */
    double len_prev = 0.0;
    for (int d = 1; d <= P->depth; ++d) {
        const osurf* x = &pb.v[d];
        const omat* m = &g->mats[x->mat];
        v3 wi = dir_to(x->p, d == 1 ? D->x0 : pb.v[d - 1].p);
        if (d >= kmin && mat_class(m) != C_DELTA) {
            v3 wl; double seg;
            double lt = light_term(g, &D->light, x, &wl, &seg);
            double fs = lt > 0 ? bsdf_f(m, x->n, wi, wl) : 0.0;
            if (fs > 0) {
                double tau = len + seg - D->o;
                int in = gated_lo_hi ? (tau >= glo && tau < ghi) : 1;
                if (in && light_visible(g, &D->light, x, P->ray_eps)) {
                    double c = beta * fs * lt;
                    if (ell_prev) {
                        double pt = pb.pdfA[d], pe = ell_pdf(g, D, &pb.v[d - 1], len_prev, glo, ghi, x);
                        c *= pt / (pt + pe);
                    }
                    sink(ctx, d, c, tau, &pb, 0);
                }
            }
        }
        const int ell_here = ell && gated_lo_hi && d < P->depth && mat_class(m) != C_DELTA && D->light.kind != 0;
        if (ell_here) {
            osurf z;
            double pe;
            if (ell_sample(g, D, seed, px, frame, tree, d, x, len, glo, ghi, &z, &pe)) {
                const omat* mz = &g->mats[z.mat];
                v3 wz = dir_to(x->p, z.p);
                double dist = vlen(vsub(z.p, x->p));
                double fx = bsdf_f(m, x->n, wi, wz);
                if (fx > 0 && dist > 0 && mat_class(mz) != C_DELTA) {
                    v3 wl; double seg;
                    double lt = light_term(g, &D->light, &z, &wl, &seg);
                    double fz = lt > 0 ? bsdf_f(mz, z.n, vmul(wz, -1.0), wl) : 0.0;
                    /* tau lies in [glo, ghi) by construction (z is on the ellipsoid of the drawn l); it is
                     * not tested again, so that rounding cannot decide it */
                    double tau = len + dist + seg - D->o;
                    if (fz > 0 && visible(g, x->p, x->n, z.p, &z.n, P->ray_eps) && light_visible(g, &D->light, &z, P->ray_eps)) {
                        double pt = bsdf_pdf(m, x->n, wi, wz) * fabs(vdot(z.n, wz)) / (dist * dist);
                        double c = beta * fx * Gterm(x, &z) * fz * lt / (pt + pe);
                        pb.v[d + 1] = z;
                        pb.cls[d + 1] = mat_class(mz);
                        pb.pdfA[d + 1] = pt;
                        sink(ctx, d + 1, c, tau, &pb, 1);
                    }
                }
            }
        }
        ell_prev = ell_here;
        len_prev = len;
        if (d == P->depth) break;
        uint32_t u[4];
        rng4(seed, px, frame, ((uint32_t)tree << 8) | (uint32_t)d, P_BSDF, u);
        v3 wo; double pdf, thr; int delta;
        if (!bsdf_sample(m, x->n, wi, u01(u[0]), u01(u[1]), &wo, &pdf, &thr, &delta)) break;
        double t;
        if (!trace_from(g, x, wo, P->ray_eps, &pb.v[d + 1], &t)) break;
        double seg = vlen(vsub(pb.v[d + 1].p, x->p));
        pb.cls[d + 1] = mat_class(&g->mats[pb.v[d + 1].mat]);
        pb.pdfA[d + 1] = delta ? 1.0 : pdf * fabs(vdot(pb.v[d + 1].n, wo)) / (seg * seg);
        len += seg;
        beta *= thr;
    }
}

typedef struct {
    const ogeom* g; const odomain* D; const oparams* P; uint64_t seed; uint32_t px, frame; int tree;
    int B; double t0, w;         /* transient: B bins of width w from t0; gated: B = 0 */
    orec* out;                   /* gated: 1 record; transient: B records */
    double* S;                   /* running weight sums (1 or B) */
    double invN;
} oinit_ctx;

static void init_sink(void* vctx, int k, double c, double tau, const opathbuf* pb, int strategy) {
    oinit_ctx* C = (oinit_ctx*)vctx;
    double w = C->invN * c;
    if (!(w > 0)) return;
    int b = 0;
    if (C->B > 0) {
        double fb = floor((tau - C->t0) / C->w);
        if (!(fb >= 0 && fb < C->B)) return;
        b = (int)fb;
    }
    uint32_t u[4];
    rng4(C->seed, C->px, C->frame, ((uint32_t)C->tree << 8) | (uint32_t)k, strategy ? P_ELL_RIS : P_RIS, u);
    if (ris_accept(&C->S[b], w, u01(u[0])))
        build_rec(C->g, C->D, pb, k, C->tree, C->px, C->frame, tau, C->P, &C->out[b]);
}

/* ============================================================================================
 * initial sampling with the path-length shrink mapping (Sec. 4.4), gated rendering.
 * Trees t >= N_A = shrink_fine draw their candidates in the gate widened K times about its
 * centre c = L0 + dL/2 (target f 1[tau in the wide gate], w = (1/N_B) f/p, N_B = n_cand - N_A)
 * and keep their RIS winner x_B with W_B; the winner alone is shrunk into the gate,
 * y_B = T(x_B) with tau' = c + (tau - c)/K and |dT/dx| = det(dxi'/dxi)/K.  Trees t < N_A keep
 * their candidates in the gate itself (canonical winner y_A with W_A).  The two are combined as a
 * GRIS merge with the generalized balance heuristic and confidences N_A, N_B:
 *   m_A(y_A) = N_A p(y_A) / (N_A p(y_A) + N_B p_wide(T^-1(y_A)) |dT^-1/dy|),
 *   m_B(y_B) = N_B p_wide(x_B)/|dT/dx| / (N_A p(y_B) + N_B p_wide(x_B)/|dT/dx|),
 *   w = m p(y) W |J| (|J| = 1 for A), selection with one uniform each, W = (w_A + w_B) / p(y).
 * With N_A = 0 (R = 1, the paper's practical setting) m_B = 1 and W = W_B |dT/dx|: biased where
 * the shrink fails or the shrunk samples do not cover the gate (the paper's darkening); with
 * N_A > 0 the canonical samples cover the whole gate and the estimate is unbiased.
 * ==========================================================================================*/
static void initial_shrink(const ogeom* g, const odomain* D, const oparams* P, uint64_t seed, uint32_t px, uint32_t frame,
                           double L0, double dL, orec* out) {
    const int NA = P->shrink_fine, NB = P->n_cand - P->shrink_fine;
    const double K = P->shrink_k, c = L0 + 0.5 * dL, half = 0.5 * K * dL;
    orec xa = EMPTY_REC, xb = EMPTY_REC;
    double Sa = 0.0, Sb = 0.0;
    oinit_ctx Ca = {g, D, P, seed, px, frame, 0, 0, L0, dL, &xa, &Sa, NA > 0 ? 1.0 / NA : 0.0};
    oinit_ctx Cb = {g, D, P, seed, px, frame, 0, 0, L0, dL, &xb, &Sb, 1.0 / NB};
    for (int t = 0; t < P->n_cand; ++t) {
        if (t < NA) { Ca.tree = t; trace_tree(g, D, P, seed, px, frame, t, 1, L0, L0 + dL, 0, init_sink, &Ca); }
        else { Cb.tree = t; trace_tree(g, D, P, seed, px, frame, t, 1, c - half, c + half, 0, init_sink, &Cb); }
    }
    const double Wa = (xa.valid && xa.phat > 0) ? ris_W(Sa, xa.phat) : 0.0;
    const double Wb = (xb.valid && xb.phat > 0) ? ris_W(Sb, xb.phat) : 0.0;
    const ogatemap to_gate = {1.0 / K, c, L0, L0 + dL}, to_wide = {K, c, c - half, c + half};
    orec yb = EMPTY_REC;
    double pyb = 0.0, Jb = 0.0;
    int okb = Wb > 0 && shift_rec_g(&xb, D, D, P, seed, 1, &yb, &pyb, &Jb, NULL, &to_gate);
    double w[2] = {0.0, 0.0};
    if (NA == 0) {
        if (okb) w[1] = pyb * Wb * Jb;
    } else {
        if (Wa > 0) {
            orec tmp;
            double pe = 0.0, Je = 0.0;
            double pb_at_a = shift_rec_g(&xa, D, D, P, seed, 1, &tmp, &pe, &Je, NULL, &to_wide) ? pe * Je : 0.0;
            double ma = NA * xa.phat / (NA * xa.phat + NB * pb_at_a);
            w[0] = ma * xa.phat * Wa;
        }
        if (okb) {
            double nb = NB * xb.phat / Jb;
            double mb = nb / (NA * pyb + nb);
            w[1] = mb * pyb * Wb * Jb;
        }
    }
    double S = 0.0;
    int sel = -1;
    for (int s = 0; s < 2; ++s) {
        if (!(w[s] > 0) || !isfinite(w[s])) continue;
        uint32_t u[4];
        rng4(seed, px, frame, (0xFFu << 8) | (uint32_t)s, P_MERGE, u);
        if (ris_accept(&S, w[s], u01(u[0]))) sel = s;
    }
    *out = EMPTY_REC;
    if (sel == 0) { *out = xa; out->valid = 1; out->W = ris_W(S, xa.phat); }
    else if (sel == 1) { *out = yb; out->valid = 1; out->W = ris_W(S, pyb); }
    out->M = P->n_cand;
}

/* ============================================================================================
 * GRIS merge (Sec. 3.2: w_i = m_i(y_i) p_hat(y_i) W_i |dS_i/dx_i|, generalized balance
 * heuristic m_i(y_i) = M_i p_hat_{<-i}(y_i) / sum_j M_j p_hat_{<-j}(y_i), with the denominator
 * evaluated at the same y_i for every j, and p_hat_{<-i}(y_i) = p_hat_i(x_i) / |dS_i/dx_i|).
 * Slot 0 is the canonical sample.  Selection streams over the slots with one uniform each.
 * ==========================================================================================*/
typedef struct { const odomain* D; const orec* x; double M; int geom_static; } oslot;

static double merge(const oslot* sl, int n, const oparams* P, uint64_t seed, uint32_t px, uint32_t frame, int pass,
                    int bin, orec* out, ostats* st) {
    orec y[16];
    double py[16], J[16], w[16];
    int ok[16];
    double Msum = 0.0;
    for (int s = 0; s < n; ++s) {
        Msum += sl[s].M;
        ok[s] = 0; w[s] = 0.0;
        if (!sl[s].x->valid) continue;
        if (s == 0) { y[0] = *sl[0].x; py[0] = sl[0].x->phat; J[0] = 1.0; ok[0] = py[0] > 0; continue; }
        ok[s] = shift_rec(sl[s].x, sl[s].D, sl[0].D, P, seed, sl[s].geom_static, &y[s], &py[s], &J[s], st);
    }
    /* MIS weight of each candidate from the targets of every domain at its own y_s (gris_mis):
     * T_0 = p_hat_0(y_s); T_s = p_hat_s(x_s) / |dS_s/dx_s| (the candidate's own domain); T_j for the
     * other domains by the inverse shift of y_s into j with its Jacobian (0 if it fails).  Pairwise
     * MIS needs only T_0 and T_s for a reused candidate, and every T_i for the canonical one. */
    const int pairwise = (P->flags & F_PAIRWISE) && n > 1;
    double Mv[16], T[16];
    for (int j = 0; j < n; ++j) Mv[j] = sl[j].M;
    for (int s = 0; s < n; ++s) {
        if (!ok[s]) continue;
        T[0] = py[s];
        for (int j = 1; j < n; ++j) {
            T[j] = 0.0;
            if (j == s) { T[j] = sl[s].x->phat / J[s]; continue; }
            if (pairwise && s != 0) continue;
            orec tmp; double pj, Jj;
            if (shift_rec(&y[s], sl[0].D, sl[j].D, P, seed, sl[j].geom_static, &tmp, &pj, &Jj, NULL))
                T[j] = pj * Jj;
        }
        double m = gris_mis(Mv, T, n, s, pairwise);
        w[s] = m * py[s] * sl[s].x->W * J[s];
        if (!(w[s] > 0) || !isfinite(w[s])) w[s] = 0.0;
    }
    double S = 0.0;
    int sel = -1;
    for (int s = 0; s < n; ++s) {
        if (!(w[s] > 0)) continue;
        uint32_t u[4];
        rng4(seed, px, frame, ((uint32_t)pass << 8) | (uint32_t)s, P_MERGE | ((uint32_t)bin << 8), u);
        if (ris_accept(&S, w[s], u01(u[0]))) sel = s;
    }
    if (sel >= 0) {
        *out = y[sel];
        out->valid = 1;
        out->W = ris_W(S, py[sel]);
    } else {
        *out = EMPTY_REC;
    }
    out->M = Msum;
    return S;
}

/* spatial neighbour of slot s in pass `pass`: uniform integer offset in the disk of radius R
 * (excluding the centre) by rejection from the square, up to 8 tries; -1 if none / off-image */
static int pick_neighbor(uint64_t seed, uint32_t px, uint32_t frame, int pass, int slot, int W, int H, int R) {
    int ix = (int)(px % (uint32_t)W), iy = (int)(px / (uint32_t)W);
    uint32_t side = 2u * (uint32_t)R + 1u;
    for (int a = 0; a < 4; ++a) {
        uint32_t u[4];
        rng4(seed, px, frame, ((uint32_t)pass << 8) | (uint32_t)slot, P_NEIGHBOR | ((uint32_t)a << 8), u);
        for (int h = 0; h < 2; ++h) {
            int dx = (int)(u[2 * h] % side) - R, dy = (int)(u[2 * h + 1] % side) - R;
            if (dx * dx + dy * dy > R * R || (dx == 0 && dy == 0)) continue;
            int nx = ix + dx, ny = iy + dy;
            if (nx < 0 || ny < 0 || nx >= W || ny >= H) return -1;
            return ny * W + nx;
        }
    }
    return -1;
}

static int xf_equal(const ogeom* a, const ogeom* b) {
    if (a == b) return 1;
    if (a->nobj != b->nobj) return 0;
    return memcmp(a->xf, b->xf, sizeof(double) * 12 * (size_t)a->nobj) == 0;
}

/* ============================================================================================
 * one frame of the pipeline (Sec. 3.2 stages (1)-(4)).  Gated when B == 0 (gate [L0, L0+dL)),
 * transient with B bins [L0 + b dL, L0 + (b+1) dL) otherwise.  Pixels outside the region of
 * interest [x0, x1) x [y0, y1) are not computed; any result that depends on one of them is
 * marked not-ok in ok_out.
 * ==========================================================================================*/
int or_render_frame(oview* v, const ogeom* g, const osensor* s, const oemitter* e, double L0, double dL, int B,
                    const oparams* P, uint64_t seed, uint32_t frame, int x0, int y0, int x1, int y1,
                    double* out, uint8_t* ok_out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int W = v->W, H = v->H;
    const int Bn = B > 0 ? B : 1;
    if (Bn != v->Bn || s->W != W || s->H != H) return -1;
    if (P->depth < 1 || P->depth > MAXD - 2 || P->n_cand < 1 || P->n_spatial > 15) return -1;
    if ((P->flags & F_ELLIPSOID) && B == 0 && P->shrink_k > 1.0) return -1;   /* one initial sampler at a time */
    int prev = v->cur;
    int cur = v->has_prev ? 1 - v->cur : v->cur;
    oframe* F = &v->fr[cur];
    oframe* Fp = &v->fr[prev];
    const int have_prev = v->has_prev && P->temporal;
    F->g = g; F->s = *s; F->e = *e; F->L0 = L0; F->dL = dL; F->B = B; F->frame = frame;
    memset(&F->laser, 0, sizeof(F->laser));
    if (e->type == 1) {
        osurf dummy; memset(&dummy, 0, sizeof(dummy));
        v3 o = vload(e->pos), d = vnorm(vload(e->dir));
        int tri; double b1, b2, t;
        if (trace(g, o, d, 1e30, 0, &tri, &b1, &b2, &t)) {
            F->laser.kind = 2; F->laser.s = surf_at(g, tri, b1, b2); F->laser.I = e->power;
            F->laser.to_origin = vmul(d, -1.0); F->laser.emit_len = t; F->laser.pos = F->laser.s.p;
        }
    }
    const int geom_static = have_prev ? xf_equal(Fp->g, g) : 1;

    /* G-buffer */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int pix = 0; pix < W * H; ++pix) {
        int ix = pix % W, iy = pix / W;
        F->ok[pix] = (ix >= x0 && ix < x1 && iy >= y0 && iy < y1);
        F->gb[pix].valid = 0;
        if (!F->ok[pix]) continue;
        uint32_t u[4];
        rng4(seed, (uint32_t)pix, frame, 0, P_JITTER, u);
        v3 o, d;
        primary_ray(s, ix, iy, u01(u[0]), u01(u[1]), &o, &d);
        int tri; double b1, b2, t;
        if (trace(g, o, d, 1e30, 0, &tri, &b1, &b2, &t)) {
            F->gb[pix].valid = 1;
            F->gb[pix].s = surf_at(g, tri, b1, b2);
            F->gb[pix].t = vlen(vsub(F->gb[pix].s.p, o));
        }
    }

    /* initial candidates */
    orec* R0 = (orec*)calloc((size_t)W * H * Bn, sizeof(orec));
    const int shrink = B == 0 && P->shrink_k > 1.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int pix = 0; pix < W * H; ++pix) {
        /* pixels outside the region of interest are never touched: their reservoirs stay zero
         * (empty), and every result that depends on them is marked not-ok */
        if (!F->ok[pix]) continue;
        orec* rr = &R0[(size_t)pix * Bn];
        for (int b = 0; b < Bn; ++b) { rr[b] = EMPTY_REC; rr[b].M = P->n_cand; }
        if (!F->gb[pix].valid) continue;
        odomain D = make_domain(F, pix, P, L0, dL);
        if (shrink) {
            initial_shrink(g, &D, P, seed, (uint32_t)pix, frame, L0, dL, rr);
            continue;
        }
        double* S = (double*)calloc((size_t)Bn, sizeof(double));
        oinit_ctx C = {g, &D, P, seed, (uint32_t)pix, frame, 0, B, L0, dL, rr, S, 1.0 / P->n_cand};
        for (int t = 0; t < P->n_cand; ++t) {
            C.tree = t;
            const int ell = (P->flags & F_ELLIPSOID) != 0;
            if (B > 0) trace_tree(g, &D, P, seed, (uint32_t)pix, frame, t, 1, L0, L0 + B * dL, ell, init_sink, &C);
            else trace_tree(g, &D, P, seed, (uint32_t)pix, frame, t, 1, L0, L0 + dL, ell, init_sink, &C);
        }
        for (int b = 0; b < Bn; ++b) {
            if (rr[b].valid && rr[b].phat > 0) { rr[b].W = ris_W(S[b], rr[b].phat); rr[b].M = P->n_cand; }
            else { rr[b] = EMPTY_REC; rr[b].M = P->n_cand; }
        }
        free(S);
    }

    /* bin gate of bin b */
#define GATE_L0(b) (B > 0 ? L0 + (b) * dL : L0)
    /* temporal reuse (stage (2)): previous reservoir at the back-projected pixel */
    /* Confidence weights are per pixel and shared by every bin: they follow from the reuse
     * structure alone (N after the initial stage, then sums of capped inputs), never from whether
     * a reservoir happens to hold a sample -- a sample-dependent M would bias the generalized
     * balance heuristic. */
    double* Mc = (double*)malloc(sizeof(double) * (size_t)W * H);
    for (int pix = 0; pix < W * H; ++pix) Mc[pix] = P->n_cand;
    orec* R1 = R0;
    uint8_t* ok1 = (uint8_t*)malloc((size_t)W * H);
    memcpy(ok1, F->ok, (size_t)W * H);
    if (have_prev) {
        double* Mt = (double*)malloc(sizeof(double) * (size_t)W * H);
        R1 = (orec*)calloc((size_t)W * H * Bn, sizeof(orec));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
        for (int pix = 0; pix < W * H; ++pix) {
            Mt[pix] = Mc[pix];
            if (!F->ok[pix]) continue;
            orec* dst = &R1[(size_t)pix * Bn];
            memcpy(dst, &R0[(size_t)pix * Bn], sizeof(orec) * Bn);
            if (!F->gb[pix].valid) continue;
            int q = -1;
            if (s->mode == 1) q = pix;
            else {
                osurf sp = surf_at(Fp->g, F->gb[pix].s.tri, F->gb[pix].s.b1, F->gb[pix].s.b2);
                int qx, qy;
                if (project(&Fp->s, sp.p, &qx, &qy)) q = qy * W + qx;
            }
            if (q < 0) continue;
            if (!Fp->ok[q]) { ok1[pix] = 0; continue; }
            double Mprev = fmin(Fp->M[q], P->m_cap);
            Mt[pix] = Mc[pix] + Mprev;
            for (int b = 0; b < Bn; ++b) {
                const orec* xc = &R0[(size_t)pix * Bn + b];
                const orec* xt = &Fp->res[(size_t)q * Bn + b];
                if (B > 0 && !xc->valid && !xt->valid) continue;
                odomain Dc = make_domain(F, pix, P, GATE_L0(b), dL);
                odomain Dt = make_domain(Fp, q, P, Fp->B > 0 ? Fp->L0 + b * Fp->dL : Fp->L0, Fp->dL);
                oslot sl[2];
                sl[0].D = &Dc; sl[0].x = xc; sl[0].M = Mc[pix]; sl[0].geom_static = 1;
                sl[1].D = &Dt; sl[1].x = xt; sl[1].M = Mprev; sl[1].geom_static = geom_static;
                merge(sl, 2, P, seed, (uint32_t)pix, frame, 0, b, &dst[b], &v->st);
            }
        }
        free(Mc);
        Mc = Mt;
    }

    /* bin reuse (Sec. 4.5: the histogram's extra reuse axis), transient views with F_BIN_REUSE: one
     * pass after temporal reuse in which the reservoir of bin b reuses the same pixel's bins b - 1
     * and b + 1, shifted into bin b's gate by the gate translation (delta = -+ w).  Bins outside
     * [0, B) are not domains (no candidate was ever drawn for them): they take no part in the MIS.
     * The stored per-pixel confidence counts both neighbours for every bin -- any structural
     * confidence keeps the balance heuristic a partition of unity. */
    if (B > 0 && (P->flags & F_BIN_REUSE)) {
        orec* Rb = (orec*)calloc((size_t)W * H * Bn, sizeof(orec));
        double* Mb = (double*)malloc(sizeof(double) * (size_t)W * H);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
        for (int pix = 0; pix < W * H; ++pix) {
            const double Mn = fmin(Mc[pix], P->m_cap);
            Mb[pix] = Mc[pix] + 2.0 * Mn;
            if (!ok1[pix]) continue;
            orec* dst = &Rb[(size_t)pix * Bn];
            memcpy(dst, &R1[(size_t)pix * Bn], sizeof(orec) * Bn);
            if (!F->gb[pix].valid) continue;
            for (int b = 0; b < Bn; ++b) {
                const orec* xc = &R1[(size_t)pix * Bn + b];
                int any = xc->valid;
                if (b >= 1) any |= R1[(size_t)pix * Bn + b - 1].valid;
                if (b + 1 < Bn) any |= R1[(size_t)pix * Bn + b + 1].valid;
                if (!any) continue;
                /* slots 0 (bin b), 1 (bin b - 1), 2 (bin b + 1); an absent bin is an empty slot with
                 * confidence 0, so it adds nothing to any MIS weight */
                odomain Dc = make_domain(F, pix, P, GATE_L0(b), dL);
                odomain Dn[2];
                oslot sl[3];
                sl[0].D = &Dc; sl[0].x = xc; sl[0].M = Mc[pix]; sl[0].geom_static = 1;
                for (int k = 0; k < 2; ++k) {
                    int bb = k == 0 ? b - 1 : b + 1;
                    int present = bb >= 0 && bb < Bn;
                    Dn[k] = make_domain(F, pix, P, GATE_L0(bb), dL);
                    sl[1 + k].D = &Dn[k];
                    sl[1 + k].x = present ? &R1[(size_t)pix * Bn + bb] : &EMPTY_REC;
                    sl[1 + k].M = present ? Mn : 0.0;
                    sl[1 + k].geom_static = 1;
                }
                merge(sl, 3, P, seed, (uint32_t)pix, frame, 8, b, &dst[b], &v->st);
            }
        }
        if (R1 != R0) free(R1);
        R1 = Rb;
        free(Mc);
        Mc = Mb;
    }

    /* spatial reuse (stage (3)) */
    orec* Rcur = R1;
    uint8_t* okc = ok1;
    for (int it = 0; it < P->n_spatial_iters && P->n_spatial > 0; ++it) {
        orec* Rn = (orec*)calloc((size_t)W * H * Bn, sizeof(orec));
        uint8_t* okn = (uint8_t*)malloc((size_t)W * H);
        double* Mn = (double*)malloc(sizeof(double) * (size_t)W * H);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
        for (int pix = 0; pix < W * H; ++pix) {
            okn[pix] = okc[pix];
            Mn[pix] = Mc[pix];
            if (!okc[pix]) continue;
            orec* dst = &Rn[(size_t)pix * Bn];
            memcpy(dst, &Rcur[(size_t)pix * Bn], sizeof(orec) * Bn);
            if (!F->gb[pix].valid) continue;
            int nb[16], nn = 0;
            for (int sI = 1; sI <= P->n_spatial; ++sI) {
                int q = pick_neighbor(seed, (uint32_t)pix, frame, 1 + it, sI, W, H, P->radius);
                if (q < 0) continue;
                if (!okc[q]) { okn[pix] = 0; }
                nb[nn++] = q;
            }
            if (!okn[pix]) continue;
            for (int a = 0; a < nn; ++a) Mn[pix] += fmin(Mc[nb[a]], P->m_cap);
            for (int b = 0; b < Bn; ++b) {
                const orec* xc = &Rcur[(size_t)pix * Bn + b];
                if (B > 0) {
                    int any = xc->valid;
                    for (int a = 0; a < nn; ++a) any |= Rcur[(size_t)nb[a] * Bn + b].valid;
                    if (!any) continue;
                }
                odomain Dc = make_domain(F, pix, P, GATE_L0(b), dL);
                odomain Dn[16];
                oslot sl[16];
                sl[0].D = &Dc; sl[0].x = xc; sl[0].M = Mc[pix]; sl[0].geom_static = 1;
                for (int a = 0; a < nn; ++a) {
                    Dn[a] = make_domain(F, nb[a], P, GATE_L0(b), dL);
                    sl[1 + a].D = &Dn[a];
                    sl[1 + a].x = &Rcur[(size_t)nb[a] * Bn + b];
                    sl[1 + a].M = fmin(Mc[nb[a]], P->m_cap);
                    sl[1 + a].geom_static = 1;
                }
                merge(sl, 1 + nn, P, seed, (uint32_t)pix, frame, 1 + it, b, &dst[b], &v->st);
            }
        }
        if (Rcur != R0 && Rcur != R1) free(Rcur);
        if (okc != ok1) free(okc);
        Rcur = Rn;
        okc = okn;
        free(Mc);
        Mc = Mn;
    }

    /* final shading (stage (4)): f(y) W_y (= the merge's weight sum for a box gate) */
    for (int pix = 0; pix < W * H; ++pix) {
        for (int b = 0; b < Bn; ++b) {
            const orec* rr = &Rcur[(size_t)pix * Bn + b];
            out[(size_t)pix * Bn + b] = (okc[pix] && rr->valid) ? rr->phat * rr->W : 0.0;
        }
        ok_out[pix] = okc[pix];
        /* the frame's reservoirs (read by the next frame only where this frame is ok) */
        if (okc[pix]) memcpy(&F->res[(size_t)pix * Bn], &Rcur[(size_t)pix * Bn], sizeof(orec) * Bn);
    }
    memcpy(F->ok, okc, (size_t)W * H);
    memcpy(F->M, Mc, sizeof(double) * (size_t)W * H);
    free(Mc);
    if (Rcur != R0) free(Rcur);
    if (R1 != R0 && R1 != Rcur) free(R1);
    free(R0);
    if (okc != ok1) free(okc);
    free(ok1);
    v->cur = cur;
    v->has_prev = 1;
    return 0;
#undef GATE_L0
}

/* ============================================================================================
 * plain path tracing (the "path tracing without any reuse" comparison of Sec. 6): spp paths
 * per pixel, each with its own jitter, every NEE path of length kmin..depth splatted with
 * f / p into the gate (B == 0) or its bin.
 * ==========================================================================================*/
typedef struct { int B; double t0, w; double* acc; double scale; } opt_ctx;
static void pt_sink(void* vctx, int k, double c, double tau, const opathbuf* pb, int strategy) {
    (void)k; (void)pb; (void)strategy;
    opt_ctx* C = (opt_ctx*)vctx;
    if (C->B > 0) {
        double fb = floor((tau - C->t0) / C->w);
        if (!(fb >= 0 && fb < C->B)) return;
        C->acc[(int)fb] += C->scale * c;
    } else {
        C->acc[0] += C->scale * c;
    }
}

int or_render_pt(const ogeom* g, const osensor* s, const oemitter* e, double L0, double dL, int B, const oparams* P,
                 uint64_t seed, uint32_t frame, int spp, int x0, int y0, int x1, int y1, double* out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int W = s->W, H = s->H, Bn = B > 0 ? B : 1;
    olight laser; memset(&laser, 0, sizeof(laser));
    if (e->type == 1) {
        v3 o = vload(e->pos), d = vnorm(vload(e->dir));
        int tri; double b1, b2, t;
        if (trace(g, o, d, 1e30, 0, &tri, &b1, &b2, &t)) {
            laser.kind = 2; laser.s = surf_at(g, tri, b1, b2); laser.I = e->power;
            laser.to_origin = vmul(d, -1.0); laser.emit_len = t; laser.pos = laser.s.p;
        }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int pix = 0; pix < W * H; ++pix) {
        double* acc = &out[(size_t)pix * Bn];
        for (int b = 0; b < Bn; ++b) acc[b] = 0.0;
        int ix = pix % W, iy = pix / W;
        if (!(ix >= x0 && ix < x1 && iy >= y0 && iy < y1)) continue;
        for (int sm = 0; sm < spp; ++sm) {
            uint32_t u[4];
            rng4(seed, (uint32_t)pix, frame, (uint32_t)sm, P_JITTER, u);
            v3 o, d;
            primary_ray(s, ix, iy, u01(u[0]), u01(u[1]), &o, &d);
            int tri; double b1, b2, t;
            if (!trace(g, o, d, 1e30, 0, &tri, &b1, &b2, &t)) continue;
            odomain D; memset(&D, 0, sizeof(D));
            D.g = g; D.valid = 1; D.x0 = o; D.y1 = surf_at(g, tri, b1, b2);
            double tp = vlen(vsub(D.y1.p, o));
            D.o = s->mode == 1 ? 2.0 * tp : 0.0;
            if (e->type == 0) { D.light.kind = 1; D.light.pos = vload(e->pos); D.light.I = e->power; }
            else if (e->type == 1) D.light = laser;
            else {
                D.light.kind = 2; D.light.s = D.y1; D.light.I = e->power;
                D.light.to_origin = vnorm(vsub(vload(e->pos), D.y1.p));
                D.light.emit_len = vlen(vsub(vload(e->pos), D.y1.p)); D.light.pos = D.y1.p;
            }
            opt_ctx C = {B, L0, dL, acc, 1.0 / spp};
            if (B > 0) trace_tree(g, &D, P, seed, (uint32_t)pix, frame, sm, 1, L0, L0 + B * dL, 0, pt_sink, &C);
            else trace_tree(g, &D, P, seed, (uint32_t)pix, frame, sm, 1, L0, L0 + dL, 0, pt_sink, &C);
        }
    }
    return 0;
}

/* ============================================================================================
 * small exported hooks for the pins (tests call these on explicit inputs)
 * ==========================================================================================*/
/* streaming selection over n weights with uniforms u: returns the selected index or -1 */
int or_stream_select(const double* w, const double* u, int n, double* S_out) {
    double S = 0.0;
    int sel = -1;
    for (int i = 0; i < n; ++i) {
        if (!(w[i] > 0)) continue;
        if (ris_accept(&S, w[i], u[i])) sel = i;
    }
    *S_out = S;
    return sel;
}
/* the pipeline's resampling primitives on explicit inputs (exhaustive-enumeration pins) */
int or_ris_accept(double S_in, double w, double u, double* S_out) {
    double S = S_in;
    int a = ris_accept(&S, w, u);
    *S_out = S;
    return a;
}
double or_ris_W(double S, double phat) { return ris_W(S, phat); }
double or_gris_mis(const double* M, const double* T, int n, int s, int pairwise) {
    if (n < 1 || n > 16 || s < 0 || s >= n) return -1.0;
    return gris_mis(M, T, n, s, pairwise);
}

/* BSDF sampling hook: returns ok; wo[3], pdf, thr */
int or_bsdf_sample(int type, double albedo, double alpha, const double* n, const double* wi, double u0, double u1,
                   double* wo, double* pdf, double* thr) {
    omat m = {type, albedo, alpha};
    v3 w; int delta;
    int ok = bsdf_sample(&m, vload(n), vload(wi), u0, u1, &w, pdf, thr, &delta);
    wo[0] = w.x; wo[1] = w.y; wo[2] = w.z;
    return ok;
}
double or_bsdf_pdf(int type, double albedo, double alpha, const double* n, const double* wi, const double* wo) {
    omat m = {type, albedo, alpha};
    return bsdf_pdf(&m, vload(n), vload(wi), vload(wo));
}

/* read a stored reservoir (for record-level tests): fills W, M, phat, tau, k, r, valid */
int or_view_reservoir(const oview* v, int pix, int b, double out[4], int iout[3]) {
    const orec* r = &v->fr[v->cur].res[(size_t)pix * v->Bn + b];
    out[0] = r->W; out[1] = r->M; out[2] = r->phat; out[3] = r->tau;
    iout[0] = r->k; iout[1] = r->r; iout[2] = r->valid;
    return 0;
}

/* exercise the full shift on a stored reservoir: shift the record of pixel `src` (current
 * frame) into the domain of pixel `dst` and back.  Returns 1 if both succeed; outputs the
 * forward and inverse Jacobians and the round-trip barycentric error. */
int or_shift_roundtrip(const oview* v, const oparams* P, uint64_t seed, int src, int dst, double out[6]) {
    const oframe* F = &v->fr[v->cur];
    const orec* x = &F->res[(size_t)src * v->Bn];
    odomain Ds = make_domain(F, src, P, F->L0, F->dL);
    odomain Dd = make_domain(F, dst, P, F->L0, F->dL);
    orec y, z;
    double py, J, pz, Jz;
    for (int i = 0; i < 6; ++i) out[i] = 0;
    if (!shift_rec(x, &Ds, &Dd, P, seed, 1, &y, &py, &J, NULL)) return 0;
    if (!shift_rec(&y, &Dd, &Ds, P, seed, 1, &z, &pz, &Jz, NULL)) return -1;
    out[0] = J; out[1] = Jz; out[2] = fabs(z.p_b1 - x->p_b1) + fabs(z.p_b2 - x->p_b2);
    out[3] = py; out[4] = pz; out[5] = x->phat;
    return 1;
}

/* exercise the shrink mapping of Sec. 4.4 on a stored gated reservoir: expand the record of pixel
 * `pix` (current frame) from its gate into the gate widened K times about the same centre, then
 * shrink the result back.  Returns 1 if both succeed; out = (J_expand, J_shrink, round-trip
 * barycentric error, tau, tau after expanding, tau after shrinking back, p_hat, p_hat expanded). */
int or_shrink_roundtrip(const oview* v, const oparams* P, uint64_t seed, int pix, double K, double out[8]) {
    const oframe* F = &v->fr[v->cur];
    const orec* x = &F->res[(size_t)pix * v->Bn];
    odomain D = make_domain(F, pix, P, F->L0, F->dL);
    const double c = F->L0 + 0.5 * F->dL, half = 0.5 * K * F->dL;
    const ogatemap to_wide = {K, c, c - half, c + half}, to_gate = {1.0 / K, c, F->L0, F->L0 + F->dL};
    orec y, z;
    double py, Jy, pz, Jz;
    for (int i = 0; i < 8; ++i) out[i] = 0;
    if (!x->valid) return 0;
    if (!shift_rec_g(x, &D, &D, P, seed, 1, &y, &py, &Jy, NULL, &to_wide)) return 0;
    if (!shift_rec_g(&y, &D, &D, P, seed, 1, &z, &pz, &Jz, NULL, &to_gate)) return -1;
    out[0] = Jy; out[1] = Jz; out[2] = fabs(z.p_b1 - x->p_b1) + fabs(z.p_b2 - x->p_b2);
    out[3] = x->tau; out[4] = y.tau; out[5] = z.tau; out[6] = x->phat; out[7] = py;
    return 1;
}
