// tof_device.cuh -- device functions of the ToF ReSTIR hot path (sm_103a, FP32).
//
// Layering: float3 algebra -> Philox streams -> BSDFs -> LBVH traversal -> domains and lights ->
// path trees (initial candidates) -> path-length-aware shift -> GRIS merge.
// The method follows Kim, Jarosz, Pediredla, "ToF ReSTIR" (ACM TOG 45(4), 2026); each function
// names the section or equation it implements.
#pragma once
#include <stdint.h>

#include "tof_internal.h"

namespace tof {

// ============================================================================================
// float3 algebra
// ============================================================================================
static __device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
static __device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
static __device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
static __device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
static __device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static __device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static __device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }
static __device__ __forceinline__ float3 norm3(float3 a) {
    float l = len3(a);
    return l > 0.f ? a * (1.0f / l) : f3(0.f, 0.f, 0.f);
}
static __device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }
static __device__ __forceinline__ float3 dir_to(float3 from, float3 to) { return norm3(to - from); }

// ============================================================================================
// Philox4x32-10 (Salmon et al., SC 2011) counter-based streams.  Key = 64-bit seed; counter =
// (pixel, frame, stream word, purpose word).  Uniform u = (x >> 8) * 2^-24.
// ============================================================================================
enum : uint32_t { P_JITTER = 1, P_BSDF = 2, P_RIS = 3, P_NEIGHBOR = 4, P_MERGE = 5,
                  P_ELL_RIS = 6,   // selection of an ellipsoidal candidate
                  P_ELL = 7 };     // P_ELL + q, q = 0..5: the ellipsoidal connection's draws

static __device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}
static __device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ============================================================================================
// materials (Sec. 6: diffuse, glossy, specular).  Class: rough (Lambert, GGX alpha >= 0.2),
// glossy (GGX alpha < 0.2), delta (mirror).
// ============================================================================================
enum { M_LAMBERT = 0, M_GGX = 1, M_MIRROR = 2 };
enum { C_ROUGH = 0, C_GLOSSY = 1, C_DELTA = 2 };
constexpr float kPi = 3.14159265358979323846f;

struct Mat { int type; float albedo, alpha; };
static __device__ __forceinline__ Mat load_mat(const GeomDev& g, int id) {
    float4 m = __ldg(&g.mats[id]);
    Mat r; r.type = (int)m.x; r.albedo = m.y; r.alpha = m.z;
    return r;
}
static __device__ __forceinline__ int mat_class(const Mat& m) {
    if (m.type == M_MIRROR) return C_DELTA;
    if (m.type == M_GGX && m.alpha < 0.2f) return C_GLOSSY;
    return C_ROUGH;
}
static __device__ __forceinline__ float ggx_D(float nh, float a) {
    float a2 = a * a, t = nh * nh * (a2 - 1.0f) + 1.0f;
    return a2 / (kPi * t * t);
}
static __device__ __forceinline__ float ggx_G1(float nv, float a) {
    float a2 = a * a;
    return 2.0f * nv / (nv + sqrtf(a2 + (1.0f - a2) * nv * nv));
}
// f_s(wi, wo): wi toward the previous vertex, wo toward the next; reflection only
static __device__ float bsdf_f(const Mat& m, float3 n, float3 wi, float3 wo) {
    float ci = dot3(n, wi), co = dot3(n, wo);
    if (ci * co <= 0.f) return 0.f;
    if (ci < 0.f) { ci = -ci; co = -co; n = n * -1.0f; }
    if (m.type == M_LAMBERT) return m.albedo / kPi;
    if (m.type == M_GGX) {
        float3 h = norm3(wi + wo);
        float nh = dot3(n, h);
        if (nh <= 0.f) return 0.f;
        return m.albedo * ggx_D(nh, m.alpha) * ggx_G1(ci, m.alpha) * ggx_G1(co, m.alpha) / (4.0f * ci * co);
    }
    return 0.f;
}
static __device__ float bsdf_pdf(const Mat& m, float3 n, float3 wi, float3 wo) {
    float ci = dot3(n, wi), co = dot3(n, wo);
    if (ci * co <= 0.f) return 0.f;
    if (ci < 0.f) { co = -co; n = n * -1.0f; }
    if (m.type == M_LAMBERT) return co / kPi;
    if (m.type == M_GGX) {
        float3 h = norm3(wi + wo);
        float nh = dot3(n, h), oh = dot3(wo, h);
        if (nh <= 0.f || oh <= 0.f) return 0.f;
        return ggx_D(nh, m.alpha) * nh / (4.0f * oh);
    }
    return 0.f;
}
// tangent frame (t, b, n): t = normalize(a x n), b = n x t, with the reference axis a one of two
// fixed generic unit vectors (a2 perpendicular to a1, used when |n.a1| >= 0.6); the frame's
// unavoidable discontinuity sits on a cone that axis-aligned or symmetric mesh normals do not
// meet exactly, so the branch taken does not depend on rounding
static __device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
    const float3 a1 = f3(0.4140355211239282f, 0.731736150464251f, 0.5414210869105452f);
    const float3 a2 = f3(0.0f, 0.5947978113475719f, -0.8038753408434284f);
    float3 a = fabsf(dot3(n, a1)) < 0.6f ? a1 : a2;
    t = norm3(cross3(a, n));
    b = cross3(n, t);
}
// sample wo given wi; thr = f_s |cos_o| / pdf (albedo for the mirror)
static __device__ bool bsdf_sample(const Mat& m, float3 n, float3 wi, float u0, float u1, float3& wo, float& pdf,
                            float& thr, bool& delta) {
    if (dot3(n, wi) < 0.f) n = n * -1.0f;
    delta = false;
    if (m.type == M_MIRROR) {
        wo = n * (2.0f * dot3(wi, n)) - wi;
        pdf = 1.0f; thr = m.albedo; delta = true;
        return true;
    }
    float3 t, b;
    onb(n, t, b);
    if (m.type == M_LAMBERT) {
        float r = sqrtf(u0), ph = 2.0f * kPi * u1;
        float lz = sqrtf(fmaxf(0.f, 1.0f - u0));
        float s, c;
        sincosf(ph, &s, &c);
        wo = t * (r * c) + b * (r * s) + n * lz;
    } else {
        float a = m.alpha;
        float tan2 = a * a * u0 / (1.0f - u0);
        float ct = 1.0f / sqrtf(1.0f + tan2), st = sqrtf(fmaxf(0.f, 1.0f - ct * ct)), ph = 2.0f * kPi * u1;
        float s, c;
        sincosf(ph, &s, &c);
        float3 h = t * (st * c) + b * (st * s) + n * ct;
        wo = h * (2.0f * dot3(wi, h)) - wi;
    }
    float co = dot3(n, wo);
    if (co <= 0.f) return false;
    pdf = bsdf_pdf(m, n, wi, wo);
    float f = bsdf_f(m, n, wi, wo);
    if (!(pdf > 0.f) || !(f > 0.f)) return false;
    thr = f * co / pdf;
    return true;
}

// ============================================================================================
// geometry: surface points, Moller-Trumbore, LBVH traversal, visibility
// ============================================================================================
struct Surf { int tri; float b1, b2; float3 p, n; int mat; };

static __device__ __forceinline__ Surf surf_at(const GeomDev& g, int tri, float b1, float b2) {
    float4 a = __ldg(&g.tri[3 * tri]), e1 = __ldg(&g.tri[3 * tri + 1]), e2 = __ldg(&g.tri[3 * tri + 2]);
    Surf s;
    s.tri = tri; s.b1 = b1; s.b2 = b2;
    float3 E1 = xyz(e1), E2 = xyz(e2);
    s.p = xyz(a) + (E1 * b1 + E2 * b2);
    s.n = norm3(cross3(E1, E2));
    s.mat = __float_as_int(a.w);
    return s;
}
static __device__ __forceinline__ float3 offset_point(float3 p, float3 n, float3 dir, float eps) {
    return dot3(n, dir) >= 0.f ? p + n * eps : p - n * eps;
}

// Moller-Trumbore with barycentric tests inclusive by kBaryEps, so that a ray through an edge
// shared by two triangles hits at least one of them whatever the rounding (no cracks)
constexpr float kBaryEps = 1e-6f;
static __device__ __forceinline__ bool tri_test(const float4* __restrict__ L, int leaf, float3 o, float3 d, float tmax, float& t,
                                         float& b1, float& b2, int& orig) {
    float4 a = __ldg(&L[3 * leaf]), e1v = __ldg(&L[3 * leaf + 1]), e2v = __ldg(&L[3 * leaf + 2]);
    float3 e1 = xyz(e1v), e2 = xyz(e2v);
    float3 pv = cross3(d, e2);
    float det = dot3(e1, pv);
    if (fabsf(det) < 1e-20f) return false;
    float inv = 1.0f / det;
    float3 tv = o - xyz(a);
    float u = dot3(tv, pv) * inv;
    if (u < -kBaryEps || u > 1.f + kBaryEps) return false;
    float3 qv = cross3(tv, e1);
    float w = dot3(d, qv) * inv;
    if (w < -kBaryEps || u + w > 1.f + kBaryEps) return false;
    float tt = dot3(e2, qv) * inv;
    if (!(tt > 0.f && tt <= tmax)) return false;
    t = tt; b1 = u; b2 = w; orig = __float_as_int(a.w);
    return true;
}
// closest-hit acceptance: nearer, or equally near with a lower triangle id (order-independent)
static __device__ __forceinline__ bool closer(bool found, float t, int id, float best, int best_id) {
    return !found || t < best || (t == best && id < best_id);
}

// closest hit (any_hit = false) or first hit (any_hit = true) of o + t d, t in (0, tmax).
// Kept out of line: one copy of the loop serves every call site (replay, visibility, NEE), which
// keeps the shift kernels' code small and lets lanes from different call sites share it.
template <bool kAny>
static __device__ __noinline__ bool traverse(const GeomDev& g, float3 o, float3 d, float tmax, int& tri, float& b1, float& b2, float& tout) {
    // the loop reads the hierarchy through these copies and makes no store that could alias them;
    // an overflow is only noted here and published in the error word after the loop
    const float4* __restrict__ nodes = g.nodes;
    const float4* __restrict__ leaf = g.leaf;
    const int nt = g.nt;
    if (nt <= 0) return false;
    bool found = false;
    float best = tmax;
    if (nt == 1) {
        int orig;
        if (tri_test(leaf, 0, o, d, best, tout, b1, b2, orig) && tout < tmax) { tri = orig; return true; }
        return false;
    }
    float3 id = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    float3 ood = f3(o.x * id.x, o.y * id.y, o.z * id.z);
    int stack[kStack];
    int sp = 0;
    int node = 0;
    unsigned fault = 0u;
    // a valid hierarchy visits each of its nt - 1 internal nodes at most once per ray; the cap
    // only guards against a malformed one, and running into it is reported in the error word
    int budget = nt + 64;
    while (true) {
        if (--budget < 0) {
            fault |= kErrVisitBudget;
            break;
        }
        const float4* N = nodes + 4 * node;
        float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
        float a0 = n0.x * id.x - ood.x, a1 = n0.y * id.x - ood.x;
        float b0 = n0.z * id.y - ood.y, bb1 = n0.w * id.y - ood.y;
        float c0 = n2.x * id.z - ood.z, c1 = n2.y * id.z - ood.z;
        float lo0 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, bb1)), fmaxf(fminf(c0, c1), 0.f));
        float hi0 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, bb1)), fminf(fmaxf(c0, c1), best));
        float d0 = n1.x * id.x - ood.x, d1 = n1.y * id.x - ood.x;
        float e0 = n1.z * id.y - ood.y, e1 = n1.w * id.y - ood.y;
        float f0 = n2.z * id.z - ood.z, f1 = n2.w * id.z - ood.z;
        float lo1 = fmaxf(fmaxf(fminf(d0, d1), fminf(e0, e1)), fmaxf(fminf(f0, f1), 0.f));
        float hi1 = fminf(fminf(fmaxf(d0, d1), fmaxf(e0, e1)), fminf(fmaxf(f0, f1), best));
        bool h0 = lo0 <= hi0, h1 = lo1 <= hi1;
        int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
        if (h0 && ch0 < 0) {
            float t, u, w; int orig;
            if (tri_test(leaf, ~ch0, o, d, best, t, u, w, orig) && (found || t < tmax) && closer(found, t, orig, best, tri)) {
                best = t; tri = orig; b1 = u; b2 = w; found = true;
                if (kAny) { tout = t; return true; }
            }
            h0 = false;
        }
        if (h1 && ch1 < 0) {
            float t, u, w; int orig;
            if (tri_test(leaf, ~ch1, o, d, best, t, u, w, orig) && (found || t < tmax) && closer(found, t, orig, best, tri)) {
                best = t; tri = orig; b1 = u; b2 = w; found = true;
                if (kAny) { tout = t; return true; }
            }
            h1 = false;
        }
        if (h0 && h1) {
            int nearc = lo0 <= lo1 ? ch0 : ch1, farc = lo0 <= lo1 ? ch1 : ch0;
            if (sp < kStack) stack[sp++] = farc;
            else fault |= kErrStackOverflow;   // the far subtree is skipped: reported below
            node = nearc;
        } else if (h0) {
            node = ch0;
        } else if (h1) {
            node = ch1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    if (fault && g.err) atomicOr(g.err, fault);
    if (found) tout = best;
    return found;
}

static __device__ __forceinline__ bool trace_from(const GeomDev& g, const Surf& s, float3 d, float eps, Surf& hit) {
    float3 o = offset_point(s.p, s.n, d, eps);
    int tri; float b1, b2, t;
    if (!traverse<false>(g, o, d, 3.0e38f, tri, b1, b2, t)) return false;
    hit = surf_at(g, tri, b1, b2);
    return true;
}
// mutual visibility of surface point a and surface point b (bsurf) or point b
static __device__ bool visible(const GeomDev& g, float3 a, float3 an, float3 b, const float3* bn, float eps) {
    float3 ao = offset_point(a, an, b - a, eps);
    float3 bo = bn ? offset_point(b, *bn, a - b, eps) : b;
    float3 d = bo - ao;
    float dist = len3(d);
    if (!(dist > 0.f)) return true;
    d = d * (1.0f / dist);
    int tri; float b1, b2, t;
    return !traverse<true>(g, ao, d, dist, tri, b1, b2, t);
}

// Deferred visibility: a shift kernel hands its visibility segments to a queue instead of tracing
// them in place, and a separate kernel (vis_kernel) traces the queue with every lane of a warp on
// a ray.  A queued ray carries the index of the float result it guards (a shifted target or an MIS
// term); an occluded ray zeroes that result.  The traced segment is exactly the one visible()
// traces, so deferring it changes no result.  A full queue falls back to tracing in place.
struct VisQ {
    float4* rays;        // 2 float4 per ray: (origin, tmax), (direction, target index bits)
    uint32_t* counter;   // rays reserved so far (may exceed cap)
    uint32_t cap;
    uint32_t target;     // index of the guarded result
};

// one atomic for whichever lanes are converged here (any subset of the warp); every lane of the
// mask runs the same straight-line sequence of shuffles, so all of them meet
static __device__ __forceinline__ uint32_t reserve_coalesced(uint32_t* counter, uint32_t n) {
    const uint32_t mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t prefix = 0, total = 0;
    // rolled: unrolled copies of this loop at every queueing call site inflated the shift
    // kernels' code (4.63 against 4.85 ms per 512 x 512 frame)
#pragma unroll 1
    for (int k = 0; k < 32; ++k) {
        if (!((mask >> k) & 1u)) continue;   // uniform over the group
        uint32_t v = __shfl_sync(mask, n, k);
        total += v;
        if (k < lane) prefix += v;
    }
    uint32_t base = 0;
    if (lane == leader && total) base = atomicAdd(counter, total);
    base = __shfl_sync(mask, base, leader);
    return base + prefix;
}

// one slot for each lane converged here: a ballot, one atomic by the lowest lane, and each lane's
// rank among the converged ones -- the slots reserve_coalesced(counter, 1) gives, in the same order,
// without its loop over the warp
static __device__ __forceinline__ uint32_t reserve_one(uint32_t* counter) {
    const uint32_t mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + (uint32_t)__popc(mask & ((1u << lane) - 1u));
}

// visible(), or the same segment queued for vis_kernel (returns true: not known to be occluded)
static __device__ bool visible_q(const VisQ* q, const GeomDev& g, float3 a, float3 an, float3 b, const float3* bn, float eps) {
    if (!q) return visible(g, a, an, b, bn, eps);
    float3 ao = offset_point(a, an, b - a, eps);
    float3 bo = bn ? offset_point(b, *bn, a - b, eps) : b;
    float3 d = bo - ao;
    float dist = len3(d);
    if (!(dist > 0.f)) return true;
    d = d * (1.0f / dist);
    uint32_t i = reserve_one(q->counter);
    if (i >= q->cap) {
        int tri; float b1, b2, t;
        return !traverse<true>(g, ao, d, dist, tri, b1, b2, t);
    }
    q->rays[2 * (size_t)i] = make_float4(ao.x, ao.y, ao.z, dist);
    q->rays[2 * (size_t)i + 1] = make_float4(d.x, d.y, d.z, __uint_as_float(q->target));
    return true;
}

// ============================================================================================
// sensor rays and back-projection
// ============================================================================================
static __device__ void primary_ray(const FrameDev& F, int ix, int iy, float u0, float u1, float3& o, float3& d) {
    o = F.pos;
    if (F.mode == 1) {
        float3 w = F.wall_o + (F.wall_u * ((ix + 0.5f) / F.W) + F.wall_v * ((iy + 0.5f) / F.H));
        d = norm3(w - o);
        return;
    }
    float3 f = norm3(F.fwd);
    float3 rt = norm3(cross3(f, F.up));
    float3 up = cross3(rt, f);
    float th = tanf(0.5f * F.fov_y), asp = (float)F.W / (float)F.H;
    float sx = (2.0f * (ix + u0) / F.W - 1.0f) * th * asp;
    float sy = (1.0f - 2.0f * (iy + u1) / F.H) * th;
    d = norm3(f + (rt * sx + up * sy));
}
static __device__ bool project(const FrameDev& F, float3 p, int& ix, int& iy) {
    float3 f = norm3(F.fwd);
    float3 rt = norm3(cross3(f, F.up));
    float3 up = cross3(rt, f);
    float3 d = p - F.pos;
    float z = dot3(d, f);
    if (!(z > 0.f)) return false;
    float th = tanf(0.5f * F.fov_y), asp = (float)F.W / (float)F.H;
    float sx = dot3(d, rt) / z / (th * asp), sy = dot3(d, up) / z / th;
    float fx = (sx + 1.0f) * 0.5f * F.W, fy = (1.0f - sy) * 0.5f * F.H;
    if (!(fx >= 0.f && fy >= 0.f)) return false;
    int x = (int)floorf(fx), y = (int)floorf(fy);
    if (x >= F.W || y >= F.H) return false;
    ix = x; iy = y;
    return true;
}

// ============================================================================================
// domains and lights (Sec. 3.2: each pixel of each frame is an integration domain with its own
// target; Sec. 5: point light with NEE, laser spot as a secondary emitter)
// ============================================================================================
struct Domain {
    const FrameDev* F;
    bool valid;
    float3 x0;
    Surf y1;
    float o, L0, dL;
    LightDev light;
    float3 spot_n;   // spot surface normal (kind 2)
    int spot_mat;
};

static __device__ void resolve_spot(const GeomDev& g, LightDev& L, float3& sn, int& smat) {
    Surf s = surf_at(g, L.s_tri, L.s_b1, L.s_b2);
    L.pos = s.p; sn = s.n; smat = s.mat;
}

static __device__ Domain make_domain(const FrameDev* F, int pix, float L0, float dL) {
    Domain D;
    D.F = F;
    D.x0 = F->pos;
    D.L0 = L0; D.dL = dL;
    D.light.kind = 0;
    float4 gb = __ldg(&F->gb[pix]);
    uint32_t tri = __float_as_uint(gb.x);
    D.valid = tri != kNoHit;
    D.o = 0.f;
    D.spot_n = f3(0.f, 0.f, 1.f);
    D.spot_mat = 0;
    if (!D.valid) return D;
    D.y1 = surf_at(F->g, (int)tri, gb.y, gb.z);
    D.o = F->mode == 1 ? 2.0f * gb.w : 0.f;
    if (F->etype == 0) {
        D.light.kind = 1; D.light.pos = F->epos; D.light.I = F->epower;
    } else if (F->etype == 1) {
        D.light = *F->laser;
        if (D.light.kind == 2) resolve_spot(F->g, D.light, D.spot_n, D.spot_mat);
    } else {
        D.light.kind = 2; D.light.s_tri = D.y1.tri; D.light.s_b1 = D.y1.b1; D.light.s_b2 = D.y1.b2;
        D.light.I = F->epower;
        D.light.to_origin = dir_to(D.y1.p, F->epos);
        D.light.emit_len = len3(F->epos - D.y1.p);
        D.light.pos = D.y1.p;
        D.spot_n = D.y1.n; D.spot_mat = D.y1.mat;
    }
    return D;
}

// domain of a pixel whose primary hit is (tri, b1, b2) at distance t from the sensor
static __device__ __forceinline__ Domain make_domain_hit(const FrameDev* F, bool valid, int tri, float b1, float b2, float t, float L0, float dL) {
    Domain D;
    D.F = F;
    D.x0 = F->pos;
    D.L0 = L0; D.dL = dL;
    D.light.kind = 0;
    D.valid = valid;
    D.o = 0.f;
    D.spot_n = f3(0.f, 0.f, 1.f);
    D.spot_mat = 0;
    if (!valid) return D;
    D.y1 = surf_at(F->g, tri, b1, b2);
    D.o = F->mode == 1 ? 2.0f * t : 0.f;
    if (F->etype == 0) {
        D.light.kind = 1; D.light.pos = F->epos; D.light.I = F->epower;
    } else if (F->etype == 1) {
        D.light = *F->laser;
        if (D.light.kind == 2) resolve_spot(F->g, D.light, D.spot_n, D.spot_mat);
    } else {
        D.light.kind = 2; D.light.s_tri = D.y1.tri; D.light.s_b1 = D.y1.b1; D.light.s_b2 = D.y1.b2;
        D.light.I = F->epower;
        D.light.to_origin = dir_to(D.y1.p, F->epos);
        D.light.emit_len = len3(F->epos - D.y1.p);
        D.light.pos = D.y1.p;
        D.spot_n = D.y1.n; D.spot_mat = D.y1.mat;
    }
    return D;
}

static __device__ __forceinline__ bool light_same(const LightDev& a, const LightDev& b) {
    if (a.kind != b.kind) return false;
    if (a.kind == 0) return true;
    if (a.pos.x != b.pos.x || a.pos.y != b.pos.y || a.pos.z != b.pos.z || a.I != b.I) return false;
    if (a.kind == 2) {
        if (a.s_tri != b.s_tri || a.s_b1 != b.s_b1 || a.s_b2 != b.s_b2) return false;
        if (a.to_origin.x != b.to_origin.x || a.to_origin.y != b.to_origin.y || a.to_origin.z != b.to_origin.z) return false;
        if (a.emit_len != b.emit_len) return false;
    }
    return true;
}

// light factor I_e |cos_x| / d^2 of a path ending at x (no BSDF, no visibility); wl, seg out
static __device__ float light_term(const Domain& D, const Surf& x, float3& wl, float& seg) {
    const LightDev& L = D.light;
    float3 lp = L.pos;
    float I = 0.f;
    if (L.kind == 1) I = L.I;
    else if (L.kind == 2) {
        float3 w = dir_to(L.pos, x.p);
        Mat sm = load_mat(D.F->g, D.spot_mat);
        I = L.I * bsdf_f(sm, D.spot_n, L.to_origin, w) * fabsf(dot3(D.spot_n, w));
    }
    float3 dd = lp - x.p;
    float dist = len3(dd);
    if (!(dist > 0.f) || !(I > 0.f)) return 0.f;
    wl = dd * (1.0f / dist);
    seg = dist + (L.kind == 2 ? L.emit_len : 0.f);
    return I * fabsf(dot3(x.n, wl)) / (dist * dist);
}
static __device__ __forceinline__ bool light_visible(const Domain& D, const GeomDev& g, const Surf& x, float eps,
                                                     const VisQ* q = nullptr) {
    if (D.light.kind == 2) return visible_q(q, g, x.p, x.n, D.light.pos, &D.spot_n, eps);
    return visible_q(q, g, x.p, x.n, D.light.pos, nullptr, eps);
}

static __device__ __forceinline__ float Gterm(const Surf& a, const Surf& b) {
    float3 d = b.p - a.p;
    float d2 = dot3(d, d);
    if (!(d2 > 0.f)) return 0.f;
    float3 w = d * (1.0f / sqrtf(d2));
    return fabsf(dot3(a.n, w)) * fabsf(dot3(b.n, w)) / d2;
}

// ============================================================================================
// reservoir records: decoded form and the 6-plane float4 encoding
//   P0 (W, phat, tau, Lsuf)   P1 (key_px, key_frame, meta, pdf_pre)   P2 (xprev.xyz, p_tri)
//   P3 (p_b1, p_b2, s0_tri, s0_b1)   P4 (s0_b2, s1_tri, s1_b1, s1_b2)   P5 (s2_tri, s2_b1, s2_b2, 0)
//   (six planes, or six consecutive words per entry: see ResDev)
//   meta: tree [0,8) | k [8,11) | r [11,14) | ns [14,16) | class of x_1..x_4, 2 bits each [16,24)
// (Sec. 5: the reservoir stores the vertex after the reconnection vertex; the reconnection
//  radiance Lsuf is attached to it)
// ============================================================================================
struct Rec {
    float W, phat, tau, Lsuf;
    uint32_t key_px, key_frame, meta;
    float pdf_pre;
    float3 xprev;
    int p_tri;
    float p_b1, p_b2;
    int s_tri[3];
    float s_b1[3], s_b2[3];
};
static __device__ __forceinline__ int rec_tree(const Rec& r) { return (int)(r.meta & 0xFFu); }
static __device__ __forceinline__ int rec_k(const Rec& r) { return (int)((r.meta >> 8) & 7u); }
static __device__ __forceinline__ int rec_r(const Rec& r) { return (int)((r.meta >> 11) & 7u); }
static __device__ __forceinline__ int rec_ns(const Rec& r) { return (int)((r.meta >> 14) & 3u); }
static __device__ __forceinline__ int rec_cls(const Rec& r, int j) { return (int)((r.meta >> (16 + 2 * (j - 1))) & 3u); }

// word k of entry idx (SoA or AoS, see ResDev)
static __device__ __forceinline__ float4* res_at(const ResDev& R, int k, size_t idx) {
    return R.planes + (size_t)k * R.stride + idx * R.estride;
}
static __device__ __forceinline__ void rec_store(const ResDev& R, size_t idx, const Rec& r) {
    *res_at(R, 0, idx) = make_float4(r.W, r.phat, r.tau, r.Lsuf);
    *res_at(R, 1, idx) = make_float4(__uint_as_float(r.key_px), __uint_as_float(r.key_frame), __uint_as_float(r.meta), r.pdf_pre);
    if (rec_r(r) >= 2) {
        *res_at(R, 2, idx) = make_float4(r.xprev.x, r.xprev.y, r.xprev.z, __int_as_float(r.p_tri));
        *res_at(R, 3, idx) = make_float4(r.p_b1, r.p_b2, __int_as_float(r.s_tri[0]), r.s_b1[0]);
        int ns = rec_ns(r);
        if (ns >= 2) *res_at(R, 4, idx) = make_float4(r.s_b2[0], __int_as_float(r.s_tri[1]), r.s_b1[1], r.s_b2[1]);
        else if (ns == 1) *res_at(R, 4, idx) = make_float4(r.s_b2[0], 0.f, 0.f, 0.f);
        if (ns >= 3) *res_at(R, 5, idx) = make_float4(__int_as_float(r.s_tri[2]), r.s_b1[2], r.s_b2[2], 0.f);
    }
}
static __device__ __forceinline__ void rec_load(const ResDev& R, size_t idx, Rec& r) {
    float4 a = *res_at(R, 0, idx), b = *res_at(R, 1, idx);
    r.W = a.x; r.phat = a.y; r.tau = a.z; r.Lsuf = a.w;
    r.key_px = __float_as_uint(b.x); r.key_frame = __float_as_uint(b.y); r.meta = __float_as_uint(b.z); r.pdf_pre = b.w;
    if (rec_r(r) >= 2) {
        float4 c = *res_at(R, 2, idx), d = *res_at(R, 3, idx);
        r.xprev = f3(c.x, c.y, c.z); r.p_tri = __float_as_int(c.w);
        r.p_b1 = d.x; r.p_b2 = d.y; r.s_tri[0] = __float_as_int(d.z); r.s_b1[0] = d.w;
        int ns = rec_ns(r);
        if (ns >= 1) {
            float4 e = *res_at(R, 4, idx);
            r.s_b2[0] = e.x; r.s_tri[1] = __float_as_int(e.y); r.s_b1[1] = e.z; r.s_b2[1] = e.w;
        }
        if (ns >= 3) {
            float4 f = *res_at(R, 5, idx);
            r.s_tri[2] = __float_as_int(f.x); r.s_b1[2] = f.y; r.s_b2[2] = f.z;
        }
    }
}
static __device__ __forceinline__ bool occ_get(const ResDev& R, int pix, int b) {
    return (R.occ[(size_t)pix * R.words + (b >> 5)] >> (b & 31)) & 1u;
}

// ============================================================================================
// path trees (Sec. 3.2 stage (1); Sec. 5 light source): BSDF-sampled paths with NEE to the
// delta light at every vertex; the candidate of length k is the NEE path ending at x_k.
// ============================================================================================
struct TreeVerts {
    Surf v[kMaxDepth + 1];     // v[1..depth]
    float pdfA[kMaxDepth + 1];
    int cls[kMaxDepth + 1];
};

// reconnectability of vertex i of x_1..x_k (Sec. 4.1: first consecutive diffuse pair; the
// perturbation re-evaluates the BSDF after p, so that vertex must be rough or be the light)
static __device__ __forceinline__ bool connectable(const int* cls, const float3* pos, int k, int i, float dmin) {
    if (cls[i - 1] != C_ROUGH || cls[i] != C_ROUGH) return false;
    if (len3(pos[i - 1] - pos[i]) <= dmin) return false;
    if (i < k) {
        if (cls[i + 1] != C_ROUGH) return false;
        if (len3(pos[i] - pos[i + 1]) <= dmin) return false;
    }
    return true;
}
static __device__ __forceinline__ int find_r(const int* cls, const float3* pos, int k, float dmin) {
    for (int i = 2; i <= k; ++i)
        if (connectable(cls, pos, k, i, dmin)) return i;
    return 0;
}

// f(x) in area measure of the NEE path x_1..x_k (no visibility)
static __device__ float path_f(const Domain& D, const TreeVerts& T, int k) {
    const GeomDev& g = D.F->g;
    float f = 1.0f;
    for (int j = 1; j <= k; ++j) {
        Mat m = load_mat(g, T.v[j].mat);
        float3 wi = dir_to(T.v[j].p, j == 1 ? D.x0 : T.v[j - 1].p);
        if (j < k) {
            if (mat_class(m) == C_DELTA) f *= m.albedo;
            else f *= bsdf_f(m, T.v[j].n, wi, dir_to(T.v[j].p, T.v[j + 1].p)) * Gterm(T.v[j], T.v[j + 1]);
        } else {
            float3 wl; float seg;
            float lt = light_term(D, T.v[k], wl, seg);
            f *= bsdf_f(m, T.v[k].n, wi, wl) * lt;
        }
    }
    return f;
}

// reservoir record of the candidate of length k from tree `tree` (P0's W is filled later); out of
// line: every RIS selection calls it, and inlined at each candidate site it bloats the path-tree
// loop (0.25 ms of the ellipsoidal initial kernel on the 512 x 512 workload)
static __device__ __noinline__ void build_rec(const Domain& D, const TreeVerts& T, int k, int tree, uint32_t px, uint32_t frame, float tau,
                          const ParamsDev& P, Rec& R) {
    const GeomDev& g = D.F->g;
    R.W = 0.f;
    R.tau = tau;
    R.key_px = px; R.key_frame = frame;
    R.phat = path_f(D, T, k);
    R.Lsuf = 0.f;
    R.pdf_pre = 1.0f;
    float3 pos[kMaxDepth + 1];
    for (int j = 1; j <= k; ++j) pos[j] = T.v[j].p;
    int r = find_r(T.cls, pos, k, P.d_min);
    uint32_t meta = (uint32_t)tree | ((uint32_t)k << 8) | ((uint32_t)r << 11);
    if (r == 0) { R.meta = meta; return; }
    for (int j = 1; j < r; ++j) meta |= (uint32_t)T.cls[j] << (16 + 2 * (j - 1));
    int ns = k - r;
    meta |= (uint32_t)ns << 14;
    R.meta = meta;
    R.xprev = T.v[r - 1].p;
    for (int j = 2; j <= r - 1; ++j) R.pdf_pre *= T.pdfA[j];
    R.p_tri = T.v[r].tri; R.p_b1 = T.v[r].b1; R.p_b2 = T.v[r].b2;
    for (int q = 0; q < 3; ++q) { R.s_tri[q] = 0; R.s_b1[q] = 0.f; R.s_b2[q] = 0.f; }
    for (int q = 0; q < ns; ++q) { R.s_tri[q] = T.v[r + 1 + q].tri; R.s_b1[q] = T.v[r + 1 + q].b1; R.s_b2[q] = T.v[r + 1 + q].b2; }
    if (ns > 0) {
        float Ls = 1.0f;
        for (int j = r + 2; j <= k; ++j) {
            Mat m = load_mat(g, T.v[j].mat);
            float gg = T.cls[j - 1] == C_DELTA ? 1.0f : Gterm(T.v[j - 1], T.v[j]);
            if (mat_class(m) == C_DELTA) { Ls *= gg * m.albedo; continue; }
            float3 wi = dir_to(T.v[j].p, T.v[j - 1].p);
            float3 wo;
            if (j < k) wo = dir_to(T.v[j].p, T.v[j + 1].p);
            else { float seg; light_term(D, T.v[k], wo, seg); }
            Ls *= gg * bsdf_f(m, T.v[j].n, wi, wo);
        }
        float3 wl; float seg;
        Ls *= light_term(D, T.v[k], wl, seg);
        R.Lsuf = Ls;
    }
}

// ============================================================================================
// path-length derivatives (Sec. 4.3 "Gradient and Hessian Evaluation"):
//   L(p) = |p1 - p| + |p2 - p|, grad_p L = -(d1 + d2), hess_p L = A = sum (I - d d^T)/|p_i - p|,
//   grad_xi L = J^T grad_p L, hess_xi L = J^T A J (Q = 0 on flat triangles)
// ============================================================================================
struct Frame2 { float3 o, t, b; };
static __device__ __forceinline__ Frame2 tri_frame(const GeomDev& g, int tri) {
    float4 a = __ldg(&g.tri[3 * tri]), e1 = __ldg(&g.tri[3 * tri + 1]), e2 = __ldg(&g.tri[3 * tri + 2]);
    Frame2 f;
    f.o = xyz(a);
    f.t = norm3(xyz(e1));
    float3 n = norm3(cross3(xyz(e1), xyz(e2)));
    f.b = cross3(n, f.t);
    return f;
}
static __device__ __forceinline__ float3 frame_point(const Frame2& f, float x0, float x1) { return f.o + (f.t * x0 + f.b * x1); }

static __device__ __forceinline__ void length_derivs(float3 p1, float3 p2, const Frame2& f, float x0, float x1, float& L,
                                              float g[2], float h[3]) {
    float3 p = frame_point(f, x0, x1);
    float3 a1 = p1 - p, a2 = p2 - p;
    float l1 = len3(a1), l2 = len3(a2);
    float3 d1 = a1 * (1.0f / l1), d2 = a2 * (1.0f / l2);
    float3 s = d1 + d2;
    L = l1 + l2;
    g[0] = -dot3(f.t, s);
    g[1] = -dot3(f.b, s);
    float d1t = dot3(d1, f.t), d1b = dot3(d1, f.b), d2t = dot3(d2, f.t), d2b = dot3(d2, f.b);
    h[0] = (1.0f - d1t * d1t) / l1 + (1.0f - d2t * d2t) / l2;
    h[1] = (-d1t * d1b) / l1 + (-d2t * d2b) / l2;
    h[2] = (1.0f - d1b * d1b) / l1 + (1.0f - d2b * d2b) / l2;
}

// gauge of the Newton system: the paper's average gradient, or a comparison gauge of Sec. 4.3
// (fixed axis: the vertex moves along t or along b; gradient at the start point only)
enum { G_AVERAGE = 0, G_AXIS_T = 1, G_AXIS_B = 2, G_START = 3 };
static __device__ __forceinline__ int gauge_of(uint32_t flags) {
    return (flags & 8u) ? G_AXIS_T : (flags & 16u) ? G_AXIS_B : (flags & 32u) ? G_START : G_AVERAGE;
}
struct NewtonGeo { float3 p1x, p2x; Frame2 fx; float3 p1y, p2y; Frame2 fy; int gauge; };

// F(xi, xi') = [L_y(xi') - L_x(xi) - delta ; (R m)^T (xi' - xi)], m = (grad L_x(xi) + grad L_y(xi'))/2,
// R = 90-degree rotation; each gradient on its own path (Sec. 4.3, average-gradient gauge)
static __device__ __forceinline__ void newton_F_f(const NewtonGeo& N, const Frame2& fy, const float xi[2], float Lx, const float gx[2],
                                           float delta, const float xp[2], float F[2], float gy[2], float hy[3], float m[2]) {
    float Ly;
    length_derivs(N.p1y, N.p2y, fy, xp[0], xp[1], Ly, gy, hy);
    m[0] = 0.5f * (gx[0] + gy[0]);
    m[1] = 0.5f * (gx[1] + gy[1]);
    F[0] = Ly - Lx - delta;
    if (N.gauge == G_AVERAGE) F[1] = -m[1] * (xp[0] - xi[0]) + m[0] * (xp[1] - xi[1]);
    else if (N.gauge == G_AXIS_T) F[1] = xp[1] - xi[1];
    else if (N.gauge == G_AXIS_B) F[1] = xp[0] - xi[0];
    else F[1] = -gx[1] * (xp[0] - xi[0]) + gx[0] * (xp[1] - xi[1]);
}
static __device__ __forceinline__ void newton_F(const NewtonGeo& N, const float xi[2], float Lx, const float gx[2], float delta,
                                         const float xp[2], float F[2], float gy[2], float hy[3], float m[2]) {
    newton_F_f(N, N.fy, xi, Lx, gx, delta, xp, F, gy, hy, m);
}
// dF/dxi' rows: (grad L_y(xi'), R m - 0.5 H_y R (xi' - xi)); dF/dxi rows: (-grad L_x(xi), -(R m + 0.5 H_x R (xi' - xi)))
// comparison gauges: fixed axis rows (0, 1) / (1, 0); start gradient dF2/dxi' = R g_x,
// dF2/dxi = -(R g_x + H_x R (xi' - xi))
static __device__ __forceinline__ void newton_J(int gauge, const float xi[2], const float xp[2], const float gx[2], const float hx[3],
                                         const float gy[2], const float hy[3], const float m[2], float A[4], float Bm[4]) {
    float Rm0 = -m[1], Rm1 = m[0];
    float dd0 = xp[0] - xi[0], dd1 = xp[1] - xi[1];
    float Rd0 = -dd1, Rd1 = dd0;
    float HyRd0 = hy[0] * Rd0 + hy[1] * Rd1, HyRd1 = hy[1] * Rd0 + hy[2] * Rd1;
    float HxRd0 = hx[0] * Rd0 + hx[1] * Rd1, HxRd1 = hx[1] * Rd0 + hx[2] * Rd1;
    A[0] = gy[0]; A[1] = gy[1];
    Bm[0] = -gx[0]; Bm[1] = -gx[1];
    if (gauge == G_AVERAGE) {
        A[2] = Rm0 - 0.5f * HyRd0; A[3] = Rm1 - 0.5f * HyRd1;
        Bm[2] = -(Rm0 + 0.5f * HxRd0); Bm[3] = -(Rm1 + 0.5f * HxRd1);
    } else if (gauge == G_AXIS_T) {
        A[2] = 0.f; A[3] = 1.f; Bm[2] = 0.f; Bm[3] = -1.f;
    } else if (gauge == G_AXIS_B) {
        A[2] = 1.f; A[3] = 0.f; Bm[2] = -1.f; Bm[3] = 0.f;
    } else {
        A[2] = -gx[1]; A[3] = gx[0];
        Bm[2] = -(-gx[1] + HxRd0); Bm[3] = -(gx[0] + HxRd1);
    }
}

// Newton iteration with backtracking (Sec. 4.3); returns success, xi', |det(dxi'/dxi)| and the
// iteration count.  Stops at |F|_inf <= tol_stop (after one polishing step there) or after
// max_iter (up to 2 max_iter while |F|_inf <= tol_succ, the paper's 1 %-of-the-gate band);
// success if converged, |F|_inf <= tol_stop.
static __device__ bool newton_solve(const NewtonGeo& N, const float xi[2], float delta, int max_iter, float tol_stop,
                             float tol_succ, float xp[2], float& jdet, int& iters) {
    float Lx, gx[2], hx[3];
    length_derivs(N.p1x, N.p2x, N.fx, xi[0], xi[1], Lx, gx, hx);
    xp[0] = xi[0]; xp[1] = xi[1];
    float F[2], gy[2], hy[3], m[2];
    newton_F(N, xi, Lx, gx, delta, xp, F, gy, hy, m);
    int it = 0;
    bool polished = false;
    // loops kept rolled: the unrolled copies of the line search cost more in instruction-cache misses
    // than they save (4.9 against 5.1 ms per 512 x 512 frame)
    // the paper's budget is max_iter iterations; a solve that spends it inside the success band
    // (|F| <= tol_succ) short of convergence continues toward the root, at most max_iter more, so
    // that an accepted shift is the root F = 0 and not a point of the band that depends on rounding
#pragma unroll 1
    while (it < 2 * max_iter) {
        float nF = fmaxf(fabsf(F[0]), fabsf(F[1]));
        if (it >= max_iter && !(nF <= tol_succ)) break;
        bool polish = false;
        if (nF <= tol_stop) {
            // converged: one more full Newton step at the root, kept if |F| does not grow, so that the
            // result is the root itself (to FP32 rounding) and not the first iterate under the
            // tolerance, which FP32 and FP64 reach at different distances from it (not counted)
            if (polished || !(nF > 0.f)) break;
            polish = polished = true;
        }
        float A[4], Bm[4];
        newton_J(N.gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
        float det = A[0] * A[3] - A[1] * A[2];
        if (!(fabsf(det) > 1e-30f)) break;
        float s0 = -(A[3] * F[0] - A[1] * F[1]) / det, s1 = -(-A[2] * F[0] + A[0] * F[1]) / det;
        float lam = 1.0f;
        bool accepted = false;
#pragma unroll 1
        for (int ls = 0; ls < (polish ? 1 : 5); ++ls) {
            float c[2] = {xp[0] + lam * s0, xp[1] + lam * s1};
            float Fc[2], gyc[2], hyc[3], mc[2];
            newton_F(N, xi, Lx, gx, delta, c, Fc, gyc, hyc, mc);
            if (polish ? fmaxf(fabsf(Fc[0]), fabsf(Fc[1])) <= nF : fmaxf(fabsf(Fc[0]), fabsf(Fc[1])) < nF) {
                xp[0] = c[0]; xp[1] = c[1];
                F[0] = Fc[0]; F[1] = Fc[1];
                gy[0] = gyc[0]; gy[1] = gyc[1]; hy[0] = hyc[0]; hy[1] = hyc[1]; hy[2] = hyc[2];
                m[0] = mc[0]; m[1] = mc[1];
                accepted = true;
                break;
            }
            lam *= 0.5f;
        }
        if (!accepted) break;
        if (!polish) ++it;
    }
    iters = it;
    // success: converged (|F| <= tol_stop), so that the shift satisfies its constraint and stays
    // invertible; a solve stalled inside the band (ill-conditioned: L nearly stationary at the
    // vertex) is rejected, in FP32 as in FP64, instead of ending at a rounding-dependent point
    if (!(fmaxf(fabsf(F[0]), fabsf(F[1])) <= tol_stop)) return false;
    float A[4], Bm[4];
    newton_J(N.gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
    float dA = A[0] * A[3] - A[1] * A[2], dB = Bm[0] * Bm[3] - Bm[1] * Bm[2];
    if (!(fabsf(dA) > 0.f)) return false;
    jdet = fabsf(dB / dA);
    return isfinite(jdet);
}

// ============================================================================================
// cross-triangle walk of the reconnection vertex (TOF_FLAG_TRIANGLE_WALK; the paper
// parameterises p on the surface, Sec. 4.2, without saying what happens at a triangle's edge).
// The Newton unknown xi' lives in a 2-D chart: the plane of p's triangle, into which each
// neighbour entered is unfolded about the shared edge (an isometry: lengths, gradients and |det|
// carry over).  A candidate that leaves the current triangle crosses its exit edge into the
// neighbour; the walk fails at a boundary or after kMaxCross crossings.  Two developments of a
// triangle strip differ by a rigid motion, under which the average-gradient gauge is invariant,
// so the shift stays reversible.
// ============================================================================================
constexpr int kMaxCross = 3;   // re-solves on neighbouring triangles per shift (and crossings per walk)
struct Walk { int tri; Frame2 f; };   // f: chart -> 3-D on tri (corners found from the triangle record)

static __device__ __forceinline__ float3 tri_corner(const GeomDev& g, int tri, int j) {
    float3 v0 = xyz(__ldg(&g.tri[3 * tri]));
    if (j == 0) return v0;
    return v0 + xyz(__ldg(&g.tri[3 * tri + j]));
}
static __device__ __forceinline__ void walk_init(const GeomDev& g, int tri, Walk& W) {
    W.tri = tri;
    W.f = tri_frame(g, tri);
}
// corner j of W's triangle in the chart
static __device__ __forceinline__ void walk_corner(const GeomDev& g, const Walk& W, int j, float& q0, float& q1) {
    float3 d = tri_corner(g, W.tri, j) - W.f.o;
    q0 = dot3(d, W.f.t);
    q1 = dot3(d, W.f.b);
}
// out of line: called from several sites of the walking Newton; inlined copies cost the walking shift
// kernels 0.37 ms of instruction fetch per 512 x 512 frame
static __device__ __noinline__ void walk_bary(const GeomDev& g, const Walk& W, float c0, float c1, float lam[3]) {
    float q00, q01, q10, q11, q20, q21;
    walk_corner(g, W, 0, q00, q01);
    walk_corner(g, W, 1, q10, q11);
    walk_corner(g, W, 2, q20, q21);
    float a0 = q10 - q00, a1 = q11 - q01;
    float b0 = q20 - q00, b1 = q21 - q01;
    float d0 = c0 - q00, d1 = c1 - q01;
    float det = a0 * b1 - a1 * b0;
    lam[1] = (d0 * b1 - d1 * b0) / det;
    lam[2] = (a0 * d1 - a1 * d0) / det;
    lam[0] = 1.0f - lam[1] - lam[2];
}
// move W along the chart segment from -> to (from inside W) to the triangle holding `to`
static __device__ bool walk_locate(const GeomDev& g, Walk& W, const float from_in[2], const float to[2]) {
    float from[2] = {from_in[0], from_in[1]};
    for (int k = 0; k <= kMaxCross; ++k) {
        float lt[3], lf[3];
        walk_bary(g, W, to[0], to[1], lt);
        if (lt[0] >= -kBaryEps && lt[1] >= -kBaryEps && lt[2] >= -kBaryEps) return true;
        if (k == kMaxCross || !g.adj) break;
        walk_bary(g, W, from[0], from[1], lf);
        int ex = -1;
        float sbest = 3.0e38f;
        for (int i = 0; i < 3; ++i) {
            if (!(lt[i] < -kBaryEps)) continue;
            float den = lf[i] - lt[i];
            float sx = den > 0.f ? lf[i] / den : 0.f;
            if (sx < 0.f) sx = 0.f;
            if (sx < sbest) { sbest = sx; ex = i; }
        }
        if (ex < 0) return false;
        int n = __ldg(&g.adj[3 * W.tri + ex]);
        if (n < 0) return false;
        const int nb = n >> 2, opp = n & 3;
        const int ia = ex == 2 ? 0 : ex + 1, ib = ex == 0 ? 2 : ex - 1;
        float3 A = tri_corner(g, W.tri, ia), B = tri_corner(g, W.tri, ib), C = tri_corner(g, nb, opp);
        float a0, a1, b0, b1, e0, e1;
        walk_corner(g, W, ia, a0, a1);
        walk_corner(g, W, ib, b0, b1);
        walk_corner(g, W, ex, e0, e1);
        // 3-D: edge direction U and in-plane normal toward the neighbour's third corner; chart: edge
        // direction u and normal away from the current triangle's third corner
        float3 U = norm3(B - A);
        float3 CA = C - A;
        float3 Nv = norm3(CA - U * dot3(CA, U));
        float ul = sqrtf((b0 - a0) * (b0 - a0) + (b1 - a1) * (b1 - a1));
        float u0 = (b0 - a0) / ul, u1 = (b1 - a1) / ul;
        float n0 = -u1, n1 = u0;
        if ((e0 - a0) * n0 + (e1 - a1) * n1 > 0.f) { n0 = -n0; n1 = -n1; }
        W.tri = nb;
        W.f.t = U * u0 + Nv * n0;
        W.f.b = U * u1 + Nv * n1;
        W.f.o = A - (U * (a0 * u0 + a1 * u1) + Nv * (a0 * n0 + a1 * n1));
        from[0] += sbest * (to[0] - from[0]);
        from[1] += sbest * (to[1] - from[1]);
    }
    return false;
}

// Newton with the offset vertex walking across triangles (W: its triangle and chart).  Newton runs
// on the plane of W's triangle exactly as without the walk; when the converged point lies outside
// the triangle, W walks along the chart segment from the solve's start to it (unfolding each
// neighbour it crosses) and Newton continues from that point on the new triangle's plane, with a
// fresh iteration budget, for at most kMaxCross re-solves.  Shifts that stay on their triangle
// cost what they cost without the walk.
static __device__ bool newton_solve_walk(const GeomDev& gi, const NewtonGeo& N, Walk& W, const float xi[2], float delta,
                                         int max_iter, float tol_stop, float tol_succ, float xp[2], float& jdet, int& iters) {
    float Lx, gx[2], hx[3];
    length_derivs(N.p1x, N.p2x, N.fx, xi[0], xi[1], Lx, gx, hx);
    xp[0] = xi[0]; xp[1] = xi[1];
    float start[2] = {xi[0], xi[1]};
    float F[2], gy[2], hy[3], m[2];
    int total = 0;
#pragma unroll 1
    for (int cross = 0;; ++cross) {
        newton_F_f(N, W.f, xi, Lx, gx, delta, xp, F, gy, hy, m);
        int it = 0;
        bool polished = false;
#pragma unroll 1
        while (it < 2 * max_iter) {   // budget as in newton_solve
            float nF = fmaxf(fabsf(F[0]), fabsf(F[1]));
            if (it >= max_iter && !(nF <= tol_succ)) break;
            bool polish = false;
            if (nF <= tol_stop) {   // converged: one polishing step, as in newton_solve
                if (polished || !(nF > 0.f)) break;
                polish = polished = true;
            }
            float A[4], Bm[4];
            newton_J(N.gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
            float det = A[0] * A[3] - A[1] * A[2];
            if (!(fabsf(det) > 1e-30f)) break;
            float s0 = -(A[3] * F[0] - A[1] * F[1]) / det, s1 = -(-A[2] * F[0] + A[0] * F[1]) / det;
            float lam = 1.0f;
            bool accepted = false;
#pragma unroll 1
            for (int ls = 0; ls < (polish ? 1 : 5); ++ls) {
                float c[2] = {xp[0] + lam * s0, xp[1] + lam * s1};
                float Fc[2], gyc[2], hyc[3], mc[2];
                newton_F_f(N, W.f, xi, Lx, gx, delta, c, Fc, gyc, hyc, mc);
                if (polish ? fmaxf(fabsf(Fc[0]), fabsf(Fc[1])) <= nF : fmaxf(fabsf(Fc[0]), fabsf(Fc[1])) < nF) {
                    xp[0] = c[0]; xp[1] = c[1];
                    F[0] = Fc[0]; F[1] = Fc[1];
                    gy[0] = gyc[0]; gy[1] = gyc[1]; hy[0] = hyc[0]; hy[1] = hyc[1]; hy[2] = hyc[2];
                    m[0] = mc[0]; m[1] = mc[1];
                    accepted = true;
                    break;
                }
                lam *= 0.5f;
            }
            if (!accepted) break;
            if (!polish) ++it;
        }
        total += it;
        if (!(fmaxf(fabsf(F[0]), fabsf(F[1])) <= tol_stop)) break;   // converged, as in newton_solve
        float lm[3];
        walk_bary(gi, W, xp[0], xp[1], lm);
        if (lm[0] >= -kBaryEps && lm[1] >= -kBaryEps && lm[2] >= -kBaryEps) {
            iters = total;
            float A[4], Bm[4];
            newton_J(N.gauge, xi, xp, gx, hx, gy, hy, m, A, Bm);
            float dA = A[0] * A[3] - A[1] * A[2], dB = Bm[0] * Bm[3] - Bm[1] * Bm[2];
            if (!(fabsf(dA) > 0.f)) return false;
            jdet = fabsf(dB / dA);
            return isfinite(jdet);
        }
        if (cross == kMaxCross) break;
        // the plane's solution lies outside the triangle: walk there and solve again
        if (!walk_locate(gi, W, start, xp)) break;
        start[0] = xp[0]; start[1] = xp[1];
    }
    iters = total;
    return false;
}

// ============================================================================================
// ellipsoidal path connection for NEE (Sec. 4.4 "Initialization with Ellipsoidal Path
// Connection", Sec. 5 "Ellipsoidal Path Connection"; Pediredla et al. 2019).  From a rough vertex
// x whose prefix has length len, a vertex z is placed so that x -> z -> light lands in the gate:
//   (1) l = |x - z| + |z - q| (q the light position) uniform on [l_a, l_b), the interval the gate
//       leaves (l_a raised to |x - q|);
//   (2) a triangle by a top-down walk of the implicit binary hierarchy over triangle index ranges
//       (GeomDev::enode): at each node the child is taken with probability proportional to its
//       weight, the area below it, or zero where its box cannot meet the ellipsoid with foci x, q
//       and major axis l (the paper's heuristic weights; the distances of x and q to the box bound
//       l from below, their distances to the box's farthest points from above);
//   (3) on the triangle's plane the ellipsoid cuts an ellipse; z is uniform in its parametric
//       angle phi over the arcs inside the triangle (total angle Phi).
// Area density (coarea formula, dA = dl ds / |grad_plane l|, ds = |dz/dphi| dphi):
//   p(z) = P(tri | l) / (l_b - l_a) / Phi * |grad_plane l(z)| / |dz/dphi|.
// Ellipsoids thinner than b = 0.05 a (l within about 1.25e-3 l of |x - q|) place no vertex, in the
// sampler and the density alike (the MIS with the path tree covers those paths): there z depends on
// l - |x - q|, a difference of path lengths FP32 resolves to ~1e-6 m.  The hierarchy depends on the scene alone, so the
// density is a function of the scene, not of how the ray-tracing hierarchy was built.
// ============================================================================================

static __device__ __forceinline__ float enode_w(const float4* node, int n, float3 x, float3 q, float ell) {
    const float4 lo = __ldg(&node[2 * n]), hi = __ldg(&node[2 * n + 1]);
    if (!(lo.w > 0.f)) return 0.f;
    float ax = x.x - fminf(fmaxf(x.x, lo.x), hi.x), ay = x.y - fminf(fmaxf(x.y, lo.y), hi.y), az = x.z - fminf(fmaxf(x.z, lo.z), hi.z);
    float bx = q.x - fminf(fmaxf(q.x, lo.x), hi.x), by = q.y - fminf(fmaxf(q.y, lo.y), hi.y), bz = q.z - fminf(fmaxf(q.z, lo.z), hi.z);
    float lb = sqrtf(ax * ax + ay * ay + az * az) + sqrtf(bx * bx + by * by + bz * bz);
    if (lb > ell) return 0.f;
    float fx = fmaxf(fabsf(x.x - lo.x), fabsf(x.x - hi.x)), fy = fmaxf(fabsf(x.y - lo.y), fabsf(x.y - hi.y)),
          fz = fmaxf(fabsf(x.z - lo.z), fabsf(x.z - hi.z));
    float gx = fmaxf(fabsf(q.x - lo.x), fabsf(q.x - hi.x)), gy = fmaxf(fabsf(q.y - lo.y), fabsf(q.y - hi.y)),
          gz = fmaxf(fabsf(q.z - lo.z), fabsf(q.z - hi.z));
    float ub = sqrtf(fx * fx + fy * fy + fz * fz) + sqrtf(gx * gx + gy * gy + gz * gz);
    return ell <= ub ? lo.w : 0.f;
}

static __device__ __forceinline__ int elog2(int P) { return 31 - __clz(P); }   // P a power of two

// step (2): the triangle (or -1) and its probability.  The draws are the words 2, 3, ... of the
// Philox blocks P_ELL + k (4 words each); r0 is block 0, the later blocks are generated as the walk
// reaches them (one rolled call per 4 levels keeps the code small).
static __device__ int etree_pick(const GeomDev& g, float3 x, float3 q, float ell, uint4 r0, uint32_t c0, uint32_t c1,
                                 uint32_t c2, uint64_t seed, float& prob) {
    int n = 1;
    uint32_t j = 2;   // word index of the next draw
    uint4 r = r0;
    float p = 1.0f;
#pragma unroll 1
    while (n < g.eP) {
        if ((j & 3u) == 0u) r = philox(c0, c1, c2, P_ELL + (j >> 2), seed);
        const uint32_t w = (j & 3u) == 0u ? r.x : (j & 3u) == 1u ? r.y : (j & 3u) == 2u ? r.z : r.w;
        ++j;
        float w0 = enode_w(g.enode, 2 * n, x, q, ell), w1 = enode_w(g.enode, 2 * n + 1, x, q, ell);
        float s = w0 + w1;
        if (!(s > 0.f)) return -1;
        if (u01(w) * s < w0) { n = 2 * n; p *= w0 / s; }
        else { n = 2 * n + 1; p *= w1 / s; }
    }
    prob = p;
    return n - g.eP;
}
// P(tri | l) of step (2) along the root-to-leaf path of tri
static __device__ float etree_prob(const GeomDev& g, int tri, float3 x, float3 q, float ell) {
    const int L = elog2(g.eP), leaf = g.eP + tri;
    float p = 1.0f;
#pragma unroll 1
    for (int i = 0; i < L; ++i) {
        int n = leaf >> (L - i), next = leaf >> (L - i - 1);
        float w0 = enode_w(g.enode, 2 * n, x, q, ell), w1 = enode_w(g.enode, 2 * n + 1, x, q, ell);
        float s = w0 + w1, w = next == 2 * n ? w0 : w1;
        if (!(s > 0.f) || !(w > 0.f)) return 0.f;
        p *= w / s;
    }
    return p;
}

// step (3): the ellipse in the triangle's frame (o = v0, t, b): xi = xo + w0 + R1 cos(phi) g1 +
// R2 sin(phi) g2, and its arcs inside the triangle.  With m the centre, a = l/2, c = |q - x|/2,
// b^2 = a^2 - c^2, d the focal axis, n the normal and h = (m - v0).n, the plane's points
// m - h n + w1 t + w2 b satisfy |r|^2 + beta (r.d)^2 = b^2 (beta = -c^2/a^2): centre
// w0 = beta h (d.n) g / gamma with g = (d.t, d.b), gamma = 1 + beta |g|^2, level
// kappa = b^2 (1 - h^2 / (a^2 gamma)), radii sqrt(kappa / gamma) along g, sqrt(kappa) across.
struct Ellip {
    float xo0, xo1, w00, w01, g10, g11, R1, R2;
    int narc;
    float a0[6], alen[6];
    float Phi;
};

static __device__ __forceinline__ bool ellip_inside(const float c[3][2], float orient, float px, float py) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = i == 2 ? 0 : i + 1;
        float cr = (c[j][0] - c[i][0]) * (py - c[i][1]) - (c[j][1] - c[i][1]) * (px - c[i][0]);
        if (cr * orient < 0.f) return false;
    }
    return true;
}

// zp: a point known to lie on the ellipse (the density at a vertex placed by other means), or
// null.  With a point, kappa is the ellipse's quadratic form at it: the same value without the
// cancellation of the expression above where the plane nearly touches the ellipsoid (the point near
// the plane's mirror point of x and q, where l is minimal), which FP32 cannot resolve.
static __device__ bool ellip_on_tri(const GeomDev& g, int tri, float3 x, float3 q, float ell, const Frame2& f, Ellip& E,
                                    const float3* zp = nullptr) {
    float3 n = cross3(f.t, f.b);
    float3 m = (x + q) * 0.5f;
    float a = 0.5f * ell, c = 0.5f * len3(q - x);
    float b2 = a * a - c * c;
    if (!(b2 >= 2.5e-3f * a * a)) return false;
    float3 d = c > 0.f ? (q - x) * (0.5f / c) : f3(0.f, 0.f, 0.f);
    float beta = -(c * c) / (a * a);
    float dt = dot3(d, f.t), db = dot3(d, f.b), dn = dot3(d, n);
    float3 mo = m - f.o;
    float h = dot3(mo, n);
    float gamma = 1.0f + beta * (dt * dt + db * db);
    E.xo0 = dot3(mo, f.t);
    E.xo1 = dot3(mo, f.b);
    E.w00 = beta * h * dn * dt / gamma;
    E.w01 = beta * h * dn * db / gamma;
    float kappa;
    if (zp) {
        float3 dz = *zp - f.o;
        float d0 = dot3(dz, f.t) - E.xo0 - E.w00, d1 = dot3(dz, f.b) - E.xo1 - E.w01;
        float gd = dt * d0 + db * d1;
        kappa = d0 * d0 + d1 * d1 + beta * gd * gd;
    } else {
        kappa = b2 * (1.0f - h * h / (a * a * gamma));
    }
    if (!(kappa > 0.f)) return false;
    float gl = sqrtf(dt * dt + db * db);
    if (gl > 1e-12f) { E.g10 = dt / gl; E.g11 = db / gl; }
    else { E.g10 = 1.0f; E.g11 = 0.0f; }
    E.R1 = sqrtf(kappa / gamma);
    E.R2 = sqrtf(kappa);
    // corners in the unit-circle coordinates of the ellipse (g2 = (-g11, g10))
    float cc[3][2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float3 dv = tri_corner(g, tri, i) - f.o;
        float w0 = dot3(dv, f.t) - E.xo0 - E.w00, w1 = dot3(dv, f.b) - E.xo1 - E.w01;
        cc[i][0] = (w0 * E.g10 + w1 * E.g11) / E.R1;
        cc[i][1] = (-w0 * E.g11 + w1 * E.g10) / E.R2;
    }
    float orient = (cc[1][0] - cc[0][0]) * (cc[2][1] - cc[0][1]) - (cc[1][1] - cc[0][1]) * (cc[2][0] - cc[0][0]);
    if (orient == 0.f) return false;
    float ph[6];
    int np = 0;
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
        const int j = i == 2 ? 0 : i + 1;
        float e0 = cc[j][0] - cc[i][0], e1 = cc[j][1] - cc[i][1];
        float A2 = e0 * e0 + e1 * e1, B2 = cc[i][0] * e0 + cc[i][1] * e1, C2 = cc[i][0] * cc[i][0] + cc[i][1] * cc[i][1] - 1.0f;
        float disc = B2 * B2 - A2 * C2;
        if (!(disc > 0.f) || !(A2 > 0.f)) continue;
        float sq = sqrtf(disc);
        float s0 = (-B2 - sq) / A2, s1 = (-B2 + sq) / A2;
        if (s0 >= 0.f && s0 <= 1.f) ph[np++] = atan2f(cc[i][1] + s0 * e1, cc[i][0] + s0 * e0);
        if (s1 >= 0.f && s1 <= 1.f) ph[np++] = atan2f(cc[i][1] + s1 * e1, cc[i][0] + s1 * e0);
    }
    for (int i = 1; i < np; ++i)
        for (int j = i; j > 0 && ph[j - 1] > ph[j]; --j) { float t = ph[j]; ph[j] = ph[j - 1]; ph[j - 1] = t; }
    E.narc = 0;
    E.Phi = 0.f;
    if (np == 0) {
        if (ellip_inside(cc, orient, 1.0f, 0.0f)) { E.narc = 1; E.a0[0] = 0.f; E.alen[0] = 2.0f * kPi; E.Phi = 2.0f * kPi; }
    } else {
        for (int i = 0; i < np; ++i) {
            float s0 = ph[i], s1 = i + 1 < np ? ph[i + 1] : ph[0] + 2.0f * kPi;
            if (!(s1 > s0)) continue;
            float mid = 0.5f * (s0 + s1);
            if (!ellip_inside(cc, orient, cosf(mid), sinf(mid))) continue;
            E.a0[E.narc] = s0; E.alen[E.narc] = s1 - s0; E.narc++;
            E.Phi += s1 - s0;
        }
    }
    return E.Phi > 0.f;
}

// [l_a, l_b) of l = |x - z| + |z - q| that puts the path in [glo, ghi); false if empty
static __device__ __forceinline__ bool ell_range(const Domain& D, float3 x, float len, float glo, float ghi, float3& q,
                                                 float& la, float& lb) {
    if (D.light.kind == 0) return false;
    q = D.light.pos;
    float e = D.light.kind == 2 ? D.light.emit_len : 0.f;
    la = fmaxf(glo + D.o - len - e, len3(x - q));
    lb = ghi + D.o - len - e;
    return lb > la;
}

// |grad_plane l(z)| / |dz/dphi| at z on the ellipse E of frame f
static __device__ float ell_point_factor(const Ellip& E, const Frame2& f, float3 z, float3 x, float3 q) {
    float3 gr = dir_to(x, z) + dir_to(q, z);
    float gt = dot3(gr, f.t), gb = dot3(gr, f.b);
    float gp = sqrtf(gt * gt + gb * gb);
    float3 dz = z - f.o;
    float w0 = dot3(dz, f.t) - E.xo0 - E.w00, w1 = dot3(dz, f.b) - E.xo1 - E.w01;
    float c0 = (w0 * E.g10 + w1 * E.g11) / E.R1, c1 = (-w0 * E.g11 + w1 * E.g10) / E.R2;
    float cl = sqrtf(c0 * c0 + c1 * c1);
    if (!(cl > 0.f)) return 0.f;
    c0 /= cl; c1 /= cl;
    float dphi = sqrtf(E.R1 * E.R1 * c1 * c1 + E.R2 * E.R2 * c0 * c0);
    return dphi > 0.f ? gp / dphi : 0.f;
}

// place z from vertex x (prefix length len) of path tree `tree` at vertex index d; true if placed.
// Kept out of line (with ell_pdf): inlined into the path-tree loop, the walk and the ellipse code
// thrash the instruction cache of the divergent warps.
static __device__ __noinline__ bool ell_sample(const Domain& D, const ParamsDev& P, uint32_t px, uint32_t frame, int tree, int d,
                                               const Surf& x, float len, float glo, float ghi, Surf& z, float& pdf) {
    const GeomDev& g = D.F->g;
    if (g.nt < 1 || elog2(g.eP) > kEllMaxLevels) return false;
    float3 q;
    float la, lb;
    if (!ell_range(D, x.p, len, glo, ghi, q, la, lb)) return false;
    const uint32_t c2 = ((uint32_t)tree << 8) | (uint32_t)d;
    const uint4 r0 = philox(px, frame, c2, P_ELL, P.seed);
    float ell = la + u01(r0.x) * (lb - la);
    float ptri;
    int tri = etree_pick(g, x.p, q, ell, r0, px, frame, c2, P.seed, ptri);
    if (tri < 0) return false;
    Frame2 f = tri_frame(g, tri);
    Ellip E;
    if (!ellip_on_tri(g, tri, x.p, q, ell, f, E)) return false;
    float t = u01(r0.y) * E.Phi, cum = 0.f, phi = 0.f;
    for (int i = 0; i < E.narc; ++i) {
        if (t < cum + E.alen[i] || i == E.narc - 1) { phi = E.a0[i] + fminf(t - cum, E.alen[i]); break; }
        cum += E.alen[i];
    }
    float cp = cosf(phi), sp = sinf(phi);
    float xi0 = E.xo0 + E.w00 + E.R1 * cp * E.g10 - E.R2 * sp * E.g11;
    float xi1 = E.xo1 + E.w01 + E.R1 * cp * E.g11 + E.R2 * sp * E.g10;
    float4 e1v = __ldg(&g.tri[3 * tri + 1]), e2v = __ldg(&g.tri[3 * tri + 2]);
    float3 e1 = xyz(e1v), e2 = xyz(e2v);
    float e1t = dot3(e1, f.t), e2t = dot3(e2, f.t), e2b = dot3(e2, f.b);
    float b2 = xi1 / e2b, b1 = (xi0 - b2 * e2t) / e1t;
    z = surf_at(g, tri, b1, b2);
    pdf = ptri / (lb - la) / E.Phi * ell_point_factor(E, f, z.p, x.p, q);
    return pdf > 0.f;
}

// p_ell(z) of a vertex z reached from x by other means (0 where the sampler cannot place it)
static __device__ __noinline__ float ell_pdf(const Domain& D, const Surf& x, float len, float glo, float ghi, const Surf& z) {
    const GeomDev& g = D.F->g;
    if (g.nt < 1 || elog2(g.eP) > kEllMaxLevels) return 0.f;
    float3 q;
    float la, lb;
    if (!ell_range(D, x.p, len, glo, ghi, q, la, lb)) return 0.f;
    float ell = len3(z.p - x.p) + len3(q - z.p);
    if (!(ell >= la && ell < lb)) return 0.f;
    float ptri = etree_prob(g, z.tri, x.p, q, ell);
    if (!(ptri > 0.f)) return 0.f;
    Frame2 f = tri_frame(g, z.tri);
    Ellip E;
    if (!ellip_on_tri(g, z.tri, x.p, q, ell, f, E, &z.p)) return 0.f;
    return ptri / (lb - la) / E.Phi * ell_point_factor(E, f, z.p, x.p, q);
}

// ============================================================================================
// the shift map (Sec. 4.1-4.3): hybrid shift of the record x from domain Dj to domain Di --
// random replay of x_2..x_{r-1} from y_1, reconnection at p = x_r, path-length-aware
// perturbation of p on its triangle -- returning the offset record, its target in Di and the
// Jacobian |dS/dx| (replay pdf ratios times the Newton determinant; the in-plane frames are
// orthonormal, so the frame factor is 1).
// ============================================================================================
struct ShiftStats { uint32_t newton_calls, newton_iters, newton_ok, shift_calls, shift_ok; };

// Sec. 4.4 path-length shrink mapping: instead of keeping the sample's position inside the target
// gate, the offset path's gated length becomes tau' = centre + scale (tau - centre), accepted in
// [lo, hi).  scale = 1/K shrinks a sample drawn in a gate K times wider into the gate, scale = K
// expands it back; the constraint row of dF/dxi scales by `scale`, and so does the Jacobian.
struct GateMap { float scale, centre, lo, hi; };

// kOut = false: only the target value and the Jacobian are wanted (the MIS terms), not the record.
// vq: the visibility segments of a shift that passes every other test are queued there (vis_kernel
// zeroes the guarded result when one is occluded); null: they are traced in place.
// gm: the gate map of the shrink mapping (null: translation between gates).  kWalk: the
// reconnection vertex may walk across triangle edges (TOF_FLAG_TRIANGLE_WALK), compiled apart so
// that the default shift keeps its code size and registers.
template <bool kOut, bool kWalk = false>
static __device__ bool shift_rec(const Rec& x, const Domain& Dj, const Domain& Di, const ParamsDev& P, bool geom_static, Rec& y,
                          float& phat_out, float& jac_out, ShiftStats* st, const VisQ* vq = nullptr,
                          const GateMap* gm = nullptr) {
    const int r = rec_r(x);
    if (r < 2 || !Di.valid || !Dj.valid) return false;
    const GeomDev& gi = Di.F->g;
    const GeomDev& gj = Dj.F->g;
    const int k = rec_k(x), ns = rec_ns(x), tree = rec_tree(x);
    const float eps = P.ray_eps;
    if (st) st->shift_calls++;

    // (1) random replay with the base path's random numbers
    Surf yv[kMaxDepth];
    yv[1] = Di.y1;
    float plen = len3(Di.x0 - yv[1].p);
    float fpre = 1.0f, pdfy = 1.0f;
    for (int j = 1; j <= r - 2; ++j) {
        uint4 u = philox(x.key_px, x.key_frame, ((uint32_t)tree << 8) | (uint32_t)j, P_BSDF, P.seed);
        float3 wi = dir_to(yv[j].p, j == 1 ? Di.x0 : yv[j - 1].p);
        Mat m = load_mat(gi, yv[j].mat);
        if (mat_class(m) != rec_cls(x, j)) return false;
        float3 wo; float pdf, thr; bool delta;
        if (!bsdf_sample(m, yv[j].n, wi, u01(u.x), u01(u.y), wo, pdf, thr, delta)) return false;
        if (!trace_from(gi, yv[j], wo, eps, yv[j + 1])) return false;
        float seg = len3(yv[j + 1].p - yv[j].p);
        plen += seg;
        if (delta) fpre *= m.albedo;
        else {
            fpre *= bsdf_f(m, yv[j].n, wi, wo) * Gterm(yv[j], yv[j + 1]);
            pdfy *= pdf * fabsf(dot3(yv[j + 1].n, wo)) / (seg * seg);
        }
    }
    if (mat_class(load_mat(gi, yv[r - 1].mat)) != rec_cls(x, r - 1)) return false;

    // (2) suffix and light in the target domain
    Surf sv[3];
    for (int q = 0; q < ns; ++q) sv[q] = surf_at(gi, x.s_tri[q], x.s_b1[q], x.s_b2[q]);
    if (Di.light.kind == 0) return false;
    float3 lpos_i = Di.light.pos;
    float emit_i = Di.light.kind == 2 ? Di.light.emit_len : 0.f;
    float slen = 0.f;
    for (int q = 0; q + 1 < ns; ++q) slen += len3(sv[q].p - sv[q + 1].p);
    if (ns > 0) slen += len3(sv[ns - 1].p - lpos_i) + emit_i;
    else slen += emit_i;
    float3 p2y = ns > 0 ? sv[0].p : lpos_i;

    // (3) base-path quantities in the record's own frame
    NewtonGeo N;
    N.fx = tri_frame(gj, x.p_tri);
    Surf pbase = surf_at(gj, x.p_tri, x.p_b1, x.p_b2);
    float3 p2x = ns > 0 ? surf_at(gj, x.s_tri[0], x.s_b1[0], x.s_b2[0]).p : Dj.light.pos;
    float xi[2];
    {
        float3 dd = pbase.p - N.fx.o;
        xi[0] = dot3(dd, N.fx.t);
        xi[1] = dot3(dd, N.fx.b);
    }
    N.p1x = x.xprev; N.p2x = p2x; N.gauge = gauge_of(P.flags);
    N.p1y = yv[r - 1].p; N.p2y = p2y; N.fy = tri_frame(gi, x.p_tri);

    // (4) Newton solve of L(y') = L(x) + delta (eq. path_length_constraint), delta keeping the
    // sample at the same position inside the target gate
    float Lx_seg = len3(x.xprev - pbase.p) + len3(p2x - pbase.p);
    float tau_t = 0.f;   // target gated length under a gate map
    float ell;
    if (gm) {
        tau_t = gm->centre + gm->scale * (x.tau - gm->centre);
        ell = tau_t + Di.o - plen - slen;
    } else {
        ell = x.tau - Dj.L0 + Di.L0 + Di.o - plen - slen;
    }
    float delta = ell - Lx_seg;
    float xp[2];
    float jn = 1.0f;
    const bool walk = kWalk && !(P.flags & 2u);
    Walk W;
    if (walk) walk_init(gi, x.p_tri, W);
    if (P.flags & 2u) {
        xp[0] = xi[0]; xp[1] = xi[1];
    } else {
        int iters = 0;
        float tol_stop = gm ? 1e-6f * fabsf(tau_t + Di.o) : 1e-6f * fabsf(x.tau + Di.o + Di.L0 - Dj.L0);
        float tol_succ = P.newton_tol_frac * (gm ? gm->hi - gm->lo : Di.dL);
        bool ok = walk ? newton_solve_walk(gi, N, W, xi, delta, P.newton_max_iter, tol_stop, tol_succ, xp, jn, iters)
                       : newton_solve(N, xi, delta, P.newton_max_iter, tol_stop, tol_succ, xp, jn, iters);
        if (st) { st->newton_calls++; st->newton_iters += iters; if (ok) st->newton_ok++; }
        if (!ok) return false;
        if (!(jn >= 1.0f / P.jac_max && jn <= P.jac_max)) return false;
    }
    float nb1, nb2;
    int ptri = x.p_tri;
    if (walk) {
        float lam[3];
        walk_bary(gi, W, xp[0], xp[1], lam);
        ptri = W.tri; nb1 = lam[1]; nb2 = lam[2];
    } else {
        float4 a = __ldg(&gi.tri[3 * x.p_tri]), e1v = __ldg(&gi.tri[3 * x.p_tri + 1]), e2v = __ldg(&gi.tri[3 * x.p_tri + 2]);
        (void)a;
        float3 e1 = xyz(e1v), e2 = xyz(e2v);
        float e1t = dot3(e1, N.fy.t), e2t = dot3(e2, N.fy.t), e2b = dot3(e2, N.fy.b);
        nb2 = xp[1] / e2b;
        nb1 = (xp[0] - nb2 * e2t) / e1t;
    }
    if (!(nb1 >= -kBaryEps && nb2 >= -kBaryEps && nb1 + nb2 <= 1.0f + kBaryEps)) return false;
    Surf pp = surf_at(gi, ptri, nb1, nb2);

    // (5) the offset path must reconnect at the same index
    {
        int cls[kMaxDepth + 2];
        float3 pos[kMaxDepth + 2];
        for (int j = 1; j <= r - 1; ++j) { cls[j] = mat_class(load_mat(gi, yv[j].mat)); pos[j] = yv[j].p; }
        cls[r] = mat_class(load_mat(gi, pp.mat)); pos[r] = pp.p;
        for (int q = 0; q < ns; ++q) { cls[r + 1 + q] = mat_class(load_mat(gi, sv[q].mat)); pos[r + 1 + q] = sv[q].p; }
        if (find_r(cls, pos, k, P.d_min) != r) return false;
    }

    // (6) target function in Di without the suffix radiance, the gate and the Jacobian: cheap
    // rejections, taken before any ray is traced (the result is the same in either order)
    float3 wprev = dir_to(yv[r - 1].p, r - 1 == 1 ? Di.x0 : yv[r - 2].p);
    float f = fpre;
    f *= bsdf_f(load_mat(gi, yv[r - 1].mat), yv[r - 1].n, wprev, dir_to(yv[r - 1].p, pp.p));
    f *= Gterm(yv[r - 1], pp);
    Mat mp = load_mat(gi, pp.mat);
    if (ns == 0) {
        float3 wl; float seg;
        float lt = light_term(Di, pp, wl, seg);
        f *= bsdf_f(mp, pp.n, dir_to(pp.p, yv[r - 1].p), wl) * lt;
    } else {
        f *= bsdf_f(mp, pp.n, dir_to(pp.p, yv[r - 1].p), dir_to(pp.p, sv[0].p));
        f *= Gterm(pp, sv[0]);
        float3 wnext = ns > 1 ? dir_to(sv[0].p, sv[1].p) : dir_to(sv[0].p, lpos_i);
        f *= bsdf_f(load_mat(gi, sv[0].mat), sv[0].n, dir_to(sv[0].p, pp.p), wnext);
    }
    if (!(f > 0.f) || !isfinite(f)) return false;
    float Lnew = plen + len3(yv[r - 1].p - pp.p) + len3(pp.p - p2y) + slen;
    float tau = Lnew - Di.o;
    if (gm) {
        if (!(tau >= gm->lo && tau < gm->hi)) return false;
    } else if (!(tau >= Di.L0 && tau < Di.L0 + Di.dL)) return false;
    float jac = (x.pdf_pre / pdfy) * jn;
    if (gm) jac *= gm->scale;
    if (!(jac > 0.f) || !isfinite(jac)) return false;

    // (7) suffix radiance: cached, or re-evaluated when the scene or light differs (Sec. 5); the
    // re-evaluated suffix's segments must be unoccluded too (tested in (8))
    float Lsuf_i = x.Lsuf;
    bool suffix_eval = false;
    if (ns > 0) {
        bool cache_ok = geom_static && light_same(Dj.light, Di.light);
        if (!cache_ok) {
            suffix_eval = true;
            float Ls = 1.0f;
            for (int q = 1; q < ns; ++q) {
                Mat mq = load_mat(gi, sv[q].mat);
                float gg = mat_class(load_mat(gi, sv[q - 1].mat)) == C_DELTA ? 1.0f : Gterm(sv[q - 1], sv[q]);
                if (mat_class(mq) == C_DELTA) {
                    if (!geom_static) return false;
                    Ls *= gg * mq.albedo;
                } else {
                    float3 wn = q + 1 < ns ? dir_to(sv[q].p, sv[q + 1].p) : dir_to(sv[q].p, lpos_i);
                    Ls *= gg * bsdf_f(mq, sv[q].n, dir_to(sv[q].p, sv[q - 1].p), wn);
                }
            }
            float3 wl; float seg;
            Ls *= light_term(Di, sv[ns - 1], wl, seg);
            Lsuf_i = Ls;
        }
        f *= Lsuf_i;
    }
    if (!(f > 0.f) || !isfinite(f)) return false;

    // (8) visibility of the two reconnection segments and of a re-evaluated suffix, last: every
    // other test has passed, so only shifts that visibility alone decides queue segments
    if (!visible_q(vq, gi, yv[r - 1].p, yv[r - 1].n, pp.p, &pp.n, eps)) return false;
    if (ns > 0) { if (!visible_q(vq, gi, pp.p, pp.n, sv[0].p, &sv[0].n, eps)) return false; }
    else if (!light_visible(Di, gi, pp, eps, vq)) return false;
    if (suffix_eval) {
        for (int q = 1; q < ns; ++q)
            if (!visible_q(vq, gi, sv[q - 1].p, sv[q - 1].n, sv[q].p, &sv[q].n, eps)) return false;
        if (!light_visible(Di, gi, sv[ns - 1], eps, vq)) return false;
    }

    if (kOut) {
        y = x;
        y.tau = tau;
        y.xprev = yv[r - 1].p;
        y.pdf_pre = pdfy;
        y.p_tri = ptri; y.p_b1 = nb1; y.p_b2 = nb2;
        y.Lsuf = Lsuf_i;
        y.phat = f;
    }
    phat_out = f;
    jac_out = jac;
    if (st) st->shift_ok++;
    return true;
}

// --------------------------------------------------------------------------------------------
// batched launches (tof_render_batch): the instance of this block, blk0[j] <= blockIdx.x < blk0[j + 1],
// and its argument record copied to shared memory by the whole block
__device__ __forceinline__ int batch_job(const int* __restrict__ blk0, int n) {
    int lo = 0, hi = n - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&blk0[mid]) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
template <class T>
__device__ __forceinline__ void block_copy(T* dst, const T* src) {
    static_assert(sizeof(T) % 4 == 0, "4-byte words");
    const uint32_t* s = (const uint32_t*)src;
    uint32_t* d = (uint32_t*)dst;
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}


}  // namespace tof
