// tof_kernels.cu -- per-frame kernels of the ToF ReSTIR hot path (sm_103a).
//
//   gbuffer_kernel   primary visibility, one jittered ray per pixel            (Sec. 3.2 setup)
//   initial_kernel   path trees with NEE, streaming RIS into per-bin reservoirs (stage (1), Sec. 4.5);
//                    direct gated renders run it as a bounce wavefront (tw_*_kernel)
//   (temporal and spatial reuse, stages (2) and (3), are in tof_reuse.cu)
//   splat_kernel     transient histogram H[px, b] = f(y_b) W_b                  (stage (4), Sec. 4.5)
//   pt_kernel        plain gated / transient path tracing (the comparison of Sec. 6)
//   laser_kernel     resolves the collimated laser's spot (Sec. 5 "Light Source")
// The gated image is written by the last stage's kernels (final shading fused into them).
#include "tof_device.cuh"

namespace tof {

// --------------------------------------------------------------------------------------------
// shared helpers
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ float gate_L0(const FrameDev& F, int b) { return F.B > 0 ? F.L0 + b * F.dL : F.L0; }

// The ellipsoidal candidate from vertex x (incident direction wi, prefix length len): places z and
// returns f / (p_tree + p_ell) without the prefix throughput (cf), its tau and the tree's density of
// z (pt).  Out of line: inlined, its BSDF, light and visibility code doubles the path-tree loop and
// thrashes the instruction cache of the divergent warps.  q: its two visibility segments are queued
// there (vis_kernel zeroes the guarded weight when one is occluded) instead of traced in place.
static __device__ __noinline__ bool ell_connect(const Domain& D, const ParamsDev& P, uint32_t px, uint32_t frame, int tree, int d,
                                                const Surf& x, float3 wi, float len, float glo, float ghi, Surf& z, float& cf,
                                                float& tau, float& pt, const VisQ* q = nullptr) {
    const GeomDev& g = D.F->g;
    float pe;
    if (!ell_sample(D, P, px, frame, tree, d, x, len, glo, ghi, z, pe)) return false;
    Mat m = load_mat(g, x.mat), mz = load_mat(g, z.mat);
    float3 wz = dir_to(x.p, z.p);
    float dist = len3(z.p - x.p);
    float fx = bsdf_f(m, x.n, wi, wz);
    if (!(fx > 0.f) || !(dist > 0.f) || mat_class(mz) == C_DELTA) return false;
    float3 wl; float seg;
    float lt = light_term(D, z, wl, seg);
    float fz = lt > 0.f ? bsdf_f(mz, z.n, wz * -1.0f, wl) : 0.f;
    if (!(fz > 0.f)) return false;
    // tau lies in [glo, ghi) by construction (z is on the ellipsoid of the drawn l); it is not tested
    // again, so that rounding cannot decide it
    tau = len + dist + seg - D.o;
    if (!visible_q(q, g, x.p, x.n, z.p, &z.n, P.ray_eps) || !light_visible(D, g, z, P.ray_eps, q)) return false;
    pt = bsdf_pdf(m, x.n, wi, wz) * fabsf(dot3(z.n, wz)) / (dist * dist);
    cf = fx * Gterm(x, z) * fz * lt / (pt + pe);
    return true;
}

// NEE at surface vertex x entered from direction wi: the BSDF value towards the light (0 when the
// light does not reach x) and, through lt / seg, the light factor and the light segment's length.
// Out of line, so that every caller -- the path-tree loop of the single kernels and the start and
// shade kernels of the bounce wavefront -- evaluates it with the same code, and a candidate's
// weight does not depend on which of them drew it.
static __device__ __noinline__ float nee_eval(const Domain& D, const Surf& x, const Mat& m, float3 wi, float& lt, float& seg) {
    float3 wl;
    lt = light_term(D, x, wl, seg);
    return lt > 0.f ? bsdf_f(m, x.n, wi, wl) : 0.f;
}

// One path tree; Sink(k, c, tau, T, strategy) receives each NEE candidate of length k in
// [kmin, depth] whose tau lies in [glo, ghi) and whose light segment is unoccluded (c = f / p, no
// gate; strategy 0).  With kEll every rough vertex x_d (d < depth) also places a vertex z by the
// ellipsoidal connection, a candidate of length d + 1 (strategy 1); it and the tree's NEE
// candidate of the same length (whose last vertex x_{d+1} the tree sampled from x_d) are combined
// by the balance heuristic over the two densities of that vertex (Sec. 5: MIS between the direct
// and the ellipsoidal connection):  c_tree *= p_tree / (p_tree + p_ell),  c_ell = f / (p_tree + p_ell).
// kEll = 1 places the ellipsoidal vertex in place; kEll = 2 (the wavefront) only records every
// vertex (sink.vertex) and the ellipsoidal requests (sink.request) for a later pass.
template <int kEll = 0, class Sink>
__device__ void trace_tree(const Domain& D, const ParamsDev& P, uint32_t px, uint32_t frame, int tree, float glo, float ghi,
                           TreeVerts& T, Sink& sink) {
    const GeomDev& g = D.F->g;
    T.v[1] = D.y1;
    T.cls[1] = mat_class(load_mat(g, D.y1.mat));
    T.pdfA[1] = 1.0f;
    float len = len3(D.x0 - D.y1.p);
    float beta = 1.0f;
    const int kmin = (P.flags & 1u) ? 1 : 2;
    bool ell_prev = false;   // the ellipsoidal connection was available at x_{d-1}
    float len_prev = 0.f;
    for (int d = 1; d <= P.depth; ++d) {
        const Surf& x = T.v[d];
        Mat m = load_mat(g, x.mat);
        float3 wi = dir_to(x.p, d == 1 ? D.x0 : T.v[d - 1].p);
        if constexpr (kEll == 2) sink.vertex(d, T, beta, len);
        if (d >= kmin && mat_class(m) != C_DELTA) {
            float lt, seg;
            const float fs = nee_eval(D, x, m, wi, lt, seg);
            if (fs > 0.f) {
                float tau = len + seg - D.o;
                if (tau >= glo && tau < ghi && light_visible(D, g, x, P.ray_eps)) {
                    float c = beta * fs * lt;
                    if (kEll != 0 && ell_prev) {
                        float pt = T.pdfA[d], pe = ell_pdf(D, T.v[d - 1], len_prev, glo, ghi, x);
                        c *= pt / (pt + pe);
                    }
                    sink(d, c, tau, T, 0);
                }
            }
        }
        if constexpr (kEll != 0) {
            const bool ell_here = d < P.depth && mat_class(m) != C_DELTA && D.light.kind != 0;
            if constexpr (kEll == 2) {
                if (ell_here) sink.request(d);
            } else {
                Surf z;
                float cf, tau, pt;
                if (ell_here && ell_connect(D, P, px, frame, tree, d, x, wi, len, glo, ghi, z, cf, tau, pt)) {
                    T.v[d + 1] = z;
                    T.cls[d + 1] = mat_class(load_mat(g, z.mat));
                    T.pdfA[d + 1] = pt;
                    sink(d + 1, beta * cf, tau, T, 1);
                }
            }
            ell_prev = ell_here;
            len_prev = len;
        }
        if (d == P.depth) break;
        uint4 u = philox(px, frame, ((uint32_t)tree << 8) | (uint32_t)d, P_BSDF, P.seed);
        float3 wo; float pdf, thr; bool delta;
        if (!bsdf_sample(m, x.n, wi, u01(u.x), u01(u.y), wo, pdf, thr, delta)) break;
        if (!trace_from(g, x, wo, P.ray_eps, T.v[d + 1])) break;
        float seg = len3(T.v[d + 1].p - x.p);
        T.cls[d + 1] = mat_class(load_mat(g, T.v[d + 1].mat));
        T.pdfA[d + 1] = delta ? 1.0f : pdf * fabsf(dot3(T.v[d + 1].n, wo)) / (seg * seg);
        len += seg;
        beta *= thr;
    }
}

__device__ __forceinline__ void stats_flush(StatsDev* S, const ShiftStats& s) {
    if (!S) return;
    unsigned long long v[5] = {s.newton_calls, s.newton_iters, s.newton_ok, s.shift_calls, s.shift_ok};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        unsigned long long x = v[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&S->v[i], x);
    }
}

__device__ __forceinline__ void store_tail(const ResDev& R, size_t idx, const Rec& r) {
    *res_at(R, 1, idx) = make_float4(__uint_as_float(r.key_px), __uint_as_float(r.key_frame), __uint_as_float(r.meta), r.pdf_pre);
    if (rec_r(r) >= 2) {
        *res_at(R, 2, idx) = make_float4(r.xprev.x, r.xprev.y, r.xprev.z, __int_as_float(r.p_tri));
        *res_at(R, 3, idx) = make_float4(r.p_b1, r.p_b2, __int_as_float(r.s_tri[0]), r.s_b1[0]);
        int ns = rec_ns(r);
        if (ns >= 1) *res_at(R, 4, idx) = make_float4(r.s_b2[0], __int_as_float(r.s_tri[1]), r.s_b1[1], r.s_b2[1]);
        if (ns >= 3) *res_at(R, 5, idx) = make_float4(__int_as_float(r.s_tri[2]), r.s_b1[2], r.s_b2[2], 0.f);
    }
}

// pixel of this thread in tile (bx, by) of tile_w x (blockDim.x / tile_w) pixels (tile_w a power of
// two); a direct launch passes (blockIdx.x, blockIdx.y), a batched one the tile within its instance
__device__ __forceinline__ void tile_pixel(int tile_w, int bx, int by, int& ix, int& iy) {
    const int sh = __ffs(tile_w) - 1;
    ix = bx * tile_w + (int)(threadIdx.x & (unsigned)(tile_w - 1));
    iy = by * (int)(blockDim.x >> sh) + (int)(threadIdx.x >> sh);
}
__device__ __forceinline__ void tile_pixel(int tile_w, int& ix, int& iy) { tile_pixel(tile_w, blockIdx.x, blockIdx.y, ix, iy); }

// --------------------------------------------------------------------------------------------
// G-buffer: one jittered primary ray per pixel -> (tri, b1, b2, |x1 - x0|)
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void gbuffer_body(const GbufArgs& a, int bx, int by) {
    const FrameDev& F = a.F;
    int ix, iy;
    tile_pixel(a.tile_w, bx, by, ix, iy);
    if (ix >= F.W || iy >= F.H) return;
    int pix = iy * F.W + ix;
    uint4 u = philox((uint32_t)pix, F.frame, 0u, P_JITTER, a.P.seed);
    float3 o, d;
    primary_ray(F, ix, iy, u01(u.x), u01(u.y), o, d);
    int tri; float b1, b2, t;
    float4 out = make_float4(__uint_as_float(kNoHit), 0.f, 0.f, 0.f);
    if (traverse<false>(F.g, o, d, 3.0e38f, tri, b1, b2, t)) {
        Surf s = surf_at(F.g, tri, b1, b2);
        out = make_float4(__int_as_float(tri), b1, b2, len3(s.p - o));
    }
    a.gb[pix] = out;
}
__global__ void __launch_bounds__(128) gbuffer_kernel(const __grid_constant__ GbufArgs a) { gbuffer_body(a, blockIdx.x, blockIdx.y); }
// all instances of a batch: blocks blk0[j] .. blk0[j + 1] - 1 tile instance j
__global__ void __launch_bounds__(128) gbuffer_batch_kernel(const GbufArgs* __restrict__ A, const int* __restrict__ blk0, int n) {
    __shared__ GbufArgs s;
    const int j = batch_job(blk0, n);
    block_copy(&s, &A[j]);
    __syncthreads();
    const int lb = (int)blockIdx.x - __ldg(&blk0[j]);
    const int tx = (s.F.W + s.tile_w - 1) / s.tile_w;
    gbuffer_body(s, lb % tx, lb / tx);
}

// --------------------------------------------------------------------------------------------
// initial candidates (stage (1)): N path trees, each NEE path of length k a candidate with
// w = (1/N) f / p; gated: one reservoir per pixel; transient: each candidate streamed into the
// reservoir of its own bin (Sec. 4.5, "path reuse" deposit of Jarabo 2014)
// --------------------------------------------------------------------------------------------
struct InitSink {
    const ResDev* R;
    const Domain* D;
    const ParamsDev* P;
    uint32_t px, frame;
    int tree, B;
    float t0, w, invN;
    int n;
    int bin[kMaxBinsPerPixel];
    float S[kMaxBinsPerPixel], phat[kMaxBinsPerPixel], tau[kMaxBinsPerPixel], Lsuf[kMaxBinsPerPixel];
    bool overflow;
    __device__ void operator()(int k, float c, float tauv, const TreeVerts& T, int strategy) {
        float wv = invN * c;
        if (!(wv > 0.f)) return;
        int b = 0;
        if (B > 0) {
            float fb = floorf((tauv - t0) / w);
            if (!(fb >= 0.f && fb < (float)B)) return;
            b = (int)fb;
        }
        int e = 0;
        while (e < n && bin[e] != b) ++e;
        if (e == n) {
            if (n == kMaxBinsPerPixel) { overflow = true; return; }
            bin[n] = b; S[n] = 0.f; phat[n] = 0.f; ++n;
        }
        uint4 u = philox(px, frame, ((uint32_t)tree << 8) | (uint32_t)k, strategy ? P_ELL_RIS : P_RIS, P->seed);
        S[e] += wv;
        if (u01(u.x) * S[e] < wv) {
            Rec r;
            build_rec(*D, T, k, tree, px, frame, tauv, *P, r);
            size_t idx = (size_t)px * (B > 0 ? B : 1) + b;
            store_tail(*R, idx, r);
            phat[e] = r.phat; tau[e] = tauv; Lsuf[e] = r.Lsuf;
        }
    }
};

// gated sink: one running reservoir in registers (the transient sink's per-bin tables live in
// local memory, which every candidate of a gated pixel paid for)
struct GatedSink {
    const ResDev* R;
    const Domain* D;
    const ParamsDev* P;
    uint32_t px, frame;
    int tree;
    float invN;
    float S, phat, tau, Lsuf;
    __device__ void operator()(int k, float c, float tauv, const TreeVerts& T, int strategy) {
        float wv = invN * c;
        if (!(wv > 0.f)) return;
        uint4 u = philox(px, frame, ((uint32_t)tree << 8) | (uint32_t)k, strategy ? P_ELL_RIS : P_RIS, P->seed);
        S += wv;
        if (u01(u.x) * S < wv) {
            Rec r;
            build_rec(*D, T, k, tree, px, frame, tauv, *P, r);
            store_tail(*R, (size_t)px, r);
            phat = r.phat; tau = tauv; Lsuf = r.Lsuf;
        }
    }
};

// gated views: the same trees, candidates, order and uniforms as initial_kernel, into GatedSink
template <bool kEll>
__device__ __forceinline__ void initial_gated_body(const InitArgs& a, int bx, int by) {
    const FrameDev& F = a.F;
    int ix, iy;
    tile_pixel(a.tile_w, bx, by, ix, iy);
    if (ix >= F.W || iy >= F.H) return;
    const int pix = iy * F.W + ix;
    const ParamsDev& P = a.P;
    a.dst.M[pix] = (float)P.n_cand;
    float4 gb = F.gb[pix];
    uint32_t tri = __float_as_uint(gb.x);
    Domain D = make_domain_hit(&F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, F.L0, F.dL);
    if (!D.valid) {
        a.dst.occ[pix] = 0u;
        if (a.out) a.out[pix] = 0.f;
        return;
    }
    GatedSink sink;
    sink.R = &a.dst; sink.D = &D; sink.P = &P; sink.px = (uint32_t)pix; sink.frame = F.frame;
    sink.invN = 1.0f / (float)P.n_cand;
    sink.S = 0.f; sink.phat = 0.f; sink.tau = 0.f; sink.Lsuf = 0.f;
    TreeVerts T;
    for (int t = 0; t < P.n_cand; ++t) {
        sink.tree = t;
        trace_tree<kEll ? 1 : 0>(D, P, (uint32_t)pix, F.frame, t, F.L0, F.L0 + F.dL, T, sink);
    }
    float outv = 0.f;
    uint32_t occ = 0u;
    if (sink.phat > 0.f) {
        const float W = sink.S / sink.phat;
        *res_at(a.dst, 0, (size_t)pix) = make_float4(W, sink.phat, sink.tau, sink.Lsuf);
        occ = 1u;
        outv = sink.phat * W;
    }
    a.dst.occ[pix] = occ;
    if (a.out) a.out[pix] = outv;
}
template <bool kEll>
__global__ void __launch_bounds__(128, kEll ? 4 : 6) initial_gated_kernel(const __grid_constant__ InitArgs a) {
    initial_gated_body<kEll>(a, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(128, 6) initial_gated_batch_kernel(const InitArgs* __restrict__ A, const int* __restrict__ blk0,
                                                                     int n) {
    __shared__ InitArgs s;
    const int j = batch_job(blk0, n);
    block_copy(&s, &A[j]);
    __syncthreads();
    if (s.wave) return;   // launched as the bounce wavefront after this kernel (the whole block)
    const int lb = (int)blockIdx.x - __ldg(&blk0[j]);
    const int tx = (s.F.W + s.tile_w - 1) / s.tile_w;
    initial_gated_body<false>(s, lb % tx, lb / tx);
}

// 6 resident blocks per SM (80 registers): 1.08 against 1.11 ms at 5 blocks (96 registers) on the
// 512 x 512 dynamic workload; 8 blocks (64 registers, more spills) were slower.  kEll: with the
// ellipsoidal connection (TOF_FLAG_ELLIPSOID), compiled apart so the default keeps its registers.
template <bool kEll>
__global__ void __launch_bounds__(128, kEll ? 4 : 6) initial_kernel(const __grid_constant__ InitArgs a, unsigned* err) {
    const FrameDev& F = a.F;
    int ix, iy;
    tile_pixel(a.tile_w, ix, iy);
    if (ix >= F.W || iy >= F.H) return;
    const int pix = iy * F.W + ix;
    const ParamsDev& P = a.P;
    const int Bn = F.B > 0 ? F.B : 1;
    uint32_t* occ = a.dst.occ + (size_t)pix * a.dst.words;
    for (int w = 0; w < a.dst.words; ++w) occ[w] = 0u;
    a.dst.M[pix] = (float)P.n_cand;
    float4 gb = F.gb[pix];
    uint32_t tri = __float_as_uint(gb.x);
    Domain D = make_domain_hit(&F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, F.L0, F.dL);
    if (!D.valid) {
        if (a.out) a.out[pix] = 0.f;
        return;
    }
    InitSink sink;
    sink.R = &a.dst; sink.D = &D; sink.P = &P; sink.px = (uint32_t)pix; sink.frame = F.frame;
    sink.B = F.B; sink.t0 = F.L0; sink.w = F.dL; sink.invN = 1.0f / (float)P.n_cand; sink.n = 0; sink.overflow = false;
    float glo = F.L0, ghi = F.B > 0 ? F.L0 + F.B * F.dL : F.L0 + F.dL;
    TreeVerts T;
    for (int t = 0; t < P.n_cand; ++t) {
        sink.tree = t;
        trace_tree<kEll ? 1 : 0>(D, P, (uint32_t)pix, F.frame, t, glo, ghi, T, sink);
    }
    if (sink.overflow && err) atomicOr(err, kErrBinOverflow);
    float outv = 0.f;
    for (int e = 0; e < sink.n; ++e) {
        if (!(sink.phat[e] > 0.f)) continue;
        float W = sink.S[e] / sink.phat[e];
        size_t idx = (size_t)pix * Bn + sink.bin[e];
        *res_at(a.dst, 0, idx) = make_float4(W, sink.phat[e], sink.tau[e], sink.Lsuf[e]);
        occ[sink.bin[e] >> 5] |= 1u << (sink.bin[e] & 31);
        outv = sink.phat[e] * W;
    }
    if (a.out) a.out[pix] = outv;
}

// --------------------------------------------------------------------------------------------
// gated initial candidates with the ellipsoidal connection as a wavefront (EllWaveDev): the same
// candidates, weights, uniforms and order as initial_kernel<true>, so the same reservoirs, but the
// ellipsoidal vertices are placed in one coherent pass instead of inside the divergent path-tree
// loop (whose mixed tree / walk / traversal code stalled on instruction fetch):
//   ell_trees_kernel   the path trees: every vertex, every NEE candidate (with its MIS weight),
//                      every ellipsoidal request
//   ell_place_kernel   one thread per request: the walk, the ellipse clip, the candidate's weight;
//                      its two visibility segments queued for vis_kernel (which zeroes the weight of
//                      an occluded one)
//   tree_select_kernel<true>  the streaming RIS per pixel in the trees' order (tree-major; at vertex d the
//                      NEE candidate, then the ellipsoidal one), then the winner's record alone
// --------------------------------------------------------------------------------------------
struct RecordSink {
    const EllWaveDev* w;
    size_t base;   // slot of (pixel, tree, vertex 1)
    __device__ void operator()(int k, float c, float tauv, const TreeVerts& T, int strategy) {
        (void)T; (void)strategy;   // only the tree's own NEE candidates arrive here
        w->acand[base + k - 1] = make_float2(c, tauv);
    }
    __device__ void vertex(int d, const TreeVerts& T, float beta, float len) {
        const Surf& v = T.v[d];
        w->vtx[base + d - 1] = make_float4(__int_as_float(v.tri), v.b1, v.b2, T.pdfA[d]);
        w->vtx2[base + d - 1] = make_float2(beta, len);
    }
    __device__ void request(int d) {
        const uint32_t i = reserve_one(&w->counters[0]);
        if (i < w->req_cap) w->req[i] = (uint32_t)(base + d - 1);
    }
};

__global__ void __launch_bounds__(128, 6) ell_trees_kernel(const __grid_constant__ InitArgs a, const EllWaveDev w) {
    const FrameDev& F = a.F;
    int ix, iy;
    tile_pixel(a.tile_w, ix, iy);
    if (ix >= F.W || iy >= F.H) return;
    const int pix = iy * F.W + ix;
    const ParamsDev& P = a.P;
    float4 gb = F.gb[pix];
    uint32_t tri = __float_as_uint(gb.x);
    Domain D = make_domain_hit(&F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, F.L0, F.dL);
    if (!D.valid) return;
    RecordSink sink;
    sink.w = &w;
    TreeVerts T;
    for (int t = 0; t < P.n_cand; ++t) {
        sink.base = ((size_t)pix * w.nc + t) * w.depth;
        for (int d = 0; d < w.depth; ++d) {
            w.acand[sink.base + d] = make_float2(0.f, 0.f);
            w.bw[sink.base + d] = 0.f;
        }
        trace_tree<2>(D, P, (uint32_t)pix, F.frame, t, F.L0, F.L0 + F.dL, T, sink);
    }
}

// 6 resident blocks per SM: 1.96 ms for the ellipsoidal stage against 2.04 at the 4 its 117
// registers allow (the walk's dependent node loads wait on L2; 8 blocks: 1.97)
__global__ void __launch_bounds__(128, 6) ell_place_kernel(const __grid_constant__ InitArgs a, const EllWaveDev w) {
    const FrameDev& F = a.F;
    const ParamsDev& P = a.P;
    const uint32_t n = min(w.counters[0], w.req_cap);
    const uint32_t per = (uint32_t)(w.nc * w.depth);
    VisQ q;
    q.rays = w.rays; q.counter = &w.counters[2]; q.cap = w.ray_cap;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t slot = w.req[i];
        const int pix = (int)(slot / per), t = (int)((slot / (uint32_t)w.depth) % (uint32_t)w.nc), d = (int)(slot % (uint32_t)w.depth) + 1;
        float4 gb = F.gb[pix];
        Domain D = make_domain_hit(&F, true, (int)__float_as_uint(gb.x), gb.y, gb.z, gb.w, F.L0, F.dL);
        float4 v = w.vtx[slot];
        Surf x = surf_at(F.g, __float_as_int(v.x), v.y, v.z);
        float3 prev = D.x0;
        if (d > 1) {
            float4 u = w.vtx[slot - 1];
            prev = surf_at(F.g, __float_as_int(u.x), u.y, u.z).p;
        }
        const float2 bl = w.vtx2[slot];
        q.target = slot;
        Surf z;
        float cf, tau, pt;
        if (ell_connect(D, P, (uint32_t)pix, F.frame, t, d, x, dir_to(x.p, prev), bl.y, F.L0, F.L0 + F.dL, z, cf, tau, pt, &q)) {
            w.bw[slot] = bl.x * cf;
            w.bz[slot] = make_float4(__int_as_float(z.tri), z.b1, z.b2, tau);
            w.bpt[slot] = pt;
        } else {
            w.bw[slot] = 0.f;
        }
    }
}

// kEll = false: the tree wavefront (TreeWaveDev), whose trees are the only candidates
template <bool kEll, class Wave>
__global__ void __launch_bounds__(128) tree_select_kernel(const __grid_constant__ InitArgs a, const Wave w) {
    const FrameDev& F = a.F;
    int ix, iy;
    tile_pixel(a.tile_w, ix, iy);
    if (ix >= F.W || iy >= F.H) return;
    const int pix = iy * F.W + ix;
    const ParamsDev& P = a.P;
    a.dst.occ[pix] = 0u;
    a.dst.M[pix] = (float)P.n_cand;
    float4 gb = F.gb[pix];
    uint32_t tri = __float_as_uint(gb.x);
    Domain D = make_domain_hit(&F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, F.L0, F.dL);
    float outv = 0.f;
    if (D.valid) {
        const int kmin = (P.flags & 1u) ? 1 : 2;
        const float invN = 1.0f / (float)P.n_cand;
        float S = 0.f, sel_tau = 0.f;
        int sel_t = -1, sel_k = 0, sel_s = 0;
        for (int t = 0; t < P.n_cand; ++t) {
            const size_t base = ((size_t)pix * w.nc + t) * w.depth;
            for (int d = 1; d <= P.depth; ++d) {
                if (d >= kmin) {
                    const float2 ac = w.acand[base + d - 1];
                    const float wv = invN * ac.x;
                    if (wv > 0.f) {
                        uint4 u = philox((uint32_t)pix, F.frame, ((uint32_t)t << 8) | (uint32_t)d, P_RIS, P.seed);
                        S += wv;
                        if (u01(u.x) * S < wv) { sel_t = t; sel_k = d; sel_s = 0; sel_tau = ac.y; }
                    }
                }
                if constexpr (kEll) if (d < P.depth) {
                    const float wv = invN * w.bw[base + d - 1];
                    if (wv > 0.f) {
                        uint4 u = philox((uint32_t)pix, F.frame, ((uint32_t)t << 8) | (uint32_t)(d + 1), P_ELL_RIS, P.seed);
                        S += wv;
                        if (u01(u.x) * S < wv) { sel_t = t; sel_k = d + 1; sel_s = 1; sel_tau = w.bz[base + d - 1].w; }
                    }
                }
            }
        }
        if (sel_t >= 0) {
            // the winner's path as the tree held it when the candidate streamed by
            const GeomDev& g = F.g;
            const size_t base = ((size_t)pix * w.nc + sel_t) * w.depth;
            TreeVerts T;
            T.v[1] = D.y1;
            T.cls[1] = mat_class(load_mat(g, D.y1.mat));
            T.pdfA[1] = 1.0f;
            const int ntree = sel_s ? sel_k - 1 : sel_k;   // vertices from the tree itself
            for (int j = 2; j <= ntree; ++j) {
                float4 v = w.vtx[base + j - 1];
                T.v[j] = surf_at(g, __float_as_int(v.x), v.y, v.z);
                T.cls[j] = mat_class(load_mat(g, T.v[j].mat));
                T.pdfA[j] = v.w;
            }
            if constexpr (kEll) if (sel_s) {
                float4 zb = w.bz[base + sel_k - 2];
                T.v[sel_k] = surf_at(g, __float_as_int(zb.x), zb.y, zb.z);
                T.cls[sel_k] = mat_class(load_mat(g, T.v[sel_k].mat));
                T.pdfA[sel_k] = w.bpt[base + sel_k - 2];
            }
            Rec r;
            build_rec(D, T, sel_k, sel_t, (uint32_t)pix, F.frame, sel_tau, P, r);
            if (r.phat > 0.f) {
                const float W = S / r.phat;
                store_tail(a.dst, (size_t)pix, r);
                *res_at(a.dst, 0, (size_t)pix) = make_float4(W, r.phat, sel_tau, r.Lsuf);
                a.dst.occ[pix] = 1u;
                outv = r.phat * W;
            }
        }
    }
    if (a.out) a.out[pix] = outv;
}

// --------------------------------------------------------------------------------------------
// gated initial candidates as a bounce wavefront (TreeWaveDev): the same trees, candidates,
// uniforms and order as initial_gated_kernel<false>, so the same reservoirs, with every lane of a
// warp on the same step.  In the single kernel a warp's 32 path trees diverge in depth, in
// traversal length and in whether a candidate needs a light segment, and most lanes idle:
//   tw_start_kernel   one thread per path: vertex 1 (the G-buffer hit), its NEE candidate, the
//                     first bounce
//   tw_hit_kernel     per round, the closest hits of the round's bounce rays (persistent, each lane
//                     refilled with the next ray between rounds of kHitSteps node visits)
//   tw_shade_kernel   per round, one thread per hit: the vertex record, the NEE candidate (its light
//                     segment queued for vis_kernel) and the next bounce
//   vis_kernel        the light segments; an occluded one zeroes its candidate's weight
//   tree_select_kernel<false>  the streaming RIS per pixel in the trees' order, then the winner's record
// --------------------------------------------------------------------------------------------
// vertex d of path p (tree t of pixel pix) at x, entered from direction wi with prefix throughput
// beta and length len (area density pdfA, prefix length len_prev at vertex d - 1): its NEE candidate
// and, below the depth, the bounce towards vertex d + 1.  kEll (the ellipsoidal connection, the tree
// part of its wavefront; w.vtx / w.acand are then the EllWaveDev tables): the vertex's throughput
// and length are recorded, the NEE candidate takes the balance-heuristic factor against the
// ellipsoidal vertex placed from x_{d-1}, and a vertex that can place one is queued as a request --
// the steps of trace_tree<2> with its recording sink.
template <bool kEll>
__device__ __forceinline__ void tw_vertex(const InitArgs& a, const TreeWaveDev& w, const EllWaveDev& e, const Domain& D, uint32_t p,
                                          int pix, int t, int d, const Surf& x, float3 wi, float beta, float len, float pdfA,
                                          float len_prev, VisQ& q) {
    const FrameDev& F = a.F;
    const ParamsDev& P = a.P;
    const GeomDev& g = F.g;
    const size_t slot = (size_t)p * (size_t)w.depth + (size_t)(d - 1);
    Mat m = load_mat(g, x.mat);
    if constexpr (kEll) e.vtx2[slot] = make_float2(beta, len);
    const int kmin = (P.flags & 1u) ? 1 : 2;
    if (d >= kmin && mat_class(m) != C_DELTA) {
        float lt, seg;
        const float fs = nee_eval(D, x, m, wi, lt, seg);
        if (fs > 0.f) {
            float tau = len + seg - D.o;
            if (tau >= F.L0 && tau < F.L0 + F.dL) {
                float c = beta * fs * lt;
                if constexpr (kEll) {
                    if (d > 1) {
                        // the ellipsoidal connection was available at x_{d-1} when that vertex was rough
                        const float4 pv = w.vtx[slot - 1];
                        const Surf xp = surf_at(g, __float_as_int(pv.x), pv.y, pv.z);
                        if (mat_class(load_mat(g, xp.mat)) != C_DELTA && D.light.kind != 0) {
                            const float pe = ell_pdf(D, xp, len_prev, F.L0, F.L0 + F.dL, x);
                            c *= pdfA / (pdfA + pe);
                        }
                    }
                }
                q.target = (uint32_t)(2 * slot);   // the float index of the candidate's weight
                if (light_visible(D, g, x, P.ray_eps, &q)) w.acand[slot] = make_float2(c, tau);
            }
        }
    }
    if constexpr (kEll) {
        if (d < P.depth && mat_class(m) != C_DELTA && D.light.kind != 0) {
            const uint32_t i = reserve_one(&e.counters[0]);
            if (i < e.req_cap) e.req[i] = (uint32_t)slot;
        }
    }
    if (d >= P.depth) return;
    uint4 u = philox((uint32_t)pix, F.frame, ((uint32_t)t << 8) | (uint32_t)d, P_BSDF, P.seed);
    float3 wo; float pdf, thr; bool delta;
    if (!bsdf_sample(m, x.n, wi, u01(u.x), u01(u.y), wo, pdf, thr, delta)) return;
    const float3 o = offset_point(x.p, x.n, wo, P.ray_eps);
    // each path sends at most one ray per round, so a round's rays never exceed the paths
    const uint32_t i = reserve_one(&w.counters[d + 1]);
    if (i >= w.path_cap) return;
    float4* r = w.rays[(d + 1) & 1];
    r[2 * (size_t)i] = make_float4(o.x, o.y, o.z, 3.0e38f);
    r[2 * (size_t)i + 1] = make_float4(wo.x, wo.y, wo.z, __uint_as_float(p));
    w.ps0[p] = make_float4(beta * thr, len, delta ? -1.0f : pdf, 0.f);
    w.ps1[p] = make_float4(x.p.x, x.p.y, x.p.z, 0.f);
}

template <bool kEll>
__global__ void __launch_bounds__(128) tw_start_kernel(const __grid_constant__ InitArgs a, const TreeWaveDev w, const EllWaveDev e) {
    const FrameDev& F = a.F;
    const uint32_t npath = (uint32_t)F.W * (uint32_t)F.H * (uint32_t)w.nc;
    VisQ q;
    q.rays = w.srays; q.counter = &w.counters[14]; q.cap = w.sray_cap; q.target = 0u;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < npath; p += gridDim.x * blockDim.x) {
        const int pix = (int)(p / (uint32_t)w.nc), t = (int)(p % (uint32_t)w.nc);
        float2* ac = w.acand + (size_t)p * w.depth;
        for (int d = 0; d < w.depth; ++d) ac[d] = make_float2(0.f, 0.f);
        if constexpr (kEll)
            for (int d = 0; d < w.depth; ++d) e.bw[(size_t)p * w.depth + d] = 0.f;
        float4 gb = F.gb[pix];
        uint32_t tri = __float_as_uint(gb.x);
        if (tri == kNoHit) continue;
        Domain D = make_domain_hit(&F, true, (int)tri, gb.y, gb.z, gb.w, F.L0, F.dL);
        if constexpr (kEll) w.vtx[(size_t)p * w.depth] = make_float4(__int_as_float(D.y1.tri), D.y1.b1, D.y1.b2, 1.0f);
        tw_vertex<kEll>(a, w, e, D, p, pix, t, 1, D.y1, dir_to(D.y1.p, D.x0), 1.0f, len3(D.x0 - D.y1.p), 1.0f, 0.f, q);
    }
}

// closest hits of the rays of one round: the loop of traverse<false> with the vis_kernel's lane
// refill; hits[i] = (tri, b1, b2, t) of ray i, or kNoHit
constexpr int kHitSteps = 32;
__global__ void __launch_bounds__(128, 8) tw_hit_kernel(const GeomDev gref, const float4* __restrict__ rays, const uint32_t* counter,
                                                     uint32_t cap, uint32_t* fetch, float4* __restrict__ hits) {
    GeomDev g;
    g.nodes = gref.nodes; g.leaf = gref.leaf; g.nt = gref.nt; g.err = gref.err;
    const uint32_t n = min(*counter, cap);
    const int lane = threadIdx.x & 31;
    unsigned fault = 0u;
    bool has = false, done = false, found = false;
    float3 o = f3(0.f, 0.f, 0.f), d = o, id = o, ood = o;
    float tmax = 0.f, best = 0.f, bb1 = 0.f, bb2 = 0.f;
    int btri = 0;
    uint32_t cur = 0;
    int node = 0, sp = 0, budget = 0;
    int stack[kStack];
    while (true) {
        const bool need = !has && !done;
        const uint32_t want = __ballot_sync(0xFFFFFFFFu, need);
        if (want) {
            const int leader = __ffs(want) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(fetch, (uint32_t)__popc(want));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (need) {
                const uint32_t i = base + (uint32_t)__popc(want & ((1u << lane) - 1u));
                if (i < n) {
                    float4 ra = rays[2 * (size_t)i], rb = rays[2 * (size_t)i + 1];
                    o = f3(ra.x, ra.y, ra.z); d = f3(rb.x, rb.y, rb.z); tmax = ra.w;
                    id = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
                    ood = f3(o.x * id.x, o.y * id.y, o.z * id.z);
                    cur = i; found = false; best = tmax;
                    node = 0; sp = 0; budget = g.nt + 64;
                    has = true;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(0xFFFFFFFFu, done)) break;
        bool fin = false;
        for (int step = 0; step < kHitSteps && has; ++step) {
            if (g.nt <= 1) {
                float t, u, v; int orig;
                if (g.nt == 1 && tri_test(g.leaf, 0, o, d, best, t, u, v, orig) && t < tmax) {
                    found = true; best = t; btri = orig; bb1 = u; bb2 = v;
                }
                has = false; fin = true;
                break;
            }
            if (--budget < 0) {
                fault |= kErrVisitBudget;
                has = false; fin = true;
                break;
            }
            const float4* N = g.nodes + 4 * node;
            float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
            float a0 = n0.x * id.x - ood.x, a1 = n0.y * id.x - ood.x;
            float b0 = n0.z * id.y - ood.y, c1y = n0.w * id.y - ood.y;
            float c0 = n2.x * id.z - ood.z, c1 = n2.y * id.z - ood.z;
            float lo0 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, c1y)), fmaxf(fminf(c0, c1), 0.f));
            float hi0 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, c1y)), fminf(fmaxf(c0, c1), best));
            float d0 = n1.x * id.x - ood.x, d1 = n1.y * id.x - ood.x;
            float e0 = n1.z * id.y - ood.y, e1 = n1.w * id.y - ood.y;
            float f0 = n2.z * id.z - ood.z, f1 = n2.w * id.z - ood.z;
            float lo1 = fmaxf(fmaxf(fminf(d0, d1), fminf(e0, e1)), fmaxf(fminf(f0, f1), 0.f));
            float hi1 = fminf(fminf(fmaxf(d0, d1), fmaxf(e0, e1)), fminf(fmaxf(f0, f1), best));
            bool h0 = lo0 <= hi0, h1 = lo1 <= hi1;
            int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
            if (h0 && ch0 < 0) {
                float t, u, v; int orig;
                if (tri_test(g.leaf, ~ch0, o, d, best, t, u, v, orig) && (found || t < tmax) && closer(found, t, orig, best, btri)) {
                    best = t; btri = orig; bb1 = u; bb2 = v; found = true;
                }
                h0 = false;
            }
            if (h1 && ch1 < 0) {
                float t, u, v; int orig;
                if (tri_test(g.leaf, ~ch1, o, d, best, t, u, v, orig) && (found || t < tmax) && closer(found, t, orig, best, btri)) {
                    best = t; btri = orig; bb1 = u; bb2 = v; found = true;
                }
                h1 = false;
            }
            if (h0 && h1) {
                int nearc = lo0 <= lo1 ? ch0 : ch1, farc = lo0 <= lo1 ? ch1 : ch0;
                if (sp < kStack) stack[sp++] = farc;
                else fault |= kErrStackOverflow;   // the far subtree is skipped: reported after the loop
                node = nearc;
            } else if (h0) {
                node = ch0;
            } else if (h1) {
                node = ch1;
            } else {
                if (sp == 0) { has = false; fin = true; break; }
                node = stack[--sp];
            }
        }
        if (fin) hits[cur] = found ? make_float4(__int_as_float(btri), bb1, bb2, best) : make_float4(__uint_as_float(kNoHit), 0.f, 0.f, 0.f);
    }
    if (fault && g.err) atomicOr(g.err, fault);
}

// the hits of the round towards vertex d: one thread per ray
template <bool kEll>
__global__ void __launch_bounds__(128) tw_shade_kernel(const __grid_constant__ InitArgs a, const TreeWaveDev w, const EllWaveDev e,
                                                       int d) {
    const FrameDev& F = a.F;
    const uint32_t n = min(w.counters[d], w.path_cap);
    const float4* __restrict__ rays = w.rays[d & 1];
    VisQ q;
    q.rays = w.srays; q.counter = &w.counters[14]; q.cap = w.sray_cap; q.target = 0u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 h = w.hits[i];
        if (__float_as_uint(h.x) == kNoHit) continue;
        const float4 rd = rays[2 * (size_t)i + 1];
        const uint32_t p = __float_as_uint(rd.w);
        const int pix = (int)(p / (uint32_t)w.nc), t = (int)(p % (uint32_t)w.nc);
        const float4 s0 = w.ps0[p], s1 = w.ps1[p];
        const Surf x = surf_at(F.g, __float_as_int(h.x), h.y, h.z);
        const float3 prev = f3(s1.x, s1.y, s1.z), wo = f3(rd.x, rd.y, rd.z);
        const float seg = len3(x.p - prev);
        const float pdfA = s0.z < 0.f ? 1.0f : s0.z * fabsf(dot3(x.n, wo)) / (seg * seg);
        w.vtx[(size_t)p * w.depth + (size_t)(d - 1)] = make_float4(h.x, h.y, h.z, pdfA);
        const float4 gb = F.gb[pix];
        Domain D = make_domain_hit(&F, true, (int)__float_as_uint(gb.x), gb.y, gb.z, gb.w, F.L0, F.dL);
        tw_vertex<kEll>(a, w, e, D, p, pix, t, d, x, dir_to(x.p, prev), s0.x, s0.y + seg, pdfA, s0.y, q);
    }
}

// --------------------------------------------------------------------------------------------
// initial candidates with the path-length shrink mapping (Sec. 4.4), gated views.  Trees from
// N_A = shrink_fine on draw in the gate widened K times about its centre c and keep their RIS
// winner x_B (W_B); the winner alone is shrunk into the gate, y_B = T(x_B), tau' = c + (tau - c)/K,
// |dT/dx| = det(dxi'/dxi)/K.  Trees below N_A draw in the gate itself (winner y_A, W_A).  The two
// are combined by the generalized balance heuristic with confidences N_A and N_B = n_cand - N_A:
//   m_A = N_A p(y_A) / (N_A p(y_A) + N_B p_wide(T^-1(y_A)) |dT^-1/dy|)
//   m_B = N_B p_wide(x_B)/|dT/dx| / (N_A p(y_B) + N_B p_wide(x_B)/|dT/dx|)
// With N_A = 0 (every tree widened) W = W_B |dT/dx|.
// --------------------------------------------------------------------------------------------
struct ShrinkSink {
    const Domain* D;
    const ParamsDev* P;
    uint32_t px, frame;
    int tree;
    float invN, S;
    bool has;
    Rec rec;
    __device__ void operator()(int k, float c, float tauv, const TreeVerts& T, int strategy) {
        (void)strategy;
        float wv = invN * c;
        if (!(wv > 0.f)) return;
        uint4 u = philox(px, frame, ((uint32_t)tree << 8) | (uint32_t)k, P_RIS, P->seed);
        S += wv;
        if (u01(u.x) * S < wv) {
            build_rec(*D, T, k, tree, px, frame, tauv, *P, rec);
            has = true;
        }
    }
};

template <bool kWalk>
__global__ void __launch_bounds__(128) initial_shrink_kernel(const __grid_constant__ InitArgs a) {
    const FrameDev& F = a.F;
    int ix, iy;
    tile_pixel(a.tile_w, ix, iy);
    if (ix >= F.W || iy >= F.H) return;
    const int pix = iy * F.W + ix;
    const ParamsDev& P = a.P;
    a.dst.occ[pix] = 0u;
    a.dst.M[pix] = (float)P.n_cand;
    float4 gb = F.gb[pix];
    uint32_t tri = __float_as_uint(gb.x);
    Domain D = make_domain_hit(&F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, F.L0, F.dL);
    if (!D.valid) {
        if (a.out) a.out[pix] = 0.f;
        return;
    }
    const int NA = P.shrink_fine, NB = P.n_cand - P.shrink_fine;
    const float K = P.shrink_k, c = F.L0 + 0.5f * F.dL, half = 0.5f * K * F.dL;
    ShrinkSink sa, sb;
    sa.D = sb.D = &D; sa.P = sb.P = &P; sa.px = sb.px = (uint32_t)pix; sa.frame = sb.frame = F.frame;
    sa.invN = NA > 0 ? 1.0f / (float)NA : 0.f; sb.invN = 1.0f / (float)NB;
    sa.S = sb.S = 0.f; sa.has = sb.has = false;
    TreeVerts T;
    for (int t = 0; t < P.n_cand; ++t) {
        if (t < NA) { sa.tree = t; trace_tree(D, P, (uint32_t)pix, F.frame, t, F.L0, F.L0 + F.dL, T, sa); }
        else { sb.tree = t; trace_tree(D, P, (uint32_t)pix, F.frame, t, c - half, c + half, T, sb); }
    }
    const float Wa = (sa.has && sa.rec.phat > 0.f) ? sa.S / sa.rec.phat : 0.f;
    const float Wb = (sb.has && sb.rec.phat > 0.f) ? sb.S / sb.rec.phat : 0.f;
    GateMap to_gate, to_wide;
    to_gate.scale = 1.0f / K; to_gate.centre = c; to_gate.lo = F.L0; to_gate.hi = F.L0 + F.dL;
    to_wide.scale = K; to_wide.centre = c; to_wide.lo = c - half; to_wide.hi = c + half;
    Rec yb;
    float pyb = 0.f, Jb = 0.f;
    const bool okb = Wb > 0.f && shift_rec<true, kWalk>(sb.rec, D, D, P, true, yb, pyb, Jb, nullptr, nullptr, &to_gate);
    float w[2] = {0.f, 0.f};
    if (NA == 0) {
        if (okb) w[1] = pyb * Wb * Jb;
    } else {
        if (Wa > 0.f) {
            Rec tmp;
            float pe = 0.f, Je = 0.f;
            float pba = shift_rec<false, kWalk>(sa.rec, D, D, P, true, tmp, pe, Je, nullptr, nullptr, &to_wide) ? pe * Je : 0.f;
            float ma = NA * sa.rec.phat / (NA * sa.rec.phat + NB * pba);
            w[0] = ma * sa.rec.phat * Wa;
        }
        if (okb) {
            float nb = NB * sb.rec.phat / Jb;
            float mb = nb / (NA * pyb + nb);
            w[1] = mb * pyb * Wb * Jb;
        }
    }
    float S = 0.f;
    int sel = -1;
    for (int q = 0; q < 2; ++q) {
        if (!(w[q] > 0.f) || !isfinite(w[q])) continue;
        uint4 u = philox((uint32_t)pix, F.frame, (0xFFu << 8) | (uint32_t)q, P_MERGE, P.seed);
        S += w[q];
        if (u01(u.x) * S < w[q]) sel = q;
    }
    float outv = 0.f;
    if (sel >= 0) {
        Rec& r = sel == 0 ? sa.rec : yb;
        const float ph = sel == 0 ? sa.rec.phat : pyb;
        r.W = S / ph;
        r.phat = ph;
        rec_store(a.dst, (size_t)pix, r);
        a.dst.occ[pix] = 1u;
        outv = ph * r.W;
    }
    if (a.out) a.out[pix] = outv;
}

// --------------------------------------------------------------------------------------------
// transient splat (stage (4)): H[px, b] = f(y_b) W_b for occupied bins, 0 elsewhere; one warp
// per pixel so that the histogram row is written with coalesced stores
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) splat_kernel(const __grid_constant__ SplatArgs a) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= a.npix) return;
    const int pix = warp, B = a.B;
    const uint32_t* occ = a.src.occ + (size_t)pix * a.src.words;
    float* row = a.out + (size_t)pix * B;
    for (int w = 0; w < a.src.words; ++w) {
        uint32_t m = occ[w];
        int b = (w << 5) + lane;
        if (b >= B) break;
        float v = 0.f;
        if ((m >> lane) & 1u) { float4 p = *res_at(a.src, 0, (size_t)pix * B + b); v = p.y * p.x; }
        row[b] = v;
    }
}

// --------------------------------------------------------------------------------------------
// plain path tracing (comparison method of Sec. 6)
// --------------------------------------------------------------------------------------------
struct PtSink {
    float* row;
    int B;
    float t0, w, scale;
    __device__ void operator()(int k, float c, float tau, const TreeVerts& T, int strategy) {
        (void)k; (void)T; (void)strategy;
        if (B > 0) {
            float fb = floorf((tau - t0) / w);
            if (!(fb >= 0.f && fb < (float)B)) return;
            row[(int)fb] += scale * c;
        } else {
            row[0] += scale * c;
        }
    }
};

__global__ void __launch_bounds__(128) pt_kernel(const __grid_constant__ PtArgs a) {
    const FrameDev& F = a.F;
    int ix = blockIdx.x * 16 + (threadIdx.x & 15), iy = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (ix >= F.W || iy >= F.H) return;
    const int pix = iy * F.W + ix;
    const int Bn = F.B > 0 ? F.B : 1;
    float* row = a.out + (size_t)pix * Bn;
    float acc = 0.f;
    for (int b = 0; b < Bn; ++b) row[b] = 0.f;
    PtSink sink;
    sink.B = F.B; sink.t0 = F.L0; sink.w = F.dL; sink.scale = 1.0f / (float)a.spp;
    sink.row = F.B > 0 ? row : &acc;
    float glo = F.L0, ghi = F.B > 0 ? F.L0 + F.B * F.dL : F.L0 + F.dL;
    TreeVerts T;
    for (int s = 0; s < a.spp; ++s) {
        uint4 u = philox((uint32_t)pix, F.frame, (uint32_t)s, P_JITTER, a.P.seed);
        float3 o, d;
        primary_ray(F, ix, iy, u01(u.x), u01(u.y), o, d);
        int tri; float b1, b2, t;
        if (!traverse<false>(F.g, o, d, 3.0e38f, tri, b1, b2, t)) continue;
        Surf s1 = surf_at(F.g, tri, b1, b2);
        Domain D = make_domain_hit(&F, true, tri, b1, b2, len3(s1.p - o), F.L0, F.dL);
        D.x0 = o;
        trace_tree(D, a.P, (uint32_t)pix, F.frame, s, glo, ghi, T, sink);
    }
    if (F.B == 0) row[0] = acc;
}

// --------------------------------------------------------------------------------------------
// laser spot: first hit of the collimated beam (Sec. 5: a light ray is traced first)
// --------------------------------------------------------------------------------------------
__global__ void laser_kernel(GeomDev g, float3 o, float3 dir, float power, LightDev* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    LightDev L;
    L.kind = 0; L.pos = f3(0.f, 0.f, 0.f); L.I = power; L.s_tri = 0; L.s_b1 = 0.f; L.s_b2 = 0.f;
    L.to_origin = f3(0.f, 0.f, 0.f); L.emit_len = 0.f;
    float3 d = norm3(dir);
    int tri; float b1, b2, t;
    if (traverse<false>(g, o, d, 3.0e38f, tri, b1, b2, t)) {
        Surf s = surf_at(g, tri, b1, b2);
        L.kind = 2; L.s_tri = tri; L.s_b1 = b1; L.s_b2 = b2; L.pos = s.p;
        L.to_origin = d * -1.0f; L.emit_len = t;
    }
    *out = L;
}

// --------------------------------------------------------------------------------------------
// host-side launchers
// --------------------------------------------------------------------------------------------
static inline dim3 pix_grid(int W, int H) { return dim3((W + 15) / 16, (H + 7) / 8); }
static inline dim3 tile_grid(int W, int H, int tw, int th) { return dim3((W + tw - 1) / tw, (H + th - 1) / th); }

// tile_w x tile_h pixel tiles, tile_w a power of two in [4, 32], tile_w * tile_h = 64 or 128
cudaError_t launch_gbuffer(const GbufArgs& a, int tile_h, cudaStream_t s) {
    note_launch();
    gbuffer_kernel<<<tile_grid(a.F.W, a.F.H, a.tile_w, tile_h), a.tile_w * tile_h, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_initial(const InitArgs& a, int tile_h, unsigned* err, cudaStream_t s) {
    note_launch();
    const dim3 grid = tile_grid(a.F.W, a.F.H, a.tile_w, tile_h);
    const int threads = a.tile_w * tile_h;
    if (a.F.B == 0) {
        if (a.P.flags & kFlagEllipsoid) initial_gated_kernel<true><<<grid, threads, 0, s>>>(a);
        else initial_gated_kernel<false><<<grid, threads, 0, s>>>(a);
    } else {
        if (a.P.flags & kFlagEllipsoid) initial_kernel<true><<<grid, threads, 0, s>>>(a, err);
        else initial_kernel<false><<<grid, threads, 0, s>>>(a, err);
    }
    return cudaGetLastError();
}
cudaError_t launch_vis_queue(const GeomDev& g, const float4* rays, const uint32_t* counter, uint32_t cap, uint32_t* fetch,
                             float* target, int blocks, cudaStream_t s);   // tof_reuse.cu

// batched G-buffer and gated initial stages over the instances of a batch (device argument tables,
// blk0: first block of each instance, `blocks` in all)
cudaError_t launch_gbuffer_batch(const GbufArgs* A, const int* blk0, int n, int blocks, cudaStream_t s) {
    note_launch();
    gbuffer_batch_kernel<<<blocks, 128, 0, s>>>(A, blk0, n);
    return cudaGetLastError();
}
cudaError_t launch_initial_batch(const InitArgs* A, const int* blk0, int n, int blocks, cudaStream_t s) {
    note_launch();
    initial_gated_batch_kernel<<<blocks, 128, 0, s>>>(A, blk0, n);
    return cudaGetLastError();
}

// resident blocks of ell_place_kernel on every SM (its grid strides over the requests)
cudaError_t ell_place_blocks(int* out) {
    int dev = 0, sms = 0, b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ell_place_kernel, 128, 0);
    *out = sms * (b > 0 ? b : 1);
    return cudaGetLastError();
}

cudaError_t launch_initial_ell_wave(const InitArgs& a, const EllWaveDev& w, int tile_h, int place_blocks, int vis_blocks,
                                    cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(w.counters, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const dim3 grid = tile_grid(a.F.W, a.F.H, a.tile_w, tile_h);
    const int threads = a.tile_w * tile_h;
    note_launch();
    ell_trees_kernel<<<grid, threads, 0, s>>>(a, w);
    note_launch();
    ell_place_kernel<<<place_blocks, 128, 0, s>>>(a, w);
    e = launch_vis_queue(a.F.g, w.rays, &w.counters[2], w.ray_cap, &w.counters[3], w.bw, vis_blocks, s);
    if (e != cudaSuccess) return e;
    note_launch();
    tree_select_kernel<true><<<grid, threads, 0, s>>>(a, w);
    return cudaGetLastError();
}
// resident blocks of tw_hit_kernel on every SM (its lanes pull rays until the round's queue is empty)
cudaError_t tree_hit_blocks(int* out) {
    int dev = 0, sms = 0, b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tw_hit_kernel, 128, 0);
    *out = sms * (b > 0 ? b : 1);
    return cudaGetLastError();
}

// depth - 1 rounds of (closest hits, shading) after the start, then the light segments and the
// selection: 2 * depth + 1 kernels and one counter reset
cudaError_t launch_initial_tree_wave(const InitArgs& a, const TreeWaveDev& w, int tile_h, int hit_blocks, int vis_blocks,
                                     cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(w.counters, 0, kTreeWaveCounters * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const unsigned npath = (unsigned)a.F.W * (unsigned)a.F.H * (unsigned)w.nc;
    const EllWaveDev none = {};
    note_launch();
    tw_start_kernel<false><<<(npath + 127) / 128, 128, 0, s>>>(a, w, none);
    for (int d = 2; d <= a.P.depth; ++d) {
        note_launch(2);
        tw_hit_kernel<<<hit_blocks, 128, 0, s>>>(a.F.g, w.rays[d & 1], &w.counters[d], w.path_cap, &w.counters[8 + d], w.hits);
        tw_shade_kernel<false><<<hit_blocks, 128, 0, s>>>(a, w, none, d);
    }
    e = launch_vis_queue(a.F.g, w.srays, &w.counters[14], w.sray_cap, &w.counters[15], reinterpret_cast<float*>(w.acand),
                         vis_blocks, s);
    if (e != cudaSuccess) return e;
    note_launch();
    tree_select_kernel<false><<<tile_grid(a.F.W, a.F.H, a.tile_w, tile_h), a.tile_w * tile_h, 0, s>>>(a, w);
    return cudaGetLastError();
}

// the ellipsoidal connection's initial wavefront with its path trees as bounce rounds: the tree
// kernels write the EllWaveDev vertex, throughput, candidate and request tables (the same slots
// as ell_trees_kernel), then placement, the two visibility queues and the selection as in
// launch_initial_ell_wave
cudaError_t launch_initial_ell_tree_wave(const InitArgs& a, const TreeWaveDev& tw, const EllWaveDev& ell, int tile_h, int hit_blocks,
                                         int place_blocks, int vis_blocks, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tw.counters, 0, kTreeWaveCounters * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ell.counters, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    TreeWaveDev w = tw;
    w.vtx = ell.vtx;
    w.acand = ell.acand;
    const unsigned npath = (unsigned)a.F.W * (unsigned)a.F.H * (unsigned)w.nc;
    note_launch();
    tw_start_kernel<true><<<(npath + 127) / 128, 128, 0, s>>>(a, w, ell);
    for (int d = 2; d <= a.P.depth; ++d) {
        note_launch(2);
        tw_hit_kernel<<<hit_blocks, 128, 0, s>>>(a.F.g, w.rays[d & 1], &w.counters[d], w.path_cap, &w.counters[8 + d], w.hits);
        tw_shade_kernel<true><<<hit_blocks, 128, 0, s>>>(a, w, ell, d);
    }
    e = launch_vis_queue(a.F.g, w.srays, &w.counters[14], w.sray_cap, &w.counters[15], reinterpret_cast<float*>(w.acand),
                         vis_blocks, s);
    if (e != cudaSuccess) return e;
    note_launch();
    ell_place_kernel<<<place_blocks, 128, 0, s>>>(a, ell);
    e = launch_vis_queue(a.F.g, ell.rays, &ell.counters[2], ell.ray_cap, &ell.counters[3], ell.bw, vis_blocks, s);
    if (e != cudaSuccess) return e;
    note_launch();
    tree_select_kernel<true><<<tile_grid(a.F.W, a.F.H, a.tile_w, tile_h), a.tile_w * tile_h, 0, s>>>(a, ell);
    return cudaGetLastError();
}
cudaError_t launch_initial_shrink(const InitArgs& a, int tile_h, cudaStream_t s) {
    note_launch();
    if (a.P.flags & kFlagTriangleWalk)
        initial_shrink_kernel<true><<<tile_grid(a.F.W, a.F.H, a.tile_w, tile_h), a.tile_w * tile_h, 0, s>>>(a);
    else
        initial_shrink_kernel<false><<<tile_grid(a.F.W, a.F.H, a.tile_w, tile_h), a.tile_w * tile_h, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_splat(const SplatArgs& a, cudaStream_t s) {
    long long threads = (long long)a.npix * 32;
    note_launch();
    splat_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_pt(const PtArgs& a, cudaStream_t s) {
    note_launch();
    pt_kernel<<<pix_grid(a.F.W, a.F.H), 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_laser(const GeomDev& g, float3 o, float3 d, float power, LightDev* out, cudaStream_t s) {
    note_launch();
    laser_kernel<<<1, 32, 0, s>>>(g, o, d, power, out);
    return cudaGetLastError();
}

}  // namespace tof
