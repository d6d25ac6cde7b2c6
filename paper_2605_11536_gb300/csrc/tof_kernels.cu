// tof_kernels.cu -- per-frame kernels of the ToF ReSTIR hot path (sm_103a).
//
//   gbuffer_kernel   primary visibility, one jittered ray per pixel            (Sec. 3.2 setup)
//   initial_kernel   path trees with NEE, streaming RIS into per-bin reservoirs (stage (1), Sec. 4.5)
//   reuse_kernel     temporal or spatial GRIS merge through the path-length shift (stages (2), (3))
//   splat_kernel     transient histogram H[px, b] = f(y_b) W_b                  (stage (4), Sec. 4.5)
//   pt_kernel        plain gated / transient path tracing (the comparison of Sec. 6)
//   laser_kernel     resolves the collimated laser's spot (Sec. 5 "Light Source")
// The gated image is written by the last stage's kernel (final shading fused into it).
#include "tof_device.cuh"

namespace tof {

// --------------------------------------------------------------------------------------------
// shared helpers
// --------------------------------------------------------------------------------------------
__device__ Domain make_domain_hit(const FrameDev* F, bool valid, int tri, float b1, float b2, float t, float L0, float dL) {
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

__device__ __forceinline__ float gate_L0(const FrameDev& F, int b) { return F.B > 0 ? F.L0 + b * F.dL : F.L0; }

// One path tree; Sink(k, c, tau, T) receives each NEE candidate of length k in [kmin, depth]
// whose tau lies in [glo, ghi) and whose light segment is unoccluded (c = f / p, no gate).
template <class Sink>
__device__ void trace_tree(const Domain& D, const ParamsDev& P, uint32_t px, uint32_t frame, int tree, float glo, float ghi,
                           TreeVerts& T, Sink& sink) {
    const GeomDev& g = D.F->g;
    T.v[1] = D.y1;
    T.cls[1] = mat_class(load_mat(g, D.y1.mat));
    T.pdfA[1] = 1.0f;
    float len = len3(D.x0 - D.y1.p);
    float beta = 1.0f;
    const int kmin = (P.flags & 1u) ? 1 : 2;
    for (int d = 1; d <= P.depth; ++d) {
        const Surf& x = T.v[d];
        Mat m = load_mat(g, x.mat);
        float3 wi = dir_to(x.p, d == 1 ? D.x0 : T.v[d - 1].p);
        if (d >= kmin && mat_class(m) != C_DELTA) {
            float3 wl; float seg;
            float lt = light_term(D, x, wl, seg);
            float fs = lt > 0.f ? bsdf_f(m, x.n, wi, wl) : 0.f;
            if (fs > 0.f) {
                float tau = len + seg - D.o;
                if (tau >= glo && tau < ghi && light_visible(D, g, x, P.ray_eps)) sink(d, beta * fs * lt, tau, T);
            }
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
    float4* Pl = R.planes;
    const size_t s = R.stride;
    Pl[s + idx] = make_float4(__uint_as_float(r.key_px), __uint_as_float(r.key_frame), __uint_as_float(r.meta), r.pdf_pre);
    if (rec_r(r) >= 2) {
        Pl[2 * s + idx] = make_float4(r.xprev.x, r.xprev.y, r.xprev.z, __int_as_float(r.p_tri));
        Pl[3 * s + idx] = make_float4(r.p_b1, r.p_b2, __int_as_float(r.s_tri[0]), r.s_b1[0]);
        int ns = rec_ns(r);
        if (ns >= 1) Pl[4 * s + idx] = make_float4(r.s_b2[0], __int_as_float(r.s_tri[1]), r.s_b1[1], r.s_b2[1]);
        if (ns >= 3) Pl[5 * s + idx] = make_float4(__int_as_float(r.s_tri[2]), r.s_b1[2], r.s_b2[2], 0.f);
    }
}

// --------------------------------------------------------------------------------------------
// G-buffer: one jittered primary ray per pixel -> (tri, b1, b2, |x1 - x0|)
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) gbuffer_kernel(const __grid_constant__ GbufArgs a) {
    const FrameDev& F = a.F;
    int ix = blockIdx.x * 16 + (threadIdx.x & 15), iy = blockIdx.y * 8 + (threadIdx.x >> 4);
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
    __device__ void operator()(int k, float c, float tauv, const TreeVerts& T) {
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
        uint4 u = philox(px, frame, ((uint32_t)tree << 8) | (uint32_t)k, P_RIS, P->seed);
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

__global__ void __launch_bounds__(128) initial_kernel(const __grid_constant__ InitArgs a, int* err) {
    const FrameDev& F = a.F;
    int ix = blockIdx.x * 16 + (threadIdx.x & 15), iy = blockIdx.y * 8 + (threadIdx.x >> 4);
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
        trace_tree(D, P, (uint32_t)pix, F.frame, t, glo, ghi, T, sink);
    }
    if (sink.overflow && err) atomicOr(err, 1);
    float outv = 0.f;
    for (int e = 0; e < sink.n; ++e) {
        if (!(sink.phat[e] > 0.f)) continue;
        float W = sink.S[e] / sink.phat[e];
        size_t idx = (size_t)pix * Bn + sink.bin[e];
        a.dst.planes[idx] = make_float4(W, sink.phat[e], sink.tau[e], sink.Lsuf[e]);
        occ[sink.bin[e] >> 5] |= 1u << (sink.bin[e] & 31);
        outv = sink.phat[e] * W;
    }
    if (a.out) a.out[pix] = outv;
}

// --------------------------------------------------------------------------------------------
// reuse (stages (2) and (3)): GRIS merge (eq. GRIS_resampling_weight) with the generalized
// balance heuristic (eq. GRIS_MIS_weight, denominators evaluated at the same y_i for every
// domain, p_hat_{<-i}(y_i) = p_hat_i(x_i) / |dS_i/dx_i|); slot 0 is the canonical sample.
// Confidence weights are per pixel and shared by every bin.
// --------------------------------------------------------------------------------------------
struct Slot {
    const FrameDev* F;
    const ResDev* R;
    int pix;
    float M;
    bool geom_static;
};

__device__ __forceinline__ int pick_neighbor(uint64_t seed, uint32_t px, uint32_t frame, int pass, int slot, int W, int H, int R) {
    int ix = (int)(px % (uint32_t)W), iy = (int)(px / (uint32_t)W);
    uint32_t side = 2u * (uint32_t)R + 1u;
    for (int a = 0; a < 4; ++a) {
        uint4 u = philox(px, frame, ((uint32_t)pass << 8) | (uint32_t)slot, P_NEIGHBOR | ((uint32_t)a << 8), seed);
        uint32_t uu[4] = {u.x, u.y, u.z, u.w};
        for (int h = 0; h < 2; ++h) {
            int dx = (int)(uu[2 * h] % side) - R, dy = (int)(uu[2 * h + 1] % side) - R;
            if (dx * dx + dy * dy > R * R || (dx == 0 && dy == 0)) continue;
            int nx = ix + dx, ny = iy + dy;
            if (nx < 0 || ny < 0 || nx >= W || ny >= H) return -1;
            return ny * W + nx;
        }
    }
    return -1;
}

__device__ __forceinline__ Domain slot_domain(const Slot& s, int b) {
    float4 gb = __ldg(&s.F->gb[s.pix]);
    uint32_t tri = __float_as_uint(gb.x);
    return make_domain_hit(s.F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, gate_L0(*s.F, b), s.F->dL);
}

// merge of bin b over n slots; returns true and the merged record if any candidate survives
__device__ bool merge_bin(const ReuseArgs& a, const Slot* sl, int n, int b, uint32_t pix, Rec& out, ShiftStats& st) {
    const ParamsDev& P = a.P;
    const int Bn0 = sl[0].F->B > 0 ? sl[0].F->B : 1;
    Rec y[kMaxSlots];
    float py[kMaxSlots], J[kMaxSlots], ph[kMaxSlots], Wx[kMaxSlots], w[kMaxSlots];
    bool ok[kMaxSlots];
    Domain D0 = slot_domain(sl[0], b);
    for (int s = 0; s < n; ++s) {
        ok[s] = false; w[s] = 0.f;
        int Bs = sl[s].F->B > 0 ? sl[s].F->B : 1;
        if (!occ_get(*sl[s].R, sl[s].pix, b)) continue;
        size_t idx = (size_t)sl[s].pix * Bs + b;
        if (s == 0) {
            rec_load(*sl[0].R, idx, y[0]);
            py[0] = y[0].phat; J[0] = 1.0f; ph[0] = y[0].phat; Wx[0] = y[0].W;
            ok[0] = py[0] > 0.f;
            continue;
        }
        Rec x;
        rec_load(*sl[s].R, idx, x);
        ph[s] = x.phat; Wx[s] = x.W;
        Domain Ds = slot_domain(sl[s], b);
        ok[s] = shift_rec(x, Ds, D0, P, sl[s].geom_static, y[s], py[s], J[s], &st);
    }
    (void)Bn0;
    for (int s = 0; s < n; ++s) {
        if (!ok[s]) continue;
        float num = s == 0 ? sl[0].M * py[0] : sl[s].M * ph[s] / J[s];
        float den = sl[0].M * py[s];
        for (int j = 1; j < n; ++j) {
            if (j == s) { den += sl[s].M * ph[s] / J[s]; continue; }
            Domain Dj = slot_domain(sl[j], b);
            Rec tmp; float pj, Jj;
            if (shift_rec(y[s], D0, Dj, P, sl[j].geom_static, tmp, pj, Jj, nullptr)) den += sl[j].M * pj * Jj;
        }
        float m = den > 0.f ? num / den : 0.f;
        w[s] = m * py[s] * Wx[s] * J[s];
        if (!(w[s] > 0.f) || !isfinite(w[s])) w[s] = 0.f;
    }
    float S = 0.f;
    int sel = -1;
    for (int s = 0; s < n; ++s) {
        if (!(w[s] > 0.f)) continue;
        uint4 u = philox(pix, sl[0].F->frame, ((uint32_t)a.pass << 8) | (uint32_t)s, P_MERGE | ((uint32_t)b << 8), P.seed);
        S += w[s];
        if (u01(u.x) * S < w[s]) sel = s;
    }
    if (sel < 0) return false;
    out = y[sel];
    out.W = S / py[sel];
    return true;
}

__global__ void __launch_bounds__(128) reuse_kernel(const __grid_constant__ ReuseArgs a) {
    const FrameDev& C = a.cur;
    int ix = blockIdx.x * 16 + (threadIdx.x & 15), iy = blockIdx.y * 8 + (threadIdx.x >> 4);
    ShiftStats st = {0, 0, 0, 0, 0};
    bool active = ix < C.W && iy < C.H;
    if (active) {
        const int pix = iy * C.W + ix;
        const ParamsDev& P = a.P;
        const int Bn = C.B > 0 ? C.B : 1;
        const int words = a.dst.words;
        uint32_t* docc = a.dst.occ + (size_t)pix * words;
        const uint32_t* socc = a.src.occ + (size_t)pix * words;
        Slot sl[kMaxSlots];
        int n = 1;
        sl[0].F = &a.cur; sl[0].R = &a.src; sl[0].pix = pix; sl[0].M = a.src.M[pix]; sl[0].geom_static = true;
        bool gb_valid = __float_as_uint(C.gb[pix].x) != kNoHit;
        if (gb_valid) {
            if (a.temporal) {
                int q = -1;
                if (C.mode == 1) q = pix;
                else {
                    float4 gb = C.gb[pix];
                    Surf sp = surf_at(a.prev.g, __float_as_int(gb.x), gb.y, gb.z);
                    int qx, qy;
                    if (project(a.prev, sp.p, qx, qy)) q = qy * C.W + qx;
                }
                if (q >= 0) {
                    sl[1].F = &a.prev; sl[1].R = &a.prv; sl[1].pix = q; sl[1].M = fminf(a.prv.M[q], P.m_cap);
                    sl[1].geom_static = a.geom_static != 0;
                    n = 2;
                }
            } else {
                for (int s = 1; s <= P.n_spatial; ++s) {
                    int q = pick_neighbor(P.seed, (uint32_t)pix, C.frame, a.pass, s, C.W, C.H, P.radius);
                    if (q < 0) continue;
                    sl[n].F = &a.cur; sl[n].R = &a.src; sl[n].pix = q; sl[n].M = fminf(a.src.M[q], P.m_cap);
                    sl[n].geom_static = true;
                    ++n;
                }
            }
        }
        float Msum = 0.f;
        for (int s = 0; s < n; ++s) Msum += sl[s].M;
        a.dst.M[pix] = Msum;
        float outv = 0.f;
        if (n == 1) {
            // no reuse candidate: the canonical reservoir carries over unchanged
            for (int w = 0; w < words; ++w) {
                uint32_t m = socc[w];
                docc[w] = m;
                while (m) {
                    int bit = __ffs(m) - 1;
                    m &= m - 1;
                    size_t idx = (size_t)pix * Bn + (w << 5) + bit;
                    for (int k = 0; k < 6; ++k) a.dst.planes[k * a.dst.stride + idx] = a.src.planes[k * a.src.stride + idx];
                    if (C.B == 0) { float4 p0 = a.src.planes[idx]; outv = p0.y * p0.x; }
                }
            }
        } else {
            for (int w = 0; w < words; ++w) {
                uint32_t m = 0u;
                for (int s = 0; s < n; ++s) m |= sl[s].R->occ[(size_t)sl[s].pix * sl[s].R->words + w];
                uint32_t res = 0u;
                while (m) {
                    int bit = __ffs(m) - 1;
                    m &= m - 1;
                    int b = (w << 5) + bit;
                    if (b >= Bn) break;
                    Rec r;
                    if (merge_bin(a, sl, n, b, (uint32_t)pix, r, st)) {
                        size_t idx = (size_t)pix * Bn + b;
                        rec_store(a.dst, idx, r);
                        res |= 1u << bit;
                        if (C.B == 0) outv = r.phat * r.W;
                    }
                }
                docc[w] = res;
            }
        }
        if (a.out) a.out[pix] = outv;
    }
    stats_flush(a.stats, st);
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
    const float4* P0 = a.src.planes + (size_t)pix * B;
    for (int w = 0; w < a.src.words; ++w) {
        uint32_t m = occ[w];
        int b = (w << 5) + lane;
        if (b >= B) break;
        float v = 0.f;
        if ((m >> lane) & 1u) { float4 p = P0[b]; v = p.y * p.x; }
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
    __device__ void operator()(int k, float c, float tau, const TreeVerts& T) {
        (void)k; (void)T;
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

cudaError_t launch_gbuffer(const GbufArgs& a, cudaStream_t s) {
    gbuffer_kernel<<<pix_grid(a.F.W, a.F.H), 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_initial(const InitArgs& a, int* err, cudaStream_t s) {
    initial_kernel<<<pix_grid(a.F.W, a.F.H), 128, 0, s>>>(a, err);
    return cudaGetLastError();
}
cudaError_t launch_reuse(const ReuseArgs& a, cudaStream_t s) {
    reuse_kernel<<<pix_grid(a.cur.W, a.cur.H), 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_splat(const SplatArgs& a, cudaStream_t s) {
    long long threads = (long long)a.npix * 32;
    splat_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_pt(const PtArgs& a, cudaStream_t s) {
    pt_kernel<<<pix_grid(a.F.W, a.F.H), 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_laser(const GeomDev& g, float3 o, float3 d, float power, LightDev* out, cudaStream_t s) {
    laser_kernel<<<1, 32, 0, s>>>(g, o, d, power, out);
    return cudaGetLastError();
}

}  // namespace tof
