// tof_reuse.cu -- temporal and spatial reuse (Sec. 3.2 stages (2) and (3)) as a wavefront of
// shift tasks.
//
// One GRIS merge (eq. GRIS_resampling_weight with the generalized balance heuristic of
// eq. GRIS_MIS_weight) needs, for a pixel's (or a pixel-bin's) canonical sample and k reused
// samples, k forward shifts into the pixel's domain and, for every surviving candidate, one
// inverse shift into each other reused domain.  Run as one thread per pixel, the shifts of the
// few pixels that hold samples serialise while the rest of the warp idles, so the pass is split:
//   reuse_slots_kernel   per pixel: slots (neighbours or the back-projected previous pixel) and
//                        capped confidences
//   reuse_units_kernel   per (pixel, 32-bin word): merge units (pixel, bin), forward-shift tasks
//                        and the canonical sample's inverse-shift tasks
//   shift_fwd_kernel     persistent over forward tasks: shift slot s's sample into the unit's
//                        domain, queueing its visibility segments
//   vis_kernel           traces the queued segments, zeroing the results of occluded shifts
//   emit_inv_kernel      per surviving shifted candidate: its inverse-shift tasks
//   shift_inv_kernel     persistent over inverse tasks: shift candidate s's offset path into
//                        domain j -> the term M_j p_hat_j(S_j^-1(y_s)) |dS_j^-1/dy_s|
//                        (visibility queued again, then vis_kernel)
//   reuse_merge_kernel   persistent over units: MIS weights, streaming selection, output
// Task lists are compacted with atomics, read by the next kernel in stream order; no kernel
// waits on another's progress.
#include "tof_device.cuh"

namespace tof {

__device__ __forceinline__ float gate_L0r(const FrameDev& F, int b) { return F.B > 0 ? F.L0 + b * F.dL : F.L0; }

__device__ __forceinline__ const FrameDev* slot_frame(const ReuseArgs& a, int s) {
    return (a.temporal && s == 1) ? &a.prev : &a.cur;
}
__device__ __forceinline__ const ResDev* slot_res(const ReuseArgs& a, int s) {
    return (a.temporal && s == 1) ? &a.prv : &a.src;
}

// bin of slot s for the unit of bin b: the bin pass reuses the same pixel's bins b - 1 (slot 1)
// and b + 1 (slot 2); bins outside [0, B) are not domains (no candidate was drawn for them)
__device__ __forceinline__ int slot_bin(const ReuseArgs& a, int s, int b) {
    return a.binpass ? (s == 1 ? b - 1 : s == 2 ? b + 1 : b) : b;
}
__device__ __forceinline__ bool slot_present(const ReuseArgs& a, int s, int b) {
    if (!a.binpass) return true;
    const int sb = slot_bin(a, s, b);
    return sb >= 0 && sb < a.cur.B;
}
__device__ __forceinline__ bool slot_occ(const ReuseArgs& a, int s, int q, int b) {
    if (!slot_present(a, s, b)) return false;
    return occ_get(*slot_res(a, s), q, slot_bin(a, s, b));
}

__device__ __forceinline__ Domain pix_domain(const FrameDev* F, int pix, int b) {
    float4 gb = __ldg(&F->gb[pix]);
    uint32_t tri = __float_as_uint(gb.x);
    return make_domain_hit(F, tri != kNoHit, (int)tri, gb.y, gb.z, gb.w, gate_L0r(*F, b), F->dL);
}

__device__ __forceinline__ int pick_nb(uint64_t seed, uint32_t px, uint32_t frame, int pass, int slot, int W, int H, int R) {
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

// warp-aggregated reservation of `n` consecutive slots in a counter
__device__ __forceinline__ uint32_t reserve(uint32_t* counter, uint32_t n) {
    const uint32_t mask = __activemask();
    const int lane = threadIdx.x & 31;
    uint32_t incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(mask, incl, o);
        if (lane >= o && ((mask >> (lane - o)) & 1u)) incl += v;
    }
    // the highest active lane holds the warp total only if all lanes are active; fall back to a
    // per-thread atomic for partially active warps
    if (mask != 0xFFFFFFFFu) return n ? atomicAdd(counter, n) : 0u;
    uint32_t total = __shfl_sync(mask, incl, 31);
    uint32_t base = 0;
    if (lane == 31) base = total ? atomicAdd(counter, total) : 0u;
    base = __shfl_sync(mask, base, 31);
    return base + incl - n;
}

__device__ __forceinline__ void store_rec(float4* P, size_t stride, size_t idx, const Rec& r) {
    ResDev R;
    R.planes = P; R.stride = stride; R.estride = 1;
    rec_store(R, idx, r);
}

// --------------------------------------------------------------------------------------------
// per pixel: slots (the pixel, its reused pixels) and capped confidences
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void reuse_slots_body(const ReuseArgs& a, const WaveDev& w, int p0, int p1, int blk) {
    const FrameDev& C = a.cur;
    const int pix = p0 + blk * blockDim.x + threadIdx.x;
    if (pix >= p1) return;
    const ParamsDev& P = a.P;
    int n = 1;
    int sp[kMaxSlots];
    float sM[kMaxSlots];
    sp[0] = pix;
    sM[0] = a.src.M[pix];
    bool gb_valid = __float_as_uint(C.gb[pix].x) != kNoHit;
    if (gb_valid) {
        if (a.binpass) {
            // the same pixel's neighbouring bins: confidence capped like any reused domain
            sp[1] = sp[2] = pix;
            sM[1] = sM[2] = fminf(sM[0], P.m_cap);
            n = 3;
        } else if (a.temporal) {
            int q = -1;
            if (C.mode == 1) q = pix;
            else {
                float4 gb = C.gb[pix];
                Surf sp0 = surf_at(a.prev.g, __float_as_int(gb.x), gb.y, gb.z);
                int qx, qy;
                if (project(a.prev, sp0.p, qx, qy)) q = qy * C.W + qx;
            }
            if (q >= 0) { sp[1] = q; sM[1] = fminf(a.prv.M[q], P.m_cap); n = 2; }
        } else {
            for (int s = 1; s <= P.n_spatial; ++s) {
                int q = pick_nb(P.seed, (uint32_t)pix, C.frame, a.pass, s, C.W, C.H, P.radius);
                if (q < 0) continue;
                sp[n] = q; sM[n] = fminf(a.src.M[q], P.m_cap); ++n;
            }
        }
    }
    float Msum = 0.f;
    for (int s = 0; s < n; ++s) Msum += sM[s];
    a.dst.M[pix] = Msum;
    const int S = w.slots;
    w.nslot[pix] = (uint8_t)n;
    for (int s = 0; s < n; ++s) { w.slot_pix[(size_t)pix * S + s] = sp[s]; w.slot_M[(size_t)pix * S + s] = sM[s]; }
}
__global__ void __launch_bounds__(128) reuse_slots_kernel(const __grid_constant__ ReuseArgs a, const __grid_constant__ WaveDev w,
                                                          int p0, int p1) {
    reuse_slots_body(a, w, p0, p1, blockIdx.x);
}

// --------------------------------------------------------------------------------------------
// per (pixel, 32-bin occupancy word): merge units and their tasks. One thread per word keeps the
// transient passes parallel over bins (a pixel may occupy hundreds of bins); gated views have one
// word per pixel.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void reuse_units_body(const ReuseArgs& a, const WaveDev& w, int p0, int p1, int blk) {
    const FrameDev& C = a.cur;
    const int Bn = C.B > 0 ? C.B : 1;
    const int words = a.dst.words;
    const long long t = (long long)blk * blockDim.x + threadIdx.x;
    const bool active = t < (long long)(p1 - p0) * words;
    const int pix = active ? p0 + (int)(t / words) : 0;
    const int wd = active ? (int)(t % words) : 0;
    const int S = w.slots;
    int n = 0;
    int sp[kMaxSlots];
    uint32_t m = 0u;
    float outv = 0.f;
    if (active) {
        n = w.nslot[pix];
        for (int s = 0; s < n; ++s) sp[s] = w.slot_pix[(size_t)pix * S + s];
        uint32_t* docc = a.dst.occ + (size_t)pix * words;
        if (n == 1) {
            // no reuse candidates: the reservoirs copy through
            uint32_t c = a.src.occ[(size_t)pix * words + wd];
            docc[wd] = c;
            while (c) {
                int bit = __ffs(c) - 1;
                c &= c - 1;
                size_t idx = (size_t)pix * Bn + (wd << 5) + bit;
                for (int k = 0; k < 6; ++k) *res_at(a.dst, k, idx) = *res_at(a.src, k, idx);
                if (C.B == 0) { float4 p0v = *res_at(a.src, 0, idx); outv = p0v.y * p0v.x; }
            }
        } else if (a.binpass) {
            // units: bins whose own, lower or upper neighbour's reservoir holds a sample
            docc[wd] = 0u;
            const uint32_t* o = a.src.occ + (size_t)pix * words;
            const uint32_t c = o[wd];
            const uint32_t lo = wd > 0 ? o[wd - 1] : 0u, hi = wd + 1 < words ? o[wd + 1] : 0u;
            m = c | (c << 1) | (lo >> 31) | (c >> 1) | (hi << 31);
            const int rem = C.B - (wd << 5);
            if (rem < 32) m &= (1u << rem) - 1u;
        } else {
            docc[wd] = 0u;
            for (int s = 0; s < n; ++s) {
                const ResDev* R = slot_res(a, s);
                m |= R->occ[(size_t)sp[s] * R->words + wd];
            }
        }
    }
    // one unit per set bit. Reserve the units, then count and reserve the forward tasks and the
    // canonical inverse tasks of the units inside the capacity, then write them: three warp-wide
    // atomics instead of two per unit.
    const uint32_t nu = __popc(m);
    const uint32_t ubase = reserve(&w.counters[0], nu);
    const uint32_t nvalid = ubase >= (uint32_t)w.cap_units ? 0u : min(nu, (uint32_t)w.cap_units - ubase);
    if (nvalid < nu) atomicOr(&w.counters[3], 1u);
    uint32_t nf_tot = 0, ni_tot = 0;
    {
        uint32_t mm = m;
        for (uint32_t k = 0; k < nvalid; ++k) {
            int b = (wd << 5) + __ffs(mm) - 1;
            mm &= mm - 1;
            for (int s = 1; s < n; ++s)
                if (slot_occ(a, s, sp[s], b)) ++nf_tot;
            if (n > 1 && occ_get(a.src, pix, b))
                for (int j = 1; j < n; ++j) ni_tot += slot_present(a, j, b) ? 1u : 0u;
        }
    }
    uint32_t fb = reserve(&w.counters[1], nf_tot);
    uint32_t ib = reserve(&w.counters[2], ni_tot);
    for (uint32_t k = 0; k < nvalid; ++k) {
        int b = (wd << 5) + __ffs(m) - 1;
        m &= m - 1;
        uint32_t u = ubase + k;
        w.units[u] = make_int2(pix, b);
        for (int s = 1; s < n; ++s)
            if (slot_occ(a, s, sp[s], b)) w.fwd[fb++] = (u << 4) | (uint32_t)s;
        if (n > 1 && occ_get(a.src, pix, b)) {
            for (int j = 1; j < n; ++j)
                if (slot_present(a, j, b)) w.inv[ib++] = (u << 8) | (uint32_t)j;
        }
    }
    // gated (one word per pixel): pixels that form a unit get their value from the merge
    if (active && a.out) a.out[pix] = n == 1 ? outv : 0.f;
}
__global__ void __launch_bounds__(128) reuse_units_kernel(const __grid_constant__ ReuseArgs a, const __grid_constant__ WaveDev w,
                                                          int p0, int p1) {
    reuse_units_body(a, w, p0, p1, blockIdx.x);
}

// --------------------------------------------------------------------------------------------
// forward shifts: slot s's sample into the unit's domain
// --------------------------------------------------------------------------------------------
template <bool kWalk>
__device__ __forceinline__ void shift_fwd_body(const ReuseArgs& a, const WaveDev& w) {
    ShiftStats st = {0, 0, 0, 0, 0};
    const uint32_t ntask = min(w.counters[1], (uint32_t)w.cap_units * (uint32_t)(w.slots - 1));
    const int S = w.slots;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntask; t += gridDim.x * blockDim.x) {
        uint32_t task = w.fwd[t];
        uint32_t u = task >> 4;
        int s = (int)(task & 15u);
        int2 ub = w.units[u];
        int pix = ub.x, b = ub.y;
        int q = w.slot_pix[(size_t)pix * S + s];
        const FrameDev* Fs = slot_frame(a, s);
        const ResDev* Rs = slot_res(a, s);
        int Bs = Fs->B > 0 ? Fs->B : 1;
        Rec x;
        const int sb = slot_bin(a, s, b);
        rec_load(*Rs, (size_t)q * Bs + sb, x);
        Domain Ds = pix_domain(Fs, q, sb);
        Domain D0 = pix_domain(&a.cur, pix, b);
        Rec y;
        float py = 0.f, J = 1.f;
        bool geom_static = (a.temporal && s == 1) ? a.geom_static != 0 : true;
        size_t ui = (size_t)u * S + s;
        VisQ vq;
        vq.rays = w.rays; vq.counter = &w.counters[4]; vq.cap = w.ray_cap; vq.target = (uint32_t)ui;
        bool ok = shift_rec<true, kWalk>(x, Ds, D0, a.P, geom_static, y, py, J, &st, &vq);
        // visibility is settled by vis_kernel, which zeroes py of an occluded shift
        w.py[ui] = ok ? py : 0.f;
        w.jac[ui] = ok ? J : 1.f;
        if (ok) {
            store_rec(w.yrec, (size_t)w.cap_units * (S - 1), (size_t)u * (S - 1) + (s - 1), y);
        }
    }
    // warp-level flush of the shift statistics
    if (a.stats) {
        // counters 0..4 and 6 (spatial forward calls); counter 5 belongs to the inverse kernel
        unsigned long long v[7] = {st.newton_calls, st.newton_iters, st.newton_ok, st.shift_calls, st.shift_ok, 0ull,
                                   a.temporal ? 0ull : (unsigned long long)st.shift_calls};
        for (int i = 0; i < 7; ++i) {
            unsigned long long x = v[i];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
            if ((threadIdx.x & 31) == 0 && x) atomicAdd(&a.stats->v[i], x);
        }
    }
}
template <bool kWalk>
__global__ void __launch_bounds__(128, 8) shift_fwd_kernel(const __grid_constant__ ReuseArgs a, const __grid_constant__ WaveDev w) {
    shift_fwd_body<kWalk>(a, w);
}

// --------------------------------------------------------------------------------------------
// visibility segments queued by a shift kernel; an occluded segment zeroes the result it guards.
// Persistent, with dynamic fetch: a lane whose segment is settled takes the next queued one
// between rounds of at most kVisSteps node visits, so lanes do not idle while the warp's longest
// traversal (grazing segments over a heightfield visit many nodes) runs to its end.  Each
// segment's node visits are those of traverse<true> in the same order, so the answer is the same.
// stat >= 0: the stats counter that counted the guarded shifts as successes (one decrement per
// shift, however many of its segments are occluded); ray_stat >= 0: the counter of segments.
// --------------------------------------------------------------------------------------------
constexpr int kVisSteps = 32;   // 8: 4.63, 16: 4.52, 32: 4.49-4.51, 64 / 128: 4.50 ms per 512 x 512 frame

__device__ __forceinline__ void vis_body(const GeomDev& gref, const float4* __restrict__ rays, const uint32_t* counter,
                                         uint32_t cap, uint32_t* fetch, float* target, StatsDev* stats, int stat, int ray_stat) {
    // the hierarchy in registers (a batched launch passes the instance's GeomDev in shared memory)
    GeomDev g;
    g.nodes = gref.nodes; g.leaf = gref.leaf; g.nt = gref.nt; g.err = gref.err;
    const uint32_t n = min(*counter, cap);
    if (stats && ray_stat >= 0 && blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(&stats->v[ray_stat], (unsigned long long)n);
    const int lane = threadIdx.x & 31;
    unsigned long long lost = 0;
    unsigned fault = 0u;         // traversal overflows of this lane, published after the loop
    bool has = false, done = false;
    float3 o = f3(0.f, 0.f, 0.f), d = o, id = o, ood = o;
    float tmax = 0.f;
    uint32_t tgt = 0;
    int node = 0, sp = 0, budget = 0;
    int stack[kStack];
    while (true) {
        // refill: every lane of the warp takes part (uniform control flow around the ballot)
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
                    float4 a = rays[2 * (size_t)i], b = rays[2 * (size_t)i + 1];
                    o = f3(a.x, a.y, a.z); d = f3(b.x, b.y, b.z); tmax = a.w; tgt = __float_as_uint(b.w);
                    id = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
                    ood = f3(o.x * id.x, o.y * id.y, o.z * id.z);
                    node = 0; sp = 0; budget = g.nt + 64;
                    has = true;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(0xFFFFFFFFu, done)) break;
        bool hit = false;
        for (int step = 0; step < kVisSteps && has; ++step) {
            if (g.nt <= 0) { has = false; break; }
            if (g.nt == 1) {
                float t, u, w; int orig;
                hit = tri_test(g.leaf, 0, o, d, tmax, t, u, w, orig) && t < tmax;
                has = false;
                break;
            }
            if (--budget < 0) {
                fault |= kErrVisitBudget;
                has = false;
                break;
            }
            const float4* N = g.nodes + 4 * node;
            float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
            float a0 = n0.x * id.x - ood.x, a1 = n0.y * id.x - ood.x;
            float b0 = n0.z * id.y - ood.y, bb1 = n0.w * id.y - ood.y;
            float c0 = n2.x * id.z - ood.z, c1 = n2.y * id.z - ood.z;
            float lo0 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, bb1)), fmaxf(fminf(c0, c1), 0.f));
            float hi0 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, bb1)), fminf(fmaxf(c0, c1), tmax));
            float d0 = n1.x * id.x - ood.x, d1 = n1.y * id.x - ood.x;
            float e0 = n1.z * id.y - ood.y, e1 = n1.w * id.y - ood.y;
            float f0 = n2.z * id.z - ood.z, f1 = n2.w * id.z - ood.z;
            float lo1 = fmaxf(fmaxf(fminf(d0, d1), fminf(e0, e1)), fmaxf(fminf(f0, f1), 0.f));
            float hi1 = fminf(fminf(fmaxf(d0, d1), fmaxf(e0, e1)), fminf(fmaxf(f0, f1), tmax));
            bool h0 = lo0 <= hi0, h1 = lo1 <= hi1;
            int ch0 = __float_as_int(n3.x), ch1 = __float_as_int(n3.y);
            if (h0 && ch0 < 0) {
                float t, u, w; int orig;
                if (tri_test(g.leaf, ~ch0, o, d, tmax, t, u, w, orig) && t < tmax) { hit = true; has = false; break; }
                h0 = false;
            }
            if (h1 && ch1 < 0) {
                float t, u, w; int orig;
                if (tri_test(g.leaf, ~ch1, o, d, tmax, t, u, w, orig) && t < tmax) { hit = true; has = false; break; }
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
                if (sp == 0) { has = false; break; }
                node = stack[--sp];
            }
        }
        if (hit) {
            float old = atomicExch(&target[tgt], 0.f);
            if (old != 0.f) ++lost;
        }
    }
    if (fault && g.err) atomicOr(g.err, fault);
    if (stats && stat >= 0) {
        unsigned long long x = lost;
        for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o2);
        if (lane == 0 && x) atomicAdd(&stats->v[stat], 0ull - x);
    }
}
__global__ void __launch_bounds__(128, 8) vis_kernel(const GeomDev g, const float4* __restrict__ rays, const uint32_t* counter,
                                                  uint32_t cap, uint32_t* fetch, float* target, StatsDev* stats, int stat,
                                                  int ray_stat) {
    vis_body(g, rays, counter, cap, fetch, target, stats, stat, ray_stat);
}

// --------------------------------------------------------------------------------------------
// after the forward shifts' visibility: each surviving shifted candidate's inverse shifts into
// the other reused domains (pairwise MIS needs none: it pairs the canonical domain with each
// reused one)
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void emit_inv_body(const ReuseArgs& a, const WaveDev& w) {
    const uint32_t ntask = min(w.counters[1], (uint32_t)w.cap_units * (uint32_t)(w.slots - 1));
    const int S = w.slots;
    const bool pairwise = (a.P.flags & kFlagPairwiseMis) != 0u;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntask; t += gridDim.x * blockDim.x) {
        uint32_t task = w.fwd[t];
        uint32_t u = task >> 4;
        int s = (int)(task & 15u);
        int2 ub = w.units[u];
        const int pix = ub.x, b = ub.y;
        const int n = w.nslot[pix];
        const bool ok = w.py[(size_t)u * S + s] > 0.f;
        uint32_t ne = 0u;
        if (ok && n > 2 && !pairwise)
            for (int j = 1; j < n; ++j) ne += (j != s && slot_present(a, j, b)) ? 1u : 0u;
        uint32_t ib = reserve_coalesced(&w.counters[2], ne);
        for (int j = 1; j < n && ne; ++j)
            if (j != s && slot_present(a, j, b)) w.inv[ib++] = (u << 8) | ((uint32_t)s << 4) | (uint32_t)j;
    }
}
__global__ void __launch_bounds__(128) emit_inv_kernel(const __grid_constant__ ReuseArgs a, const __grid_constant__ WaveDev w) {
    emit_inv_body(a, w);
}

// --------------------------------------------------------------------------------------------
// inverse shifts: candidate s's offset path (in the unit's domain) into domain j
// --------------------------------------------------------------------------------------------
// tasks [t0, t1) of the list; their visibility segments go to `rays` (counter rcount, capacity rcap)
template <bool kWalk>
__device__ __forceinline__ void shift_inv_body(const ReuseArgs& a, const WaveDev& w, uint32_t t0, uint32_t t1, float4* rays,
                                               uint32_t* rcount, uint32_t rcap) {
    const int S = w.slots;
    const int Bn = a.cur.B > 0 ? a.cur.B : 1;
    unsigned long long ninv = 0;
    for (uint32_t t = t0 + blockIdx.x * blockDim.x + threadIdx.x; t < t1; t += gridDim.x * blockDim.x) {
        ++ninv;
        uint32_t task = w.inv[t];
        uint32_t u = task >> 8;
        int s = (int)((task >> 4) & 15u), j = (int)(task & 15u);
        int2 ub = w.units[u];
        int pix = ub.x, b = ub.y;
        Rec y;
        if (s == 0) {
            rec_load(a.src, (size_t)pix * Bn + b, y);
        } else {
            ResDev R;
            R.planes = w.yrec; R.stride = (size_t)w.cap_units * (S - 1); R.estride = 1;
            rec_load(R, (size_t)u * (S - 1) + (s - 1), y);
        }
        int q = w.slot_pix[(size_t)pix * S + j];
        Domain D0 = pix_domain(&a.cur, pix, b);
        Domain Dj = pix_domain(slot_frame(a, j), q, slot_bin(a, j, b));
        bool geom_static = (a.temporal && j == 1) ? a.geom_static != 0 : true;
        Rec tmp;
        float pj = 0.f, Jj = 1.f;
        float term = 0.f;
        const size_t ti = ((size_t)u * S + s) * S + j;
        VisQ vq;
        vq.rays = rays; vq.counter = rcount; vq.cap = rcap; vq.target = (uint32_t)ti;
        if (slot_present(a, j, b) && shift_rec<false, kWalk>(y, D0, Dj, a.P, geom_static, tmp, pj, Jj, nullptr, &vq))
            term = w.slot_M[(size_t)pix * S + j] * pj * Jj;
        w.terms[ti] = term;
    }
    if (a.stats) {
        unsigned long long x = ninv;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if ((threadIdx.x & 31) == 0 && x) {
            atomicAdd(&a.stats->v[5], x);
            if (!a.temporal) atomicAdd(&a.stats->v[7], x);
        }
    }
}
__device__ __forceinline__ uint32_t inv_task_cap(const WaveDev& w) {
    return (uint32_t)w.cap_units * (uint32_t)w.slots * (uint32_t)(w.slots - 1);
}
// tasks [*lo, *hi) (lo null: from 0), read when the kernel starts
template <bool kWalk>
__global__ void __launch_bounds__(128, 8) shift_inv_kernel(const __grid_constant__ ReuseArgs a, const __grid_constant__ WaveDev w,
                                                          const uint32_t* lo, const uint32_t* hi, float4* rays, uint32_t* rcount,
                                                          uint32_t rcap) {
    const uint32_t cap = inv_task_cap(w);
    shift_inv_body<kWalk>(a, w, lo ? min(*lo, cap) : 0u, min(*hi, cap), rays, rcount, rcap);
}

// --------------------------------------------------------------------------------------------
// merge: MIS weights, streaming selection, output record.  One group of G lanes per unit (G the
// power of two >= slots, so 2, 4, 8 or 16 units per warp): lane s reads slot s's slot-table
// entries, source P0 word, shifted target and Jacobian and its row of MIS terms (each unit's
// arrays are contiguous, so a group's loads coalesce and are all in flight at once), computes its
// candidate's weight, and the group forms the streaming selection by shuffles in slot order (the
// same running sum and comparisons as one thread would make); the group then copies the selected
// record plane by plane.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void reuse_merge_body(const ReuseArgs& a, const WaveDev& w) {
    const uint32_t nunits = min(w.counters[0], (uint32_t)w.cap_units);
    const int S = w.slots;
    const FrameDev& C = a.cur;
    const int Bn = C.B > 0 ? C.B : 1;
    const bool pairwise = (a.P.flags & kFlagPairwiseMis) != 0u;
    const int G = S <= 2 ? 2 : S <= 4 ? 4 : S <= 8 ? 8 : 16;
    const int lane = threadIdx.x & 31;
    const int s = lane & (G - 1);                 // this lane's slot
    const int g0 = lane & ~(G - 1);               // first lane of the group
    const unsigned gmask = (G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u)) << g0;
    const uint32_t groups = gridDim.x * (blockDim.x / G);
    const uint32_t first = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    // every lane of a warp runs the same number of iterations (the group index advances by the same
    // stride for all groups of the warp), so the warp-synchronous shuffles below see full groups
    const uint32_t warp_first = (blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) / G;
    for (uint32_t base = warp_first; base < nunits; base += groups) {
        const uint32_t u = first + (base - warp_first);
        const bool unit_ok = u < nunits;
        // loads in three dependent rounds instead of five: everything indexed by the unit first
        // (its pixel and bin, this slot's shifted target and Jacobian, this candidate's row of MIS
        // terms), then the pixel's slot count with this slot's table entries, then the slot
        // pixel's occupancy word with its P0 word
        int2 ub = make_int2(0, 0);
        float pyu = 0.f, ju = 0.f;
        float Trow[kMaxSlots];
#pragma unroll
        for (int j = 0; j < kMaxSlots; ++j) Trow[j] = 0.f;
        if (unit_ok) {
            ub = w.units[u];
            if (s < S) {
                if (s > 0) { pyu = w.py[(size_t)u * S + s]; ju = w.jac[(size_t)u * S + s]; }
                const float* T = w.terms + ((size_t)u * S + s) * S;
#pragma unroll
                for (int j = 0; j < kMaxSlots; ++j)
                    if (j < S) Trow[j] = T[j];
            }
        }
        const int pix = ub.x, b = ub.y;
        int n = 0, q = 0;
        float Mraw = 0.f;
        if (unit_ok) {
            n = (int)w.nslot[pix];
            if (s < S) { q = w.slot_pix[(size_t)pix * S + s]; Mraw = w.slot_M[(size_t)pix * S + s]; }
        }
        const bool mine = s < n;
        // this lane's slot: confidence, source P0 word, shifted target and Jacobian
        float M = 0.f, py = 0.f, J = 0.f, ph = 0.f, Wx = 0.f;
        bool ok = false;
        if (mine) {
            // an absent domain (a bin outside the histogram) takes no part in the MIS
            const bool present = slot_present(a, s, b);
            M = present ? Mraw : 0.f;
            const ResDev* R = slot_res(a, s);
            const FrameDev* Fs = slot_frame(a, s);
            const int Bs = Fs->B > 0 ? Fs->B : 1;
            const int sb = slot_bin(a, s, b);
            uint32_t word = 0u;
            float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (present) {
                word = R->occ[(size_t)q * R->words + (sb >> 5)];
                p0 = *res_at(*R, 0, (size_t)q * Bs + sb);
            }
            if ((word >> (sb & 31)) & 1u) {
                ph = p0.y; Wx = p0.x;
                if (s == 0) { py = p0.y; J = 1.f; }
                else { py = pyu; J = ju; }
                ok = py > 0.f;
            }
        }
        // every shuffle below runs on the whole warp in loops bounded by S (uniform per launch):
        // the groups of a warp hold units with different slot counts n <= S
        const float M0 = __shfl_sync(0xFFFFFFFFu, M, g0);
        const float py0 = __shfl_sync(0xFFFFFFFFu, py, g0);
        const bool pw = pairwise && n > 1;
        // pairwise MIS: pair i = {canonical with confidence M_0/k, domain i with M_i}, a two-technique
        // balance heuristic at the same y weighted by (M_i + M_0/k) / sum M.  Explicitly rounded
        // operations (no contraction into FMAs), so that pairwise MIS with one reused domain
        // reproduces the balance heuristic.
        float Msum = 0.f;
        for (int i = 0; i < S; ++i) {
            const float Mi = __shfl_sync(0xFFFFFFFFu, M, g0 + i);
            if (i < n) Msum = __fadd_rn(Msum, Mi);
        }
        const float Mck = pw ? __fdiv_rn(M0, (float)(n - 1)) : 0.f;
        float mpw0 = 0.f;   // the canonical candidate's pairwise weight (lane 0 of the group)
        for (int i = 1; i < S; ++i) {
            const float Mi = __shfl_sync(0xFFFFFFFFu, M, g0 + i);
            if (pw && s == 0 && ok && i < n) {
                const float pc = __fmul_rn(Mck, py0);
                float alpha = __fdiv_rn(__fadd_rn(Mi, Mck), Msum);
                float ti = 0.f;
#pragma unroll
                for (int j = 1; j < kMaxSlots; ++j)
                    if (j == i) ti = slot_present(a, i, b) ? Trow[j] : 0.f;
                mpw0 = __fadd_rn(mpw0, __fmul_rn(alpha, __fdiv_rn(pc, __fadd_rn(pc, ti))));
            }
        }
        float wv = 0.f;
        if (ok) {
            float m;
            if (pw) {
                if (s == 0) {
                    m = mpw0;
                } else {
                    float alpha = __fdiv_rn(__fadd_rn(M, Mck), Msum);
                    float pi = __fdiv_rn(__fmul_rn(M, ph), J);
                    float pc = __fmul_rn(Mck, py);
                    m = __fmul_rn(alpha, __fdiv_rn(pi, __fadd_rn(pc, pi)));
                }
            } else {
                // generalized balance heuristic: this candidate's row of inverse-shift terms
                float num = s == 0 ? __fmul_rn(M0, py0) : __fdiv_rn(__fmul_rn(M, ph), J);
                float den = __fmul_rn(M0, py);
#pragma unroll
                for (int j = 1; j < kMaxSlots; ++j)
                    if (j < n)
                        den = __fadd_rn(den, (j == s) ? __fdiv_rn(__fmul_rn(M, ph), J) : slot_present(a, j, b) ? Trow[j] : 0.f);
                m = den > 0.f ? __fdiv_rn(num, den) : 0.f;
            }
            wv = m * py * Wx * J;
            if (!(wv > 0.f) || !isfinite(wv)) wv = 0.f;
        }
        // streaming selection in slot order: every lane forms the running sum up to its own slot
        float Ssum = 0.f, Sat = 0.f;
        for (int i = 0; i < S; ++i) {
            const float wi = __shfl_sync(0xFFFFFFFFu, wv, g0 + i);
            if (i < n && wi > 0.f) Ssum += wi;
            if (i == s) Sat = Ssum;
        }
        bool acc = false;
        if (mine && wv > 0.f) {
            const uint4 r = philox((uint32_t)pix, C.frame, ((uint32_t)a.pass << 8) | (uint32_t)s, P_MERGE | ((uint32_t)b << 8),
                                   a.P.seed);
            acc = u01(r.x) * Sat < wv;
        }
        const unsigned accm = __ballot_sync(0xFFFFFFFFu, acc) & gmask;
        const int sel = accm ? 31 - __clz(accm) - g0 : -1;
        const float pysel = __shfl_sync(0xFFFFFFFFu, py, g0 + (sel >= 0 ? sel : 0));
        if (unit_ok && sel >= 0) {
            // the selected record, planes s, s + G, ... copied by lane s (P0 takes the new W and target)
            const size_t dst = (size_t)pix * Bn + b;
            for (int k = s; k < 6; k += G) {
                float4 v;
                if (sel == 0) v = *res_at(a.src, k, dst);
                else v = w.yrec[(size_t)k * ((size_t)w.cap_units * (S - 1)) + (size_t)u * (S - 1) + (sel - 1)];
                if (k == 0) { v.x = Ssum / pysel; v.y = pysel; }
                *res_at(a.dst, k, dst) = v;
            }
            if (s == 0) atomicOr(&a.dst.occ[(size_t)pix * a.dst.words + (b >> 5)], 1u << (b & 31));
        }
        if (unit_ok && s == 0 && a.out) a.out[pix] = sel >= 0 ? pysel * (Ssum / pysel) : 0.f;
    }
}
__global__ void __launch_bounds__(128) reuse_merge_kernel(const __grid_constant__ ReuseArgs a, const __grid_constant__ WaveDev w) {
    reuse_merge_body(a, w);
}

// --------------------------------------------------------------------------------------------
// a reuse pass over all instances of a batch (tof_render_batch): one launch per stage.  Per-pixel
// stages map each block to its instance through blk0 (first block of each instance); persistent
// stages run over the instances one after another, every block pulling its share of each instance's
// tasks (the instances are independent, so no block waits for another).  Each block copies the
// instance's argument record to shared memory.
// --------------------------------------------------------------------------------------------
__global__ void reuse_reset_batch_kernel(const ReuseJob* __restrict__ J, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * kWaveCounters; t += gridDim.x * blockDim.x)
        J[t / kWaveCounters].w.counters[t % kWaveCounters] = 0u;
}
__global__ void __launch_bounds__(128) reuse_slots_batch_kernel(const ReuseJob* __restrict__ J, const int* __restrict__ blk0, int n) {
    __shared__ ReuseJob s;
    const int j = batch_job(blk0, n);
    block_copy(&s, &J[j]);
    __syncthreads();
    reuse_slots_body(s.a, s.w, s.p0, s.p1, (int)blockIdx.x - __ldg(&blk0[j]));
}
__global__ void __launch_bounds__(128) reuse_units_batch_kernel(const ReuseJob* __restrict__ J, const int* __restrict__ blk0, int n) {
    __shared__ ReuseJob s;
    const int j = batch_job(blk0, n);
    block_copy(&s, &J[j]);
    __syncthreads();
    reuse_units_body(s.a, s.w, s.p0, s.p1, (int)blockIdx.x - __ldg(&blk0[j]));
}
// stage k of the persistent part: 0 forward shifts, 1 their visibility, 2 inverse-task emission,
// 3 inverse shifts, 4 their visibility, 5 merge
template <int kStage>
__global__ void __launch_bounds__(128, 8) reuse_persist_batch_kernel(const ReuseJob* __restrict__ J, int n) {
    __shared__ ReuseJob s;
    for (int j = 0; j < n; ++j) {
        __syncthreads();
        block_copy(&s, &J[j]);
        __syncthreads();
        const ReuseArgs& a = s.a;
        const WaveDev& w = s.w;
        if constexpr (kStage == 0) shift_fwd_body<false>(a, w);
        else if constexpr (kStage == 1)
            vis_body(a.cur.g, w.rays, &w.counters[4], w.ray_cap, &w.counters[6], w.py, a.stats, 4, a.temporal ? -1 : 8);
        else if constexpr (kStage == 2) emit_inv_body(a, w);
        else if constexpr (kStage == 3)
            shift_inv_body<false>(a, w, 0u, min(w.counters[2], inv_task_cap(w)), w.rays, &w.counters[5], w.ray_cap);
        else if constexpr (kStage == 4)
            vis_body(a.temporal ? a.prev.g : a.cur.g, w.rays, &w.counters[5], w.ray_cap, &w.counters[7], w.terms, a.stats, -1,
                     a.temporal ? -1 : 9);
        else reuse_merge_body(a, w);
    }
}

cudaError_t launch_reuse_batch(const ReuseJob* J, int n, const int* blk_slots, int nblk_slots, const int* blk_units,
                               int nblk_units, int persist_blocks, int vis_blocks, cudaStream_t s) {
    note_launch(9);
    reuse_reset_batch_kernel<<<(n * kWaveCounters + 127) / 128, 128, 0, s>>>(J, n);
    reuse_slots_batch_kernel<<<nblk_slots, 128, 0, s>>>(J, blk_slots, n);
    reuse_units_batch_kernel<<<nblk_units, 128, 0, s>>>(J, blk_units, n);
    reuse_persist_batch_kernel<0><<<persist_blocks, 128, 0, s>>>(J, n);
    reuse_persist_batch_kernel<1><<<vis_blocks, 128, 0, s>>>(J, n);
    reuse_persist_batch_kernel<2><<<persist_blocks, 128, 0, s>>>(J, n);
    reuse_persist_batch_kernel<3><<<persist_blocks, 128, 0, s>>>(J, n);
    reuse_persist_batch_kernel<4><<<vis_blocks, 128, 0, s>>>(J, n);
    reuse_persist_batch_kernel<5><<<persist_blocks, 128, 0, s>>>(J, n);
    return cudaGetLastError();
}

// ev (optional): 7 events recorded around the stages (setup | forward shifts | their visibility and
// the inverse-task emission | inverse shifts | their visibility | merge) for per-stage timing
// One reuse pass.  With a second queue (w.rays2) and a second stream s2, the canonical samples'
// inverse shifts -- listed by the units kernel, independent of the forward shifts -- and their
// visibility run on s2 beside the forward shifts, their visibility and the inverse-task emission
// (fork / join events); the emitted inverse shifts follow after the join.  The shifts and
// segments are the same ones, so the results are those of the single sequence, which runs without
// rays2 (spatial passes, batches, the allocation-free form).  Small passes gain: their persistent
// kernels wait on a few long dependent chains while most of the GPU idles.
cudaError_t launch_reuse_wave(const ReuseArgs& a, const WaveDev& w, int p0, int p1, int persist_blocks, int vis_blocks,
                              cudaEvent_t* ev, cudaStream_t s, cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join) {
    cudaError_t e = cudaMemsetAsync(w.counters, 0, kWaveCounters * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int np = p1 - p0;
    if (np <= 0) return cudaSuccess;
    const bool beside = w.rays2 && s2 && fork && join;
    const GeomDev ginv = a.temporal ? a.prev.g : a.cur.g;   // inverse shifts land in the reused domain
    // only the generalized balance heuristic over three or more slots emits inverse shifts for the
    // shifted candidates (emit_inv_body); otherwise every inverse shift is a canonical one
    const bool emits = w.slots > 2 && !(a.P.flags & kFlagPairwiseMis);
    if (ev) cudaEventRecord(ev[0], s);
    note_launch();
    reuse_slots_kernel<<<(np + 127) / 128, 128, 0, s>>>(a, w, p0, p1);
    const long long nw = (long long)np * a.dst.words;
    note_launch();
    reuse_units_kernel<<<(unsigned)((nw + 127) / 128), 128, 0, s>>>(a, w, p0, p1);
    if (ev) cudaEventRecord(ev[1], s);
    const bool walk = (a.P.flags & kFlagTriangleWalk) != 0u;
    if (beside) {
        // the canonical inverse tasks are those listed so far
        e = cudaMemcpyAsync(&w.counters[8], &w.counters[2], sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, fork, 0);
        if (e != cudaSuccess) return e;
        note_launch(2);
        if (walk) shift_inv_kernel<true><<<persist_blocks, 128, 0, s2>>>(a, w, nullptr, &w.counters[8], w.rays2, &w.counters[9], w.ray2_cap);
        else shift_inv_kernel<false><<<persist_blocks, 128, 0, s2>>>(a, w, nullptr, &w.counters[8], w.rays2, &w.counters[9], w.ray2_cap);
        vis_kernel<<<vis_blocks, 128, 0, s2>>>(ginv, w.rays2, &w.counters[9], w.ray2_cap, &w.counters[10], w.terms, a.stats, -1,
                                               a.temporal ? -1 : 9);
        e = cudaEventRecord(join, s2);
        if (e != cudaSuccess) return e;
    }
    if (walk) { note_launch(); shift_fwd_kernel<true><<<persist_blocks, 128, 0, s>>>(a, w); }
    else { note_launch(); shift_fwd_kernel<false><<<persist_blocks, 128, 0, s>>>(a, w); }
    if (ev) cudaEventRecord(ev[2], s);
    // forward shifts land in the current frame; counter 4 of the stats counted them as successes
    note_launch();
    vis_kernel<<<vis_blocks, 128, 0, s>>>(a.cur.g, w.rays, &w.counters[4], w.ray_cap, &w.counters[6], w.py, a.stats, 4,
                                          a.temporal ? -1 : 8);
    if (emits) {
        note_launch();
        emit_inv_kernel<<<persist_blocks, 128, 0, s>>>(a, w);
    }
    if (ev) cudaEventRecord(ev[3], s);
    if (beside) {
        e = cudaStreamWaitEvent(s, join, 0);
        if (e != cudaSuccess) return e;
    }
    if (emits || !beside) {   // beside with nothing emitted: the second stream did every inverse shift
        const uint32_t* lo = beside ? &w.counters[8] : nullptr;
        if (walk) { note_launch(); shift_inv_kernel<true><<<persist_blocks, 128, 0, s>>>(a, w, lo, &w.counters[2], w.rays, &w.counters[5], w.ray_cap); }
        else { note_launch(); shift_inv_kernel<false><<<persist_blocks, 128, 0, s>>>(a, w, lo, &w.counters[2], w.rays, &w.counters[5], w.ray_cap); }
    }
    if (ev) cudaEventRecord(ev[4], s);
    if (emits || !beside) {
        note_launch();
        vis_kernel<<<vis_blocks, 128, 0, s>>>(ginv, w.rays, &w.counters[5], w.ray_cap, &w.counters[7], w.terms, a.stats, -1,
                                              a.temporal ? -1 : 9);
    }
    if (ev) cudaEventRecord(ev[5], s);
    note_launch();
    reuse_merge_kernel<<<persist_blocks, 128, 0, s>>>(a, w);
    if (ev) cudaEventRecord(ev[6], s);
    return cudaGetLastError();
}

// visibility segments queued by another stage (the ellipsoidal connection's initial wavefront)
cudaError_t launch_vis_queue(const GeomDev& g, const float4* rays, const uint32_t* counter, uint32_t cap, uint32_t* fetch,
                             float* target, int blocks, cudaStream_t s) {
    note_launch();
    vis_kernel<<<blocks, 128, 0, s>>>(g, rays, counter, cap, fetch, target, nullptr, -1, -1);
    return cudaGetLastError();
}

cudaError_t reuse_persist_blocks(int* out, int* vis_out) {
    int dev = 0, sms = 0, b1 = 0, b2 = 0, b3 = 0, b4 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, shift_fwd_kernel<false>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, shift_inv_kernel<false>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, reuse_merge_kernel, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, vis_kernel, 128, 0);
    int b = b1;
    if (b2 < b) b = b2;
    if (b3 < b) b = b3;
    *out = sms * (b > 0 ? b : 1);
    *vis_out = sms * (b4 > 0 ? b4 : 1);
    return cudaGetLastError();
}

}  // namespace tof
