// tof_bvh.cu -- GPU LBVH for the ToF ReSTIR hot path (sm_103a).
//
// The paper traces rays with DXR hardware BVHs (Sec. 6, Falcor on an RTX 3090); GB300 has no
// RT cores, so visibility runs on a software LBVH built here:
//   xform_kernel    rigid 3x4 object transform of every triangle corner, per frame
//   bounds / morton 30-bit Morton codes of triangle centroids in the centroid bounds (cubic cells)
//   radix sort      4 stable 8-bit LSD passes (tile histograms, one scan, ranked scatter)
//   karras_kernel   binary radix tree over the sorted codes (Karras, HPG 2012), ties broken by index
//   refit_kernel    leaf records in leaf order and bottom-up child boxes (one atomic per node;
//                   the second arriving thread continues, no thread waits)
//   etree_*_kernel  the ellipsoidal connection's hierarchy over triangle index ranges (boxes and
//                   areas, bottom-up: 8 levels per block in shared memory, then one block)
#include <cstdio>

#include <cooperative_groups.h>

#include "tof_internal.h"

namespace tof {

__device__ __forceinline__ float3 fx3(const float* M, float3 p, int r) {
    (void)r;
    return make_float3(M[0] * p.x + M[1] * p.y + M[2] * p.z + M[3], M[4] * p.x + M[5] * p.y + M[6] * p.z + M[7],
                       M[8] * p.x + M[9] * p.y + M[10] * p.z + M[11]);
}

// per triangle: world corners -> (v0, mat), (e1), (e2); centroid
__global__ void xform_kernel(int nt, const float* __restrict__ vloc, const uint32_t* __restrict__ tris,
                             const uint32_t* __restrict__ triobj, const uint32_t* __restrict__ objmat,
                             const float* __restrict__ xf, float4* __restrict__ tri_out, float4* __restrict__ cent) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    uint32_t o = triobj[t];
    const float* M = xf + 12 * (size_t)o;
    float3 v[3];
    for (int c = 0; c < 3; ++c) {
        uint32_t vi = tris[3 * (size_t)t + c];
        float3 p = make_float3(vloc[3 * (size_t)vi], vloc[3 * (size_t)vi + 1], vloc[3 * (size_t)vi + 2]);
        v[c] = fx3(M, p, 0);
    }
    float3 e1 = make_float3(v[1].x - v[0].x, v[1].y - v[0].y, v[1].z - v[0].z);
    float3 e2 = make_float3(v[2].x - v[0].x, v[2].y - v[0].y, v[2].z - v[0].z);
    tri_out[3 * (size_t)t] = make_float4(v[0].x, v[0].y, v[0].z, __int_as_float((int)objmat[o]));
    tri_out[3 * (size_t)t + 1] = make_float4(e1.x, e1.y, e1.z, 0.f);
    tri_out[3 * (size_t)t + 2] = make_float4(e2.x, e2.y, e2.z, 0.f);
    if (cent) cent[t] = make_float4((v[0].x + v[1].x + v[2].x) / 3.0f, (v[0].y + v[1].y + v[2].y) / 3.0f,
                                    (v[0].z + v[1].z + v[2].z) / 3.0f, 0.f);
}

// order-preserving float <-> uint for atomic min / max
__device__ __forceinline__ uint32_t fenc(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fdec(uint32_t u) { return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u); }

__global__ void bounds_kernel(int n, const float4* __restrict__ cent, uint32_t* __restrict__ bb) {
    __shared__ uint32_t s[6];
    if (threadIdx.x < 3) s[threadIdx.x] = 0xFFFFFFFFu;
    else if (threadIdx.x < 6) s[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 c = cent[i];
        atomicMin(&s[0], fenc(c.x)); atomicMin(&s[1], fenc(c.y)); atomicMin(&s[2], fenc(c.z));
        atomicMax(&s[3], fenc(c.x)); atomicMax(&s[4], fenc(c.y)); atomicMax(&s[5], fenc(c.z));
    }
    __syncthreads();
    if (threadIdx.x < 3) atomicMin(&bb[threadIdx.x], s[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&bb[threadIdx.x], s[threadIdx.x]);
}

__device__ __forceinline__ uint32_t expand10(uint32_t v) {
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void morton_kernel(int n, const float4* __restrict__ cent, const uint32_t* __restrict__ bb,
                              uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float lo[3] = {fdec(bb[0]), fdec(bb[1]), fdec(bb[2])}, hi[3] = {fdec(bb[3]), fdec(bb[4]), fdec(bb[5])};
    float4 c = cent[i];
    float cc[3] = {c.x, c.y, c.z};
    uint32_t q[3];
    // one scale for all axes (the largest extent): in a flat scene the top-level splits then cut
    // the long axes, instead of slicing the thin one into wide, flat boxes that every grazing ray
    // crosses (about 11 % lower SAH cost on a 20 m x 12.5 m x 2 m terrain scene)
    const float ext = fmaxf(fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]), 1e-20f);
    for (int k = 0; k < 3; ++k) {
        float t = (cc[k] - lo[k]) / ext * 1024.0f;
        q[k] = (uint32_t)fminf(fmaxf(t, 0.f), 1023.f);
    }
    keys[i] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    vals[i] = (uint32_t)i;
}

// ---- radix sort: 2048-key tiles --------------------------------------------------------------
constexpr int kTile = 2048;

__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t* __restrict__ keys, int n, int shift,
                                                         uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    int base = blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += 256) {
        int g = base + i;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of n words in place (single block of 1024 threads)
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* __restrict__ data, int n) {
    __shared__ uint32_t part[1024];
    int per = (n + 1023) / 1024;
    int b = threadIdx.x * per, e = min(n, b + per);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += data[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int i = b; i < e; ++i) { uint32_t v = data[i]; data[i] = run; run += v; }
}

__global__ void __launch_bounds__(256) radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                            uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int n,
                                                            int shift, const uint32_t* __restrict__ offs, int ntiles) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[8][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[tid * ntiles + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kTile / 256; ++r) {
        for (int k = 0; k < 8; ++k) wc[k][tid] = 0u;
        __syncthreads();
        int i = blockIdx.x * kTile + r * 256 + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t dg = (key >> shift) & 255u;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, valid ? dg : 256u + (uint32_t)lane);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wc[warp][dg] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = base[dg] + rank;
            for (int w = 0; w < warp; ++w) off += wc[w][dg];
            kout[off] = key;
            vout[off] = vin[i];
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < 8; ++w) tot += wc[w][tid];
        base[tid] += tot;
        __syncthreads();
    }
}

// The same four passes in one cooperative launch of one block per tile (all resident): per pass
// the tile histograms, a grid-wide sync, each block's digit offsets -- the digit totals' exclusive
// scan plus the digit's count in the earlier tiles, the global scan above restated per block --
// the same stable scatter, and a grid-wide sync.  Sorted keys and values are those of the
// separate launches (after four passes back in k0 / v0).
__global__ void __launch_bounds__(256) radix_sort_coop_kernel(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int n,
                                                              uint32_t* __restrict__ hist, int ntiles) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ uint32_t h[256];
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[8][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int shift = 0; shift < 32; shift += 8) {
        h[tid] = 0u;
        __syncthreads();
        const int t0 = blockIdx.x * kTile;
        for (int i = tid; i < kTile; i += 256) {
            const int g = t0 + i;
            if (g < n) atomicAdd(&h[(__ldcg(&ki[g]) >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[tid * ntiles + blockIdx.x] = h[tid];
        __threadfence();
        grid.sync();
        uint32_t tot = 0u, before = 0u;
        for (int t = 0; t < ntiles; ++t) {
            const uint32_t c = __ldcg(&hist[tid * ntiles + t]);
            tot += c;
            if (t < (int)blockIdx.x) before += c;
        }
        h[tid] = tot;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {   // inclusive scan of the digit totals
            const uint32_t v = tid >= off ? h[tid - off] : 0u;
            __syncthreads();
            h[tid] += v;
            __syncthreads();
        }
        base[tid] = h[tid] - tot + before;
        for (int r = 0; r < kTile / 256; ++r) {
            for (int k = 0; k < 8; ++k) wc[k][tid] = 0u;
            __syncthreads();
            const int i = t0 + r * 256 + tid;
            const bool valid = i < n;
            const uint32_t key = valid ? __ldcg(&ki[i]) : 0u;
            const uint32_t dg = (key >> shift) & 255u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, valid ? dg : 256u + (uint32_t)lane);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0) wc[warp][dg] = __popc(peers);
            __syncthreads();
            if (valid) {
                uint32_t off = base[dg] + rank;
                for (int w = 0; w < warp; ++w) off += wc[w][dg];
                ko[off] = key;
                vo[off] = __ldcg(&vi[i]);
            }
            __syncthreads();
            uint32_t add = 0;
            for (int w = 0; w < 8; ++w) add += wc[w][tid];
            base[tid] += add;
            __syncthreads();
        }
        __threadfence();
        grid.sync();
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
}

// ---- Karras 2012 hierarchy --------------------------------------------------------------------
__device__ __forceinline__ int delta(const uint32_t* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    uint32_t a = k[i], b = k[j];
    if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clz(a ^ b);
}

__global__ void karras_kernel(int n, const uint32_t* __restrict__ keys, int* __restrict__ child, int* __restrict__ parent_int,
                              int* __restrict__ parent_leaf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0;
    int div = 2;
    int t = (l + div - 1) / div;
    while (true) {
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
        if (t == 1) break;
        div <<= 1;
        t = (l + div - 1) / div;
    }
    int g = i + s * d + (d < 0 ? -1 : 0);
    int left = min(i, j) == g ? ~g : g;
    int right = max(i, j) == g + 1 ? ~(g + 1) : g + 1;
    child[2 * i] = left;
    child[2 * i + 1] = right;
    if (left < 0) parent_leaf[~left] = i; else parent_int[left] = i;
    if (right < 0) parent_leaf[~right] = i; else parent_int[right] = i;
    if (i == 0) parent_int[0] = -1;
}

struct Box { float lo[3], hi[3]; };

__device__ __forceinline__ Box tri_box(const float4* __restrict__ tri, int t) {
    float4 a = tri[3 * (size_t)t], e1 = tri[3 * (size_t)t + 1], e2 = tri[3 * (size_t)t + 2];
    float v[3][3] = {{a.x, a.y, a.z}, {a.x + e1.x, a.y + e1.y, a.z + e1.z}, {a.x + e2.x, a.y + e2.y, a.z + e2.z}};
    Box b;
    for (int k = 0; k < 3; ++k) {
        float lo = fminf(v[0][k], fminf(v[1][k], v[2][k])), hi = fmaxf(v[0][k], fmaxf(v[1][k], v[2][k]));
        float pad = 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-6f;   // conservative against rounding
        b.lo[k] = lo - pad; b.hi[k] = hi + pad;
    }
    return b;
}
__device__ __forceinline__ Box node_box(const float4* N) {
    float4 n0 = __ldcg(N), n1 = __ldcg(N + 1), n2 = __ldcg(N + 2);
    Box b;
    b.lo[0] = fminf(n0.x, n1.x); b.hi[0] = fmaxf(n0.y, n1.y);
    b.lo[1] = fminf(n0.z, n1.z); b.hi[1] = fmaxf(n0.w, n1.w);
    b.lo[2] = fminf(n2.x, n2.z); b.hi[2] = fmaxf(n2.y, n2.w);
    return b;
}

// arrival counter of a node: acquire-release at device scope, so that the second arrival sees the
// node the first arrival wrote below it (release of its writes, acquire of the sibling's)
__device__ __forceinline__ uint32_t arrive_acq_rel(uint32_t* p) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__global__ void refit_kernel(int n, const uint32_t* __restrict__ prim, const float4* __restrict__ tri, float4* __restrict__ leaf,
                             float4* nodes, const int* __restrict__ child, const int* __restrict__ parent_int,
                             const int* __restrict__ parent_leaf, uint32_t* __restrict__ counter) {
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= n) return;
    int t = (int)prim[L];
    float4 a = tri[3 * (size_t)t];
    leaf[3 * (size_t)L] = make_float4(a.x, a.y, a.z, __int_as_float(t));
    leaf[3 * (size_t)L + 1] = tri[3 * (size_t)t + 1];
    leaf[3 * (size_t)L + 2] = tri[3 * (size_t)t + 2];
    if (n == 1) return;
    int p = parent_leaf[L];
    int guard = n;   // depth of a valid hierarchy is below n
    while (p >= 0 && --guard >= 0) {
        if (arrive_acq_rel(&counter[p]) == 0u) return;   // first arrival: the sibling finishes p
        int c[2] = {child[2 * p], child[2 * p + 1]};
        Box b[2];
        for (int k = 0; k < 2; ++k) b[k] = c[k] < 0 ? tri_box(tri, (int)prim[~c[k]]) : node_box(nodes + 4 * (size_t)c[k]);
        float4* N = nodes + 4 * (size_t)p;
        N[0] = make_float4(b[0].lo[0], b[0].hi[0], b[0].lo[1], b[0].hi[1]);
        N[1] = make_float4(b[1].lo[0], b[1].hi[0], b[1].lo[1], b[1].hi[1]);
        N[2] = make_float4(b[0].lo[2], b[0].hi[2], b[1].lo[2], b[1].hi[2]);
        N[3] = make_float4(__int_as_float(c[0]), __int_as_float(c[1]), 0.f, 0.f);
        p = parent_int[p];
    }
}

// ---- ellipsoidal-connection hierarchy (Sec. 5 "Ellipsoidal Path Connection": nodes weighted by
// the area of the triangles below them).  The implicit binary tree over triangle index ranges
// (GeomDev::enode): eP leaves (a power of two >= nt), node n with children 2n and 2n + 1.
constexpr int kEllBlock = 256;

__device__ __forceinline__ void enode_merge(float4 alo, float4 ahi, float4 blo, float4 bhi, float4& lo, float4& hi) {
    lo = make_float4(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z), alo.w + blo.w);
    hi = make_float4(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z), 0.f);
}

// leaves and the `levels` levels above them, one block per blockDim.x leaves (blockDim.x divides P)
__global__ void __launch_bounds__(kEllBlock) etree_low_kernel(int nt, int P, int levels, const float4* __restrict__ tri,
                                                              float4* __restrict__ node) {
    __shared__ float4 slo[kEllBlock], shi[kEllBlock];
    const int t = threadIdx.x;
    const int i = blockIdx.x * blockDim.x + t;
    float4 lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f), hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
    if (i < nt) {
        float4 a = tri[3 * (size_t)i], b = tri[3 * (size_t)i + 1], c = tri[3 * (size_t)i + 2];
        float3 v0 = make_float3(a.x, a.y, a.z), e1 = make_float3(b.x, b.y, b.z), e2 = make_float3(c.x, c.y, c.z);
        float3 v1 = make_float3(v0.x + e1.x, v0.y + e1.y, v0.z + e1.z), v2 = make_float3(v0.x + e2.x, v0.y + e2.y, v0.z + e2.z);
        float cx = e1.y * e2.z - e1.z * e2.y, cy = e1.z * e2.x - e1.x * e2.z, cz = e1.x * e2.y - e1.y * e2.x;
        lo = make_float4(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)),
                         0.5f * sqrtf(cx * cx + cy * cy + cz * cz));
        hi = make_float4(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)), 0.f);
    }
    node[2 * (size_t)(P + i)] = lo;
    node[2 * (size_t)(P + i) + 1] = hi;
    slo[t] = lo;
    shi[t] = hi;
    for (int h = 1; h <= levels; ++h) {
        __syncthreads();
        const int cnt = (int)blockDim.x >> h;
        float4 nlo, nhi;
        if (t < cnt) enode_merge(slo[2 * t], shi[2 * t], slo[2 * t + 1], shi[2 * t + 1], nlo, nhi);
        __syncthreads();
        if (t < cnt) {
            slo[t] = nlo;
            shi[t] = nhi;
            const size_t n = (size_t)((P + (int)(blockIdx.x * blockDim.x)) >> h) + t;
            node[2 * n] = nlo;
            node[2 * n + 1] = nhi;
        }
    }
}

// the levels above: nodes [cnt, 2 cnt) for cnt = lowest / 2, ..., 1, one block
__global__ void __launch_bounds__(1024) etree_top_kernel(int lowest, float4* node) {
    for (int cnt = lowest >> 1; cnt >= 1; cnt >>= 1) {
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const size_t n = (size_t)cnt + t;
            float4 lo, hi;
            enode_merge(node[4 * n], node[4 * n + 1], node[4 * n + 2], node[4 * n + 3], lo, hi);
            node[2 * n] = lo;
            node[2 * n + 1] = hi;
        }
        __syncthreads();
    }
}

// ---- host launchers --------------------------------------------------------------------------
static inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_xform(int nt, const float* vloc, const uint32_t* tris, const uint32_t* triobj, const uint32_t* objmat,
                         const float* xf, float4* tri_out, float4* cent, cudaStream_t s) {
    note_launch();
    xform_kernel<<<blocks(nt, 256), 256, 0, s>>>(nt, vloc, tris, triobj, objmat, xf, tri_out, cent);
    return cudaGetLastError();
}

// full build of the hierarchy (prim order, children, parents) from the centroids
cudaError_t launch_build_topology(int n, const float4* cent, uint32_t* bb, uint32_t* keys, uint32_t* vals, uint32_t* keys2,
                                  uint32_t* vals2, uint32_t* hist, int* child, int* parent_int, int* parent_leaf,
                                  uint32_t** prim_out, cudaStream_t s) {
    // centroid bounds start empty: encoded minima at 0xFFFFFFFF, maxima at 0
    cudaError_t e = cudaMemsetAsync(bb, 0xFF, 3 * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bb + 3, 0, 3 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    note_launch();
    bounds_kernel<<<min(1024u, blocks(n, 256)), 256, 0, s>>>(n, cent, bb);
    note_launch();
    morton_kernel<<<blocks(n, 256), 256, 0, s>>>(n, cent, bb, keys, vals);
    int ntiles = (n + kTile - 1) / kTile;
    uint32_t *ki = keys, *vi = vals, *ko = keys2, *vo = vals2;
    // one cooperative launch when every tile's block can be resident at once
    // resident blocks of the cooperative sort on each device (found once per device and process)
    static std::atomic<int> coop_blocks[64];
    static std::atomic<bool> coop_known[64];
    int dev = 0;
    cudaGetDevice(&dev);
    int coop_cap = 0;
    if (dev >= 0 && dev < 64) {
        if (!coop_known[dev].load()) {
            int sms = 0, per = 0, coop = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, radix_sort_coop_kernel, 256, 0);
            cudaGetLastError();
            coop_blocks[dev].store(coop ? sms * per : 0);
            coop_known[dev].store(true);
        }
        coop_cap = coop_blocks[dev].load();
    }
    if (ntiles <= coop_cap) {
        int nn = n, nt = ntiles;
        void* args[] = {&ki, &vi, &ko, &vo, &nn, &hist, &nt};
        note_launch();
        e = cudaLaunchCooperativeKernel((const void*)radix_sort_coop_kernel, dim3(ntiles), dim3(256), args, 0, s);
        if (e != cudaSuccess) return e;
        if (n > 1) { note_launch(); karras_kernel<<<blocks(n - 1, 256), 256, 0, s>>>(n, ki, child, parent_int, parent_leaf); }
        *prim_out = vi;
        return cudaGetLastError();
    }
    for (int shift = 0; shift < 32; shift += 8) {
        note_launch();
        radix_hist_kernel<<<ntiles, 256, 0, s>>>(ki, n, shift, hist, ntiles);
        note_launch();
        scan_kernel<<<1, 1024, 0, s>>>(hist, 256 * ntiles);
        note_launch();
        radix_scatter_kernel<<<ntiles, 256, 0, s>>>(ki, vi, ko, vo, n, shift, hist, ntiles);
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    // after 4 passes the sorted keys / prims are back in keys / vals
    if (n > 1) { note_launch(); karras_kernel<<<blocks(n - 1, 256), 256, 0, s>>>(n, ki, child, parent_int, parent_leaf); }
    *prim_out = vi;
    return cudaGetLastError();
}

cudaError_t launch_refit(int n, const uint32_t* prim, const float4* tri, float4* leaf, float4* nodes, const int* child,
                         const int* parent_int, const int* parent_leaf, uint32_t* counter, cudaStream_t s) {
    if (n > 1) {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t) * (size_t)(n - 1), s);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    refit_kernel<<<blocks(n, 256), 256, 0, s>>>(n, prim, tri, leaf, nodes, child, parent_int, parent_leaf, counter);
    return cudaGetLastError();
}

cudaError_t launch_etree(int nt, int P, const float4* tri, float4* node, cudaStream_t s) {
    const int bs = P < kEllBlock ? P : kEllBlock;
    int levels = 0;
    while ((1 << levels) < bs) ++levels;
    note_launch();
    etree_low_kernel<<<P / bs, bs, 0, s>>>(nt, P, levels, tri, node);
    if (P / bs > 1) { note_launch(); etree_top_kernel<<<1, 1024, 0, s>>>(P / bs, node); }
    return cudaGetLastError();
}

}  // namespace tof
