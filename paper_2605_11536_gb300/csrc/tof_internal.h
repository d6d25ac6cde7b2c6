// tof_internal.h -- device-visible data layouts shared by the kernels and the host runtime of
// libtof.so (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

// number of objects of a scene (server -> context); hidden from the library's exports
extern "C" __attribute__((visibility("hidden"))) int tof_internal_scene_objects(struct tof_ctx* c, int32_t scene);

namespace tof {

constexpr int kMaxDepth = 5;        // surface vertices per path
constexpr int kMaxCand = 64;        // path trees per pixel
constexpr int kMaxNb = 8;           // spatial neighbours per pass
constexpr int kMaxSlots = 1 + kMaxNb;
constexpr int kStack = 64;          // BVH traversal stack
constexpr int kMaxBinsPerPixel = 32;  // distinct transient bins a pixel's initial candidates may hit
constexpr uint32_t kNoHit = 0xFFFFFFFFu;
constexpr uint32_t kFlagPairwiseMis = 4u;  // TOF_FLAG_PAIRWISE_MIS
constexpr uint32_t kFlagTriangleWalk = 64u;  // TOF_FLAG_TRIANGLE_WALK
constexpr uint32_t kFlagEllipsoid = 256u;    // TOF_FLAG_ELLIPSOID
constexpr int kEllMaxLevels = 22;           // ellipsoidal-connection hierarchies of up to 2^22 triangles

// bits of the context's device error word (read back by the host at the next synchronising call)
constexpr unsigned kErrBinOverflow = 1u;    // a pixel's initial candidates hit more distinct bins than it holds
constexpr unsigned kErrStackOverflow = 2u;  // a BVH traversal stack was full (a far child would have been dropped)
constexpr unsigned kErrVisitBudget = 4u;    // a BVH traversal visited more nodes than a valid hierarchy has

// kernel launches issued by the library in this process (every launch wrapper counts its kernels;
// a kernel recorded into a graph counts once, when it is recorded)
inline std::atomic<unsigned long long> g_kernel_launches{0};
inline void note_launch(unsigned n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// material record: (type, albedo, alpha, unused)
// triangle record (original order): 3 float4 = (v0.xyz, material id bits), (e1.xyz, 0), (e2.xyz, 0)
// triangle record (leaf order):     3 float4 = (v0.xyz, original id bits), (e1.xyz, 0), (e2.xyz, 0)
// internal node: 4 float4 = (c0 lo.x, hi.x, lo.y, hi.y), (c1 lo.x, hi.x, lo.y, hi.y),
//                           (c0 lo.z, hi.z, c1 lo.z, hi.z), (child0 bits, child1 bits, 0, 0)
//                child >= 0: internal node, child < 0: leaf ~child.
// adjacency (original order), nt * 3: across the edge opposite vertex i of triangle t,
// 4 * neighbour + the neighbour's vertex opposite that edge, or -1
// ellipsoidal-connection hierarchy: the implicit binary tree over triangle index ranges, eP (a
// power of two >= nt) leaves, node n in [1, 2 eP) with children 2n, 2n + 1, triangle t at leaf
// eP + t; 2 float4 per node = (lo.xyz, area of the triangles below), (hi.xyz, 0); padding leaves
// have area 0
struct GeomDev {
    const float4* tri;
    const float4* leaf;
    const float4* nodes;
    const float4* mats;
    const int* adj;
    const float4* enode;
    int eP;
    int nt;
    uint32_t version;
    unsigned* err;           // the context's device error word (kErr* bits), or null
};

// resolved light of one domain (Sec. 5 "Light Source")
struct LightDev {
    int kind;          // 0 none, 1 point, 2 spot (laser / confocal)
    float3 pos;        // point position or spot position
    float I;           // intensity (point) or laser power (spot)
    int s_tri;         // spot surface
    float s_b1, s_b2;
    float3 to_origin;  // spot -> laser origin
    float emit_len;    // laser origin -> spot
};

// one frame of one view: geometry, sensor, emitter, gate, G-buffer
struct FrameDev {
    GeomDev g;
    int mode, W, H;
    float3 pos, fwd, up;
    float fov_y;
    float3 wall_o, wall_u, wall_v;
    int etype;
    float3 epos, edir;
    float epower;
    const LightDev* laser;   // resolved laser spot (etype == 1)
    float L0, dL;            // gate, or (t0, width) of the bins
    int B;                   // 0 gated, else bins
    uint32_t frame;
    const float4* gb;        // (tri bits, b1, b2, t) per pixel
};

// reservoir buffer: 6 float4 words per entry, per-pixel confidence M and one occupancy bit per
// (pixel, bin).  Word k of entry i sits at planes[k * stride + i * estride]: structure of arrays
// (stride = entries, estride = 1; each word a plane read with 16-byte vectors) or array of
// structures (stride = 1, estride = 6; an entry's 96 bytes contiguous)
struct ResDev {
    float4* planes;
    size_t stride;           // SoA: W*H*max(B,1); AoS: 1
    size_t estride;          // SoA: 1; AoS: 6
    float* M;                // W*H
    uint32_t* occ;           // W*H*words, words = ceil(max(B,1)/32)
    int words;
};

struct ParamsDev {
    int depth, n_cand, n_spatial, radius, n_spatial_iters, temporal;
    float m_cap;
    int newton_max_iter;
    float newton_tol_frac, jac_max, d_min, ray_eps;
    uint32_t flags;
    float shrink_k;          // Sec. 4.4 shrink mapping (<= 1: off)
    int shrink_fine;         // trees kept in the gate itself
    uint64_t seed;
};

// shift statistics (device, accumulated): newton calls, iterations, successes, forward shift
// calls, forward successes, inverse shift calls, spatial forward calls, spatial inverse calls,
// visibility segments traced by vis_kernel for the spatial forward / inverse shifts
struct StatsDev {
    unsigned long long v[10];
};

struct GbufArgs {
    FrameDev F;
    float4* gb;
    ParamsDev P;
    int tile_w;              // pixel tile width (a power of two); tile height = threads / tile_w
};

struct InitArgs {
    FrameDev F;
    ResDev dst;
    ParamsDev P;
    float* out;              // gated image if this is the last stage (else null)
    int tile_w;
    int wave;                // a staged batch runs this instance's initial stage as the bounce
                             // wavefront: initial_gated_batch_kernel skips it
};

struct ReuseArgs {
    FrameDev cur, prev;
    ResDev src;              // canonical reservoirs (current frame)
    ResDev prv;              // previous frame's final reservoirs (temporal)
    ResDev dst;
    ParamsDev P;
    int temporal;            // 1: temporal pass, 0: spatial pass
    int binpass;             // 1: bin pass (slots 1, 2 = the same pixel's bins b - 1, b + 1)
    int pass;                // 0 temporal, 1.. spatial, 8 bin pass
    int geom_static;         // previous and current geometry identical
    float* out;              // gated image if last stage
    StatsDev* stats;
};

// wavefront scratch of one reuse pass (tof_reuse.cu); S = slots per pixel (1 canonical + reused)
struct WaveDev {
    int slots;              // S
    int cap_units;          // merge units (pixel, bin) per launch
    int* slot_pix;          // npix * S
    float* slot_M;          // npix * S
    uint8_t* nslot;         // npix
    int2* units;            // cap_units
    uint32_t* fwd;          // cap_units * (S - 1)   forward tasks (unit << 4 | slot)
    uint32_t* inv;          // cap_units * S * (S-1) inverse tasks (unit << 8 | s << 4 | j)
    float4* yrec;           // 6 planes of cap_units * (S - 1) shifted records
    float* py;              // cap_units * S
    float* jac;             // cap_units * S
    float* terms;           // cap_units * S * S
    float4* rays;           // 2 * ray_cap: queued visibility segments of the shifts (VisQ)
    uint32_t ray_cap;
    float4* rays2;          // 2 * ray2_cap: the segments of the canonical samples' inverse shifts when
    uint32_t ray2_cap;      // those run beside the forward shifts (null: one queue, one sequence)
    uint32_t* counters;     // units, forward tasks, inverse tasks, overflow, forward rays, inverse rays,
                            // forward rays fetched, inverse rays fetched, [8] canonical inverse tasks
                            // (the task count after the units kernel), [9] / [10] their rays / fetched
};
constexpr int kWaveCounters = 12;

// wavefront of the gated initial stage with the ellipsoidal connection (tof_kernels.cu): the path
// trees record their vertices, their NEE candidates and the ellipsoidal requests; the vertices are
// placed in one pass over the requests, their visibility segments traced by vis_kernel, and the
// streaming RIS replayed per pixel in the trees' candidate order.  Slot (pixel, tree, vertex d) =
// (pixel * nc + tree) * depth + d - 1.
struct EllWaveDev {
    int nc, depth;
    float4* vtx;            // (tri bits, b1, b2, area pdf) of vertex d
    float2* vtx2;           // (prefix throughput beta, prefix length) at vertex d
    float2* acand;          // (f / p, tau) of the tree's NEE candidate ending at vertex d (0: none)
    float* bw;              // f / p of the ellipsoidal candidate from vertex d (0: none; zeroed when occluded)
    float4* bz;             // (z tri bits, b1, b2, tau) of that candidate
    float* bpt;             // the tree's area density of z (its pdf entry in the record)
    uint32_t* req;          // ellipsoidal requests (slot indices)
    uint32_t req_cap;
    float4* rays;           // 2 * ray_cap: their visibility segments (VisQ, target = slot)
    uint32_t ray_cap;
    uint32_t* counters;     // requests, request fetch, segments, segment fetch
};

// wavefront of the gated initial stage without the ellipsoidal connection (tof_kernels.cu): the
// path trees of all pixels advance one bounce per round -- a persistent closest-hit kernel with lane
// refill traces the round's bounce rays, a shade kernel records each new vertex, queues its NEE
// candidate's light segment for vis_kernel and samples the next bounce -- and the streaming RIS is
// replayed per pixel in the trees' order.  Path p = pixel * nc + tree; slot (p, d) = p * depth + d - 1.
constexpr int kTreeWaveCounters = 16;
struct TreeWaveDev {
    int nc, depth;
    float4* vtx;            // per slot: (tri bits, b1, b2, area pdf) of vertex d
    float2* acand;          // per slot: (f / p, tau) of the NEE candidate at vertex d (0: none; zeroed when occluded)
    float4* ps0;            // per path: (throughput after the sampled bounce, prefix length, its pdf or -1 for a delta, 0)
    float4* ps1;            // per path: (position of the vertex the bounce leaves, 0)
    float4* rays[2];        // bounce rays towards vertex d in rays[d & 1]: (origin, tmax), (direction, path bits)
    float4* hits;           // per ray of the round: (tri bits or kNoHit, b1, b2, t)
    uint32_t path_cap;      // npix * nc: the most rays of a round
    float4* srays;          // light segments of the NEE candidates (VisQ; target 2 * slot, the candidate's weight)
    uint32_t sray_cap;
    uint32_t* counters;     // [d]: rays towards vertex d, [8 + d]: their fetch counter, [14] light segments, [15] their fetch
};

// one instance's reuse pass in a batched launch (tof_render_batch): its arguments, its wavefront
// scratch and its pixel range
struct ReuseJob {
    ReuseArgs a;
    WaveDev w;
    int p0, p1;
};

struct SplatArgs {
    ResDev src;
    int npix, B;
    float* out;
};

struct PtArgs {
    FrameDev F;
    ParamsDev P;
    int spp;
    float* out;
};

}  // namespace tof
