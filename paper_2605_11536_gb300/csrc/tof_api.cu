// tof_api.cu -- host runtime behind the C ABI of include/tof.h.
//
// Owns the device state (scenes with double-buffered world geometry and LBVH, views with the
// reservoirs / G-buffers / confidence of the current and previous frame), validates arguments,
// accounts device memory against the context's HBM budget and orders the per-frame stages of
// the ToF ReSTIR pipeline on the caller's stream (Sec. 3.2 stages (1)-(4)).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tof.h"
#include "tof_internal.h"

namespace tof {
cudaError_t launch_gbuffer(const GbufArgs& a, int tile_h, cudaStream_t s);
cudaError_t launch_initial(const InitArgs& a, int tile_h, unsigned* err, cudaStream_t s);
cudaError_t launch_initial_ell_wave(const InitArgs& a, const EllWaveDev& w, int tile_h, int place_blocks, int vis_blocks,
                                    cudaStream_t s);
cudaError_t launch_initial_tree_wave(const InitArgs& a, const TreeWaveDev& w, int tile_h, int hit_blocks, int vis_blocks,
                                     cudaStream_t s);
cudaError_t tree_hit_blocks(int* out);
cudaError_t launch_initial_ell_tree_wave(const InitArgs& a, const TreeWaveDev& tw, const EllWaveDev& ell, int tile_h, int hit_blocks,
                                         int place_blocks, int vis_blocks, cudaStream_t s);
cudaError_t ell_place_blocks(int* out);
cudaError_t launch_initial_shrink(const InitArgs& a, int tile_h, cudaStream_t s);
cudaError_t launch_reuse_wave(const ReuseArgs& a, const WaveDev& w, int p0, int p1, int persist_blocks, int vis_blocks,
                              cudaEvent_t* ev, cudaStream_t s, cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join);
cudaError_t reuse_persist_blocks(int* out, int* vis_out);
cudaError_t launch_splat(const SplatArgs& a, cudaStream_t s);
cudaError_t launch_pt(const PtArgs& a, cudaStream_t s);
cudaError_t launch_laser(const GeomDev& g, float3 o, float3 d, float power, LightDev* out, cudaStream_t s);
cudaError_t launch_xform(int nt, const float* vloc, const uint32_t* tris, const uint32_t* triobj, const uint32_t* objmat,
                         const float* xf, float4* tri_out, float4* cent, cudaStream_t s);
cudaError_t launch_build_topology(int n, const float4* cent, uint32_t* bb, uint32_t* keys, uint32_t* vals, uint32_t* keys2,
                                  uint32_t* vals2, uint32_t* hist, int* child, int* parent_int, int* parent_leaf,
                                  uint32_t** prim_out, cudaStream_t s);
cudaError_t launch_etree(int nt, int P, const float4* tri, float4* node, cudaStream_t s);
cudaError_t launch_refit(int n, const uint32_t* prim, const float4* tri, float4* leaf, float4* nodes, const int* child,
                         const int* parent_int, const int* parent_leaf, uint32_t* counter, cudaStream_t s);
cudaError_t launch_gbuffer_batch(const GbufArgs* A, const int* blk0, int n, int blocks, cudaStream_t s);
cudaError_t launch_initial_batch(const InitArgs* A, const int* blk0, int n, int blocks, cudaStream_t s);
cudaError_t launch_reuse_batch(const ReuseJob* J, int n, const int* blk_slots, int nblk_slots, const int* blk_units,
                               int nblk_units, int persist_blocks, int vis_blocks, cudaStream_t s);
}  // namespace tof

using namespace tof;

namespace {

struct DevAlloc {
    void* p = nullptr;
    size_t bytes = 0;
};

struct SceneH {
    bool alive = false;
    int nv = 0, nt = 0, nobj = 0, nmat = 0;
    float* vloc = nullptr;
    uint32_t *tris = nullptr, *triobj = nullptr, *objmat = nullptr;
    float4* mats = nullptr;
    float* xf = nullptr;
    float4* cent = nullptr;
    uint32_t *keys = nullptr, *vals = nullptr, *keys2 = nullptr, *vals2 = nullptr, *hist = nullptr, *bb = nullptr;
    uint32_t* prim = nullptr;   // points into vals after a build
    int *child = nullptr, *parent_int = nullptr, *parent_leaf = nullptr;
    uint32_t* counter = nullptr;
    int* adj = nullptr;          // edge adjacency (original triangle order)
    float4* tri[2] = {nullptr, nullptr};
    float4* leaf[2] = {nullptr, nullptr};
    float4* nodes[2] = {nullptr, nullptr};
    float4* enode[2] = {nullptr, nullptr};   // ellipsoidal-connection hierarchy (null above 2^22 triangles)
    int eP = 0;
    uint32_t version[2] = {0, 0};
    std::vector<float> xfh[2];
    int cur = 0;
    bool built = false;
};

struct ResH {
    float4* planes = nullptr;
    float* M = nullptr;
    uint32_t* occ = nullptr;
    size_t entries = 0;
    int layout = TOF_LAYOUT_SOA;
    int words = 1;
    ResDev dev() const {
        ResDev r;
        r.planes = planes; r.M = M; r.occ = occ; r.words = words;
        r.stride = layout == TOF_LAYOUT_AOS ? 1 : entries;
        r.estride = layout == TOF_LAYOUT_AOS ? 6 : 1;
        return r;
    }
};

struct ViewH {
    bool alive = false;
    int scene = -1, W = 0, H = 0, B = 0;
    float4* gb[2] = {nullptr, nullptr};
    LightDev* laser[2] = {nullptr, nullptr};
    ResH res[3];
    FrameDev fd[2];
    int geom_slot[2] = {0, 0};
    uint32_t geom_version[2] = {0, 0};
    int cur = 0;
    int prev_final = -1;
    bool has_prev = false;
    StatsDev* stats = nullptr;
    cudaStream_t last_stream = nullptr;
    bool profile = false;
    cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ran[5] = {false, false, false, false, false};
    // wavefront scratch of the reuse passes (sized on first use)
    WaveDev wave;
    int wave_slots = 0, wave_cap = 0;
    std::vector<cudaEvent_t> kev;   // kReuseEvents events per timed spatial launch group
    size_t kev_used = 0;
    void* wave_ptrs[12] = {nullptr};
    // direct renders: the second visibility queue, stream and fork / join events that let the
    // canonical inverse shifts run beside the forward shifts (created on first use)
    float4* rays2 = nullptr;
    uint32_t ray2_cap = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    // the ellipsoidal connection's initial wavefront (gated views; sized on first use)
    EllWaveDev ell;
    size_t ell_slots = 0;        // pixels x trees x depth it holds
    void* ell_ptrs[9] = {nullptr};
    TreeWaveDev tw;              // the gated initial stage's bounce wavefront
    size_t tw_paths = 0;         // pixels x trees it holds
    void* tw_ptrs[9] = {nullptr};
    tof_tuning tune = {16, 8, 0, TOF_LAYOUT_SOA};   // launch shapes and reservoir layout (autotuner)
};

}  // namespace

constexpr int kBatchSlots = 8;   // batch graphs that may be in flight at once (launches of one graph serialise)

struct tof_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    std::string err;
    std::vector<SceneH> scenes;
    std::vector<ViewH> views;
    std::vector<DevAlloc> allocs;
    uint32_t version_counter = 0;
    unsigned* d_err = nullptr;   // device error word (kErr* bits), set by kernels
    unsigned* h_err = nullptr;   // pinned host mirror of it, copied after every render on its stream
    float* d_scratch = nullptr;  // laser spot of plain PT renders
    int persist_blocks = 0;      // resident blocks of the persistent reuse kernels (all SMs)
    int ell_blocks = 0;          // resident blocks of the ellipsoidal placement kernel (all SMs)
    int hit_blocks = 0;          // resident blocks of the wavefront closest-hit kernel (all SMs)
    int vis_blocks = 0;          // resident blocks of the visibility kernel (all SMs)
    int sms = 0;                 // streaming multiprocessors
    // batched rendering: stream pool, fork / join events, and the instantiated graph
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t batch_exec[kBatchSlots] = {};   // one instantiated graph per batch slot
    // staged batches: argument tables per slot (pinned host staging, device copy) and the event after
    // the slot's last launch (the staging buffer is rewritten only once that launch has finished)
    void* bstage[kBatchSlots] = {};
    size_t bstage_bytes[kBatchSlots] = {};
    unsigned char* btab[kBatchSlots] = {};
    size_t btab_bytes[kBatchSlots] = {};
    cudaEvent_t bdone[kBatchSlots] = {};
    bool in_batch = false;
};

static tof_status fail(tof_ctx* c, tof_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

template <class T>
static tof_status dalloc(tof_ctx* c, T** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->budget && c->used + bytes > c->budget)
        return fail(c, TOF_EBUDGET, "%s: %zu bytes exceed the HBM budget (%llu of %llu used)", what, bytes,
                    (unsigned long long)c->used, (unsigned long long)c->budget);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, TOF_ENOMEM, "%s: cudaMalloc(%zu) failed: %s", what, bytes, cudaGetErrorString(e));
    }
    c->used += bytes;
    DevAlloc a;
    a.p = q; a.bytes = bytes;
    c->allocs.push_back(a);
    *p = (T*)q;
    return TOF_OK;
}
static void dfree(tof_ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i)
        if (c->allocs[i].p == p) {
            c->used -= c->allocs[i].bytes;
            c->allocs.erase(c->allocs.begin() + (long)i);
            break;
        }
    cudaFree(p);
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t _e = (call);                                                                     \
        if (_e != cudaSuccess) return fail(c, TOF_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));   \
    } while (0)
#define TRY(call)                          \
    do {                                   \
        tof_status _s = (call);            \
        if (_s != TOF_OK) return _s;       \
    } while (0)

static float3 v3f(const float* p) { return make_float3(p[0], p[1], p[2]); }

// turn error-word bits into a status: TOF_ECUDA naming every cause, the word cleared (on the device
// too) so that each error is reported once
static tof_status report_err_bits(tof_ctx* c, unsigned bits) {
    if (!bits) return TOF_OK;
    cudaMemset(c->d_err, 0, sizeof(unsigned));
    c->h_err[0] = 0u;
    return fail(c, TOF_ECUDA, "device error word 0x%x:%s%s%s (results since the last check are unreliable)", bits,
                (bits & kErrBinOverflow) ? " transient bin table overflow;" : "",
                (bits & kErrStackOverflow) ? " BVH traversal stack overflow (a subtree was skipped);" : "",
                (bits & kErrVisitBudget) ? " BVH traversal visit budget exhausted (malformed hierarchy);" : "");
}
// errors of earlier renders whose mirror copy has already landed (no wait)
static tof_status pending_err(tof_ctx* c) {
    const unsigned bits = c->h_err ? *(volatile unsigned*)c->h_err : 0u;
    return report_err_bits(c, bits);
}
// queue the mirror copy of the error word after a render (not while a batch graph is captured:
// the next direct render or tof_sync reads the word)
static void mirror_err(tof_ctx* c, cudaStream_t s, bool capturing) {
    if (!capturing) cudaMemcpyAsync(c->h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
}

static ParamsDev to_dev(const tof_params* p, uint64_t seed) {
    ParamsDev d;
    d.depth = p->depth; d.n_cand = p->n_cand; d.n_spatial = p->n_spatial; d.radius = p->radius;
    d.n_spatial_iters = p->n_spatial_iters; d.temporal = p->temporal; d.m_cap = p->m_cap;
    d.newton_max_iter = p->newton_max_iter; d.newton_tol_frac = p->newton_tol_frac; d.jac_max = p->jac_max;
    d.d_min = p->d_min; d.ray_eps = p->ray_eps; d.flags = p->flags; d.seed = seed;
    d.shrink_k = p->shrink_k; d.shrink_fine = p->shrink_fine;
    return d;
}

static tof_status check_params(tof_ctx* c, const tof_params* p, int transient) {
    if (!p) return fail(c, TOF_EINVAL, "params is NULL");
    if (p->depth < 1 || p->depth > kMaxDepth) return fail(c, TOF_EINVAL, "depth %d outside [1, %d]", p->depth, kMaxDepth);
    if (p->n_cand < 1 || p->n_cand > kMaxCand) return fail(c, TOF_EINVAL, "n_cand %d outside [1, %d]", p->n_cand, kMaxCand);
    if (p->n_spatial < 0 || p->n_spatial > kMaxNb) return fail(c, TOF_EINVAL, "n_spatial %d outside [0, %d]", p->n_spatial, kMaxNb);
    if (p->radius < 1 || p->radius > 255) return fail(c, TOF_EINVAL, "radius %d outside [1, 255]", p->radius);
    if (p->n_spatial_iters < 0 || p->n_spatial_iters > 4) return fail(c, TOF_EINVAL, "n_spatial_iters outside [0, 4]");
    const uint32_t gauges = p->flags & (TOF_FLAG_GAUGE_AXIS_T | TOF_FLAG_GAUGE_AXIS_B | TOF_FLAG_GAUGE_START);
    if (p->flags & ~(TOF_FLAG_DIRECT | TOF_FLAG_NAIVE_SHIFT | TOF_FLAG_PAIRWISE_MIS | TOF_FLAG_TRIANGLE_WALK | TOF_FLAG_BIN_REUSE |
                     TOF_FLAG_ELLIPSOID | gauges))
        return fail(c, TOF_EINVAL, "unknown flag bits 0x%x", p->flags);
    if (gauges & (gauges - 1)) return fail(c, TOF_EINVAL, "at most one gauge flag");
    if ((p->flags & TOF_FLAG_BIN_REUSE) && !transient) return fail(c, TOF_EINVAL, "bin reuse applies to transient rendering");
    if (p->newton_max_iter < 0 || p->newton_max_iter > 16) return fail(c, TOF_EINVAL, "newton_max_iter outside [0, 16]");
    if (!(p->m_cap > 0) || !(p->jac_max >= 1) || !(p->newton_tol_frac > 0) || !(p->ray_eps > 0) || !(p->d_min >= 0))
        return fail(c, TOF_EINVAL, "m_cap, jac_max, newton_tol_frac, ray_eps must be positive, d_min >= 0");
    if (!std::isfinite(p->shrink_k) || p->shrink_k > 1000.f)
        return fail(c, TOF_EINVAL, "shrink_k must be finite and at most 1000");
    if (p->shrink_k > 1.f) {
        if (transient) return fail(c, TOF_EINVAL, "the shrink mapping applies to gated rendering only");
        if (p->flags & TOF_FLAG_ELLIPSOID) return fail(c, TOF_EINVAL, "the shrink mapping and the ellipsoidal connection exclude each other");
        if (p->shrink_fine < 0 || p->shrink_fine >= p->n_cand)
            return fail(c, TOF_EINVAL, "shrink_fine %d outside [0, n_cand - 1]", p->shrink_fine);
    }
    if (transient) {
        int kmin = (p->flags & TOF_FLAG_DIRECT) ? 1 : 2;
        int lengths = p->depth - kmin + 1;
        if (p->flags & TOF_FLAG_ELLIPSOID) lengths += p->depth - 1;   // one ellipsoidal candidate per vertex below depth
        if (lengths > 0 && p->n_cand * lengths > kMaxBinsPerPixel)
            return fail(c, TOF_EINVAL, "transient: n_cand * path lengths = %d exceeds %d candidates per pixel",
                        p->n_cand * lengths, kMaxBinsPerPixel);
    }
    return TOF_OK;
}

static tof_status check_sensor(tof_ctx* c, const tof_sensor* s, int W, int H) {
    if (!s) return fail(c, TOF_EINVAL, "sensor is NULL");
    if (s->W != W || s->H != H) return fail(c, TOF_EINVAL, "sensor %dx%d does not match the view %dx%d", s->W, s->H, W, H);
    if (s->mode != TOF_PINHOLE && s->mode != TOF_CONFOCAL) return fail(c, TOF_EINVAL, "unknown sensor mode %d", s->mode);
    if (s->mode == TOF_PINHOLE && !(s->fov_y > 0 && s->fov_y < 3.1f)) return fail(c, TOF_EINVAL, "fov_y out of range");
    return TOF_OK;
}

static FrameDev make_frame(const SceneH& S, int slot, const tof_sensor* s, const tof_emitter* e, float L0, float dL, int B,
                           uint32_t frame, float4* gb, LightDev* laser, unsigned* err) {
    FrameDev F;
    memset(&F, 0, sizeof(F));
    F.g.tri = S.tri[slot]; F.g.leaf = S.leaf[slot]; F.g.nodes = S.nodes[slot]; F.g.mats = S.mats; F.g.nt = S.nt;
    F.g.adj = S.adj;
    F.g.enode = S.enode[slot]; F.g.eP = S.eP;
    F.g.version = S.version[slot];
    F.g.err = err;
    F.mode = s->mode; F.W = s->W; F.H = s->H;
    F.pos = v3f(s->pos); F.fwd = v3f(s->fwd); F.up = v3f(s->up); F.fov_y = s->fov_y;
    F.wall_o = v3f(s->wall_o); F.wall_u = v3f(s->wall_u); F.wall_v = v3f(s->wall_v);
    F.etype = e->type; F.epos = v3f(e->pos); F.edir = v3f(e->dir); F.epower = e->power;
    F.laser = laser;
    F.L0 = L0; F.dL = dL; F.B = B;
    F.frame = frame;
    F.gb = gb;
    return F;
}

// ============================================================================================
// allocation-free gated rendering
//
// The first render of a view allocates the reuse passes' wavefront scratch (slot tables, task
// lists, shifted records, MIS terms) with cudaMalloc.  tof_render_gated_noalloc instead takes that
// scratch from the file-scope device array below, so a call allocates nothing.  The array is a
// fixed part of the library's device image: every GPU that loads libtof.so holds it until the
// process exits.  Limits: W*H <= kNoAllocMaxPix pixels and 1 + n_spatial <= kNoAllocMaxSlots.
// ============================================================================================
constexpr size_t kNoAllocMaxPix = 16384;
constexpr size_t kNoAllocMaxSlots = 6;
constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNA_U = kNoAllocMaxPix, kNA_S = kNoAllocMaxSlots;
constexpr size_t kNA_slot_pix = 0;
constexpr size_t kNA_slot_M = kNA_slot_pix + al256(sizeof(int) * kNoAllocMaxPix * kNA_S);
constexpr size_t kNA_nslot = kNA_slot_M + al256(sizeof(float) * kNoAllocMaxPix * kNA_S);
constexpr size_t kNA_units = kNA_nslot + al256(kNoAllocMaxPix);
constexpr size_t kNA_fwd = kNA_units + al256(sizeof(int2) * kNA_U);
constexpr size_t kNA_inv = kNA_fwd + al256(sizeof(uint32_t) * kNA_U * (kNA_S - 1));
constexpr size_t kNA_yrec = kNA_inv + al256(sizeof(uint32_t) * kNA_U * kNA_S * (kNA_S - 1));
constexpr size_t kNA_py = kNA_yrec + al256(sizeof(float4) * 6 * kNA_U * (kNA_S - 1));
constexpr size_t kNA_jac = kNA_py + al256(sizeof(float) * kNA_U * kNA_S);
constexpr size_t kNA_terms = kNA_jac + al256(sizeof(float) * kNA_U * kNA_S);
constexpr size_t kNA_rays = kNA_terms + al256(sizeof(float) * kNA_U * kNA_S * kNA_S);
constexpr size_t kNoAllocRays = 65536;   // queued visibility segments; the rest are traced in place
constexpr size_t kNA_counters = kNA_rays + al256(sizeof(float4) * 2 * kNoAllocRays);
constexpr size_t kNoAllocBytes = kNA_counters + 256;   // about 15.6 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// device address of g_noalloc_scratch per device, looked up once per device (with that device
// current) on the first call made on it
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];

static tof_status noalloc_wave(tof_ctx* c, WaveDev* w) {
    if (c->device < 0 || c->device >= 256) return fail(c, TOF_EINVAL, "device id out of range");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[c->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(c, TOF_ECUDA, "cudaGetSymbolAddress of the static reuse scratch failed: %s", cudaGetErrorString(e));
            g_noalloc_addr[c->device] = p;
        }
        base = g_noalloc_addr[c->device];
    }
    unsigned char* b = (unsigned char*)base;
    w->slots = (int)kNA_S;
    w->cap_units = (int)kNA_U;
    w->slot_pix = (int*)(b + kNA_slot_pix);
    w->slot_M = (float*)(b + kNA_slot_M);
    w->nslot = (uint8_t*)(b + kNA_nslot);
    w->units = (int2*)(b + kNA_units);
    w->fwd = (uint32_t*)(b + kNA_fwd);
    w->inv = (uint32_t*)(b + kNA_inv);
    w->yrec = (float4*)(b + kNA_yrec);
    w->py = (float*)(b + kNA_py);
    w->jac = (float*)(b + kNA_jac);
    w->terms = (float*)(b + kNA_terms);
    w->rays = (float4*)(b + kNA_rays);
    w->ray_cap = (uint32_t)kNoAllocRays;
    w->rays2 = nullptr;
    w->ray2_cap = 0;
    w->counters = (uint32_t*)(b + kNA_counters);
    return TOF_OK;
}

extern "C" {

tof_status tof_create(tof_ctx** out, int device, uint64_t hbm_budget_bytes) {
    if (!out) return TOF_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return TOF_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return TOF_ECUDA;
    tof_ctx* c = new tof_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (dalloc(c, &c->d_err, 64, "error word") != TOF_OK) { delete c; return TOF_ENOMEM; }
    cudaMemset(c->d_err, 0, 64);
    if (cudaHostAlloc((void**)&c->h_err, 64, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        for (auto& a : c->allocs) cudaFree(a.p);
        delete c;
        return TOF_ENOMEM;
    }
    memset(c->h_err, 0, 64);
    *out = c;
    return TOF_OK;
}

tof_status tof_destroy(tof_ctx* c) {
    if (!c) return TOF_EINVAL;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (cudaGraphExec_t& x : c->batch_exec)
        if (x) cudaGraphExecDestroy(x);
    for (int k = 0; k < kBatchSlots; ++k) {
        if (c->bstage[k]) cudaFreeHost(c->bstage[k]);
        if (c->bdone[k]) cudaEventDestroy(c->bdone[k]);
    }
    for (cudaStream_t q : c->pool) cudaStreamDestroy(q);
    for (cudaEvent_t e : c->join) cudaEventDestroy(e);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->capture) cudaStreamDestroy(c->capture);
    for (auto& a : c->allocs) cudaFree(a.p);
    if (c->h_err) cudaFreeHost(c->h_err);
    delete c;
    return TOF_OK;
}

const char* tof_last_error(tof_ctx* c) { return c ? c->err.c_str() : "no context"; }
uint64_t tof_device_bytes(tof_ctx* c) { return c ? c->used : 0; }

tof_status tof_scene_upload(tof_ctx* c, const float* verts, uint32_t nv, const uint32_t* tris, uint32_t nt,
                            const uint32_t* tri_object, const tof_material* mats, uint32_t nmat,
                            const uint32_t* object_material, uint32_t nobj, tof_scene* out) {
    if (!c || !out) return TOF_EINVAL;
    if (!verts || !tris || !tri_object || !mats || !object_material) return fail(c, TOF_EINVAL, "NULL scene array");
    if (nt == 0 || nv == 0 || nobj == 0 || nmat == 0) return fail(c, TOF_EINVAL, "empty scene");
    if (nt > (1u << 26)) return fail(c, TOF_EINVAL, "too many triangles");
    for (uint64_t i = 0; i < 3ull * nv; ++i)
        if (!std::isfinite(verts[i])) return fail(c, TOF_EINVAL, "non-finite vertex coordinate at %llu", (unsigned long long)i);
    for (uint64_t i = 0; i < 3ull * nt; ++i)
        if (tris[i] >= nv) return fail(c, TOF_EINVAL, "triangle index out of range");
    for (uint32_t i = 0; i < nt; ++i)
        if (tri_object[i] >= nobj) return fail(c, TOF_EINVAL, "tri_object out of range");
    for (uint32_t i = 0; i < nobj; ++i)
        if (object_material[i] >= nmat) return fail(c, TOF_EINVAL, "object_material out of range");
    std::vector<float4> mh(nmat);
    for (uint32_t i = 0; i < nmat; ++i) {
        if (mats[i].type < 0 || mats[i].type > 2 || !(mats[i].albedo >= 0 && mats[i].albedo <= 1))
            return fail(c, TOF_EINVAL, "material %u invalid", i);
        if (mats[i].type == TOF_GGX && !(mats[i].alpha > 0 && mats[i].alpha <= 1))
            return fail(c, TOF_EINVAL, "material %u: GGX alpha must be in (0, 1]", i);
        mh[i] = make_float4((float)mats[i].type, mats[i].albedo, mats[i].alpha, 0.f);
    }
    cudaSetDevice(c->device);
    SceneH S;
    S.nv = (int)nv; S.nt = (int)nt; S.nobj = (int)nobj; S.nmat = (int)nmat;
    TRY(dalloc(c, &S.vloc, sizeof(float) * 3 * nv, "vertices"));
    TRY(dalloc(c, &S.tris, sizeof(uint32_t) * 3 * nt, "triangles"));
    TRY(dalloc(c, &S.triobj, sizeof(uint32_t) * nt, "tri_object"));
    TRY(dalloc(c, &S.objmat, sizeof(uint32_t) * nobj, "object_material"));
    TRY(dalloc(c, &S.mats, sizeof(float4) * nmat, "materials"));
    TRY(dalloc(c, &S.xf, sizeof(float) * 12 * nobj, "transforms"));
    TRY(dalloc(c, &S.cent, sizeof(float4) * nt, "centroids"));
    TRY(dalloc(c, &S.keys, sizeof(uint32_t) * nt, "keys"));
    TRY(dalloc(c, &S.vals, sizeof(uint32_t) * nt, "vals"));
    TRY(dalloc(c, &S.keys2, sizeof(uint32_t) * nt, "keys2"));
    TRY(dalloc(c, &S.vals2, sizeof(uint32_t) * nt, "vals2"));
    int ntiles = ((int)nt + 2047) / 2048;
    TRY(dalloc(c, &S.hist, sizeof(uint32_t) * 256 * (size_t)ntiles, "histogram"));
    TRY(dalloc(c, &S.bb, sizeof(uint32_t) * 8, "bounds"));
    TRY(dalloc(c, &S.child, sizeof(int) * 2 * nt, "children"));
    TRY(dalloc(c, &S.parent_int, sizeof(int) * nt, "parents"));
    TRY(dalloc(c, &S.parent_leaf, sizeof(int) * nt, "leaf parents"));
    TRY(dalloc(c, &S.counter, sizeof(uint32_t) * nt, "refit counters"));
    for (int k = 0; k < 2; ++k) {
        TRY(dalloc(c, &S.tri[k], sizeof(float4) * 3 * nt, "triangle records"));
        TRY(dalloc(c, &S.leaf[k], sizeof(float4) * 3 * nt, "leaf records"));
        TRY(dalloc(c, &S.nodes[k], sizeof(float4) * 4 * (size_t)(nt > 1 ? nt - 1 : 1), "nodes"));
    }
    if (nt <= (1u << kEllMaxLevels)) {
        S.eP = 1;
        while ((uint32_t)S.eP < nt) S.eP <<= 1;
        for (int k = 0; k < 2; ++k) TRY(dalloc(c, &S.enode[k], sizeof(float4) * 4 * (size_t)S.eP, "ellipsoid hierarchy"));
    }
    CK(cudaMemcpy(S.vloc, verts, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S.tris, tris, sizeof(uint32_t) * 3 * nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S.triobj, tri_object, sizeof(uint32_t) * nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S.objmat, object_material, sizeof(uint32_t) * nobj, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S.mats, mh.data(), sizeof(float4) * nmat, cudaMemcpyHostToDevice));
    {
        // edge adjacency: an edge (two vertex indices) shared by exactly two triangles of one object
        struct Edge { uint32_t a, b, t, opp; };
        std::vector<Edge> E((size_t)nt * 3);
        for (uint32_t t = 0; t < nt; ++t)
            for (uint32_t i = 0; i < 3; ++i) {
                uint32_t u = tris[3 * t + (i + 1) % 3], w = tris[3 * t + (i + 2) % 3];
                E[3 * t + i] = Edge{u < w ? u : w, u < w ? w : u, t, i};
            }
        std::sort(E.begin(), E.end(), [](const Edge& x, const Edge& y) {
            return x.a != y.a ? x.a < y.a : x.b != y.b ? x.b < y.b : x.t < y.t;
        });
        std::vector<int> adj((size_t)nt * 3, -1);
        for (size_t k = 0; k < E.size();) {
            size_t m = k + 1;
            while (m < E.size() && E[m].a == E[k].a && E[m].b == E[k].b) ++m;
            if (m - k == 2 && tri_object[E[k].t] == tri_object[E[k + 1].t] && E[k].t != E[k + 1].t) {
                adj[3 * (size_t)E[k].t + E[k].opp] = (int)(4 * E[k + 1].t + E[k + 1].opp);
                adj[3 * (size_t)E[k + 1].t + E[k + 1].opp] = (int)(4 * E[k].t + E[k].opp);
            }
            k = m;
        }
        TRY(dalloc(c, &S.adj, sizeof(int) * 3 * (size_t)nt, "adjacency"));
        CK(cudaMemcpy(S.adj, adj.data(), sizeof(int) * 3 * (size_t)nt, cudaMemcpyHostToDevice));
    }
    S.alive = true;
    c->scenes.push_back(S);
    *out = (tof_scene)(c->scenes.size() - 1);
    return TOF_OK;
}

tof_status tof_scene_destroy(tof_ctx* c, tof_scene id) {
    if (!c || id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].alive) return c ? fail(c, TOF_EINVAL, "bad scene") : TOF_EINVAL;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    SceneH& S = c->scenes[id];
    void* ps[] = {S.vloc, S.tris, S.triobj, S.objmat, S.mats, S.xf, S.cent, S.keys, S.vals, S.keys2, S.vals2, S.hist, S.bb,
                  S.child, S.parent_int, S.parent_leaf, S.counter, S.tri[0], S.tri[1], S.leaf[0], S.leaf[1], S.nodes[0], S.nodes[1],
                  S.adj, S.enode[0], S.enode[1]};
    for (void* p : ps) dfree(c, p);
    S = SceneH();
    return TOF_OK;
}

tof_status tof_bvh_build(tof_ctx* c, tof_scene id, const float* xf, int refit_only, void* stream) {
    if (!c) return TOF_EINVAL;
    if (id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].alive) return fail(c, TOF_EINVAL, "bad scene handle %d", id);
    if (!xf) return fail(c, TOF_EINVAL, "object_xforms is NULL");
    SceneH& S = c->scenes[id];
    for (int i = 0; i < 12 * S.nobj; ++i)
        if (!std::isfinite(xf[i])) return fail(c, TOF_EINVAL, "non-finite transform entry %d", i);
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<float> xv(xf, xf + 12 * S.nobj);
    if (S.built && S.xfh[S.cur] == xv) return TOF_OK;   // static between frames
    int slot = S.built ? 1 - S.cur : 0;
    CK(cudaMemcpyAsync(S.xf, xf, sizeof(float) * 12 * S.nobj, cudaMemcpyHostToDevice, s));
    CK(launch_xform(S.nt, S.vloc, S.tris, S.triobj, S.objmat, S.xf, S.tri[slot], S.cent, s));
    if (!S.built || !refit_only) {
        CK(launch_build_topology(S.nt, S.cent, S.bb, S.keys, S.vals, S.keys2, S.vals2, S.hist, S.child, S.parent_int,
                                 S.parent_leaf, &S.prim, s));
    }
    CK(launch_refit(S.nt, S.prim, S.tri[slot], S.leaf[slot], S.nodes[slot], S.child, S.parent_int, S.parent_leaf, S.counter, s));
    if (S.enode[slot]) CK(launch_etree(S.nt, S.eP, S.tri[slot], S.enode[slot], s));
    S.version[slot] = ++c->version_counter;
    S.xfh[slot] = xv;
    S.cur = slot;
    S.built = true;
    return TOF_OK;
}

tof_status tof_view_create(tof_ctx* c, tof_scene scene, int32_t W, int32_t H, int32_t B, tof_view* out) {
    if (!c || !out) return TOF_EINVAL;
    if (scene < 0 || scene >= (int)c->scenes.size() || !c->scenes[scene].alive) return fail(c, TOF_EINVAL, "bad scene handle");
    if (W < 1 || H < 1 || W > 16384 || H > 16384 || B < 0 || B > 65536) return fail(c, TOF_EINVAL, "bad view size %dx%dx%d", W, H, B);
    cudaSetDevice(c->device);
    ViewH V;
    V.scene = scene; V.W = W; V.H = H; V.B = B;
    size_t npix = (size_t)W * H, Bn = B > 0 ? (size_t)B : 1;
    int words = (int)((Bn + 31) / 32);
    for (int k = 0; k < 2; ++k) {
        TRY(dalloc(c, &V.gb[k], sizeof(float4) * npix, "G-buffer"));
        TRY(dalloc(c, &V.laser[k], sizeof(LightDev), "laser spot"));
    }
    for (int k = 0; k < 3; ++k) {
        ResH& R = V.res[k];
        R.entries = npix * Bn;
        R.words = words;
        TRY(dalloc(c, &R.planes, sizeof(float4) * 6 * R.entries, "reservoirs"));
        TRY(dalloc(c, &R.M, sizeof(float) * npix, "confidence"));
        TRY(dalloc(c, &R.occ, sizeof(uint32_t) * npix * words, "occupancy"));
        CK(cudaMemset(R.occ, 0, sizeof(uint32_t) * npix * words));
    }
    TRY(dalloc(c, &V.stats, sizeof(StatsDev), "stats"));
    CK(cudaMemset(V.stats, 0, sizeof(StatsDev)));
    V.alive = true;
    c->views.push_back(V);
    *out = (tof_view)(c->views.size() - 1);
    return TOF_OK;
}

tof_status tof_view_destroy(tof_ctx* c, tof_view id) {
    if (!c || id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return c ? fail(c, TOF_EINVAL, "bad view") : TOF_EINVAL;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    ViewH& V = c->views[id];
    for (int k = 0; k < 2; ++k) { dfree(c, V.gb[k]); dfree(c, V.laser[k]); }
    for (int k = 0; k < 3; ++k) { dfree(c, V.res[k].planes); dfree(c, V.res[k].M); dfree(c, V.res[k].occ); }
    for (void* p : V.wave_ptrs) dfree(c, p);
    for (void* p : V.ell_ptrs) dfree(c, p);
    for (void* p : V.tw_ptrs) dfree(c, p);
    dfree(c, V.rays2);
    if (V.side) cudaStreamDestroy(V.side);
    if (V.side_fork) cudaEventDestroy(V.side_fork);
    if (V.side_join) cudaEventDestroy(V.side_join);
    dfree(c, V.stats);
    for (int k = 0; k < 7; ++k)
        if (V.ev[k]) cudaEventDestroy(V.ev[k]);
    for (cudaEvent_t e : V.kev) cudaEventDestroy(e);
    V = ViewH();
    return TOF_OK;
}

tof_status tof_reservoirs_reset(tof_ctx* c, tof_view id) {
    if (!c || id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return c ? fail(c, TOF_EINVAL, "bad view") : TOF_EINVAL;
    ViewH& V = c->views[id];
    V.has_prev = false;
    V.prev_final = -1;
    return TOF_OK;
}

tof_status tof_view_stats(tof_ctx* c, tof_view id, double out[10]) {
    if (!c || !out || id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return c ? fail(c, TOF_EINVAL, "bad view") : TOF_EINVAL;
    cudaSetDevice(c->device);
    ViewH& V = c->views[id];
    StatsDev h;
    CK(cudaStreamSynchronize(V.last_stream));
    CK(cudaMemcpy(&h, V.stats, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 10; ++i) out[i] = (double)h.v[i];
    unsigned bits = 0;
    CK(cudaMemcpy(&bits, c->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
    return report_err_bits(c, bits);
}

static bool g_no_marks = false;   // set while a batch is being captured (no profiling events)

// a recorded initial stage that a staged batch runs as the bounce wavefront
struct WaveRec {
    InitArgs a;
    TreeWaveDev w;
    int tile_h, hit_blocks, vis_blocks;
};
struct BatchRec {
    std::vector<GbufArgs> gbuf;
    std::vector<InitArgs> init;
    std::vector<WaveRec> wave;
    std::vector<std::vector<ReuseJob>> pass;   // pass[q]: every instance's q-th reuse pass
    size_t q = 0;                              // the current instance's next pass
};
// staged batches: while set, render() records each stage's arguments instead of launching them
static BatchRec* g_rec = nullptr;
constexpr int kReuseEvents = 7;   // events around the kernels of one reuse launch group

// resident-block counts of the persistent reuse kernels, once per context
static tof_status persist_init(tof_ctx* c) {
    if (c->persist_blocks) return TOF_OK;
    CK(reuse_persist_blocks(&c->persist_blocks, &c->vis_blocks));
    CK(ell_place_blocks(&c->ell_blocks));
    CK(tree_hit_blocks(&c->hit_blocks));
    CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
    return TOF_OK;
}

// (re)allocate the scratch of the ellipsoidal connection's initial wavefront for nc trees of the
// given depth: per (pixel, tree, vertex) 64 B of vertex, candidate and placement records, a request
// and two queued visibility segments (450 MB for 512 x 512, 4 trees, depth 4)
static tof_status ensure_ell_wave(tof_ctx* c, ViewH& V, int nc, int depth) {
    const size_t npix = (size_t)V.W * V.H, slots = npix * (size_t)nc * (size_t)depth;
    if (V.ell_slots >= slots && V.ell.nc == nc && V.ell.depth == depth) return TOF_OK;
    for (void*& p : V.ell_ptrs) { dfree(c, p); p = nullptr; }
    V.ell_slots = 0;
    EllWaveDev& w = V.ell;
    w.nc = nc; w.depth = depth;
    const size_t reqs = npix * (size_t)nc * (size_t)(depth > 1 ? depth - 1 : 1);
    TRY(dalloc(c, &w.vtx, sizeof(float4) * slots, "ellipsoid wave vertices"));
    TRY(dalloc(c, &w.vtx2, sizeof(float2) * slots, "ellipsoid wave throughputs"));
    TRY(dalloc(c, &w.acand, sizeof(float2) * slots, "ellipsoid wave tree candidates"));
    TRY(dalloc(c, &w.bw, sizeof(float) * slots, "ellipsoid wave weights"));
    TRY(dalloc(c, &w.bz, sizeof(float4) * slots, "ellipsoid wave vertices placed"));
    TRY(dalloc(c, &w.bpt, sizeof(float) * slots, "ellipsoid wave densities"));
    TRY(dalloc(c, &w.req, sizeof(uint32_t) * reqs, "ellipsoid wave requests"));
    w.req_cap = (uint32_t)reqs;
    TRY(dalloc(c, &w.rays, sizeof(float4) * 4 * reqs, "ellipsoid wave visibility queue"));
    w.ray_cap = (uint32_t)(2 * reqs);
    TRY(dalloc(c, &w.counters, sizeof(uint32_t) * 4, "ellipsoid wave counters"));
    void* ps[9] = {w.vtx, w.vtx2, w.acand, w.bw, w.bz, w.bpt, w.req, w.rays, w.counters};
    for (int k = 0; k < 9; ++k) V.ell_ptrs[k] = ps[k];
    V.ell_slots = slots;
    return TOF_OK;
}

// (re)allocate the bounce wavefront of the gated initial stage for nc trees of the given depth: per
// (pixel, tree) 24 B per vertex (record and candidate), 32 B of path state, 80 B of rays and hits
// and a queued light segment (about 240 MB for 512 x 512, 4 trees, depth 4)
static tof_status ensure_tree_wave(tof_ctx* c, ViewH& V, int nc, int depth) {
    const size_t paths = (size_t)V.W * V.H * (size_t)nc, slots = paths * (size_t)depth;
    if (V.tw_paths >= paths && V.tw.nc == nc && V.tw.depth == depth) return TOF_OK;
    for (void*& p : V.tw_ptrs) { dfree(c, p); p = nullptr; }
    V.tw_paths = 0;
    TreeWaveDev& w = V.tw;
    w.nc = nc; w.depth = depth;
    TRY(dalloc(c, &w.vtx, sizeof(float4) * slots, "tree wave vertices"));
    TRY(dalloc(c, &w.acand, sizeof(float2) * slots, "tree wave candidates"));
    TRY(dalloc(c, &w.ps0, sizeof(float4) * paths, "tree wave path throughputs"));
    TRY(dalloc(c, &w.ps1, sizeof(float4) * paths, "tree wave path vertices"));
    TRY(dalloc(c, &w.rays[0], sizeof(float4) * 2 * paths, "tree wave rays"));
    TRY(dalloc(c, &w.rays[1], sizeof(float4) * 2 * paths, "tree wave rays"));
    TRY(dalloc(c, &w.hits, sizeof(float4) * paths, "tree wave hits"));
    w.path_cap = (uint32_t)paths;
    TRY(dalloc(c, &w.srays, sizeof(float4) * 2 * paths, "tree wave light segments"));
    w.sray_cap = (uint32_t)paths;   // more segments than paths are traced in place
    TRY(dalloc(c, &w.counters, sizeof(uint32_t) * kTreeWaveCounters, "tree wave counters"));
    void* ps[9] = {w.vtx, w.acand, w.ps0, w.ps1, w.rays[0], w.rays[1], w.hits, w.srays, w.counters};
    for (int k = 0; k < 9; ++k) V.tw_ptrs[k] = ps[k];
    V.tw_paths = paths;
    return TOF_OK;
}

// a gated render without the ellipsoidal connection or the shrink mapping runs its initial stage as
// the bounce wavefront, except in the allocation-free form and beyond 16M (pixel, tree) paths (~4 GB
// of scratch); in a batch only views of kBatchWaveMinPix pixels and more do (small instances would
// pay for its 2 * depth + 1 launches each).  The rest keep the single kernel, which needs no scratch.
// Both give the same reservoirs.
static bool use_tree_wave(const ViewH& V, int B, const tof_params* p, bool fixed) {
    if (fixed || B > 0 || (p->flags & TOF_FLAG_ELLIPSOID) || p->shrink_k > 1.f) return false;
    return (double)V.W * V.H * p->n_cand <= 16.0 * 1024.0 * 1024.0;
}

// batches run a gated instance's initial stage as the bounce wavefront from this many pixels on:
// smaller ones are cheaper as blocks of the batched single kernel than as 2 * depth + 1 launches
constexpr size_t kBatchWaveMinPix = 256 * 256;
static bool use_ell_wave(const ViewH& V, int B, const tof_params* p, bool fixed);
static bool batch_tree_wave(const ViewH& V, const tof_job& J) {
    return !J.transient && (size_t)V.W * V.H >= kBatchWaveMinPix &&
           (use_tree_wave(V, 0, &J.params, false) || use_ell_wave(V, 0, &J.params, false));
}
// the view's wavefront scratch is allocated for these parameters (by prepare_job before a batch)
static bool tree_wave_ready(const ViewH& V, const tof_params* p) {
    return (size_t)V.W * V.H >= kBatchWaveMinPix && V.tw_paths >= (size_t)V.W * V.H * (size_t)p->n_cand &&
           V.tw.nc == p->n_cand && V.tw.depth == p->depth;
}

// the initial stage runs as the ellipsoidal wavefront: gated, ellipsoidal connection, not the
// allocation-free form, and at most 32M (pixel, tree, vertex) slots (~2.5 GB of scratch; larger
// views or tree counts keep the single kernel, which needs none)
static bool use_ell_wave(const ViewH& V, int B, const tof_params* p, bool fixed) {
    if (fixed || B > 0 || !(p->flags & TOF_FLAG_ELLIPSOID) || p->shrink_k > 1.f) return false;
    return (double)V.W * V.H * p->n_cand * p->depth <= 32.0 * 1024.0 * 1024.0;
}

// (re)allocate the view's wavefront scratch for S slots per pixel and cap merge units
static tof_status ensure_wave(tof_ctx* c, ViewH& V, int S, int cap) {
    if (V.wave_slots >= S && V.wave_cap >= cap) return TOF_OK;
    for (void*& p : V.wave_ptrs) { dfree(c, p); p = nullptr; }
    S = S > V.wave_slots ? S : V.wave_slots;
    cap = cap > V.wave_cap ? cap : V.wave_cap;
    size_t npix = (size_t)V.W * V.H, U = (size_t)cap;
    WaveDev& w = V.wave;
    w.slots = S; w.cap_units = cap;
    TRY(dalloc(c, &w.slot_pix, sizeof(int) * npix * S, "reuse slots"));
    TRY(dalloc(c, &w.slot_M, sizeof(float) * npix * S, "reuse confidences"));
    TRY(dalloc(c, &w.nslot, npix, "reuse slot counts"));
    TRY(dalloc(c, &w.units, sizeof(int2) * U, "merge units"));
    TRY(dalloc(c, &w.fwd, sizeof(uint32_t) * U * (S - 1), "forward shift tasks"));
    TRY(dalloc(c, &w.inv, sizeof(uint32_t) * U * S * (S - 1), "inverse shift tasks"));
    TRY(dalloc(c, &w.yrec, sizeof(float4) * 6 * U * (S - 1), "shifted records"));
    TRY(dalloc(c, &w.py, sizeof(float) * U * S, "shifted targets"));
    TRY(dalloc(c, &w.jac, sizeof(float) * U * S, "shift Jacobians"));
    TRY(dalloc(c, &w.terms, sizeof(float) * U * S * S, "MIS terms"));
    // queued visibility segments: two per inverse shift would need up to 2 U S (S - 1); a pass
    // shifts far fewer (a 512 x 512 spatial pass with 5 neighbours queues 3-6 M), and segments
    // beyond the queue are traced in place
    size_t rcap = 2 * U * S * (S - 1);
    size_t rmax = npix * 24 + ((size_t)1 << 20);
    if (rcap > rmax) rcap = rmax;
    TRY(dalloc(c, &w.rays, sizeof(float4) * 2 * rcap, "visibility queue"));
    w.ray_cap = (uint32_t)rcap;
    TRY(dalloc(c, &w.counters, sizeof(uint32_t) * kWaveCounters, "task counters"));
    void* ps[12] = {w.slot_pix, w.slot_M, w.nslot, w.units, w.fwd, w.inv, w.yrec, w.py, w.jac, w.terms, w.rays, w.counters};
    for (int k = 0; k < 12; ++k) V.wave_ptrs[k] = ps[k];
    V.wave_slots = S; V.wave_cap = cap;
    return TOF_OK;
}

// the second visibility queue of a view's direct renders (the temporal pass's canonical inverse
// shifts, at most one per pixel and bin: 4 segments per pixel, beyond which they are traced in
// place), its stream and events
static tof_status ensure_side(tof_ctx* c, ViewH& V) {
    if (V.rays2) return TOF_OK;
    const size_t cap = (size_t)V.W * V.H * 4 + ((size_t)1 << 20);
    if (!V.side) CK(cudaStreamCreateWithFlags(&V.side, cudaStreamNonBlocking));
    if (!V.side_fork) CK(cudaEventCreateWithFlags(&V.side_fork, cudaEventDisableTiming));
    if (!V.side_join) CK(cudaEventCreateWithFlags(&V.side_join, cudaEventDisableTiming));
    TRY(dalloc(c, &V.rays2, sizeof(float4) * 2 * cap, "second visibility queue"));
    V.ray2_cap = (uint32_t)cap;
    return TOF_OK;
}

// one reuse pass as a wavefront; transient passes run in pixel chunks so that a chunk's merge
// units (at most B per pixel) never exceed the scratch capacity
static tof_status reuse_pass(tof_ctx* c, ViewH& V, const ReuseArgs& ra, const WaveDev* fixed, cudaStream_t s) {
    const int S = ra.binpass ? 3 : ra.temporal ? 2 : 1 + ra.P.n_spatial;
    const size_t npix = (size_t)V.W * V.H;
    const size_t Bn = V.B > 0 ? (size_t)V.B : 1;
    const size_t kMaxUnits = (size_t)1 << 22;
    size_t cap = npix * Bn < kMaxUnits ? npix * Bn : kMaxUnits;
    if (cap < npix && V.B == 0) cap = npix;
    if (!fixed) TRY(ensure_wave(c, V, S, (int)cap));
    TRY(persist_init(c));
    WaveDev w = fixed ? *fixed : V.wave;
    w.slots = S;
    // the temporal pass of a direct render runs the canonical inverse shifts beside the forward
    // shifts: both are small there and wait on a few long chains (0.52 -> 0.39 ms per 512 x 512
    // frame); in a spatial pass both fill the GPU and beside each other they were slower
    const bool beside = ra.temporal && !fixed && !g_rec && !c->in_batch;
    if (beside) TRY(ensure_side(c, V));
    w.rays2 = beside ? V.rays2 : nullptr;
    w.ray2_cap = beside ? V.ray2_cap : 0u;
    if (!fixed) w.cap_units = V.wave_cap;
    size_t chunk = V.B > 0 ? (size_t)V.wave_cap / Bn : npix;
    if (chunk < 1) chunk = 1;
    for (size_t p0 = 0; p0 < npix; p0 += chunk) {
        size_t p1 = p0 + chunk < npix ? p0 + chunk : npix;
        cudaEvent_t* ev = nullptr;
        if (V.profile && !ra.temporal && !fixed && !g_no_marks) {
            while (V.kev.size() < V.kev_used + kReuseEvents) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                V.kev.push_back(e);
            }
            ev = &V.kev[V.kev_used];
            V.kev_used += kReuseEvents;
        }
        if (g_rec) {
            if (g_rec->pass.size() <= g_rec->q) g_rec->pass.resize(g_rec->q + 1);
            ReuseJob J;
            J.a = ra; J.w = w; J.p0 = (int)p0; J.p1 = (int)p1;
            g_rec->pass[g_rec->q].push_back(J);
            continue;
        }
        int pb = c->persist_blocks, vb = c->vis_blocks;
        if (V.tune.packet > 0) {
            pb = std::min(pb, c->sms * V.tune.packet);
            vb = std::min(vb, c->sms * V.tune.packet);
        }
        CK(launch_reuse_wave(ra, w, (int)p0, (int)p1, pb, vb, ev, s, beside ? V.side : nullptr, V.side_fork, V.side_join));
    }
    if (g_rec) ++g_rec->q;
    return TOF_OK;
}

// stage boundaries: ev[0] frame start, ev[1] after G-buffer, ev[2] after initial, ev[3] after
// temporal, ev[4] after spatial, ev[5] after splat, ev[6] frame end
static void mark(ViewH& V, int k, cudaStream_t s) {
    if (V.profile && V.ev[k] && !g_no_marks) cudaEventRecord(V.ev[k], s);
}

static tof_status render(tof_ctx* c, tof_scene scene, tof_view vid, const tof_sensor* sensor, const tof_emitter* emitter,
                         float L0, float dL, int B, const tof_params* params, uint64_t seed, uint32_t frame, float* out,
                         void* stream, const WaveDev* fixed_wave = nullptr) {
    if (!c) return TOF_EINVAL;
    if (scene < 0 || scene >= (int)c->scenes.size() || !c->scenes[scene].alive) return fail(c, TOF_EINVAL, "bad scene handle");
    if (vid < 0 || vid >= (int)c->views.size() || !c->views[vid].alive) return fail(c, TOF_EINVAL, "bad view handle");
    ViewH& V = c->views[vid];
    SceneH& S = c->scenes[scene];
    if (V.scene != scene) return fail(c, TOF_EINVAL, "view %d belongs to scene %d", vid, V.scene);
    if (!S.built) return fail(c, TOF_ESTATE, "tof_bvh_build has not been called for scene %d", scene);
    if ((B > 0) != (V.B > 0) || (B > 0 && B != V.B)) return fail(c, TOF_EINVAL, "bins %d do not match the view (%d)", B, V.B);
    TRY(check_sensor(c, sensor, V.W, V.H));
    TRY(check_params(c, params, B > 0));
    if ((params->flags & TOF_FLAG_ELLIPSOID) && !S.enode[0])
        return fail(c, TOF_EINVAL, "the ellipsoidal connection supports scenes of up to 2^%d triangles", kEllMaxLevels);
    if (!emitter || emitter->type < 0 || emitter->type > 2 || !(emitter->power >= 0))
        return fail(c, TOF_EINVAL, "bad emitter");
    if (!(dL > 0) || !std::isfinite(L0)) return fail(c, TOF_EINVAL, "gate / bin width must be positive and finite");
    if (!out) return fail(c, TOF_EINVAL, "output pointer is NULL");
    cudaSetDevice(c->device);
    if (!g_no_marks) TRY(pending_err(c));
    cudaStream_t s = (cudaStream_t)stream;
    V.last_stream = s;

    const int fc = V.has_prev ? 1 - V.cur : V.cur;
    FrameDev F = make_frame(S, S.cur, sensor, emitter, L0, dL, B, frame, V.gb[fc], V.laser[fc], c->d_err);
    ParamsDev P = to_dev(params, seed);
    for (int k = 0; k < 5; ++k) V.ran[k] = false;
    V.kev_used = 0;
    mark(V, 0, s);
    if (emitter->type == TOF_EMIT_LASER) CK(launch_laser(F.g, v3f(emitter->pos), v3f(emitter->dir), emitter->power, V.laser[fc], s));
    GbufArgs ga;
    ga.F = F; ga.gb = V.gb[fc]; ga.P = P; ga.tile_w = V.tune.tile_w;
    if (g_rec) {
        g_rec->q = 0;
        g_rec->gbuf.push_back(ga);
    } else {
        CK(launch_gbuffer(ga, V.tune.tile_h, s));
    }
    mark(V, 1, s);
    V.ran[0] = true;

    // temporal reuse needs the previous frame's geometry still resident
    bool temporal = params->temporal && V.has_prev && V.prev_final >= 0 &&
                    S.version[V.geom_slot[1 - fc]] == V.geom_version[1 - fc];
    const bool binpass = B > 0 && (params->flags & TOF_FLAG_BIN_REUSE);
    int stages = 1 + (temporal ? 1 : 0) + (binpass ? 1 : 0) + (params->n_spatial > 0 ? params->n_spatial_iters : 0);
    int bufs[2], nb = 0;
    for (int k = 0; k < 3 && nb < 2; ++k)
        if (k != V.prev_final) bufs[nb++] = k;
    // stage i writes bufs[(i + off) % 2] so that the last stage lands in bufs[1]
    int off = (stages % 2 == 0) ? 0 : 1;
    auto out_of = [&](int st) { return bufs[(st + off) % 2]; };
    int stage = 0;
    InitArgs ia;
    ia.wave = 0;
    ia.F = F; ia.dst = V.res[out_of(stage)].dev(); ia.P = P;
    ia.out = (stage == stages - 1 && B == 0) ? out : nullptr;
    ia.tile_w = V.tune.tile_w;
    if (B == 0 && params->shrink_k > 1.f) {
        CK(launch_initial_shrink(ia, V.tune.tile_h, s));
    } else if (use_ell_wave(V, B, params, fixed_wave != nullptr)) {
        TRY(ensure_ell_wave(c, V, params->n_cand, params->depth));
        TRY(persist_init(c));
        int vb = c->vis_blocks, eb = c->ell_blocks;
        if (V.tune.packet > 0) {
            vb = std::min(vb, c->sms * V.tune.packet);
            eb = std::min(eb, c->sms * V.tune.packet);
        }
        if (!(c->in_batch || g_rec) || tree_wave_ready(V, params)) {
            // its path trees as bounce rounds (a batch: where prepare_job allocated that scratch)
            TRY(ensure_tree_wave(c, V, params->n_cand, params->depth));
            int hb = c->hit_blocks;
            if (V.tune.packet > 0) hb = std::min(hb, c->sms * V.tune.packet);
            CK(launch_initial_ell_tree_wave(ia, V.tw, V.ell, V.tune.tile_h, hb, eb, vb, s));
        } else {
            CK(launch_initial_ell_wave(ia, V.ell, V.tune.tile_h, eb, vb, s));
        }
    } else if (use_tree_wave(V, B, params, fixed_wave != nullptr) &&
               (!(c->in_batch || g_rec) || tree_wave_ready(V, params))) {
        // a batch uses the wavefront only where prepare_job allocated its scratch (large views)
        TRY(ensure_tree_wave(c, V, params->n_cand, params->depth));
        TRY(persist_init(c));
        int hb = c->hit_blocks, vb = c->vis_blocks;
        if (V.tune.packet > 0) {
            hb = std::min(hb, c->sms * V.tune.packet);
            vb = std::min(vb, c->sms * V.tune.packet);
        }
        if (g_rec) {
            ia.wave = 1;
            g_rec->init.push_back(ia);
            g_rec->wave.push_back(WaveRec{ia, V.tw, V.tune.tile_h, hb, vb});
        } else {
            CK(launch_initial_tree_wave(ia, V.tw, V.tune.tile_h, hb, vb, s));
        }
    } else if (g_rec) {
        g_rec->init.push_back(ia);   // staged batches hold gated views without those options only
    } else {
        CK(launch_initial(ia, V.tune.tile_h, c->d_err, s));
    }
    mark(V, 2, s);
    V.ran[1] = true;
    int src = out_of(stage);
    ++stage;
    ReuseArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.cur = F; ra.P = P; ra.stats = V.stats;
    if (temporal) {
        ra.prev = V.fd[1 - fc];
        ra.src = V.res[src].dev();
        ra.prv = V.res[V.prev_final].dev();
        ra.dst = V.res[out_of(stage)].dev();
        ra.temporal = 1; ra.pass = 0;
        ra.geom_static = V.geom_version[1 - fc] == S.version[S.cur];
        ra.out = (stage == stages - 1 && B == 0) ? out : nullptr;
        TRY(reuse_pass(c, V, ra, fixed_wave, s));
        src = out_of(stage);
        ++stage;
        V.ran[2] = true;
    }
    mark(V, 3, s);
    if (binpass) {
        // bin reuse: the same pixel's neighbouring bins (timed with the spatial stage)
        ra.prev = F;
        ra.src = V.res[src].dev();
        ra.prv = ra.src;
        ra.dst = V.res[out_of(stage)].dev();
        ra.temporal = 0; ra.binpass = 1; ra.pass = 8; ra.geom_static = 1;
        ra.out = nullptr;
        TRY(reuse_pass(c, V, ra, fixed_wave, s));
        ra.binpass = 0;
        src = out_of(stage);
        ++stage;
        V.ran[3] = true;
    }
    if (params->n_spatial > 0) {
        for (int it = 0; it < params->n_spatial_iters; ++it) {
            ra.prev = F;
            ra.src = V.res[src].dev();
            ra.prv = ra.src;
            ra.dst = V.res[out_of(stage)].dev();
            ra.temporal = 0; ra.pass = 1 + it; ra.geom_static = 1;
            ra.out = (stage == stages - 1 && B == 0) ? out : nullptr;
            TRY(reuse_pass(c, V, ra, fixed_wave, s));
            src = out_of(stage);
            ++stage;
            V.ran[3] = true;
        }
    }
    mark(V, 4, s);
    if (B > 0) {
        SplatArgs sa;
        sa.src = V.res[src].dev(); sa.npix = V.W * V.H; sa.B = B; sa.out = out;
        CK(launch_splat(sa, s));
        V.ran[4] = true;
    }
    mark(V, 5, s);
    mark(V, 6, s);
    if (!g_rec) mirror_err(c, s, g_no_marks);
    V.fd[fc] = F;
    V.geom_slot[fc] = S.cur;
    V.geom_version[fc] = S.version[S.cur];
    V.cur = fc;
    V.prev_final = src;
    V.has_prev = true;
    return TOF_OK;
}

tof_status tof_view_profile(tof_ctx* c, tof_view id, int enable) {
    if (!c || id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return c ? fail(c, TOF_EINVAL, "bad view") : TOF_EINVAL;
    cudaSetDevice(c->device);
    ViewH& V = c->views[id];
    if (enable && !V.ev[0])
        for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&V.ev[k]));
    V.profile = enable != 0;
    return TOF_OK;
}

tof_status tof_view_stage_ms(tof_ctx* c, tof_view id, float out[12]) {
    if (!c || !out || id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return c ? fail(c, TOF_EINVAL, "bad view") : TOF_EINVAL;
    ViewH& V = c->views[id];
    if (!V.profile || !V.ev[0]) return fail(c, TOF_ESTATE, "profiling is off for view %d", id);
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize(V.last_stream));
    for (int k = 0; k < 5; ++k) {
        out[k] = 0.f;
        if (V.ran[k]) CK(cudaEventElapsedTime(&out[k], V.ev[k], V.ev[k + 1]));
    }
    CK(cudaEventElapsedTime(&out[5], V.ev[0], V.ev[6]));
    for (int k = 6; k < 12; ++k) out[k] = 0.f;
    // per launch group: setup, forward shifts, forward visibility + emission, inverse shifts,
    // inverse visibility, merge
    const int slot[kReuseEvents - 1] = {6, 7, 10, 8, 11, 9};
    for (size_t g = 0; g + kReuseEvents <= V.kev_used; g += kReuseEvents)
        for (int k = 0; k < kReuseEvents - 1; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, V.kev[g + k], V.kev[g + k + 1]));
            out[slot[k]] += ms;
        }
    return TOF_OK;
}

tof_status tof_render_gated(tof_ctx* c, tof_scene scene, tof_view view, const tof_sensor* sensor, const tof_emitter* emitter,
                            const tof_gate* gate, const tof_params* params, uint64_t seed, uint32_t frame, float* out_image_dev,
                            void* stream) {
    if (!c) return TOF_EINVAL;
    if (!gate) return fail(c, TOF_EINVAL, "gate is NULL");
    return render(c, scene, view, sensor, emitter, gate->L0, gate->dL, 0, params, seed, frame, out_image_dev, stream);
}

tof_status tof_render_gated_noalloc(tof_ctx* c, tof_scene scene, tof_view view, const tof_sensor* sensor,
                                    const tof_emitter* emitter, const tof_gate* gate, const tof_params* params, uint64_t seed,
                                    uint32_t frame, float* out_image_dev, void* stream) {
    if (!c) return TOF_EINVAL;
    if (!gate) return fail(c, TOF_EINVAL, "gate is NULL");
    if (!params) return fail(c, TOF_EINVAL, "params is NULL");
    if (view < 0 || view >= (int)c->views.size() || !c->views[view].alive) return fail(c, TOF_EINVAL, "bad view handle");
    const ViewH& V = c->views[view];
    if (V.B != 0) return fail(c, TOF_EINVAL, "tof_render_gated_noalloc: the view is a transient view");
    if ((size_t)V.W * (size_t)V.H > kNoAllocMaxPix)
        return fail(c, TOF_EINVAL, "tof_render_gated_noalloc: %d x %d pixels exceed the static scratch limit of %zu pixels",
                    V.W, V.H, kNoAllocMaxPix);
    if (params->n_spatial < 0 || (size_t)(1 + params->n_spatial) > kNoAllocMaxSlots)
        return fail(c, TOF_EINVAL, "tof_render_gated_noalloc: n_spatial %d exceeds the static scratch limit of %zu",
                    params->n_spatial, kNoAllocMaxSlots - 1);
    cudaSetDevice(c->device);
    WaveDev w;
    TRY(noalloc_wave(c, &w));
    return render(c, scene, view, sensor, emitter, gate->L0, gate->dL, 0, params, seed, frame, out_image_dev, stream, &w);
}

tof_status tof_render_transient(tof_ctx* c, tof_scene scene, tof_view view, const tof_sensor* sensor,
                                const tof_emitter* emitter, const tof_bins* bins, const tof_params* params, uint64_t seed,
                                uint32_t frame, float* out_hist_dev, void* stream) {
    if (!c) return TOF_EINVAL;
    if (!bins || bins->B < 1) return fail(c, TOF_EINVAL, "bins missing or B < 1");
    return render(c, scene, view, sensor, emitter, bins->t0, bins->width, bins->B, params, seed, frame, out_hist_dev, stream);
}

// number of objects of a scene (used by the server to copy a request's transforms); -1 if invalid
__attribute__((visibility("hidden"))) int tof_internal_scene_objects(tof_ctx* c, tof_scene id) {
    if (!c || id < 0 || id >= (int)c->scenes.size() || !c->scenes[id].alive) return -1;
    return c->scenes[id].nobj;
}

// validate one job of a batch and allocate its view's scratch (allocation is not allowed inside the
// capture)
static tof_status prepare_job(tof_ctx* c, const tof_job& J, uint32_t i) {
    if (J.view < 0 || J.view >= (int)c->views.size() || !c->views[J.view].alive)
        return fail(c, TOF_EINVAL, "job %u: bad view handle", i);
    if (J.scene < 0 || J.scene >= (int)c->scenes.size() || !c->scenes[J.scene].alive)
        return fail(c, TOF_EINVAL, "job %u: bad scene handle", i);
    if (!c->scenes[J.scene].built) return fail(c, TOF_ESTATE, "job %u: scene %d has no BVH", i, J.scene);
    ViewH& V = c->views[J.view];
    TRY(check_params(c, &J.params, J.transient != 0));
    if ((J.params.flags & TOF_FLAG_ELLIPSOID) && !c->scenes[J.scene].enode[0])
        return fail(c, TOF_EINVAL, "job %u: the ellipsoidal connection supports scenes of up to 2^%d triangles", i, kEllMaxLevels);
    TRY(check_sensor(c, &J.sensor, V.W, V.H));
    if (!J.out_dev) return fail(c, TOF_EINVAL, "job %u: output pointer is NULL", i);
    const size_t npix = (size_t)V.W * V.H, Bn = V.B > 0 ? (size_t)V.B : 1;
    size_t cap = npix * Bn < ((size_t)1 << 22) ? npix * Bn : ((size_t)1 << 22);
    if (cap < npix && V.B == 0) cap = npix;
    int S = 1 + J.params.n_spatial > 2 ? 1 + J.params.n_spatial : 2;
    if (J.transient && (J.params.flags & TOF_FLAG_BIN_REUSE) && S < 3) S = 3;
    TRY(ensure_wave(c, V, S, (int)cap));
    if (use_ell_wave(V, J.transient ? V.B : 0, &J.params, false)) TRY(ensure_ell_wave(c, V, J.params.n_cand, J.params.depth));
    if (batch_tree_wave(V, J)) TRY(ensure_tree_wave(c, V, J.params.n_cand, J.params.depth));
    return TOF_OK;
}

// allocate the scratch a job's view needs (as the first batch with that job would), for callers that
// account device memory per view before launching (the served form's admission)
__attribute__((visibility("hidden"))) tof_status tof_internal_prepare_job(tof_ctx* c, const tof_job* job) {
    if (!c || !job) return TOF_EINVAL;
    cudaSetDevice(c->device);
    return prepare_job(c, *job, 0);
}

// launch a captured batch graph through the slot's executable graph (updated in place when only node
// parameters changed, else instantiated again); the graph itself is consumed
static tof_status launch_batch_graph(tof_ctx* c, cudaGraph_t graph, int slot, cudaStream_t stream) {
    cudaGraphExec_t& X = c->batch_exec[slot];
    bool updated = false;
    if (X) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(X, graph, &info) == cudaSuccess) updated = true;
        else {
            cudaGetLastError();
            cudaGraphExecDestroy(X);
            X = nullptr;
        }
    }
    if (!updated) {
        cudaError_t e = cudaGraphInstantiate(&X, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            X = nullptr;
            return fail(c, TOF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    cudaGraphDestroy(graph);
    CK(cudaGraphLaunch(X, stream));
    return TOF_OK;
}

// staged batches: jobs whose every stage has a batched kernel (gated views without the ellipsoidal
// connection, the triangle walk, the shrink mapping or a laser emitter)
static bool stageable(const tof_job& J) {
    return !J.transient && !(J.params.flags & (TOF_FLAG_ELLIPSOID | TOF_FLAG_TRIANGLE_WALK)) && !(J.params.shrink_k > 1.f) &&
           J.emitter.type != TOF_EMIT_LASER;
}
static size_t al256h(size_t b) { return (b + 255) / 256 * 256; }

// argument tables of one group of a staged batch, laid out in the slot's staging buffer from `off`
struct StagedGroup {
    BatchRec rec;
    std::vector<int> bpix;
    std::vector<std::vector<int>> bs, bu;
    size_t o_g = 0, o_i = 0, o_b = 0;
    std::vector<size_t> o_p, o_s, o_u;
};
static size_t staged_layout(StagedGroup& G, size_t off) {
    const size_t nj = G.rec.gbuf.size(), np = G.rec.pass.size();
    G.bpix.assign(nj + 1, 0);
    for (size_t j = 0; j < nj; ++j) {
        const GbufArgs& g = G.rec.gbuf[j];
        const int tw = g.tile_w, th = 128 / tw;
        G.bpix[j + 1] = G.bpix[j] + ((g.F.W + tw - 1) / tw) * ((g.F.H + th - 1) / th);
    }
    G.o_g = off;
    off = al256h(off + sizeof(GbufArgs) * nj);
    G.o_i = off;
    off = al256h(off + sizeof(InitArgs) * nj);
    G.o_b = off;
    off = al256h(off + sizeof(int) * (nj + 1));
    G.o_p.assign(np, 0); G.o_s.assign(np, 0); G.o_u.assign(np, 0);
    G.bs.assign(np, {}); G.bu.assign(np, {});
    for (size_t q = 0; q < np; ++q) {
        const std::vector<ReuseJob>& P = G.rec.pass[q];
        G.bs[q].assign(P.size() + 1, 0);
        G.bu[q].assign(P.size() + 1, 0);
        for (size_t k = 0; k < P.size(); ++k) {
            const long long npx = P[k].p1 - P[k].p0;
            G.bs[q][k + 1] = G.bs[q][k] + (int)((npx + 127) / 128);
            G.bu[q][k + 1] = G.bu[q][k] + (int)((npx * P[k].a.dst.words + 127) / 128);
        }
        G.o_p[q] = off;
        off = al256h(off + sizeof(ReuseJob) * P.size());
        G.o_s[q] = off;
        off = al256h(off + sizeof(int) * (P.size() + 1));
        G.o_u[q] = off;
        off = al256h(off + sizeof(int) * (P.size() + 1));
    }
    return off;
}
static void staged_fill(const StagedGroup& G, unsigned char* h) {
    const size_t nj = G.rec.gbuf.size();
    memcpy(h + G.o_g, G.rec.gbuf.data(), sizeof(GbufArgs) * nj);
    memcpy(h + G.o_i, G.rec.init.data(), sizeof(InitArgs) * nj);
    memcpy(h + G.o_b, G.bpix.data(), sizeof(int) * (nj + 1));
    for (size_t q = 0; q < G.rec.pass.size(); ++q) {
        memcpy(h + G.o_p[q], G.rec.pass[q].data(), sizeof(ReuseJob) * G.rec.pass[q].size());
        memcpy(h + G.o_s[q], G.bs[q].data(), sizeof(int) * G.bs[q].size());
        memcpy(h + G.o_u[q], G.bu[q].data(), sizeof(int) * G.bu[q].size());
    }
}
static cudaError_t staged_launch(tof_ctx* c, const StagedGroup& G, unsigned char* d, cudaStream_t q) {
    const int nj = (int)G.rec.gbuf.size();
    if (nj == 0) return cudaSuccess;
    cudaError_t e = launch_gbuffer_batch((const GbufArgs*)(d + G.o_g), (const int*)(d + G.o_b), nj, G.bpix[nj], q);
    if (e == cudaSuccess) e = launch_initial_batch((const InitArgs*)(d + G.o_i), (const int*)(d + G.o_b), nj, G.bpix[nj], q);
    for (size_t k = 0; k < G.rec.wave.size() && e == cudaSuccess; ++k) {
        const WaveRec& w = G.rec.wave[k];
        e = launch_initial_tree_wave(w.a, w.w, w.tile_h, w.hit_blocks, w.vis_blocks, q);
    }
    for (size_t k = 0; k < G.rec.pass.size() && e == cudaSuccess; ++k)
        e = launch_reuse_batch((const ReuseJob*)(d + G.o_p[k]), (int)G.rec.pass[k].size(), (const int*)(d + G.o_s[k]),
                               G.bs[k].back(), (const int*)(d + G.o_u[k]), G.bu[k].back(), c->persist_blocks, c->vis_blocks, q);
    return e;
}

// One graph for the whole batch: the instances are split into kStagedGroups groups of similar
// estimated work, and each group is a branch of the graph with one launch per stage over all its
// instances (per-pixel stages map each block to its instance, persistent stages pull every
// instance's tasks in turn).  render() records every instance's stage arguments (advancing the
// views' state exactly as a direct render does); the tables are copied once at the head of the
// graph.  The branches let different stages of different groups overlap on the device, which one
// stage at a time over every instance would not (latency-bound stages leave the GPU half idle).
constexpr uint32_t kStagedGroups = 4;
static tof_status render_batch_staged(tof_ctx* c, const tof_job* jobs, uint32_t n, cudaStream_t stream, int slot) {
    TRY(persist_init(c));
    if (!c->capture) CK(cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    if (!c->fork) CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    if (!c->bdone[slot]) CK(cudaEventCreateWithFlags(&c->bdone[slot], cudaEventDisableTiming));
    else CK(cudaEventSynchronize(c->bdone[slot]));   // the slot's staging buffer is free again
    const uint32_t NG = n < kStagedGroups ? n : kStagedGroups;
    while (c->pool.size() < NG) {
        cudaStream_t q;
        cudaEvent_t e;
        CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->pool.push_back(q);
        c->join.push_back(e);
    }
    // groups: longest estimated work first onto the least loaded group
    std::vector<double> cost(n), load(NG, 0.0);
    std::vector<uint32_t> order(n), group(n);
    for (uint32_t i = 0; i < n; ++i) {
        const tof_job& J = jobs[i];
        const ViewH& V = c->views[J.view];
        const double passes = 1.0 + (J.params.temporal ? 1.0 : 0.0) + J.params.n_spatial_iters * (1.0 + J.params.n_spatial);
        cost[i] = (double)V.W * V.H * J.params.depth * (J.params.n_cand + passes);
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
    for (uint32_t i : order) {
        uint32_t best = 0;
        for (uint32_t g = 1; g < NG; ++g)
            if (load[g] < load[best]) best = g;
        group[i] = best;
        load[best] += cost[i];
    }
    std::vector<StagedGroup> G(NG);
    g_no_marks = true;
    tof_status st = TOF_OK;
    for (uint32_t i = 0; i < n && st == TOF_OK; ++i) {
        const tof_job& J = jobs[i];
        g_rec = &G[group[i]].rec;
        st = render(c, J.scene, J.view, &J.sensor, &J.emitter, J.gate.L0, J.gate.dL, 0, &J.params, J.seed, J.frame, J.out_dev,
                    stream);
        if (st == TOF_OK && g_rec->init.size() != g_rec->gbuf.size())
            st = fail(c, TOF_ESTATE, "staged batch: job %u recorded no initial stage", i);
    }
    g_rec = nullptr;
    g_no_marks = false;
    TRY(st);
    size_t bytes = 0;
    for (StagedGroup& g : G) bytes = staged_layout(g, bytes);
    if (c->bstage_bytes[slot] < bytes) {
        if (c->bstage[slot]) cudaFreeHost(c->bstage[slot]);
        c->bstage[slot] = nullptr;
        c->bstage_bytes[slot] = 0;
        CK(cudaHostAlloc(&c->bstage[slot], bytes, cudaHostAllocDefault));
        c->bstage_bytes[slot] = bytes;
    }
    if (c->btab_bytes[slot] < bytes) {
        dfree(c, c->btab[slot]);
        c->btab[slot] = nullptr;
        c->btab_bytes[slot] = 0;
        TRY(dalloc(c, &c->btab[slot], bytes, "batch argument tables"));
        c->btab_bytes[slot] = bytes;
    }
    unsigned char* h = (unsigned char*)c->bstage[slot];
    for (const StagedGroup& g : G) staged_fill(g, h);
    unsigned char* d = c->btab[slot];
    c->in_batch = true;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t r = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->capture);
        if (r == cudaSuccess) r = cudaEventRecord(c->fork, c->capture);
        for (uint32_t g = 0; g < NG && r == cudaSuccess; ++g) {
            r = cudaStreamWaitEvent(c->pool[g], c->fork, 0);
            if (r == cudaSuccess) r = staged_launch(c, G[g], d, c->pool[g]);
            if (r == cudaSuccess) r = cudaEventRecord(c->join[g], c->pool[g]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(c->capture, c->join[g], 0);
        }
        e = cudaStreamEndCapture(c->capture, &graph);
        if (r != cudaSuccess) e = r;
    }
    c->in_batch = false;
    if (e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(c, TOF_ECUDA, "staged batch capture failed: %s", cudaGetErrorString(e));
    }
    TRY(launch_batch_graph(c, graph, slot, stream));
    CK(cudaEventRecord(c->bdone[slot], stream));
    mirror_err(c, stream, false);
    for (uint32_t i = 0; i < n; ++i) c->views[jobs[i].view].last_stream = stream;
    return TOF_OK;
}

static tof_status render_batch(tof_ctx* c, const tof_job* jobs, uint32_t n, void* stream, int slot) {
    if (!c) return TOF_EINVAL;
    if (!jobs || n == 0) return fail(c, TOF_EINVAL, "empty batch");
    if (slot < 0 || slot >= kBatchSlots) return fail(c, TOF_EINVAL, "batch slot %d outside [0, %d)", slot, kBatchSlots);
    if (c->in_batch) return fail(c, TOF_ESTATE, "tof_render_batch is not re-entrant");
    cudaSetDevice(c->device);
    TRY(pending_err(c));
    std::vector<int> seen;
    for (uint32_t i = 0; i < n; ++i) {
        const tof_job& J = jobs[i];
        for (int v : seen)
            if (v == J.view) return fail(c, TOF_EINVAL, "job %u: view %d used by two jobs of one batch", i, J.view);
        seen.push_back(J.view);
        TRY(prepare_job(c, J, i));
    }
    bool staged = true;
    for (uint32_t i = 0; i < n && staged; ++i) staged = stageable(jobs[i]);
    if (staged) return render_batch_staged(c, jobs, n, (cudaStream_t)stream, slot);
    TRY(persist_init(c));
    const uint32_t P = n < 16 ? n : 16;
    while (c->pool.size() < P) {
        cudaStream_t q;
        cudaEvent_t e;
        CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->pool.push_back(q);
        c->join.push_back(e);
    }
    if (!c->fork) CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    if (!c->capture) CK(cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    // stream of each job: longest estimated work first onto the least loaded stream, so that no
    // branch of the graph carries several of the largest instances (the critical path)
    std::vector<double> cost(n), load(P, 0.0);
    std::vector<uint32_t> order(n), branch(n);
    for (uint32_t i = 0; i < n; ++i) {
        const tof_job& J = jobs[i];
        const ViewH& V = c->views[J.view];
        const double passes = 1.0 + (J.params.temporal ? 1.0 : 0.0) + J.params.n_spatial_iters * (1.0 + J.params.n_spatial);
        cost[i] = (double)V.W * V.H * J.params.depth * (J.params.n_cand + passes) * (J.transient ? 8.0 : 1.0);
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
    for (uint32_t i : order) {
        uint32_t best = 0;
        for (uint32_t p = 1; p < P; ++p)
            if (load[p] < load[best]) best = p;
        branch[i] = best;
        load[best] += cost[i];
    }
    // capture: fork onto the pool, one branch per stream, join
    c->in_batch = true;
    g_no_marks = true;
    tof_status st = TOF_OK;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaEventRecord(c->fork, c->capture);
        for (uint32_t p = 0; p < P; ++p) cudaStreamWaitEvent(c->pool[p], c->fork, 0);
        for (uint32_t k = 0; k < n && st == TOF_OK; ++k) {
            const uint32_t i = order[k];
            const tof_job& J = jobs[i];
            cudaStream_t q = c->pool[branch[i]];
            if (J.transient)
                st = render(c, J.scene, J.view, &J.sensor, &J.emitter, J.bins.t0, J.bins.width, J.bins.B, &J.params, J.seed,
                            J.frame, J.out_dev, q);
            else
                st = render(c, J.scene, J.view, &J.sensor, &J.emitter, J.gate.L0, J.gate.dL, 0, &J.params, J.seed, J.frame,
                            J.out_dev, q);
        }
        for (uint32_t p = 0; p < P; ++p) {
            cudaEventRecord(c->join[p], c->pool[p]);
            cudaStreamWaitEvent(c->capture, c->join[p], 0);
        }
        e = cudaStreamEndCapture(c->capture, &graph);
    }
    g_no_marks = false;
    c->in_batch = false;
    if (st != TOF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess || !graph) {
        cudaGetLastError();
        return fail(c, TOF_ECUDA, "batch capture failed: %s", cudaGetErrorString(e));
    }
    TRY(launch_batch_graph(c, graph, slot, (cudaStream_t)stream));
    mirror_err(c, (cudaStream_t)stream, false);
    for (uint32_t i = 0; i < n; ++i) c->views[jobs[i].view].last_stream = (cudaStream_t)stream;
    return TOF_OK;
}

tof_status tof_render_batch(tof_ctx* c, const tof_job* jobs, uint32_t n, void* stream) {
    return render_batch(c, jobs, n, stream, 0);
}

// batch on graph slot `slot` (the served form keeps several batches in flight, one slot each)
__attribute__((visibility("hidden"))) tof_status tof_internal_render_batch(tof_ctx* c, const tof_job* jobs, uint32_t n,
                                                                         void* stream, int slot) {
    return render_batch(c, jobs, n, stream, slot);
}

static tof_status check_tuning(tof_ctx* c, const tof_tuning* t) {
    if (!t) return fail(c, TOF_EINVAL, "tuning is NULL");
    const int tw = t->tile_w, th = t->tile_h;
    if (tw < 4 || tw > 32 || (tw & (tw - 1)) || th < 1 || (tw * th != 64 && tw * th != 128))
        return fail(c, TOF_EINVAL, "tile %d x %d: tile_w must be a power of two in [4, 32] and tile_w * tile_h 64 or 128",
                    tw, th);
    if (t->packet < 0 || t->packet > 8) return fail(c, TOF_EINVAL, "packet %d outside [0, 8]", t->packet);
    if (t->layout != TOF_LAYOUT_SOA && t->layout != TOF_LAYOUT_AOS) return fail(c, TOF_EINVAL, "unknown layout %d", t->layout);
    return TOF_OK;
}

tof_status tof_view_set_tuning(tof_ctx* c, tof_view id, const tof_tuning* t) {
    if (!c) return TOF_EINVAL;
    if (id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return fail(c, TOF_EINVAL, "bad view handle");
    TRY(check_tuning(c, t));
    ViewH& V = c->views[id];
    if (t->layout != V.tune.layout) {
        // the stored reservoirs are in the old layout: forget them
        V.has_prev = false;
        V.prev_final = -1;
        for (int k = 0; k < 3; ++k) V.res[k].layout = t->layout;
    }
    V.tune = *t;
    return TOF_OK;
}

tof_status tof_view_get_tuning(tof_ctx* c, tof_view id, tof_tuning* out) {
    if (!c) return TOF_EINVAL;
    if (!out || id < 0 || id >= (int)c->views.size() || !c->views[id].alive) return fail(c, TOF_EINVAL, "bad view handle");
    *out = c->views[id].tune;
    return TOF_OK;
}

// instance class of a job for the autotuner: transient bins (0 = gated) and a pixel-count bucket
static std::pair<int, int> tune_class(const ViewH& V) {
    const long long np = (long long)V.W * V.H;
    int bucket = np < 128 * 128 ? 0 : np < 256 * 256 ? 1 : np < 512 * 512 ? 2 : 3;
    return std::make_pair(V.B, bucket);
}

tof_status tof_autotune(tof_ctx* c, const tof_job* jobs, uint32_t n, int32_t frames, void* stream, tof_tuning* out) {
    if (!c) return TOF_EINVAL;
    if (!jobs || n == 0) return fail(c, TOF_EINVAL, "no jobs");
    if (frames < 2 || frames > 64) return fail(c, TOF_EINVAL, "frames %d outside [2, 64]", frames);
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::map<std::pair<int, int>, std::vector<uint32_t>> classes;
    for (uint32_t i = 0; i < n; ++i) {
        const tof_job& J = jobs[i];
        if (J.view < 0 || J.view >= (int)c->views.size() || !c->views[J.view].alive)
            return fail(c, TOF_EINVAL, "job %u: bad view handle", i);
        if (J.scene < 0 || J.scene >= (int)c->scenes.size() || !c->scenes[J.scene].alive || !c->scenes[J.scene].built)
            return fail(c, TOF_EINVAL, "job %u: bad or unbuilt scene", i);
        if (c->views[J.view].scene != J.scene) return fail(c, TOF_EINVAL, "job %u: view and scene differ", i);
        classes[tune_class(c->views[J.view])].push_back(i);
    }
    // the jobs on scratch views (same scene, size and bins) with scratch outputs: the candidates are
    // timed on the whole batch, where instances of different classes run beside each other
    std::vector<tof_job> sj(jobs, jobs + n);
    std::vector<tof_view> sv;
    std::vector<float*> so;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tof_status st = TOF_OK;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        for (float* p : so) dfree(c, p);
        for (tof_view v : sv) tof_view_destroy(c, v);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    for (uint32_t i = 0; i < n && st == TOF_OK; ++i) {
        const ViewH& V = c->views[jobs[i].view];
        tof_view v = -1;
        st = tof_view_create(c, jobs[i].scene, V.W, V.H, V.B, &v);
        if (st != TOF_OK) break;
        sv.push_back(v);
        float* o = nullptr;
        st = dalloc(c, &o, sizeof(float) * (size_t)V.W * V.H * (V.B > 0 ? V.B : 1), "autotune output");
        if (st != TOF_OK) break;
        so.push_back(o);
        sj[i].view = v;
        sj[i].out_dev = o;
    }
    if (st == TOF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(c, TOF_ECUDA, "cudaEventCreate failed");
    if (st != TOF_OK) { cleanup(); return st; }
    std::map<std::pair<int, int>, tof_tuning> cur;
    for (auto& kv : classes) cur[kv.first] = tof_tuning{16, 8, 0, TOF_LAYOUT_SOA};
    // `frames` consecutive batches under the current tunings, the first untimed
    auto time_batch = [&](float* ms) -> tof_status {
        for (auto& kv : classes)
            for (uint32_t i : kv.second) {
                TRY(tof_view_set_tuning(c, sj[i].view, &cur[kv.first]));
                TRY(tof_reservoirs_reset(c, sj[i].view));
            }
        for (int f = 0; f < frames; ++f) {
            for (uint32_t i = 0; i < n; ++i) sj[i].frame = jobs[i].frame + (uint32_t)f;
            if (f == 1) CK(cudaEventRecord(e0, s));
            TRY(tof_render_batch(c, sj.data(), n, stream));
        }
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        return TOF_OK;
    };
    float best_ms = 0.f;
    st = time_batch(&best_ms);
    // classes with the most pixels first; per class tiles, then packets, then the layout
    std::vector<std::pair<long long, std::pair<int, int>>> by_size;
    for (auto& kv : classes) {
        long long px = 0;
        for (uint32_t i : kv.second) px += (long long)c->views[jobs[i].view].W * c->views[jobs[i].view].H;
        by_size.push_back(std::make_pair(px, kv.first));
    }
    std::sort(by_size.begin(), by_size.end(), [](const std::pair<long long, std::pair<int, int>>& a,
                                                 const std::pair<long long, std::pair<int, int>>& b) { return a.first > b.first; });
    const int tiles[3][2] = {{8, 8}, {32, 4}, {8, 16}};
    const int packets[3] = {8, 4, 2};
    for (auto& cl : by_size) {
        const std::pair<int, int> key = cl.second;
        auto trial = [&](const tof_tuning& t) -> tof_status {
            const tof_tuning keep = cur[key];
            cur[key] = t;
            float ms = 0.f;
            TRY(time_batch(&ms));
            if (ms < best_ms) best_ms = ms;
            else cur[key] = keep;
            return TOF_OK;
        };
        for (int k = 0; k < 3 && st == TOF_OK; ++k) {
            tof_tuning t = cur[key];
            t.tile_w = tiles[k][0]; t.tile_h = tiles[k][1];
            st = trial(t);
        }
        for (int k = 0; k < 3 && st == TOF_OK; ++k) {
            tof_tuning t = cur[key];
            t.packet = packets[k];
            st = trial(t);
        }
        if (st == TOF_OK) {
            tof_tuning t = cur[key];
            t.layout = TOF_LAYOUT_AOS;
            st = trial(t);
        }
        if (st != TOF_OK) break;
    }
    cleanup();
    if (st != TOF_OK) return st;
    for (auto& kv : classes)
        for (uint32_t i : kv.second) {
            TRY(tof_view_set_tuning(c, jobs[i].view, &cur[kv.first]));
            if (out) out[i] = cur[kv.first];
        }
    return TOF_OK;
}

tof_status tof_render_pt(tof_ctx* c, tof_scene scene, const tof_sensor* sensor, const tof_emitter* emitter, const tof_gate* gate,
                         const tof_bins* bins, const tof_params* params, uint64_t seed, uint32_t frame, int32_t spp,
                         float* out_dev, void* stream) {
    if (!c) return TOF_EINVAL;
    if (scene < 0 || scene >= (int)c->scenes.size() || !c->scenes[scene].alive) return fail(c, TOF_EINVAL, "bad scene handle");
    SceneH& S = c->scenes[scene];
    if (!S.built) return fail(c, TOF_ESTATE, "tof_bvh_build has not been called");
    if (!sensor) return fail(c, TOF_EINVAL, "sensor is NULL");
    TRY(check_sensor(c, sensor, sensor->W, sensor->H));
    TRY(check_params(c, params, 0));
    if (!emitter || emitter->type < 0 || emitter->type > 2) return fail(c, TOF_EINVAL, "bad emitter");
    if (spp < 1) return fail(c, TOF_EINVAL, "spp must be >= 1");
    if (!out_dev) return fail(c, TOF_EINVAL, "output pointer is NULL");
    if (!gate && !bins) return fail(c, TOF_EINVAL, "gate or bins required");
    float L0 = bins ? bins->t0 : gate->L0, dL = bins ? bins->width : gate->dL;
    int B = bins ? bins->B : 0;
    if (bins && B < 1) return fail(c, TOF_EINVAL, "B < 1");
    if (!(dL > 0)) return fail(c, TOF_EINVAL, "gate / bin width must be positive");
    cudaSetDevice(c->device);
    TRY(pending_err(c));
    cudaStream_t s = (cudaStream_t)stream;
    LightDev* laser = nullptr;
    if (emitter->type == TOF_EMIT_LASER) {
        if (!c->d_scratch) TRY(dalloc(c, &c->d_scratch, 256, "laser scratch"));
        laser = (LightDev*)c->d_scratch;
    }
    FrameDev F = make_frame(S, S.cur, sensor, emitter, L0, dL, B, frame, nullptr, laser, c->d_err);
    ParamsDev P = to_dev(params, seed);
    if (laser) CK(launch_laser(F.g, v3f(emitter->pos), v3f(emitter->dir), emitter->power, laser, s));
    PtArgs pa;
    pa.F = F; pa.P = P; pa.spp = spp; pa.out = out_dev;
    CK(launch_pt(pa, s));
    mirror_err(c, s, false);
    return TOF_OK;
}

tof_status tof_sync(tof_ctx* c, void* stream) {
    if (!c) return TOF_EINVAL;
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned bits = 0;
    CK(cudaMemcpy(&bits, c->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
    return report_err_bits(c, bits);
}

uint64_t tof_kernel_launches(void) { return (uint64_t)g_kernel_launches.load(std::memory_order_relaxed); }

}  // extern "C"
