/*
 * tof.h -- C ABI of the GB300 ToF ReSTIR library (libtof.so).
 *
 * The library renders time-gated images and transient histograms with the ToF ReSTIR method
 * (Kim, Jarosz, Pediredla, "ToF ReSTIR: Time-of-Flight Rendering with Spatio-temporal Reservoir
 * Resampling", ACM TOG 45(4), 2026): per-pixel RIS reservoirs of light paths under an optical
 * path-length gate, initial path-tree candidates, temporal and spatial reuse through the
 * path-length-aware shift mapping (Newton solve on the reconnection vertex with the
 * average-gradient gauge and its Jacobian), and the splat into a gated image or a transient
 * histogram.  Every stage runs as hand-written CUDA kernels for sm_103a on one GPU.
 *
 * Conventions for every entry point
 *   - Return value: TOF_OK (0) or a negative tof_status; never aborts.  tof_last_error() gives a
 *     one-line message for the last failure on that context.
 *   - Device-side errors (a BVH traversal that overflows its stack or exceeds its visit budget,
 *     a transient pixel whose candidates overflow its bin table) set bits of the context's error
 *     word instead of faulting.  The word is read back asynchronously after every render and
 *     reported (TOF_ECUDA, message naming the cause, word cleared) by the context's next render or
 *     batch call, by tof_view_stats, and by tof_sync, which waits for the stream first.
 *   - Host pointers (const T*) are read during the call only and stay owned by the caller.
 *   - Device pointers (out_*_dev) are caller-owned device memory on the context's GPU, written
 *     asynchronously on `stream` (a cudaStream_t passed as void*, NULL = legacy default stream);
 *     they are valid once the stream has been synchronised.
 *   - Scenes and views are library-owned device state named by integer handles; they persist
 *     until destroyed (or the context is destroyed).
 *   - Units are metres, optical path length uses c = 1 and refractive index 1 (Sec. 3.1).
 *   - Thread safety: one context per host thread, or external locking.
 */
#ifndef TOF_H
#define TOF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tof_status;
#define TOF_OK 0
#define TOF_EINVAL (-1)   /* invalid argument (sizes, ids, NaN geometry, unsupported option) */
#define TOF_ENOMEM (-2)   /* device allocation failed */
#define TOF_EBUDGET (-3)  /* request exceeds the context's HBM budget */
#define TOF_ECUDA (-4)    /* a CUDA runtime call or kernel launch failed */
#define TOF_ETIMEOUT (-5) /* a bounded device-side wait gave up */
#define TOF_ESTATE (-6)   /* call out of order (e.g. render before tof_bvh_build) */

typedef struct tof_ctx tof_ctx;
typedef int32_t tof_scene;
typedef int32_t tof_view;

/* material types (Sec. 6: diffuse, glossy and specular surfaces) */
#define TOF_LAMBERT 0
#define TOF_GGX 1      /* Walter et al. 2007 microfacet, Smith G1*G1, Fresnel = albedo */
#define TOF_MIRROR 2   /* perfect specular reflection */
typedef struct {
    int32_t type;
    float albedo;      /* in [0, 1] */
    float alpha;       /* GGX roughness; ignored otherwise */
} tof_material;

/* sensor: pinhole camera, or confocal scan of a planar wall (one pixel per scanned wall point;
 * the path length of each pixel is measured minus 2 |device - wall point|) */
#define TOF_PINHOLE 0
#define TOF_CONFOCAL 1
typedef struct {
    int32_t mode;
    int32_t W, H;
    float pos[3];      /* camera / device position */
    float fwd[3], up[3];
    float fov_y;       /* radians, pinhole only */
    float wall_o[3], wall_u[3], wall_v[3]; /* confocal only: wall point (i,j) = o + (i+.5)/W u + (j+.5)/H v */
} tof_sensor;

/* emitters (Sec. 5 "Light Source"): delta lights only */
#define TOF_EMIT_POINT 0     /* isotropic point light of intensity `power` at pos, NEE */
#define TOF_EMIT_LASER 1     /* collimated laser from pos along dir; its first hit is a secondary
                                emitter of intensity power * f_s * |cos| (a light ray is traced first) */
#define TOF_EMIT_CONFOCAL 2  /* laser from pos aimed at each pixel's own primary hit */
typedef struct {
    int32_t type;
    float pos[3];
    float dir[3];
    float power;
} tof_emitter;

/* gate [L0, L0 + dL) on tau = L - offset (Sec. 3.1 W_tau, a box; Sec. 6) */
typedef struct { float L0, dL; } tof_gate;

/* transient bins: bin b covers [t0 + b*width, t0 + (b+1)*width) (Sec. 3.1, Sec. 4.5) */
typedef struct { float t0, width; int32_t B; } tof_bins;

/* flags */
#define TOF_FLAG_DIRECT 1u       /* include length-1 (direct) paths; the paper reports indirect only */
#define TOF_FLAG_NAIVE_SHIFT 2u  /* hybrid shift without the path-length correction (comparison) */
/* pairwise MIS instead of the generalized balance heuristic: the canonical sample pairs with each
 * of the k reused ones; pair i is a two-technique balance heuristic between the canonical domain
 * (confidence M_c/k) and domain i (confidence M_i), weighted by (M_i + M_c/k)/sum M.  The weights
 * still sum to one (unbiased), equal the balance heuristic when k = 1 or when every domain's
 * target agrees, and need 2k shifts per merge instead of k + k^2.  Not in the paper (which states
 * the balance heuristic only); an optimisation from the ReSTIR literature. */
#define TOF_FLAG_PAIRWISE_MIS 4u
/* comparison gauges of the Newton system (Sec. 4.3 "Selecting a Good Gauge Condition"; the default
 * is the paper's average-gradient gauge): a fixed axis G(xi) = a^T xi of the reconnection
 * triangle's in-plane frame (the vertex moves along t, or along b), reversible; or the gradient at
 * the start point alone, which is not reversible (biased under MIS: the paper's counterexample).
 * At most one of the three. */
#define TOF_FLAG_GAUGE_AXIS_T 8u
#define TOF_FLAG_GAUGE_AXIS_B 16u
#define TOF_FLAG_GAUGE_START 32u
/* cross-triangle walk of the reconnection vertex: when Newton moves the vertex off its triangle,
 * it continues on the neighbour across the edge it crossed (the neighbour unfolded into the
 * triangle's plane about the shared edge), instead of failing the shift.  Neighbours share an edge
 * (two vertex indices) within one object.  Shifts stay reversible; on planar surfaces the result
 * no longer depends on the tessellation. */
#define TOF_FLAG_TRIANGLE_WALK 64u
/* transient rendering: bin reuse (Sec. 4.5, the histogram's extra reuse axis) -- one pass after
 * temporal reuse in which the reservoir of bin b also reuses the same pixel's bins b - 1 and
 * b + 1, shifted into bin b's gate by one bin width; bins outside the histogram are no domains. */
#define TOF_FLAG_BIN_REUSE 128u
/* ellipsoidal path connection for the initial candidates (Sec. 4.4 "Initialization with
 * Ellipsoidal Path Connection", Sec. 5 "Ellipsoidal Path Connection"): every rough vertex x of a
 * path tree below the maximum depth also places a vertex z with |x - z| + |z - light| drawn
 * uniformly in the interval the gate (or the histogram's range) leaves, so that the NEE path
 * through z lies in it.  z's triangle comes from an area-weighted walk of the binary hierarchy over
 * triangle index ranges (nodes whose box cannot meet the ellipsoid weigh zero; built by
 * tof_bvh_build for scenes of up to 2^22 triangles, else the flag is rejected), z itself uniformly
 * in the parametric angle of the ellipse the ellipsoid cuts from the triangle, over its arcs inside
 * the triangle.  Each such candidate and the path tree's own candidate of the same length are
 * combined by the balance heuristic over the two densities of the last vertex (the paper's MIS
 * between direct and ellipsoidal connection), so the estimate stays unbiased.  Excludes the shrink
 * mapping.  Gated views run this stage as a wavefront whose scratch the first such render allocates
 * in the view (about 112 B per pixel x tree x vertex: 450 MB for 512 x 512, 4 trees, depth 4, plus
 * the bounce wavefront's for its path trees; views above 32M such slots, transient views and
 * tof_render_gated_noalloc use a single kernel that needs none and gives the same result). */
#define TOF_FLAG_ELLIPSOID 256u

/* reuse / sampling parameters (Sec. 6: path depth, candidates, neighbours, radius, M-cap;
 * Newton tolerance 1 % of the gate width with at most 5 iterations) */
typedef struct {
    int32_t depth;            /* max surface vertices per path, 1..5 */
    int32_t n_cand;           /* path trees per pixel, 1..64 */
    int32_t n_spatial;        /* spatial neighbours per pass, 0..8 */
    int32_t radius;           /* spatial radius in pixels, 1..255 */
    int32_t n_spatial_iters;  /* spatial passes, 0..4 */
    int32_t temporal;         /* temporal reuse on (1) / off (0) */
    float m_cap;              /* confidence cap for reused reservoirs */
    int32_t newton_max_iter;  /* <= 16 */
    float newton_tol_frac;    /* success threshold as a fraction of the gate width */
    float jac_max;            /* reject shifts with |det| outside [1/jac_max, jac_max] */
    float d_min;              /* minimum reconnection segment length */
    float ray_eps;            /* ray origin offset along the normal */
    uint32_t flags;
    /* Sec. 4.4 path-length shrink mapping for initial sampling (gated rendering only): the trees
     * from shrink_fine on draw their candidates in the gate widened shrink_k times about its
     * centre c, and their RIS winner is moved into the gate by the path-length Newton solve with
     * tau' = c + (tau - c) / shrink_k (Jacobian scaled by 1 / shrink_k).  Trees below shrink_fine
     * keep drawing in the gate itself; their winner and the shrunk one are combined with the
     * generalized balance heuristic (unbiased).  shrink_fine = 0 widens every tree (the paper's
     * R = 1: lower variance, darker where shrinking fails).  shrink_k <= 1 turns it off. */
    float shrink_k;
    int32_t shrink_fine;      /* 0 .. n_cand - 1 */
} tof_params;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the device memory the
 * context may allocate for scenes and views (0 = no bound); allocations beyond it fail with
 * TOF_EBUDGET.  Not in the paper: library plumbing (the paper's renderer runs inside Falcor). */
tof_status tof_create(tof_ctx** out, int device, uint64_t hbm_budget_bytes);
tof_status tof_destroy(tof_ctx* ctx);
const char* tof_last_error(tof_ctx* ctx);
/* bytes currently allocated on the device by this context */
uint64_t tof_device_bytes(tof_ctx* ctx);

/* Upload a triangle scene (Sec. 6 scenes: triangle meshes with per-object materials).
 *   verts  [nv*3] object-local positions; tris [nt*3] vertex indices; tri_object [nt] object id;
 *   mats [nmat]; object_material [nobj] material id per object.
 * Host arrays are copied.  Rejects non-finite vertices, out-of-range ids, nt == 0. */
tof_status tof_scene_upload(tof_ctx* ctx, const float* verts, uint32_t nv, const uint32_t* tris, uint32_t nt,
                            const uint32_t* tri_object, const tof_material* mats, uint32_t nmat,
                            const uint32_t* object_material, uint32_t nobj, tof_scene* out);
tof_status tof_scene_destroy(tof_ctx* ctx, tof_scene scene);

/* Place the objects (row-major 3x4 object-to-world matrices, nobj*12 floats) and build the GPU
 * LBVH (Morton codes, radix sort, hierarchy, bounds).  Not in the paper, which traces rays with
 * the GPU's ray-tracing hardware through DXR (Sec. 6); GB300 has no such units, so the library
 * builds its own hierarchy (Karras 2012 construction over 30-bit Morton codes).  refit_only = 1 keeps the hierarchy and
 * refits bounds after rigid motion: cheaper to build, but the hierarchy's quality decays as objects
 * move away from where it was built (a full build of 66k triangles takes about 0.2 ms on GB300 and
 * pays for itself within a few frames of motion).  Call once per frame before rendering it: the library keeps
 * the geometry of the previous call resident for temporal reuse (an exact inverse shift into the
 * previous frame needs the previous scene).  Transforms identical to the current ones are a
 * no-op (the scene is static between the two frames). */
tof_status tof_bvh_build(tof_ctx* ctx, tof_scene scene, const float* object_xforms, int refit_only, void* stream);

/* Per-view device state (reservoirs of the current and previous frame, G-buffers, confidence)
 * for a W x H sensor; B = 0 for gated rendering, else the number of transient bins. */
tof_status tof_view_create(tof_ctx* ctx, tof_scene scene, int32_t W, int32_t H, int32_t B, tof_view* out);
tof_status tof_view_destroy(tof_ctx* ctx, tof_view view);

/* Render one time-gated frame (Sec. 3.2 stages (1)-(4)): G-buffer, initial path-tree RIS,
 * temporal reuse against the view's previous frame (params->temporal), params->n_spatial_iters
 * spatial passes, and the gated image out_image_dev[H*W] (row-major, float32) = f(y) W_y.
 * `frame` keys the random streams together with `seed`.  Without the ellipsoidal connection and
 * the shrink mapping, views of up to 16M pixels x trees run the initial stage as a bounce
 * wavefront whose scratch (about 240 MB for 512 x 512 x 4 trees at depth 4) the first such render
 * allocates; it gives the same reservoirs as the single kernel that small instances of a batch
 * and the allocation-free form run.  The temporal pass runs part of its work on a stream of the view
 * (created with the view's first such render), forked from `stream` by an event and joined back
 * into it before the spatial passes, so the frame completes in `stream` order as before, and a
 * capture of `stream` into a CUDA graph takes that branch in. */
tof_status tof_render_gated(tof_ctx* ctx, tof_scene scene, tof_view view, const tof_sensor* sensor,
                            const tof_emitter* emitter, const tof_gate* gate, const tof_params* params,
                            uint64_t seed, uint32_t frame, float* out_image_dev, void* stream);

/* Allocation-free variant of tof_render_gated, for callers that may not allocate device memory
 * while they render: code that records frames into a CUDA graph, real-time loops that run under
 * a fixed device-memory pool, or hosts that forbid cudaMalloc after start-up.  tof_render_gated
 * allocates a view's reuse scratch (slot tables, shift task lists, shifted records, MIS terms)
 * with cudaMalloc on the view's first frame; this entry point takes that scratch from a static
 * device array compiled into the library instead and calls no cudaMalloc, cudaFree or other
 * allocating routine.  The paper has no counterpart; the rendering it performs is exactly that
 * of tof_render_gated.
 *   - Limits: the view has W*H <= 16384 pixels (e.g. 128 x 128), is a gated view (B = 0), and
 *     params->n_spatial <= 5; larger requests fail with TOF_EINVAL and a message naming the limit.
 *   - The static array (about 15.6 MiB) belongs to the library's device image: every GPU that
 *     loads libtof.so holds it until the process exits.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress with
 *     that device current).  Under CUDA's lazy module loading (the default) that lookup is also
 *     what loads the library's host-side module and commits the array's device memory, so the
 *     first call does take memory once; later calls take none.  Make that first call at set-up,
 *     before any stream capture.
 *   - Every call shares the one array and each call overwrites it (its task counters are reset on
 *     the stream at the start of each reuse pass): calls whose work overlaps on the GPU -- on
 *     different streams, or from different threads -- race and must be serialised by the caller.
 *   - Scene, view and output are as for tof_render_gated; the view itself (tof_view_create) is
 *     allocated at set-up time. */
tof_status tof_render_gated_noalloc(tof_ctx* ctx, tof_scene scene, tof_view view, const tof_sensor* sensor,
                                    const tof_emitter* emitter, const tof_gate* gate, const tof_params* params,
                                    uint64_t seed, uint32_t frame, float* out_image_dev, void* stream);

/* Render one transient frame (Sec. 4.5): per-bin reservoirs, per-bin temporal / spatial reuse,
 * and the histogram out_hist_dev[H*W*B] (bin fastest, float32). */
tof_status tof_render_transient(tof_ctx* ctx, tof_scene scene, tof_view view, const tof_sensor* sensor,
                                const tof_emitter* emitter, const tof_bins* bins, const tof_params* params,
                                uint64_t seed, uint32_t frame, float* out_hist_dev, void* stream);

/* One render job of a batch (batched rendering of many independent instances): a gated (transient == 0) or
 * transient frame of one view, exactly as tof_render_gated / tof_render_transient would render it. */
typedef struct {
    tof_scene scene;
    tof_view view;
    tof_sensor sensor;
    tof_emitter emitter;
    tof_gate gate;            /* used when transient == 0 */
    tof_bins bins;            /* used when transient != 0 */
    int32_t transient;
    tof_params params;
    uint64_t seed;
    uint32_t frame;
    float* out_dev;           /* H*W (gated) or H*W*B (transient) floats, caller-owned device memory */
} tof_job;

/* Render n independent jobs as one CUDA graph launched on `stream`.  When every job is a gated view
 * without the ellipsoidal connection, the triangle walk, the shrink mapping or a laser emitter, the
 * jobs are split into 4 groups of similar estimated work and each group is one branch of the graph
 * with one kernel launch per stage over all of its instances (per-pixel stages map each block to its
 * instance; persistent stages pull every instance's tasks), ~20 launches per group whatever the
 * number of instances; the stage arguments travel as tables copied at the head of the graph.
 * A gated instance of 256 x 256 pixels or more runs its initial stage as the bounce wavefront on its
 * group's branch (its scratch is allocated before capture, like every view's); smaller ones are
 * blocks of the batched single kernel.
 * Otherwise every job's stage kernels form their own branch (16 concurrent branches).  Jobs must
 * use distinct views.  Results equal those of rendering each job on its own.  Scratch for every view
 * is allocated before the graph is captured (first use of a view). */
tof_status tof_render_batch(tof_ctx* ctx, const tof_job* jobs, uint32_t n, void* stream);

/* Launch shapes and reservoir layout of a view (the batched form's per-instance-class tuning).
 * None of them changes a result: every pixel's random numbers are keyed by the pixel, and the
 * merges read their inputs by index, so a frame renders to the same bits under every tuning.
 *   tile_w x tile_h: pixel tile of the per-pixel kernels (G-buffer, initial candidates), one thread
 *     per pixel; tile_w a power of two in [4, 32], tile_w * tile_h = 64 or 128.
 *   packet: blocks of 128 threads per SM that pull shift and visibility tasks in the persistent
 *     reuse kernels (the width of the task packets in flight per SM), 1..8; 0 = as many as fit.
 *     Fewer leave room for other instances of a batch to run beside this one.
 *   layout: TOF_LAYOUT_SOA (six 16-byte planes, the default) or TOF_LAYOUT_AOS (each reservoir's
 *     96 bytes contiguous).
 * In a staged batch (tof_render_batch) the per-pixel stages run blocks of 128 threads, tiles of
 * tile_w x (128 / tile_w) pixels, and the persistent stages run as many blocks as fit: there only
 * tile_w and the layout of a view's tuning apply. */
#define TOF_LAYOUT_SOA 0
#define TOF_LAYOUT_AOS 1
typedef struct {
    int32_t tile_w, tile_h;
    int32_t packet;
    int32_t layout;
} tof_tuning;

/* Set / read a view's tuning.  Changing the layout forgets the view's history (the next frame
 * renders without temporal reuse); the other fields take effect at the next frame.  TOF_EINVAL for
 * out-of-range fields. */
tof_status tof_view_set_tuning(tof_ctx* ctx, tof_view view, const tof_tuning* t);
tof_status tof_view_get_tuning(tof_ctx* ctx, tof_view view, tof_tuning* out);

/* Autotuner for batched rendering.  Groups the jobs into instance classes (gated or transient with
 * its bin count, and the pixel count: below 128^2, 256^2, 512^2, or above) and chooses each class's
 * tuning by coordinate descent -- tiles 8x8, 32x4, 8x16 against the default 16x8, then packets 8,
 * 4, 2, then the AoS layout, each kept only if it makes the whole batch faster -- with classes of
 * more pixels first.  Every candidate is timed on the whole batch (tof_render_batch, `frames`
 * consecutive frames, the first untimed), rendered on scratch views of the jobs' scenes and sizes
 * that the call creates and destroys, so the jobs' own views keep their history (unless their
 * layout changes) and the scratch views take as much device memory again while it runs.  The
 * scenes must have been built.  The chosen tunings are set on the jobs' views and, if out is not
 * NULL, written to out[i].  Synchronises `stream`; not for use during stream capture. */
tof_status tof_autotune(tof_ctx* ctx, const tof_job* jobs, uint32_t n, int32_t frames, void* stream, tof_tuning* out);

/* Served form: a request scheduler over several dynamic streams (continuous batching).  Not in the
 * paper (its renderer serves one view); the method's real-time intent (Sec. 6) served as a system.
 *   A stream is a scene plus a fixed sensor resolution (and bin count for transient streams); its
 *   view -- reservoirs, G-buffers, confidences, reuse scratch -- is created on admission and stays
 *   resident, so frames of a stream reuse their predecessors temporally.
 *   tof_server_submit queues one frame request: the job (view field ignored) and the frame's
 *   object transforms (nobj * 12 floats, copied).  tof_server_step retires batches whose GPU work
 *   has finished and admits pending requests in arrival order: at most one frame in flight per
 *   stream and per scene (streams may share a scene; its BVH is rebuilt only while no frame reads
 *   it).  A stream's first admission creates its view and scratch, measures the device bytes they
 *   took and keeps them only if the resident views fit the server's HBM budget, evicting the least
 *   recently used idle views (no frame in flight, none queued; an evicted stream's next frame
 *   renders without temporal reuse) to make room; otherwise the request waits.  The step applies
 *   each admitted stream's transforms (tof_bvh_build, full build) and launches all admitted frames
 *   as one batch graph on the next of the server's own streams (4, round robin), ordered after the
 *   work already queued on `stream`; batches of successive steps therefore overlap on the device.
 *   Requests arriving while batches run join the next step.  Times are host wall-clock:
 *   submit -> observed completion.  The server's results are those of tof_render_gated /
 *   tof_render_transient on the same views (every random number is keyed by pixel and frame). */
typedef struct tof_server tof_server;
tof_status tof_server_create(tof_ctx* ctx, uint64_t hbm_budget_bytes, tof_server** out);
tof_status tof_server_destroy(tof_server* srv);
tof_status tof_server_open_stream(tof_server* srv, tof_scene scene, int32_t W, int32_t H, int32_t B, int32_t* stream_id);
tof_status tof_server_submit(tof_server* srv, int32_t stream_id, const tof_job* job, const float* object_xforms,
                             uint64_t* ticket);
tof_status tof_server_step(tof_server* srv, void* stream);
/* state: 0 queued, 1 on the GPU, 2 done (latency_ms = submit -> completion), -1 unknown ticket */
tof_status tof_server_poll(tof_server* srv, uint64_t ticket, int32_t* state, double* latency_ms);
/* out[0] submitted, out[1] completed, out[2] launched batches, out[3] admissions deferred by the
 * budget, out[4] device bytes of resident stream views, out[5] queued, out[6] in flight */
tof_status tof_server_stats(tof_server* srv, double out[7]);

/* Plain gated (bins == NULL) or transient path tracing without reuse, spp paths per pixel each
 * with its own jitter (the comparison method of Sec. 6).  Output layout as above. */
tof_status tof_render_pt(tof_ctx* ctx, tof_scene scene, const tof_sensor* sensor, const tof_emitter* emitter,
                         const tof_gate* gate, const tof_bins* bins, const tof_params* params, uint64_t seed,
                         uint32_t frame, int32_t spp, float* out_dev, void* stream);

/* Wait for `stream` and report any device-side error recorded since the last check (TOF_ECUDA
 * with a message naming the cause; the error word is cleared).  Outputs written on `stream`
 * before the call are valid when it returns TOF_OK.  Not in the paper: error plumbing. */
tof_status tof_sync(tof_ctx* ctx, void* stream);

/* Kernel launches the library has issued in this process, across every context (a kernel recorded
 * into a batch graph counts once, when it is recorded; graph replays add nothing).  Not in the
 * paper: instrumentation for launch accounting. */
uint64_t tof_kernel_launches(void);

/* Forget the view's history (the next frame renders without temporal reuse).  Not in the paper:
 * a restart of the reservoir sequence (e.g. after a scene cut), which the method leaves to the
 * renderer. */
tof_status tof_reservoirs_reset(tof_ctx* ctx, tof_view view);

/* Shift statistics accumulated by the view since creation (Table "Newton statistics", Sec. 6):
 * out[0] Newton solves, out[1] Newton iterations, out[2] Newton successes, out[3] forward shift
 * attempts, out[4] successful forward shifts (these five over forward shifts of every reuse
 * pass), out[5] inverse (MIS) shift attempts of every pass, out[6] forward and out[7] inverse
 * shift attempts of the spatial passes alone, out[8] and out[9] visibility segments traced for
 * the spatial passes' forward and inverse shifts.  Synchronises the view's last stream. */
tof_status tof_view_stats(tof_ctx* ctx, tof_view view, double out[10]);

/* Per-stage timing of a view's frames with CUDA events recorded on the render stream
 * (enable = 1 turns it on; off by default).  tof_view_stage_ms synchronises that stream and
 * returns the device durations (ms) of the last rendered frame: out[0] G-buffer (and laser spot),
 * out[1] initial candidates, out[2] temporal reuse, out[3] spatial reuse (all passes), out[4]
 * transient splat, out[5] the whole frame, and the spatial passes' kernels summed over passes:
 * out[6] setup (slots, units, tasks), out[7] forward shifts (shift_fwd_kernel), out[8] inverse
 * (MIS) shifts (shift_inv_kernel), out[9] merge, out[10] the forward shifts' visibility and the
 * inverse-task emission, out[11] the inverse shifts' visibility.  A stage that did not run
 * reports 0. */
tof_status tof_view_profile(tof_ctx* ctx, tof_view view, int enable);
tof_status tof_view_stage_ms(tof_ctx* ctx, tof_view view, float out[12]);

#ifdef __cplusplus
}
#endif
#endif /* TOF_H */
