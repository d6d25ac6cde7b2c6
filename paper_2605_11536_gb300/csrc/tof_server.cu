// tof_server.cu -- served form of the ToF ReSTIR path (8 dynamic streams, mixed gated and transient): continuous batching of frame
// requests from several dynamic streams on one GPU.
//
// Host-side scheduler over the C ABI: it never waits on the GPU (completion is observed with
// cudaEventQuery), keeps every admitted stream's view resident for temporal reuse, bounds the
// device memory of resident views by a budget (measured per view, least recently used idle views
// evicted to make room), and launches each step's admitted frames as one batch graph on the next
// of its own streams, so that the batches of successive steps overlap on the device.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "tof.h"
#include "tof_internal.h"

extern "C" {
__attribute__((visibility("hidden"))) tof_status tof_internal_prepare_job(tof_ctx* c, const tof_job* job);
__attribute__((visibility("hidden"))) tof_status tof_internal_render_batch(tof_ctx* c, const tof_job* jobs, uint32_t n,
                                                                         void* stream, int slot);
}

namespace {

using clk = std::chrono::steady_clock;

constexpr int kLanes = 4;    // server streams (and batch graph slots): batches in flight at once

struct StreamS {
    tof_scene scene = -1;
    int32_t W = 0, H = 0, B = 0;
    tof_view view = -1;      // created on admission, destroyed by eviction
    uint64_t bytes = 0;      // device bytes of the view and its scratch (measured)
    bool busy = false;       // a frame of this stream is in flight
    uint64_t last_used = 0;  // step of its last admission (eviction order)
    int queued = 0;          // requests waiting
};

struct Request {
    uint64_t ticket = 0;
    int32_t stream = -1;
    tof_job job;
    std::vector<float> xf;
    clk::time_point t_submit;
    int32_t state = 0;       // 0 queued, 1 in flight, 2 done
    double latency_ms = 0.0;
};

struct Batch {
    cudaEvent_t done = nullptr;
    std::vector<uint64_t> tickets;
    std::vector<tof_scene> scenes;
};

}  // namespace

struct tof_server {
    tof_ctx* ctx = nullptr;
    uint64_t budget = 0;
    uint64_t resident = 0;
    std::vector<StreamS> streams;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> reqs;
    std::deque<Batch> inflight;
    std::vector<cudaEvent_t> free_events;
    cudaStream_t lanes[kLanes] = {};
    cudaEvent_t lane_after[kLanes] = {};   // the caller stream's work before a batch
    int next_lane = 0;
    std::map<tof_scene, int> scene_busy;   // frames in flight per scene (its BVH may not be rebuilt)
    uint64_t next_ticket = 1, steps = 0;
    double submitted = 0, completed = 0, batches = 0, deferred = 0, evicted = 0;
};

extern "C" {

tof_status tof_server_create(tof_ctx* ctx, uint64_t hbm_budget_bytes, tof_server** out) {
    if (!ctx || !out) return TOF_EINVAL;
    tof_server* s = new tof_server();
    s->ctx = ctx;
    s->budget = hbm_budget_bytes;
    for (int k = 0; k < kLanes; ++k)
        if (cudaStreamCreateWithFlags(&s->lanes[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->lane_after[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j <= k; ++j) {
                if (s->lanes[j]) cudaStreamDestroy(s->lanes[j]);
                if (s->lane_after[j]) cudaEventDestroy(s->lane_after[j]);
            }
            delete s;
            return TOF_ECUDA;
        }
    *out = s;
    return TOF_OK;
}

tof_status tof_server_destroy(tof_server* s) {
    if (!s) return TOF_EINVAL;
    for (Batch& b : s->inflight) {
        cudaEventSynchronize(b.done);
        cudaEventDestroy(b.done);
    }
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (StreamS& st : s->streams)
        if (st.view >= 0) tof_view_destroy(s->ctx, st.view);
    for (int k = 0; k < kLanes; ++k) {
        cudaStreamDestroy(s->lanes[k]);
        cudaEventDestroy(s->lane_after[k]);
    }
    delete s;
    return TOF_OK;
}

tof_status tof_server_open_stream(tof_server* s, tof_scene scene, int32_t W, int32_t H, int32_t B, int32_t* id) {
    if (!s || !id || W < 1 || H < 1 || B < 0) return TOF_EINVAL;
    StreamS st;
    st.scene = scene; st.W = W; st.H = H; st.B = B;
    s->streams.push_back(st);
    *id = (int32_t)s->streams.size() - 1;
    return TOF_OK;
}

tof_status tof_server_submit(tof_server* s, int32_t sid, const tof_job* job, const float* xf, uint64_t* ticket) {
    if (!s || !job || !xf || !ticket || sid < 0 || sid >= (int32_t)s->streams.size()) return TOF_EINVAL;
    StreamS& st = s->streams[sid];
    if (job->sensor.W != st.W || job->sensor.H != st.H) return TOF_EINVAL;
    if ((job->transient != 0) != (st.B > 0) || (job->transient && job->bins.B != st.B)) return TOF_EINVAL;
    if (!job->out_dev) return TOF_EINVAL;
    // the number of objects is the scene's; the caller passes nobj * 12 floats
    Request r;
    r.ticket = s->next_ticket++;
    r.stream = sid;
    r.job = *job;
    r.job.scene = st.scene;
    int nobj = tof_internal_scene_objects(s->ctx, st.scene);
    if (nobj <= 0) return TOF_EINVAL;
    r.xf.assign(xf, xf + 12 * (size_t)nobj);
    r.t_submit = clk::now();
    *ticket = r.ticket;
    st.queued += 1;
    s->queue.push_back(r.ticket);
    s->reqs.emplace(r.ticket, std::move(r));
    s->submitted += 1;
    return TOF_OK;
}

static void retire(tof_server* s) {
    while (!s->inflight.empty()) {
        Batch& b = s->inflight.front();
        cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) break;
        auto now = clk::now();
        for (uint64_t t : b.tickets) {
            auto it = s->reqs.find(t);
            if (it == s->reqs.end()) continue;
            it->second.state = 2;
            it->second.latency_ms = std::chrono::duration<double, std::milli>(now - it->second.t_submit).count();
            s->streams[it->second.stream].busy = false;
            s->completed += 1;
        }
        for (tof_scene sc : b.scenes)
            if (--s->scene_busy[sc] <= 0) s->scene_busy.erase(sc);
        s->free_events.push_back(b.done);
        s->inflight.pop_front();
    }
}

// destroy the least recently used idle view (no frame in flight, no request waiting) other than
// `keep`; false if there is none
static bool evict_one(tof_server* s, int32_t keep) {
    int best = -1;
    for (int i = 0; i < (int)s->streams.size(); ++i) {
        const StreamS& st = s->streams[i];
        if (i == keep || st.view < 0 || st.busy || st.queued > 0) continue;
        if (best < 0 || st.last_used < s->streams[best].last_used) best = i;
    }
    if (best < 0) return false;
    StreamS& st = s->streams[best];
    tof_view_destroy(s->ctx, st.view);
    s->resident -= st.bytes;
    st.view = -1;
    st.bytes = 0;
    s->evicted += 1;
    return true;
}

// first admission of a stream: create its view and the scratch its frames need, measure the device
// bytes that took, and keep it only if it fits the budget (evicting idle views if needed)
static tof_status admit_view(tof_server* s, int32_t sid, const tof_job& job, bool* fits) {
    StreamS& st = s->streams[sid];
    *fits = false;
    const uint64_t before = tof_device_bytes(s->ctx);
    tof_view v;
    tof_status rc = tof_view_create(s->ctx, st.scene, st.W, st.H, st.B, &v);
    if (rc == TOF_OK) {
        tof_job j = job;
        j.view = v;
        rc = tof_internal_prepare_job(s->ctx, &j);
        if (rc != TOF_OK) tof_view_destroy(s->ctx, v);
    }
    if (rc == TOF_EBUDGET || rc == TOF_ENOMEM) return TOF_OK;   // the context's own bound: defer
    if (rc != TOF_OK) return rc;
    const uint64_t bytes = tof_device_bytes(s->ctx) - before;
    while (s->budget && s->resident + bytes > s->budget)
        if (!evict_one(s, sid)) break;
    if (s->budget && s->resident + bytes > s->budget) {
        tof_view_destroy(s->ctx, v);
        return TOF_OK;
    }
    st.view = v;
    st.bytes = bytes;
    s->resident += bytes;
    *fits = true;
    return TOF_OK;
}

tof_status tof_server_step(tof_server* s, void* stream) {
    if (!s) return TOF_EINVAL;
    retire(s);
    s->steps += 1;
    const int lane = s->next_lane;
    cudaStream_t q = s->lanes[lane];
    std::vector<tof_job> jobs;
    std::vector<uint64_t> tickets;
    std::vector<tof_scene> scenes;
    std::deque<uint64_t> keep;
    bool ordered = false;
    while (!s->queue.empty()) {
        uint64_t t = s->queue.front();
        s->queue.pop_front();
        Request& r = s->reqs[t];
        StreamS& st = s->streams[r.stream];
        // one frame in flight per stream (temporal reuse needs its predecessor), and a scene's BVH is
        // rebuilt only while no frame reads it
        if (st.busy || s->scene_busy.count(st.scene)) { keep.push_back(t); continue; }
        if (st.view < 0) {
            bool fits = false;
            tof_status rc = admit_view(s, r.stream, r.job, &fits);
            if (rc != TOF_OK) return rc;
            if (!fits) { s->deferred += 1; keep.push_back(t); continue; }
        }
        if (!ordered) {
            // the batch runs on the server's lane, after what the caller queued on `stream`
            if (cudaEventRecord(s->lane_after[lane], (cudaStream_t)stream) != cudaSuccess ||
                cudaStreamWaitEvent(q, s->lane_after[lane], 0) != cudaSuccess)
                return TOF_ECUDA;
            ordered = true;
        }
        tof_status rc = tof_bvh_build(s->ctx, st.scene, r.xf.data(), 0, q);   // full rebuild: see tof.h
        if (rc != TOF_OK) return rc;
        r.job.view = st.view;
        r.state = 1;
        st.busy = true;
        st.queued -= 1;
        st.last_used = s->steps;
        s->scene_busy[st.scene] += 1;
        jobs.push_back(r.job);
        tickets.push_back(t);
        scenes.push_back(st.scene);
    }
    s->queue.swap(keep);
    if (jobs.empty()) return TOF_OK;
    tof_status rc = tof_internal_render_batch(s->ctx, jobs.data(), (uint32_t)jobs.size(), q, lane);
    if (rc != TOF_OK) return rc;
    Batch b;
    if (!s->free_events.empty()) {
        b.done = s->free_events.back();
        s->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
        return TOF_ECUDA;
    }
    if (cudaEventRecord(b.done, q) != cudaSuccess) return TOF_ECUDA;
    b.tickets = tickets;
    b.scenes = scenes;
    s->inflight.push_back(b);
    s->batches += 1;
    s->next_lane = (lane + 1) % kLanes;
    return TOF_OK;
}

tof_status tof_server_poll(tof_server* s, uint64_t ticket, int32_t* state, double* latency_ms) {
    if (!s || !state) return TOF_EINVAL;
    retire(s);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { *state = -1; return TOF_OK; }
    *state = it->second.state;
    if (latency_ms) *latency_ms = it->second.latency_ms;
    return TOF_OK;
}

tof_status tof_server_stats(tof_server* s, double out[7]) {
    if (!s || !out) return TOF_EINVAL;
    retire(s);
    size_t infl = 0;
    for (const Batch& b : s->inflight) infl += b.tickets.size();
    out[0] = s->submitted; out[1] = s->completed; out[2] = s->batches; out[3] = s->deferred;
    out[4] = (double)s->resident; out[5] = (double)s->queue.size(); out[6] = (double)infl;
    return TOF_OK;
}

}  // extern "C"
