// tof_server.cu -- served form of the ToF ReSTIR path (8 dynamic streams, mixed gated and transient): continuous batching of frame
// requests from several dynamic streams on one GPU.
//
// Host-side scheduler over the C ABI: it never waits on the GPU (completion is observed with
// cudaEventQuery), keeps every admitted stream's view resident for temporal reuse, bounds the
// device memory of resident views by a budget, and launches each step's admitted frames as one
// tof_render_batch graph.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "tof.h"
#include "tof_internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct StreamS {
    tof_scene scene = -1;
    int32_t W = 0, H = 0, B = 0;
    tof_view view = -1;      // created on first admission
    uint64_t bytes = 0;      // device bytes of the view
    bool busy = false;       // a frame of this stream is in flight
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
    uint64_t next_ticket = 1;
    double submitted = 0, completed = 0, batches = 0, deferred = 0;
};

extern "C" {

tof_status tof_server_create(tof_ctx* ctx, uint64_t hbm_budget_bytes, tof_server** out) {
    if (!ctx || !out) return TOF_EINVAL;
    tof_server* s = new tof_server();
    s->ctx = ctx;
    s->budget = hbm_budget_bytes;
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
        s->free_events.push_back(b.done);
        s->inflight.pop_front();
    }
}

tof_status tof_server_step(tof_server* s, void* stream) {
    if (!s) return TOF_EINVAL;
    retire(s);
    std::vector<tof_job> jobs;
    std::vector<uint64_t> tickets;
    std::deque<uint64_t> keep;
    while (!s->queue.empty()) {
        uint64_t t = s->queue.front();
        s->queue.pop_front();
        Request& r = s->reqs[t];
        StreamS& st = s->streams[r.stream];
        if (st.busy) { keep.push_back(t); continue; }
        if (st.view < 0) {
            // first admission of the stream: its view must fit the budget
            uint64_t before = tof_device_bytes(s->ctx);
            tof_view v;
            if (s->budget) {
                uint64_t Bn = st.B > 0 ? (uint64_t)st.B : 1ull, npix = (uint64_t)st.W * st.H;
                uint64_t need = npix * Bn * 96ull * 3 + npix * 64ull;
                if (s->resident + need > s->budget) { s->deferred += 1; keep.push_back(t); continue; }
            }
            tof_status rc = tof_view_create(s->ctx, st.scene, st.W, st.H, st.B, &v);
            if (rc != TOF_OK) return rc;
            st.view = v;
            st.bytes = tof_device_bytes(s->ctx) - before;
            s->resident += st.bytes;
        }
        tof_status rc = tof_bvh_build(s->ctx, st.scene, r.xf.data(), 0, stream);   // full rebuild: see tof.h
        if (rc != TOF_OK) return rc;
        r.job.view = st.view;
        r.state = 1;
        st.busy = true;
        jobs.push_back(r.job);
        tickets.push_back(t);
    }
    s->queue.swap(keep);
    if (jobs.empty()) return TOF_OK;
    tof_status rc = tof_render_batch(s->ctx, jobs.data(), (uint32_t)jobs.size(), stream);
    if (rc != TOF_OK) return rc;
    Batch b;
    if (!s->free_events.empty()) {
        b.done = s->free_events.back();
        s->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
        return TOF_ECUDA;
    }
    if (cudaEventRecord(b.done, (cudaStream_t)stream) != cudaSuccess) return TOF_ECUDA;
    b.tickets = tickets;
    s->inflight.push_back(b);
    s->batches += 1;
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
