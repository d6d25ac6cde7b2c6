"""Served form (tof_server_*): continuous batching of frame requests from several dynamic streams.
Every request's result must be the same when its stream is served alone and when it is served in
the mix with other streams (their frames share batches), and equal to rendering the stream's frames
directly; an HBM budget defers admissions that would not fit."""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes
from tests.harness import compare

pytestmark = pytest.mark.gpu

NF = 3


def _streams():
    box = scenes.box_icosphere(W=48, H=40, frames=NF)
    box.gates = [(5.0, 0.25)] * NF
    box.params.n_spatial, box.params.radius, box.params.temporal = 3, 6, 1
    hf = scenes.heightfield_spheres(W=64, H=48, frames=NF, nx=60, ny=40, n_spheres=6)
    hf.params.radius = 10
    conf = scenes.confocal_nlos(W=24, H=24, frames=NF, B=64, stacks=32, slices=32)
    conf.bins = (1.35, 0.01, 64)
    return [box, hf, conf]


def _serve(which, budget=0, order_seed=0):
    """Serve the frames of the streams in `which` (indices into _streams()) with a random interleaving
    of submissions and steps; returns {(stream, frame): image} and the server stats."""
    import torch
    from paper_2605_11536_gb300 import tof
    scs = _streams()
    ctx = tof.tof_create(0)
    rng = np.random.default_rng(order_seed)
    out = {}
    try:
        srv = tof.tof_server_create(ctx, budget)
        sids, streams, bufs = {}, {}, {}
        for i in which:
            sc = scs[i]
            sids[i] = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
            tof.tof_bvh_build(ctx, sids[i], sc.xforms[0].reshape(-1))
            W, H = sc.sensors[0]["W"], sc.sensors[0]["H"]
            B = sc.bins[2] if sc.bins else 0
            streams[i] = tof.tof_server_open_stream(srv, sids[i], W, H, B)
            for f in range(NF):
                bufs[(i, f)] = torch.zeros(W * H * max(B, 1), device="cuda")
        pending = [(i, f) for f in range(NF) for i in which]
        tickets = {}
        while pending or any(tof.tof_server_poll(srv, t)[0] != 2 for t in tickets.values()):
            for _ in range(int(rng.integers(0, 3))):
                if pending:
                    i, f = pending.pop(0)
                    sc = scs[i]
                    j = tof.job(sids[i], 0, sc.sensors[f], sc.emitters[f], sc.params, 7 + i, f, bufs[(i, f)].data_ptr(),
                                gate=None if sc.bins else sc.gates[f], bins=sc.bins)
                    tickets[(i, f)] = tof.tof_server_submit(srv, streams[i], j, sc.xforms[f].reshape(-1))
            tof.tof_server_step(srv)
            if rng.uniform() < 0.5:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        stats = tof.tof_server_stats(srv)
        for k, b in bufs.items():
            out[k] = b.cpu().numpy().astype(np.float64)
        tof.tof_server_destroy(srv)
    finally:
        tof.tof_destroy(ctx)
    return out, stats


def _direct(i):
    import torch
    from tests.harness import gpu_render
    sc = _streams()[i]
    return gpu_render(sc, list(range(NF)), seed=7 + i, B=sc.bins[2] if sc.bins else 0)


def test_results_equal_alone_and_in_the_mix():
    mix, st = _serve([0, 1, 2], order_seed=1)
    assert st["completed"] == 3 * NF and st["batches"] >= 2
    for i in range(3):
        alone, _ = _serve([i], order_seed=2)
        direct = _direct(i)
        for f in range(NF):
            a, m = alone[(i, f)], mix[(i, f)]
            assert np.count_nonzero(a) > 0, (i, f)
            fr, rm, _ = compare(m, a)
            assert fr >= 0.999 and rm <= 1e-6, (i, f, fr, rm)
            fr, rm, _ = compare(m, np.asarray(direct[f]).ravel())
            assert fr >= 0.999 and rm <= 1e-6, (i, f, fr, rm)


def test_budget_defers_admission():
    # room for the two small gated streams' views but not the transient one's
    mix, st = _serve([0, 1], budget=1 << 30, order_seed=3)
    assert st["completed"] == 2 * NF and st["deferred"] == 0
    import torch
    from paper_2605_11536_gb300 import tof
    scs = _streams()
    ctx = tof.tof_create(0)
    try:
        srv = tof.tof_server_create(ctx, 4 << 20)
        sc = scs[2]
        sid = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
        tof.tof_bvh_build(ctx, sid, sc.xforms[0].reshape(-1))
        s = tof.tof_server_open_stream(srv, sid, 24, 24, 64)
        buf = torch.zeros(24 * 24 * 64, device="cuda")
        j = tof.job(sid, 0, sc.sensors[0], sc.emitters[0], sc.params, 1, 0, buf.data_ptr(), bins=sc.bins)
        t = tof.tof_server_submit(srv, s, j, sc.xforms[0].reshape(-1))
        tof.tof_server_step(srv)
        torch.cuda.synchronize()
        assert tof.tof_server_poll(srv, t)[0] == 0
        st2 = tof.tof_server_stats(srv)
        assert st2["deferred"] >= 1 and st2["queued"] == 1
        tof.tof_server_destroy(srv)
    finally:
        tof.tof_destroy(ctx)


def test_idle_views_are_evicted_for_new_streams():
    """A budget that holds one view: admitting a second stream evicts the first (idle) one, whose
    next frame then renders without temporal history -- the same image as a direct render after
    tof_reservoirs_reset; the resident bytes never exceed the budget."""
    import torch
    from paper_2605_11536_gb300 import tof
    from tests.harness import gpu_render
    scs = [_streams()[0], scenes.box_icosphere(W=48, H=40, frames=NF, seed=5)]
    scs[1].gates = [(5.0, 0.25)] * NF
    scs[1].params.n_spatial, scs[1].params.radius, scs[1].params.temporal = 3, 6, 1
    ctx = tof.tof_create(0)
    out = {}
    try:
        sids = []
        for sc in scs:
            sids.append(tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material))
            tof.tof_bvh_build(ctx, sids[-1], sc.xforms[0].reshape(-1))

        def run(srv, streams, i, f):
            sc = scs[i]
            buf = torch.zeros(48 * 40, device="cuda")
            j = tof.job(sids[i], 0, sc.sensors[f], sc.emitters[f], sc.params, 21 + i, f, buf.data_ptr(), gate=sc.gates[f])
            t = tof.tof_server_submit(srv, streams[i], j, sc.xforms[f].reshape(-1))
            for _ in range(1000):
                tof.tof_server_step(srv)
                torch.cuda.synchronize()
                if tof.tof_server_poll(srv, t)[0] == 2:
                    break
            assert tof.tof_server_poll(srv, t)[0] == 2
            return buf.cpu().numpy().astype(np.float64)

        # the device bytes of one stream's view, measured by a server without a budget
        srv = tof.tof_server_create(ctx, 0)
        run(srv, [tof.tof_server_open_stream(srv, sids[0], 48, 40, 0)], 0, 0)
        one = tof.tof_server_stats(srv)["resident_bytes"]
        tof.tof_server_destroy(srv)
        assert one > 0
        budget = int(one * 1.5)
        srv = tof.tof_server_create(ctx, budget)
        streams = [tof.tof_server_open_stream(srv, sids[i], 48, 40, 0) for i in range(2)]
        out[(0, 0)] = run(srv, streams, 0, 0)
        out[(1, 0)] = run(srv, streams, 1, 0)      # evicts stream 0's view
        assert tof.tof_server_stats(srv)["resident_bytes"] <= budget
        out[(0, 1)] = run(srv, streams, 0, 1)      # evicts stream 1's; stream 0 starts without history
        st = tof.tof_server_stats(srv)
        assert st["resident_bytes"] <= budget and st["completed"] == 3 and st["queued"] == 0
        tof.tof_server_destroy(srv)
    finally:
        tof.tof_destroy(ctx)
    d0 = gpu_render(scs[0], [0, 1], seed=21, reset_each=True)
    d1 = gpu_render(scs[1], [0], seed=22)
    for key, ref in (((0, 0), d0[0]), ((1, 0), d1[0]), ((0, 1), d0[1])):
        assert np.count_nonzero(ref) > 0, key
        fr, rm, _ = compare(out[key], np.asarray(ref).ravel())
        assert fr >= 0.999 and rm <= 1e-6, (key, fr, rm)
    # and the evicted stream's frame 1 is not what it would have been with its history
    with_history = gpu_render(scs[0], [0, 1], seed=21)[1]
    assert not np.array_equal(out[(0, 1)], np.asarray(with_history).ravel())
