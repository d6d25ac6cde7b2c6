"""Batched rendering (tof_render_batch): many independent instances as one CUDA graph whose
branches run concurrently.  Each batched result must equal the same job rendered on its own, over
consecutive frames (temporal state carried per view), and agree with the oracle."""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes
from tests.harness import compare, oracle_render

pytestmark = pytest.mark.gpu


def _jobs_spec():
    box = scenes.box_icosphere(W=64, H=64, frames=2)
    box.gates = [(5.0, 0.25)] * 2
    hf = scenes.heightfield_spheres(W=96, H=80, frames=2, nx=60, ny=40, n_spheres=6)
    conf = scenes.confocal_nlos(W=24, H=24, frames=2, B=96, stacks=32, slices=32)
    conf.bins = (1.35, 0.008, 96)
    spec = []
    # (scene, W, H, gate, depth, n_spatial, radius, temporal, transient)
    spec.append((box, 64, 64, (5.0, 0.25), 3, 1, 8, 1, False))
    spec.append((box, 40, 24, (5.2, 0.1), 4, 3, 5, 1, False))
    spec.append((box, 17, 29, (4.8, 0.05), 2, 2, 4, 0, False))
    spec.append((hf, 96, 80, (8.0, 0.05), 4, 5, 12, 1, False))
    spec.append((hf, 48, 40, (8.0, 0.03), 5, 2, 6, 1, False))
    spec.append((conf, 24, 24, None, 4, 3, 4, 1, True))
    return spec


def _sensor(sc, f, W, H):
    return dict(sc.sensors[f], W=W, H=H)


def _run(batched, tune=None, chosen=None, flags=0):
    """Render the spec's jobs over two frames, batched or one launch per job.  tune: None (default
    tuning), a dict of tof_view_set_tuning fields for every view, or "auto" (tof_autotune on the
    first frame's jobs, chosen tunings appended to `chosen`).  flags: method flags added to the
    gated jobs."""
    import torch
    from paper_2605_11536_gb300 import tof
    spec = _jobs_spec()
    ctx = tof.tof_create(0)
    outs = []
    try:
        sids = {}
        for sc, *_ in spec:
            if id(sc) not in sids:
                sids[id(sc)] = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
        views, bufs, params = [], [], []
        for sc, W, H, gate, depth, nsp, rad, temporal, transient in spec:
            B = sc.bins[2] if transient else 0
            views.append(tof.tof_view_create(ctx, sids[id(sc)], W, H, B))
            bufs.append(torch.zeros(W * H * max(B, 1), device="cuda"))
            p = scenes.Params(**vars(sc.params))
            p.depth, p.n_spatial, p.radius, p.temporal = depth, nsp, rad, temporal
            if not transient:
                p.flags |= flags
            params.append(p)
            if isinstance(tune, dict):
                tof.tof_view_set_tuning(ctx, views[-1], **tune)
        for f in range(2):
            done = set()
            for sc, *_ in spec:
                if id(sc) not in done:
                    tof.tof_bvh_build(ctx, sids[id(sc)], sc.xforms[f].reshape(-1), refit_only=0 if f == 0 else 1)
                    done.add(id(sc))
            jobs = []
            for i, (sc, W, H, gate, depth, nsp, rad, temporal, transient) in enumerate(spec):
                s = _sensor(sc, f, W, H)
                if batched:
                    jobs.append(tof.job(sids[id(sc)], views[i], s, sc.emitters[f], params[i], 100 + i, f, bufs[i].data_ptr(),
                                        gate=None if transient else gate, bins=sc.bins if transient else None))
                elif transient:
                    tof.tof_render_transient(ctx, sids[id(sc)], views[i], s, sc.emitters[f], sc.bins, params[i], 100 + i, f,
                                             bufs[i].data_ptr())
                else:
                    tof.tof_render_gated(ctx, sids[id(sc)], views[i], s, sc.emitters[f], gate, params[i], 100 + i, f,
                                         bufs[i].data_ptr())
            if tune == "auto" and f == 0:
                auto_jobs = [tof.job(sids[id(sc)], views[i], _sensor(sc, 0, W, H), sc.emitters[0], params[i], 100 + i, 0,
                                     bufs[i].data_ptr(), gate=None if tr else gate, bins=sc.bins if tr else None)
                             for i, (sc, W, H, gate, _d, _n, _r, _t, tr) in enumerate(spec)]
                got = tof.tof_autotune(ctx, auto_jobs, frames=2)
                if chosen is not None:
                    chosen.extend(got)
            if batched:
                tof.tof_render_batch(ctx, jobs)
            torch.cuda.synchronize()
            outs.append([b.cpu().numpy().astype(np.float64) for b in bufs])
    finally:
        tof.tof_destroy(ctx)
    return outs


def test_batch_equals_individual_renders_over_two_frames():
    ind = _run(False)
    bat = _run(True)
    for f in range(2):
        for i, (a, b) in enumerate(zip(ind[f], bat[f])):
            assert np.count_nonzero(a) > 0, (f, i)
            frac, relmse, _ = compare(b, a)
            assert frac >= 0.999 and relmse <= 1e-6, (f, i, frac, relmse)


def test_batch_with_ellipsoid_pairwise_walk_equals_individual_renders():
    """The gated jobs with the ellipsoidal connection (its initial wavefront's scratch is allocated
    before the graph is captured), pairwise MIS and the walk: batched as rendered one by one."""
    flags = scenes.FLAG_ELLIPSOID | scenes.FLAG_PAIRWISE_MIS | scenes.FLAG_TRIANGLE_WALK
    ind = _run(False, flags=flags)
    bat = _run(True, flags=flags)
    for f in range(2):
        for i, (a, b) in enumerate(zip(ind[f], bat[f])):
            assert np.count_nonzero(a) > 0, (f, i)
            frac, relmse, _ = compare(b, a)
            assert frac >= 0.999 and relmse <= 1e-6, (f, i, frac, relmse)


def test_batched_instance_matches_oracle():
    spec = _jobs_spec()
    sc, W, H, gate, depth, nsp, rad, temporal, transient = spec[1]
    bat = _run(True)
    o_sc = scenes.box_icosphere(W=W, H=H, frames=2)
    o_sc.gates = [gate] * 2
    o_sc.params.depth, o_sc.params.n_spatial, o_sc.params.radius, o_sc.params.temporal = depth, nsp, rad, temporal
    o, ok, st, _ = oracle_render(o_sc, [0, 1], seed=101)
    for f in range(2):
        frac, relmse, _ = compare(bat[f][1].reshape(H, W), o[f])
        assert frac >= 0.995 and relmse <= 1e-4, (f, frac, relmse)


@pytest.mark.parametrize("tune", [dict(tile_w=8, tile_h=8, packet=0, layout=0),
                                  dict(tile_w=32, tile_h=4, packet=2, layout=1),
                                  dict(tile_w=8, tile_h=16, packet=4, layout=0),
                                  dict(tile_w=4, tile_h=16, packet=1, layout=1)])
def test_tunings_render_identical_frames(tune):
    """Pixel tiles, task packets and the reservoir layout change launch shapes and addresses only:
    every job renders to the same bits (one launch per job, two frames with temporal state)."""
    ref = _run(False)
    got = _run(False, tune=tune)
    for f in range(2):
        for i, (a, b) in enumerate(zip(ref[f], got[f])):
            assert np.count_nonzero(a) > 0, (f, i)
            assert np.array_equal(a, b), (tune, f, i, float(np.abs(a - b).max()))


def test_autotune_chooses_valid_tunings_and_keeps_results():
    chosen = []
    ref = _run(True)
    got = _run(True, tune="auto", chosen=chosen)
    assert len(chosen) == len(_jobs_spec())
    for t in chosen:
        assert t["tile_w"] * t["tile_h"] in (64, 128) and 0 <= t["packet"] <= 8 and t["layout"] in (0, 1), t
    for f in range(2):
        for i, (a, b) in enumerate(zip(ref[f], got[f])):
            frac, relmse, _ = compare(b, a)
            assert frac >= 0.999 and relmse <= 1e-6, (f, i, frac, relmse)


def test_full_size_instance_in_a_batch_matches_the_oracle():
    """A 512x512 instance of the dynamic gated workload rendered inside a batch with two small
    instances of other scenes, over 2 frames; the oracle computes a central region covering the
    dependency cone of its inner pixels, and every untainted pixel is compared at the common bar."""
    import torch
    from paper_2605_11536_gb300 import tof
    from tests.harness import PARITY_FRAC, PARITY_RELMSE
    big = scenes.heightfield_spheres(W=512, H=512, frames=2)
    box = scenes.box_icosphere(W=64, H=64, frames=2)
    box.gates = [(5.0, 0.25)] * 2
    ctx = tof.tof_create(0)
    imgs = []
    try:
        sb = tof.tof_scene_upload(ctx, big.verts, big.tris, big.tri_object, big.materials, big.object_material)
        sx = tof.tof_scene_upload(ctx, box.verts, box.tris, box.tri_object, box.materials, box.object_material)
        vb = tof.tof_view_create(ctx, sb, 512, 512, 0)
        vx = [tof.tof_view_create(ctx, sx, 64, 64, 0) for _ in range(2)]
        out = torch.zeros(512 * 512, device="cuda")
        small = [torch.zeros(64 * 64, device="cuda") for _ in range(2)]
        for f in range(2):
            tof.tof_bvh_build(ctx, sb, big.xforms[f].reshape(-1), refit_only=0 if f == 0 else 1)
            tof.tof_bvh_build(ctx, sx, box.xforms[f].reshape(-1), refit_only=0 if f == 0 else 1)
            jobs = [tof.job(sb, vb, big.sensors[f], big.emitters[f], big.params, big.seed, f, out.data_ptr(), gate=big.gates[f])]
            for k in range(2):
                jobs.append(tof.job(sx, vx[k], box.sensors[f], box.emitters[f], box.params, 40 + k, f, small[k].data_ptr(),
                                    gate=box.gates[f]))
            tof.tof_render_batch(ctx, jobs)
            tof.tof_sync(ctx)
            imgs.append(out.cpu().numpy().astype(np.float64).reshape(512, 512))
    finally:
        tof.tof_destroy(ctx)
    half = 110
    roi = (256 - half, 256 - half, 256 + half, 256 + half)
    o, oks, st, _ = oracle_render(big, [0, 1], roi=roi)
    for f in range(2):
        assert oks[f].sum() >= 40 * 40
        frac, relmse, _ = compare(imgs[f], o[f], oks[f])
        assert np.count_nonzero(o[f][oks[f]]) >= 30
        assert frac >= PARITY_FRAC and relmse <= PARITY_RELMSE, (f, frac, relmse)


def test_large_instance_runs_the_wavefront_inside_a_batch_bit_for_bit():
    """A 256x256 gated instance (large enough for its initial stage to run as the bounce wavefront
    inside a staged batch) beside two small ones (the batched single kernel): over two frames, the
    batched images equal the ones rendered one by one bit for bit."""
    import torch
    from paper_2605_11536_gb300 import tof
    big = scenes.heightfield_spheres(W=256, H=256, frames=2, nx=60, ny=40, n_spheres=6)
    box = scenes.box_icosphere(W=64, H=64, frames=2)
    box.gates = [(5.0, 0.25)] * 2

    def run(batched):
        ctx = tof.tof_create(0)
        imgs = []
        try:
            sb = tof.tof_scene_upload(ctx, big.verts, big.tris, big.tri_object, big.materials, big.object_material)
            sx = tof.tof_scene_upload(ctx, box.verts, box.tris, box.tri_object, box.materials, box.object_material)
            vb = tof.tof_view_create(ctx, sb, 256, 256, 0)
            vx = [tof.tof_view_create(ctx, sx, 64, 64, 0) for _ in range(2)]
            out = torch.zeros(256 * 256, device="cuda")
            small = [torch.zeros(64 * 64, device="cuda") for _ in range(2)]
            for f in range(2):
                tof.tof_bvh_build(ctx, sb, big.xforms[f].reshape(-1), refit_only=0)
                tof.tof_bvh_build(ctx, sx, box.xforms[f].reshape(-1), refit_only=0)
                if batched:
                    jobs = [tof.job(sb, vb, big.sensors[f], big.emitters[f], big.params, 7, f, out.data_ptr(),
                                    gate=big.gates[f])]
                    for k in range(2):
                        jobs.append(tof.job(sx, vx[k], box.sensors[f], box.emitters[f], box.params, 40 + k, f,
                                            small[k].data_ptr(), gate=box.gates[f]))
                    tof.tof_render_batch(ctx, jobs)
                else:
                    tof.tof_render_gated(ctx, sb, vb, big.sensors[f], big.emitters[f], big.gates[f], big.params, 7, f,
                                         out.data_ptr())
                    for k in range(2):
                        tof.tof_render_gated(ctx, sx, vx[k], box.sensors[f], box.emitters[f], box.gates[f], box.params,
                                             40 + k, f, small[k].data_ptr())
                tof.tof_sync(ctx)
                imgs.append([out.cpu().numpy()] + [s.cpu().numpy() for s in small])
        finally:
            tof.tof_destroy(ctx)
        return imgs

    ind, bat = run(False), run(True)
    for f in range(2):
        for i in range(3):
            assert np.count_nonzero(ind[f][i]) > 20, (f, i)
            assert np.array_equal(ind[f][i], bat[f][i]), (f, i, int(np.count_nonzero(ind[f][i] != bat[f][i])))
