"""tof_render_gated_noalloc: the gated render for callers that may not allocate device memory while
rendering (frames recorded into CUDA graphs, fixed memory pools, hosts that forbid cudaMalloc after
start-up).  It must produce what tof_render_gated produces, over consecutive frames (the second
one reuses the first temporally), while leaving the device allocations of the context and of
torch unchanged; oversized requests must fail with a message naming the limit.

This file is collected last so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes
from tests.harness import compare

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    from paper_2605_11536_gb300 import tof
    sc = scenes.box_icosphere(W=96, H=80, frames=2)
    sc.gates = [(5.0, 0.25)] * 2
    sc.params.n_spatial, sc.params.radius, sc.params.temporal = 3, 6, 1
    ctx = tof.tof_create(0)
    sid = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
    return torch, tof, sc, ctx, sid


def test_noalloc_matches_allocating_render_on_two_frames():
    torch, tof, sc, ctx, sid = _setup()
    try:
        W, H = 96, 80
        va = tof.tof_view_create(ctx, sid, W, H, 0)
        vb = tof.tof_view_create(ctx, sid, W, H, 0)
        out_a = torch.zeros(W * H, device="cuda")
        out_b = torch.zeros(W * H, device="cuda")
        for f in range(2):
            tof.tof_bvh_build(ctx, sid, sc.xforms[f].reshape(-1), refit_only=0 if f == 0 else 1)
            tof.tof_render_gated(ctx, sid, va, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 11, f,
                                 out_a.data_ptr())
            torch.cuda.synchronize()
            lib_bytes, torch_bytes = tof.tof_device_bytes(ctx), torch.cuda.memory_allocated()
            tof.tof_render_gated_noalloc(ctx, sid, vb, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 11, f,
                                         out_b.data_ptr())
            torch.cuda.synchronize()
            assert tof.tof_device_bytes(ctx) == lib_bytes
            assert torch.cuda.memory_allocated() == torch_bytes
            a = out_a.cpu().numpy().astype(np.float64)
            b = out_b.cpu().numpy().astype(np.float64)
            assert np.count_nonzero(a) > 50
            frac, relmse, _ = compare(b, a)
            assert frac >= 0.995 and relmse <= 1e-4, (f, frac, relmse)
    finally:
        tof.tof_destroy(ctx)


def test_noalloc_rejects_requests_beyond_the_static_limit():
    torch, tof, sc, ctx, sid = _setup()
    try:
        tof.tof_bvh_build(ctx, sid, sc.xforms[0].reshape(-1))
        big = tof.tof_view_create(ctx, sid, 160, 128, 0)
        s = dict(sc.sensors[0], W=160, H=128)
        out = torch.zeros(160 * 128, device="cuda")
        with pytest.raises(tof.TofError, match="exceed"):
            tof.tof_render_gated_noalloc(ctx, sid, big, s, sc.emitters[0], sc.gates[0], sc.params, 1, 0, out.data_ptr())
        small = tof.tof_view_create(ctx, sid, 96, 80, 0)
        sc.params.n_spatial = 6
        with pytest.raises(tof.TofError, match="exceed"):
            tof.tof_render_gated_noalloc(ctx, sid, small, sc.sensors[0], sc.emitters[0], sc.gates[0], sc.params, 1, 0,
                                         out.data_ptr())
    finally:
        tof.tof_destroy(ctx)
