"""tof_render_gated_noalloc: the gated render for callers that may not allocate device memory while
rendering (frames recorded into CUDA graphs, fixed memory pools, hosts that forbid cudaMalloc after
start-up).  It must produce exactly what tof_render_gated produces -- every random number is keyed
by pixel and frame and the merges read their inputs by index, so the two agree bit for bit -- over
consecutive frames (the second one reuses the first temporally), while leaving the device
allocations of the context, of torch and of the device as a whole unchanged after its first call;
oversized requests must fail with a message naming the limit.

This file is collected last so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes

pytestmark = pytest.mark.gpu


def _setup(W=96, H=80, n_spatial=3):
    import torch
    from paper_2605_11536_gb300 import tof
    sc = scenes.box_icosphere(W=W, H=H, frames=3)
    sc.gates = [(5.0, 0.25)] * 3
    sc.params.n_spatial, sc.params.radius, sc.params.temporal = n_spatial, 6, 1
    ctx = tof.tof_create(0)
    sid = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
    return torch, tof, sc, ctx, sid


@pytest.mark.parametrize("W,H,n_spatial", [(96, 80, 3), (128, 128, 5)])
def test_noalloc_matches_allocating_render_on_two_frames(W, H, n_spatial):
    """Bit-equal to tof_render_gated on consecutive frames; (128, 128, 5) fills the static scratch
    to its limits (16384 pixels, 6 slots per pixel)."""
    torch, tof, sc, ctx, sid = _setup(W, H, n_spatial)
    try:
        va = tof.tof_view_create(ctx, sid, W, H, 0)
        vb = tof.tof_view_create(ctx, sid, W, H, 0)
        out_a = torch.zeros(W * H, device="cuda")
        out_b = torch.zeros(W * H, device="cuda")
        free_after_first = None
        for f in range(3):
            tof.tof_bvh_build(ctx, sid, sc.xforms[f].reshape(-1), refit_only=0 if f == 0 else 1)
            tof.tof_render_gated(ctx, sid, va, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 11, f,
                                 out_a.data_ptr())
            tof.tof_sync(ctx)
            lib_bytes, torch_bytes = tof.tof_device_bytes(ctx), torch.cuda.memory_allocated()
            free0 = torch.cuda.mem_get_info()[0]
            tof.tof_render_gated_noalloc(ctx, sid, vb, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 11, f,
                                         out_b.data_ptr())
            tof.tof_sync(ctx)
            assert tof.tof_device_bytes(ctx) == lib_bytes
            assert torch.cuda.memory_allocated() == torch_bytes
            if free_after_first is not None:
                # the first call may load the library's module (and commit the static array); later
                # calls take no device memory at all
                assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed across a noalloc call"
            free_after_first = free0
            a = out_a.cpu().numpy()
            b = out_b.cpu().numpy()
            assert np.count_nonzero(a) > 50
            assert np.array_equal(a, b), (f, int(np.count_nonzero(a != b)))
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
