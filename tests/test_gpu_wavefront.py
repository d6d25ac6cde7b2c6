"""The gated initial stage as a bounce wavefront (direct renders) against the single kernel (which
the allocation-free entry point runs): both draw the same trees, candidates and uniforms in the same
order, so the frames must agree bit for bit.  The cases reach what the dynamic workload does not:
* a gate holding every path length, with direct candidates and depth 5, so every vertex of every
  tree queues a light segment -- up to five per path, beyond the queue's one per path, so most of
  them take the in-place fallback;
* mirror and glossy walls (delta bounces carry no area density) with 7 path trees;
* depth 2 (a single bounce round) with one tree."""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "all_lengths_direct_depth5":
        sc = scenes.box_icosphere(W=96, H=80, frames=2)
        sc.gates = [(0.5, 60.0)] * 2
        sc.params.depth, sc.params.flags = 5, scenes.FLAG_DIRECT
        sc.params.n_spatial, sc.params.radius, sc.params.temporal = 2, 6, 1
    elif name == "mirror_glossy_7_trees":
        sc = scenes.box_materials(W=96, H=80, frames=2, moving=True)
        sc.params.n_cand, sc.params.temporal = 7, 1
    else:
        sc = scenes.box_icosphere(W=64, H=48, frames=2)
        sc.gates = [(4.0, 1.0)] * 2
        sc.params.depth, sc.params.n_cand, sc.params.n_spatial = 2, 1, 0
    return sc


@pytest.mark.parametrize("name", ["all_lengths_direct_depth5", "mirror_glossy_7_trees", "depth2_one_tree"])
def test_wavefront_equals_single_kernel(name):
    import torch
    from paper_2605_11536_gb300 import tof
    sc = _case(name)
    W, H = sc.sensors[0]["W"], sc.sensors[0]["H"]
    ctx = tof.tof_create(0)
    try:
        sid = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
        va = tof.tof_view_create(ctx, sid, W, H, 0)
        vb = tof.tof_view_create(ctx, sid, W, H, 0)
        out_a = torch.zeros(W * H, device="cuda")
        out_b = torch.zeros(W * H, device="cuda")
        for f in range(2):
            tof.tof_bvh_build(ctx, sid, sc.xforms[f].reshape(-1), refit_only=0)
            tof.tof_render_gated(ctx, sid, va, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 5, f,
                                 out_a.data_ptr())
            tof.tof_render_gated_noalloc(ctx, sid, vb, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 5, f,
                                         out_b.data_ptr())
            tof.tof_sync(ctx)
            a = out_a.cpu().numpy()
            b = out_b.cpu().numpy()
            assert np.count_nonzero(a) > 50, (f, int(np.count_nonzero(a)))
            assert np.array_equal(a, b), (f, int(np.count_nonzero(a != b)))
    finally:
        tof.tof_destroy(ctx)
