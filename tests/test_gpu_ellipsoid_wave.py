"""The gated initial stage with the ellipsoidal connection runs as a wavefront (path trees that
record their vertices and candidates, one placement pass over the ellipsoidal requests, their
visibility through the queue kernel, the streaming RIS replayed per pixel).  It draws the same
candidates with the same weights, uniforms and order as the single-kernel form, which the
allocation-free entry point still uses: the two must give the same images, frame after frame
(temporal and spatial reuse of the reservoirs they leave)."""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes
from tests.harness import compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["box", "heightfield_pairwise_walk", "materials_moving"])
def test_wavefront_matches_single_kernel(case):
    import torch
    from paper_2605_11536_gb300 import tof
    nf = 3
    if case == "box":
        sc = scenes.box_icosphere(W=96, H=80, frames=nf)
        sc.gates = [(5.0, 0.25)] * nf
        sc.params.n_spatial, sc.params.radius, sc.params.temporal = 3, 6, 1
    elif case == "materials_moving":
        sc = scenes.box_materials(W=96, H=80, frames=nf, moving=True)
        sc.params.temporal = 1
    else:
        sc = scenes.heightfield_spheres(W=96, H=80, frames=nf)
        sc.params.radius = 8
        sc.params.flags |= scenes.FLAG_PAIRWISE_MIS | scenes.FLAG_TRIANGLE_WALK
    sc.params.flags |= scenes.FLAG_ELLIPSOID
    W, H = 96, 80
    ctx = tof.tof_create(0)
    try:
        sid = tof.tof_scene_upload(ctx, sc.verts, sc.tris, sc.tri_object, sc.materials, sc.object_material)
        va = tof.tof_view_create(ctx, sid, W, H, 0)
        vb = tof.tof_view_create(ctx, sid, W, H, 0)
        out_a = torch.zeros(W * H, device="cuda")
        out_b = torch.zeros(W * H, device="cuda")
        for f in range(nf):
            tof.tof_bvh_build(ctx, sid, sc.xforms[f].reshape(-1))
            tof.tof_render_gated(ctx, sid, va, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 5, f, out_a.data_ptr())
            tof.tof_render_gated_noalloc(ctx, sid, vb, sc.sensors[f], sc.emitters[f], sc.gates[f], sc.params, 5, f,
                                         out_b.data_ptr())
            torch.cuda.synchronize()
            a = out_a.cpu().numpy().astype(np.float64)
            b = out_b.cpu().numpy().astype(np.float64)
            assert np.count_nonzero(a) > 100
            frac, relmse, rel = compare(a, b)
            assert frac >= 0.999 and relmse <= 1e-6, (f, frac, relmse, np.sort(rel)[-4:])
    finally:
        tof.tof_destroy(ctx)
