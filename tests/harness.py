"""Test / bench harness: drive the CUDA path through the C ABI binding and the oracle on the
same seeded inputs, and compare.  Test infrastructure (imports the oracle)."""
from __future__ import annotations

import numpy as np

# parity bar of every GPU-vs-oracle comparison: per-value relative difference <= PARITY_TOL on at
# least PARITY_FRAC of the values (the rest being discrete branch flips between FP32 and FP64) and
# image relative MSE <= PARITY_RELMSE
PARITY_TOL, PARITY_FRAC, PARITY_RELMSE = 1e-3, 0.995, 1e-4


def gpu_render(scene, frames, seed=None, params=None, B=0, reset_each=False, collect_stats=False, device=0):
    """Render `frames` of `scene` through libtof (tof_bvh_build once per frame, then
    tof_render_gated / tof_render_transient).  Returns a list of float64 numpy images."""
    import torch
    from paper_2605_11536_gb300 import tof
    p = params if params is not None else scene.params
    seed = scene.seed if seed is None else seed
    ctx = tof.tof_create(device)
    try:
        sid = tof.tof_scene_upload(ctx, scene.verts, scene.tris, scene.tri_object, scene.materials, scene.object_material)
        s0 = scene.sensors[frames[0]]
        W, H = int(s0["W"]), int(s0["H"])
        vid = tof.tof_view_create(ctx, sid, W, H, B)
        outs = []
        first = True
        for f in frames:
            tof.tof_bvh_build(ctx, sid, scene.xforms[f].reshape(-1), refit_only=0 if first else 1)
            first = False
            if reset_each:
                tof.tof_reservoirs_reset(ctx, vid)
            out = torch.full((H * W * max(B, 1),), -1.0, device="cuda", dtype=torch.float32)
            if B > 0:
                tof.tof_render_transient(ctx, sid, vid, scene.sensors[f], scene.emitters[f], (scene.bins[0], scene.bins[1], B),
                                         p, seed, f, out.data_ptr())
            else:
                tof.tof_render_gated(ctx, sid, vid, scene.sensors[f], scene.emitters[f], scene.gates[f], p, seed, f,
                                     out.data_ptr())
            tof.tof_sync(ctx)   # raises if a kernel recorded a device-side error for this frame
            img = out.cpu().numpy().astype(np.float64)
            outs.append(img.reshape(H, W, B) if B > 0 else img.reshape(H, W))
        stats = tof.tof_view_stats(ctx, vid) if collect_stats else None
    finally:
        tof.tof_destroy(ctx)
    return (outs, stats) if collect_stats else outs


def gpu_pt(scene, frame, spp, seed=None, params=None, B=0, device=0):
    import torch
    from paper_2605_11536_gb300 import tof
    p = params if params is not None else scene.params
    seed = scene.seed if seed is None else seed
    ctx = tof.tof_create(device)
    try:
        sid = tof.tof_scene_upload(ctx, scene.verts, scene.tris, scene.tri_object, scene.materials, scene.object_material)
        tof.tof_bvh_build(ctx, sid, scene.xforms[frame].reshape(-1))
        s = scene.sensors[frame]
        W, H = int(s["W"]), int(s["H"])
        out = torch.zeros(H * W * max(B, 1), device="cuda")
        tof.tof_render_pt(ctx, sid, s, scene.emitters[frame], None if B else scene.gates[frame],
                          (scene.bins[0], scene.bins[1], B) if B else None, p, seed, frame, spp, out.data_ptr())
        tof.tof_sync(ctx)
        img = out.cpu().numpy().astype(np.float64)
    finally:
        tof.tof_destroy(ctx)
    return img.reshape(H, W, B) if B else img.reshape(H, W)


def oracle_render(scene, frames, seed=None, params=None, B=0, roi=None, nthreads=0):
    import oracle as O
    geoms = {}
    s0 = scene.sensors[frames[0]]
    v = O.View(int(s0["W"]), int(s0["H"]), B)
    outs, oks = [], []
    for f in frames:
        g = O.Geom(scene, f)
        geoms[f] = g
        img, ok = O.render_frame(v, g, scene, f, params=params, seed=seed, roi=roi, nthreads=nthreads)
        outs.append(img)
        oks.append(ok)
    # every frame's geometry stays referenced in `geoms` (the view points at the previous one)
    stats = v.stats()
    return outs, oks, stats, geoms


def compare(gpu, ref, mask=None, tol=1e-3):
    """Per-pixel relative difference |g - o| / max(|g|, |o|) (0 where both are 0) and the image
    relative MSE sum (g - o)^2 / sum o^2."""
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    if mask is not None:
        m = np.asarray(mask, dtype=bool)
        if g.ndim == 3:
            m = np.repeat(m[..., None], g.shape[2], axis=2)
        g, o = g[m], o[m]
    g, o = g.ravel(), o.ravel()
    den = np.maximum(np.abs(g), np.abs(o))
    rel = np.where(den > 0, np.abs(g - o) / np.where(den > 0, den, 1.0), 0.0)
    frac_ok = float(np.mean(rel <= tol)) if rel.size else 1.0
    s = float(np.sum(o * o))
    relmse = float(np.sum((g - o) ** 2) / s) if s > 0 else float(np.sum((g - o) ** 2))
    return frac_ok, relmse, rel


def bin_moves(gpu, ref, mask=None, tol=1e-3):
    """Transient histograms [H, W, B]: the (pixel, bin) values whose sample sits one bin apart on
    the two sides -- g[b] nonzero where o[b] is zero and o[b -/+ 1] equals g[b] (within tol) while
    g[b -/+ 1] is zero, and the mirror pair.  A path length within rounding of a bin boundary is
    binned by floor((tau - t0) / w) in each side's own precision, so both answers are correct.
    Returns a boolean array [H, W, B] marking both values of every such pair."""
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    moved = np.zeros(g.shape, dtype=bool)
    for d in (-1, 1):
        gs = np.roll(g, d, axis=2)   # gs[..., b] = g[..., b - d]
        os_ = np.roll(o, d, axis=2)
        # the GPU's value at b - d is the oracle's at b: a move by +d
        hit = (g == 0) & (os_ == 0) & (gs != 0) & (o != 0) & (np.abs(gs - o) <= tol * np.maximum(np.abs(gs), np.abs(o)))
        if d == 1:
            hit[..., 0] = False
        else:
            hit[..., -1] = False
        moved |= hit
        moved |= np.roll(hit, -d, axis=2)
    if mask is not None:
        moved &= np.asarray(mask, dtype=bool)[..., None]
    return moved

