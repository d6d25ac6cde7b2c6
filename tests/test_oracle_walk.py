"""Pins of the cross-triangle walk of the reconnection vertex in the oracle (opt-in: when Newton
moves the vertex off its triangle -- an edge case Sec. 4.2 does not address -- it continues on the
neighbour across the crossed edge, unfolded into the triangle's plane, instead of failing).

* Tessellation invariance: on planar surfaces the walk unfolds coplanar neighbours without
  change, so the box scene renders the same whether its walls are 2 or 32 triangles each (without
  the walk the finer walls fail shifts that leave a triangle, and the images differ).
* Bijectivity: forward then inverse shifts that cross edges return the base path, with
  Jacobians multiplying to 1, and succeed more often than without the walk.
* Unbiasedness of the whole pipeline against plain path tracing with the walk on.
"""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes
from tests.test_oracle_pipeline import _box, _unbiased

FLAG_WALK = 64


def _subdivide(sc, obj, levels):
    """Midpoint-subdivide object `obj`'s triangles `levels` times (same surface, shared vertices)."""
    verts = [tuple(v) for v in np.asarray(sc.verts)]
    tris, tobj = [], []
    other = [(t, o) for t, o in zip(np.asarray(sc.tris), np.asarray(sc.tri_object)) if o != obj]
    cur = [tuple(int(i) for i in t) for t, o in zip(np.asarray(sc.tris), np.asarray(sc.tri_object)) if o == obj]
    for _ in range(levels):
        mids = {}

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in mids:
                verts.append(tuple((np.array(verts[a]) + np.array(verts[b])) / 2.0))
                mids[k] = len(verts) - 1
            return mids[k]
        nxt = []
        for a, b, c in cur:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        cur = nxt
    tris = [list(t) for t in cur] + [list(t) for t, _ in other]
    tobj = [obj] * len(cur) + [int(o) for _, o in other]
    sc.verts = np.array(verts, dtype=np.float64)
    sc.tris = np.array(tris, dtype=np.uint32)
    sc.tri_object = np.array(tobj, dtype=np.uint32)
    return sc


def _render(O, sc, seed=3):
    g = O.Geom(sc, 0)
    return O.render_frame(O.View(32, 32), g, sc, 0, seed=seed, nthreads=8)[0]


def test_walk_makes_planar_walls_tessellation_invariant(oracle_lib):
    O = oracle_lib
    res = {}
    for flags in (FLAG_WALK, 0):
        imgs = []
        for levels in (0, 2):
            sc = _box(1)
            sc.params.n_spatial, sc.params.radius, sc.params.flags = 3, 8, flags
            if levels:
                _subdivide(sc, 0, levels)
            imgs.append(_render(O, sc))
        a, b = imgs
        assert np.count_nonzero(a) > 200
        res[flags] = float(np.mean(np.isclose(a, b, rtol=1e-6, atol=0)))
    assert res[FLAG_WALK] >= 0.995, res
    assert res[0] < res[FLAG_WALK] - 0.02, res


def test_walk_shift_roundtrip_on_reservoirs(oracle_lib):
    O = oracle_lib
    counts = {}
    for flags in (0, FLAG_WALK):
        sc = _subdivide(_box(1), 0, 2)
        sc.params.n_spatial, sc.params.flags = 0, flags
        g = O.Geom(sc, 0)
        rng = np.random.default_rng(0)
        fwd = inv_fail = bad = 0
        for s in range(8):
            v = O.View(32, 32)
            O.render_frame(v, g, sc, 0, seed=s)
            for pix in range(32 * 32):
                r = v.reservoir(pix)
                if not r["valid"] or r["r"] == 0:
                    continue
                dx, dy = rng.integers(-8, 9, size=2)
                q = pix + dy * 32 + dx
                if q < 0 or q >= 32 * 32 or q == pix:
                    continue
                rc, out = O.shift_roundtrip(v, sc.params, s, pix, q)
                if rc == 0:
                    continue
                fwd += 1
                if rc == -1:
                    inv_fail += 1
                elif abs(out[0] * out[1] - 1) > 1e-4 or out[2] > 1e-4:
                    bad += 1
        counts[flags] = fwd
        assert fwd > 200
        assert inv_fail <= 0.02 * fwd and bad <= 0.02 * fwd, (flags, fwd, inv_fail, bad)
    assert counts[FLAG_WALK] > 1.1 * counts[0], counts


@pytest.mark.parametrize("case", ["box_spatial_fine", "materials_moving_temporal"])
def test_pipeline_unbiased_with_walk(oracle_lib, case):
    O = oracle_lib
    if case == "box_spatial_fine":
        sc, nf = _subdivide(_box(1), 0, 2), 1
    else:
        sc, nf = scenes.box_materials(W=32, H=32, frames=3, moving=True), 3
        sc.params.temporal = 1
    sc.params.flags = FLAG_WALK
    gz, rel, z = _unbiased(O, sc, nf)
    assert abs(gz) < 3.5, (gz, rel)
    assert abs(rel) < 0.03, (gz, rel)
    assert np.max(np.abs(z)) < 4.5, z
