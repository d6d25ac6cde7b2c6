"""Closed-form pins of the oracle's estimator of the ToF path integral (Sec. 3.1).

1. Single-bounce Lambertian plane under a point light (direct paths only, the DIRECT flag):
   every plain path-tracing sample equals (rho/pi) I cos(theta_l) / d_l^2 * 1[L in gate] at the
   jittered primary hit, with L = |x1| + |x1 - light| (camera at the origin).  The sample is
   recomputed here from the camera model, an analytic ray/plane hit and the Philox jitter.
   The mean over many samples equals the exact pixel-footprint integral (2-D quadrature): the
   gate selects an ellipse band on the plane.
2. White furnace: closed Lambertian sphere of radius R, camera and point light at its centre.
   Every bounce-k path contributes rho^k I / (pi R^2) (k >= 2 for indirect-only output), and
   the two-bounce transient density is rho^2 I/(pi R^2) (L - 2R) / (2 R^2) on [2R, 4R] (chords
   of cosine-distributed directions have pdf l / (2 R^2)).
"""
import math

import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes


def _u01(x):
    return (x >> 8) * (1.0 / 16777216.0)


def _direct_sample(sc, ix, iy, u0, u1):
    """Closed-form direct sample at jitter (u0, u1) (scalars or arrays): value and L."""
    s = sc.sensors[0]
    e = sc.emitters[0]
    W, H = s["W"], s["H"]
    f = np.array(s["fwd"], float)
    f /= np.linalg.norm(f)
    rt = np.cross(f, s["up"])
    rt /= np.linalg.norm(rt)
    up = np.cross(rt, f)
    th = math.tan(0.5 * s["fov_y"])
    u0, u1 = np.asarray(u0, float), np.asarray(u1, float)
    sx = (2 * (ix + u0) / W - 1) * th * W / H
    sy = (1 - 2 * (iy + u1) / H) * th
    d = f + rt * sx[..., None] + up * sy[..., None]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    z0 = sc.verts[0, 2]
    x1 = d * (z0 / d[..., 2:3])
    lp = np.array(e["pos"], float)
    dl = np.linalg.norm(lp - x1, axis=-1)
    cos_l = np.abs((lp - x1)[..., 2]) / dl
    rho = sc.materials[0, 1]
    L = np.linalg.norm(x1, axis=-1) + dl
    L0, dL = sc.gates[0]
    val = rho / math.pi * e["power"] * cos_l / dl ** 2
    return val * ((L0 <= L) & (L < L0 + dL)), L


def test_direct_plane_per_sample_exact(oracle_lib):
    O = oracle_lib
    sc = scenes.lambert_plane()
    g = O.Geom(sc, 0)
    seed = 12345
    img = O.render_pt(g, sc, 0, spp=1, seed=seed)
    W, H = sc.sensors[0]["W"], sc.sensors[0]["H"]
    nonzero = 0
    for iy in range(H):
        for ix in range(W):
            pix = iy * W + ix
            u = O.philox([pix, 0, 0, 1], [seed & 0xFFFFFFFF, seed >> 32])
            v, L = _direct_sample(sc, ix, iy, _u01(u[0]), _u01(u[1]))
            v = float(v)
            assert img[iy, ix] == pytest.approx(v, rel=1e-10, abs=1e-14)
            nonzero += v > 0
    assert 4 < nonzero < W * H


def test_direct_plane_pixel_integral(oracle_lib):
    O = oracle_lib
    sc = scenes.lambert_plane()
    g = O.Geom(sc, 0)
    spp = 4096
    img = O.render_pt(g, sc, 0, spp=spp, seed=99, nthreads=8)
    W, H = sc.sensors[0]["W"], sc.sensors[0]["H"]
    n = 400
    grid = (np.arange(n) + 0.5) / n
    checked = 0
    for iy in range(H):
        for ix in range(W):
            A, Bg = np.meshgrid(grid, grid)
            vals = _direct_sample(sc, ix, iy, A, Bg)[0]
            exact = vals.mean()
            p_in = (vals > 0).mean()
            if exact == 0:
                assert img[iy, ix] == 0
                continue
            # per-sample standard deviation bound from the quadrature samples
            sd = vals.std() / math.sqrt(spp)
            quad_err = vals.max() * (4.0 / n)  # boundary cells of the gate's ellipse band
            assert abs(img[iy, ix] - exact) <= 4.5 * sd + quad_err, (ix, iy, p_in)
            checked += 1
    assert checked >= 8


def test_white_furnace_bounce_sums(oracle_lib):
    O = oracle_lib
    rho, R = 0.5, 1.0
    sc = scenes.white_furnace_sphere(R=R, albedo=rho, subdiv=5, W=8, H=8)
    g = O.Geom(sc, 0)
    for depth in (2, 3, 4):
        sc.params.depth = depth
        img = O.render_pt(g, sc, 0, spp=16, seed=5, nthreads=8)
        expected = sum(rho ** k for k in range(2, depth + 1)) / (math.pi * R * R)
        assert img.mean() == pytest.approx(expected, rel=1e-2)
        assert img.min() == pytest.approx(expected, rel=2e-2)


def test_white_furnace_two_bounce_transient(oracle_lib):
    O = oracle_lib
    rho, R = 0.5, 1.0
    sc = scenes.white_furnace_sphere(R=R, albedo=rho, subdiv=5, W=8, H=8)
    sc.params.depth = 2
    B, t0, w = 8, 2.0, 0.25
    sc.bins = (t0, w, B)
    g = O.Geom(sc, 0)
    spp = 4000
    hist = O.render_pt(g, sc, 0, spp=spp, seed=17, nthreads=8, B=B)
    mean = hist.reshape(-1, B).mean(axis=0)
    c = rho * rho / (math.pi * R * R)
    edges = t0 + w * np.arange(B + 1)
    expected = c * ((edges[1:] - 2 * R) ** 2 - (edges[:-1] - 2 * R) ** 2) / (4 * R * R)
    n = 64 * spp
    for b in range(B):
        p = expected[b] / c
        sd = c * math.sqrt(p * (1 - p) / n)
        assert abs(mean[b] - expected[b]) <= 4.5 * sd + 5e-3 * expected[b], (b, mean[b], expected[b])
    assert mean.sum() == pytest.approx(c, rel=5e-3)
