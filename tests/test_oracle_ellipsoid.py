"""Pins of the oracle's ellipsoidal path connection (Sec. 4.4 "Initialization with Ellipsoidal Path
Connection", Sec. 5 "Ellipsoidal Path Connection").

The sampler places a vertex z with l(z) = |x - z| + |z - q| in [l_a, l_b) and returns its area
density p(z).  What the mathematics fixes:
* sum over samples of g(z) / p(z), divided by the number of draws, is an unbiased estimate of the
  integral of g over the surface region {l(z) in [l_a, l_b)}; the region's area and first moment
  are computed here independently by uniform area sampling of the triangles;
* the density evaluated at a point reached by other means equals the density the sampler reported;
* the path-tree NEE and the ellipsoidal connection, combined by the balance heuristic, estimate the
  same integral as the tree alone: the two-bounce white furnace has a closed form, and the whole
  pipeline (initial candidates, temporal and spatial reuse) matches plain path tracing.
"""
import math

import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes
from tests.test_oracle_pipeline import _box, _unbiased


def _world_tris(sc, frame=0):
    xf = sc.xforms[frame]
    out = np.empty((len(sc.tris), 3, 3))
    for t, tri in enumerate(sc.tris):
        M = xf[sc.tri_object[t]].reshape(3, 4)
        for c in range(3):
            out[t, c] = M[:, :3] @ sc.verts[tri[c]] + M[:, 3]
    return out


def _region_integrals(tris, x, q, la, lb, n, rng):
    """Area and first moments of {z on the triangles : la <= |x - z| + |z - q| < lb} by uniform
    area sampling (n points), with their standard errors."""
    e1, e2 = tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]
    A = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    ti = rng.choice(len(A), size=n, p=A / A.sum())
    r1, r2 = rng.random(n), rng.random(n)
    s = np.sqrt(r1)
    b1, b2 = s * (1 - r2), s * r2
    P = tris[ti, 0] + e1[ti] * b1[:, None] + e2[ti] * b2[:, None]
    ell = np.linalg.norm(P - x, axis=1) + np.linalg.norm(P - q, axis=1)
    m = (ell >= la) & (ell < lb)
    vals = np.stack([m, m * P[:, 0], m * P[:, 2]], axis=1) * A.sum()
    return vals.mean(0), vals.std(0) / math.sqrt(n)


def _sampler_integrals(O, g, x, q, la, lb, n, rng):
    vals = np.zeros((n, 3))
    placed = 0
    for i in range(n):
        u = rng.integers(0, 2 ** 32, size=24, dtype=np.uint64).astype(np.uint32)
        r = O.ell_sample(g, x, q, la, lb, u)
        if r is None:
            continue
        tri, b1, b2, pdf, z = r
        ell = np.linalg.norm(z - x) + np.linalg.norm(z - q)
        assert la - 1e-9 <= ell < lb + 1e-9
        vals[i] = np.array([1.0, z[0], z[2]]) / pdf
        placed += 1
    return vals.mean(0), vals.std(0) / math.sqrt(n), placed


@pytest.mark.parametrize("case", ["box_general", "box_coincident_foci", "furnace_sphere"])
def test_density_integrates_to_region(oracle_lib, case):
    """E[g(z)/p(z)] equals the integral of g over the gated surface region (g = 1, z_x, z_z): a
    dropped factor of the density (the hierarchy walk, the length interval, the angle measure or
    the coarea Jacobian), or a region the sampler cannot reach, moves it by many standard errors."""
    O = oracle_lib
    rng = np.random.default_rng(11)
    if case == "furnace_sphere":
        sc = scenes.white_furnace_sphere(R=1.0, albedo=0.5, subdiv=3)
        x, q = np.array([0.0, 0.0, -0.999]), np.zeros(3)
        la, lb = 1.5, 2.0
    else:
        sc = scenes.box_icosphere(W=8, H=8)
        x = np.array([0.3, -0.5, -1.0])
        q = x.copy() if case == "box_coincident_foci" else np.array([-0.4, 0.6, 0.2])
        d = np.linalg.norm(x - q)
        la, lb = (2.2, 2.8) if case == "box_coincident_foci" else (d + 1.5, d + 1.9)
    g = O.Geom(sc, 0)
    est, se, placed = _sampler_integrals(O, g, x, q, la, lb, 40000, rng)
    ref, rse = _region_integrals(_world_tris(sc), x, q, la, lb, 2_000_000, rng)
    assert placed > 400
    assert ref[0] > 0.05
    for k in range(3):
        z = (est[k] - ref[k]) / math.sqrt(se[k] ** 2 + rse[k] ** 2)
        assert abs(z) < 4.5, (k, est, ref, se, rse)


def test_density_matches_sampler(oracle_lib):
    """The density at a placed point, recomputed from the point alone (the walk's probability along
    its root-to-leaf path, the ellipse through it), equals the density the sampler reported."""
    O = oracle_lib
    rng = np.random.default_rng(5)
    sc = scenes.heightfield_spheres(W=8, H=8, frames=1)
    g = O.Geom(sc, 0)
    x, q = np.array([1.0, 2.0, 0.1]), np.array([0.5, -1.0, 1.7])
    d = np.linalg.norm(x - q)
    checked = 0
    for i in range(3000):
        u = rng.integers(0, 2 ** 32, size=24, dtype=np.uint64).astype(np.uint32)
        r = O.ell_sample(g, x, q, d + 2.0, d + 2.03, u)
        if r is None:
            continue
        tri, b1, b2, pdf, z = r
        assert O.ell_pdf(g, x, q, d + 2.0, d + 2.03, tri, b1, b2) == pytest.approx(pdf, rel=1e-6)
        checked += 1
    assert checked > 100
    # outside the length interval the density is zero
    assert O.ell_pdf(g, x, q, d + 5.0, d + 5.01, tri, b1, b2) == 0.0


def test_walk_probabilities_are_a_subdistribution(oracle_lib):
    """The walk's triangle probabilities are positive exactly on reachable triangles and sum to at
    most one (the rest is the walk ending at a node whose children both miss); a triangle the
    ellipsoid passes through is always reachable."""
    O = oracle_lib
    sc = scenes.heightfield_spheres(W=8, H=8, frames=1)
    g = O.Geom(sc, 0)
    tris = _world_tris(sc)
    x, q = np.array([1.0, 2.0, 0.1]), np.array([0.5, -1.0, 1.7])
    ell = np.linalg.norm(x - q) + 2.0
    p = O.ell_tri_probs(g, x, q, ell, len(tris))
    assert 0.0 < p.sum() <= 1.0 + 1e-12
    # brute force: triangles whose corners lie on both sides of the ellipsoid are crossed by it
    lens = np.linalg.norm(tris - x, axis=2) + np.linalg.norm(tris - q, axis=2)
    crossed = (lens.min(1) < ell) & (lens.max(1) > ell)
    assert crossed.sum() > 50
    assert np.all(p[crossed] > 0)
    # and a triangle entirely inside or outside it only when its box test passes conservatively
    far = (lens.min(1) > ell + 0.5) | (lens.max(1) < ell - 0.5)
    assert np.all(p[far] == 0)


def test_two_bounce_furnace_closed_form(oracle_lib):
    """White furnace (closed Lambertian sphere, camera and point light at the centre): the gated
    two-bounce image is rho^2 I/(pi R^2) ((L1 - 2R)^2 - (L0 - 2R)^2) / (4 R^2) at every pixel.  The
    RIS estimate with the ellipsoidal connection (MIS with the path tree) matches it, as does the
    path tree alone."""
    O = oracle_lib
    rho, R = 0.5, 1.0
    sc = scenes.white_furnace_sphere(R=R, albedo=rho, subdiv=4, W=8, H=8)
    sc.params.depth, sc.params.n_cand, sc.params.n_spatial, sc.params.temporal = 2, 4, 0, 0
    L0, dL = 2.5, 0.5
    sc.gates = [(L0, dL)]
    g = O.Geom(sc, 0)
    exact = rho * rho / (math.pi * R * R) * ((L0 + dL - 2 * R) ** 2 - (L0 - 2 * R) ** 2) / (4 * R * R)
    for flags in (0, scenes.FLAG_ELLIPSOID):
        sc.params.flags = flags
        imgs = np.array([O.render_frame(O.View(8, 8), g, sc, 0, seed=s, nthreads=8)[0] for s in range(400)])
        m, se = imgs.mean(), imgs.std() / math.sqrt(imgs.size)
        assert abs(m - exact) < 4.5 * se + 5e-3 * exact, (flags, m, exact, se)


def test_ellipsoid_finds_in_gate_paths(oracle_lib):
    """On the narrow-gate heightfield workload (3 cm gate at 8 m) the path trees find an in-gate
    path in few pixels; the ellipsoidal connection, whose vertices lie in the gate by
    construction, finds one in many more, and the per-pixel variance of the initial estimate drops."""
    O = oracle_lib
    sc = scenes.heightfield_spheres(W=32, H=32, frames=1)
    sc.params.n_spatial, sc.params.temporal = 0, 0
    g = O.Geom(sc, 0)
    res = {}
    for flags in (0, scenes.FLAG_ELLIPSOID):
        sc.params.flags = flags
        res[flags] = np.array([O.render_frame(O.View(32, 32), g, sc, 0, seed=s, nthreads=8)[0] for s in range(16)])
    frac = {f: (v > 0).mean() for f, v in res.items()}
    var = {f: v.var(axis=0).mean() for f, v in res.items()}
    assert frac[scenes.FLAG_ELLIPSOID] > 4 * frac[0], frac
    assert var[scenes.FLAG_ELLIPSOID] < 0.7 * var[0], var


@pytest.mark.parametrize("case", ["box_spatial", "materials_moving_temporal"])
def test_pipeline_with_ellipsoid_unbiased(oracle_lib, case):
    """Initial candidates by both strategies, then temporal and spatial reuse (the reconnection and
    replay shifts do not depend on how a vertex was sampled): unbiased against plain path tracing
    per 8x8 tile and over the image, with Lambertian, glossy and mirror surfaces."""
    O = oracle_lib
    if case == "box_spatial":
        sc, nf = _box(1), 1
    else:
        sc, nf = scenes.box_materials(W=32, H=32, frames=3, moving=True), 3
        sc.params.temporal = 1
    sc.params.flags |= scenes.FLAG_ELLIPSOID
    gz, rel, z = _unbiased(O, sc, nf, nseeds=128)
    assert abs(gz) < 3.5, (gz, rel)
    assert abs(rel) < 0.03, (gz, rel)
    assert np.max(np.abs(z)) < 4.5, z
