"""Pins of the oracle's building blocks against things other than itself.

* Philox4x32-10 against the published known-answer vectors (tests/golden).
* The oracle's BVH closest hit against brute force over all triangles.
* BSDFs: reciprocity, sampling consistency (throughput = f cos / pdf), the GGX distribution's
  projected-area normalisation by quadrature, Lambert throughput = albedo.
* Streaming weighted selection: selection frequencies equal w_i / sum w (exhaustive small cases).
"""
import math
import os

import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle_lib):
    O = oracle_lib
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def _random_rays(rng, n, lo, hi):
    o = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


@pytest.mark.parametrize("which", ["box", "field"])
def test_bvh_matches_brute_force(oracle_lib, which):
    O = oracle_lib
    if which == "box":
        sc = scenes.box_icosphere()
        lo, hi = -1.9, 1.9
    else:
        sc = scenes.heightfield_spheres(W=8, H=8, frames=2, nx=40, ny=25, n_spheres=6)
        lo, hi = -3.0, 3.0
    g = O.Geom(sc, sc.n_frames - 1)
    rng = np.random.default_rng(7)
    o, d = _random_rays(rng, 400, lo, hi)
    nhit = 0
    for i in range(len(o)):
        a = g.intersect(o[i], d[i])
        b = g.intersect(o[i], d[i], brute=True)
        assert (a is None) == (b is None)
        if a is not None:
            nhit += 1
            assert a[1] == pytest.approx(b[1], rel=1e-12, abs=1e-12)
            if a[0] != b[0]:  # exact tie on a shared edge: same distance, different triangle
                assert abs(a[1] - b[1]) < 1e-12
    assert nhit > 50


def _unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


def test_bsdf_reciprocity_and_sampling(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(3)
    n = _unit([0.2, -0.3, 0.9])
    for typ, alpha in [(0, 0.0), (1, 0.1), (1, 0.35), (1, 0.8)]:
        for _ in range(50):
            wi = _unit(rng.normal(size=3))
            wo = _unit(rng.normal(size=3))
            a = O.bsdf_eval(typ, 0.7, alpha, n, wi, wo)
            b = O.bsdf_eval(typ, 0.7, alpha, n, wo, wi)
            assert a == pytest.approx(b, rel=1e-12, abs=1e-15)
            if np.dot(n, wi) * np.dot(n, wo) <= 0:
                assert a == 0.0
        for _ in range(200):
            wi = _unit(rng.normal(size=3))
            ok, wo, pdf, thr = O.bsdf_sample(typ, 0.7, alpha, n, wi, rng.uniform(), rng.uniform())
            if not ok:
                continue
            f = O.bsdf_eval(typ, 0.7, alpha, n, wi, wo)
            p = O.bsdf_pdf(typ, 0.7, alpha, n, wi, wo)
            assert p == pytest.approx(pdf, rel=1e-9)
            assert thr == pytest.approx(f * abs(np.dot(n, wo)) / pdf, rel=1e-9)
            if typ == 0:
                assert thr == pytest.approx(0.7, rel=1e-12)


def _hemisphere_quadrature(fn, n_theta=400, n_phi=400):
    th = (np.arange(n_theta) + 0.5) * (math.pi / 2) / n_theta
    ph = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    dA = (math.pi / 2 / n_theta) * (2 * math.pi / n_phi)
    tot = 0.0
    for t in th:
        st, ct = math.sin(t), math.cos(t)
        for p in ph:
            tot += fn(np.array([st * math.cos(p), st * math.sin(p), ct])) * st * dA
    return tot


@pytest.mark.parametrize("alpha", [0.25, 0.5])
def test_ggx_pdf_normalises(oracle_lib, alpha):
    """At normal incidence the sampled half-vector has P(tan^2 theta_h <= T) = T / (alpha^2 + T)
    (the GGX distribution with int D(h) (n.h) dh = 1, Walter et al. 2007); reflection doubles the
    polar angle, so the mass reflected above the horizon is P(theta_h < 45 deg) = 1/(1 + alpha^2)."""
    O = oracle_lib
    n = np.array([0.0, 0.0, 1.0])
    tot = _hemisphere_quadrature(lambda wo: O.bsdf_pdf(1, 1.0, alpha, n, n, wo), 600, 16)
    assert tot == pytest.approx(1.0 / (1.0 + alpha * alpha), rel=2e-3)


def test_lambert_albedo_by_quadrature(oracle_lib):
    O = oracle_lib
    n = np.array([0.0, 0.0, 1.0])
    wi = _unit([0.3, 0.1, 0.8])
    tot = _hemisphere_quadrature(lambda wo: O.bsdf_eval(0, 0.6, 0.0, n, wi, wo) * wo[2], 200, 64)
    assert tot == pytest.approx(0.6, rel=2e-3)


def test_stream_select_frequencies(oracle_lib):
    """Weighted reservoir sampling (Chao 1982, used by ReSTIR for streaming RIS, Sec. 3.2):
    candidate i is selected with probability w_i / sum_j w_j."""
    O = oracle_lib
    rng = np.random.default_rng(11)
    for n in range(1, 7):
        w = rng.uniform(0.0, 1.0, size=n)
        w[rng.uniform(size=n) < 0.2] = 0.0
        if w.sum() == 0:
            w[0] = 0.5
        cnt = np.zeros(n)
        T = 40000
        for _ in range(T):
            sel, S = O.stream_select(w, rng.uniform(size=n))
            cnt[sel] += 1
        assert S == pytest.approx(w.sum())
        p = w / w.sum()
        sigma = np.sqrt(p * (1 - p) / T)
        assert np.all(np.abs(cnt / T - p) <= 4.5 * sigma + 1e-12)


@pytest.mark.parametrize("typ,alpha", [(0, 0.0), (1, 0.15), (1, 0.45)])
def test_sampling_pdf_is_density_of_direction_map(oracle_lib, typ, alpha):
    """The replay Jacobian of the hybrid shift is the ratio of the two paths' sampling pdfs
    (Sec. 3.2 shift maps; random replay): that holds only if each pdf is the true density of its
    sampler u -> w.  Check pdf(w(u)) = 1 / |dw/du0 x dw/du1| by central differences."""
    O = oracle_lib
    rng = np.random.default_rng(5 + typ)
    n = _unit([0.1, 0.2, 0.95])
    h = 1e-6
    checked = 0
    for _ in range(60):
        wi = _unit(n + rng.normal(size=3) * 0.4)
        u0, u1 = rng.uniform(0.05, 0.95, size=2)
        ok, wo, pdf, _ = O.bsdf_sample(typ, 0.7, alpha, n, wi, u0, u1)
        oks = [O.bsdf_sample(typ, 0.7, alpha, n, wi, u0 + a, u1 + b)
               for a, b in ((h, 0), (-h, 0), (0, h), (0, -h))]
        if not ok or not all(o[0] for o in oks):
            continue
        d0 = (oks[0][1] - oks[1][1]) / (2 * h)
        d1 = (oks[2][1] - oks[3][1]) / (2 * h)
        area = np.linalg.norm(np.cross(d0, d1))
        assert pdf == pytest.approx(1.0 / area, rel=1e-4)
        checked += 1
    assert checked > 30
