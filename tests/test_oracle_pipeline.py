"""Pins of the oracle's whole ReSTIR pipeline (Sec. 3.2 stages (1)-(4) with the path-length shift
of Sec. 4 and the transient extension of Sec. 4.5).

The exact per-seed values of the pipeline have no published counterpart; what the mathematics
fixes is that the estimator is unbiased for the ToF path integral.  These tests check the
64..256-seed mean of the pipeline against plain path tracing (the plain definition, itself pinned
by the closed forms in test_oracle_closed_forms.py), per 8x8 tile and over the image, plus the
bijectivity of the shift on stored reservoirs.  The sensitivity of the unbiasedness check was
confirmed by planting an MIS-weight mistake in a copy of the oracle (|z| > 17); the shift
Jacobians are pinned separately by finite differences (test_oracle_newton.py) because the
generalized balance heuristic is only weakly sensitive to them.
"""
import numpy as np
import pytest

from paper_2605_11536_gb300 import scenes

T = 8


def _unbiased(O, sc, nframes, nseeds=256, nbatches=32, spp=128, B=0):
    F = nframes - 1
    geoms = [O.Geom(sc, f) for f in range(nframes)]
    W, H = sc.sensors[0]["W"], sc.sensors[0]["H"]
    refs = np.array([O.render_pt(geoms[F], sc, F, spp=spp, seed=7000 + b, nthreads=8, B=B) for b in range(nbatches)])
    imgs = []
    for s in range(nseeds):
        v = O.View(W, H, B)
        for f in range(nframes):
            img, ok = O.render_frame(v, geoms[f], sc, f, seed=s, nthreads=8)
        assert ok.all()
        imgs.append(img)
    imgs = np.array(imgs)
    if B > 0:   # compare the image-summed histogram per bin
        a = imgs.sum(axis=(1, 2))
        r = refs.sum(axis=(1, 2))
        se = np.sqrt(a.var(axis=0, ddof=1) / nseeds + r.var(axis=0, ddof=1) / nbatches)
        m = r.mean(0) > 0
        z = (a.mean(0)[m] - r.mean(0)[m]) / se[m]
        ga, gr = a.sum(1), r.sum(1)
    else:
        z = []
        for ty in range(0, H, T):
            for tx in range(0, W, T):
                a = imgs[:, ty:ty + T, tx:tx + T].mean(axis=(1, 2))
                r = refs[:, ty:ty + T, tx:tx + T].mean(axis=(1, 2))
                se = np.sqrt(a.var(ddof=1) / nseeds + r.var(ddof=1) / nbatches)
                if se > 0:
                    z.append((a.mean() - r.mean()) / se)
        z = np.array(z)
        ga, gr = imgs.mean(axis=(1, 2)), refs.mean(axis=(1, 2))
    gz = (ga.mean() - gr.mean()) / np.sqrt(ga.var(ddof=1) / nseeds + gr.var(ddof=1) / nbatches)
    rel = ga.mean() / gr.mean() - 1
    return gz, rel, z


def _box(nframes):
    sc = scenes.box_icosphere(W=32, H=32, frames=nframes)
    sc.gates = [(5.0, 0.25)] * nframes
    sc.params.n_spatial, sc.params.radius = 2, 4
    sc.params.temporal = int(nframes > 1)
    return sc


@pytest.mark.parametrize("case", ["box_spatial", "box_temporal", "materials_spatial", "materials_moving_temporal"])
def test_pipeline_unbiased(oracle_lib, case):
    O = oracle_lib
    if case == "box_spatial":
        sc, nf = _box(1), 1
    elif case == "box_temporal":
        sc, nf = _box(3), 3
    elif case == "materials_spatial":
        sc, nf = scenes.box_materials(W=32, H=32), 1
    else:
        sc, nf = scenes.box_materials(W=32, H=32, frames=3, moving=True), 3
        sc.params.temporal = 1
    gz, rel, z = _unbiased(O, sc, nf)
    assert abs(gz) < 3.5, (gz, rel)
    assert abs(rel) < 0.03, (gz, rel)
    assert np.max(np.abs(z)) < 4.5, z


def test_transient_pipeline_unbiased(oracle_lib):
    """Per-bin reservoirs with per-bin reuse (Sec. 4.5) are unbiased for every bin."""
    O = oracle_lib
    sc = scenes.box_icosphere(W=16, H=16, frames=2)
    sc.params.n_spatial, sc.params.radius, sc.params.temporal = 2, 4, 1
    sc.bins = (4.4, 0.1, 16)
    gz, rel, z = _unbiased(O, sc, 2, nseeds=128, nbatches=32, spp=64, B=16)
    assert abs(gz) < 3.5, (gz, rel)
    assert abs(rel) < 0.03
    assert np.max(np.abs(z)) < 4.5, z


def test_shift_bijective_on_reservoirs(oracle_lib):
    """Forward shift followed by the inverse shift returns the base path and the Jacobians
    multiply to 1 (the average-gradient gauge is reversible, Sec. 4.3); the identity shift into
    the record's own domain returns it unchanged with unit Jacobian."""
    O = oracle_lib
    sc = _box(1)
    sc.params.n_spatial = 0
    g = O.Geom(sc, 0)
    W = H = 32
    rng = np.random.default_rng(0)
    fwd = inv_fail = bad = ident = 0
    for s in range(12):
        v = O.View(W, H)
        O.render_frame(v, g, sc, 0, seed=s)
        for pix in range(W * H):
            r = v.reservoir(pix)
            if not r["valid"] or r["r"] == 0:
                continue
            rc, out = O.shift_roundtrip(v, sc.params, s, pix, pix)
            assert rc == 1 and out[0] == pytest.approx(1.0, rel=1e-9) and out[2] < 1e-9
            assert out[3] == pytest.approx(r["phat"], rel=1e-9)
            ident += 1
            dx, dy = rng.integers(-4, 5, size=2)
            q = pix + dy * W + dx
            if q < 0 or q >= W * H or q == pix:
                continue
            rc, out = O.shift_roundtrip(v, sc.params, s, pix, q)
            if rc == 0:
                continue
            fwd += 1
            if rc == -1:
                inv_fail += 1
                continue
            if abs(out[0] * out[1] - 1) > 1e-4 or out[2] > 1e-4:
                bad += 1
    assert ident > 100 and fwd > 300
    assert inv_fail <= 0.01 * fwd
    assert bad <= 0.01 * fwd


def test_newton_statistics_in_paper_range(oracle_lib):
    """Context check against Table "Newton statistics" (Sec. 6): a few iterations on average and
    a Newton success rate well above 0.8 for reuse within a few pixels."""
    O = oracle_lib
    sc = _box(1)
    g = O.Geom(sc, 0)
    v = O.View(32, 32)
    for s in range(16):
        O.render_frame(v, g, sc, 0, seed=s)
    st = v.stats()
    assert st["newton_calls"] > 500
    assert 1.0 <= st["newton_iters"] / st["newton_calls"] <= 3.0
    assert st["newton_ok"] / st["newton_calls"] > 0.8


def test_pairwise_mis_equals_balance_heuristic_for_one_reused_domain(oracle_lib):
    """With one reused domain (k = 1) pairwise MIS is the two-technique balance heuristic: a
    spatial pass with one neighbour and a temporal pass give the same images bit for bit."""
    O = oracle_lib
    for nf, temporal in [(1, 0), (2, 1)]:
        sc = scenes.box_icosphere(W=24, H=24, frames=nf)
        sc.gates = [(5.0, 0.25)] * nf
        sc.params.n_spatial, sc.params.radius, sc.params.temporal = 1, 4, temporal
        geoms = [O.Geom(sc, f) for f in range(nf)]
        out = []
        for flags in (0, scenes.FLAG_PAIRWISE_MIS):
            sc.params.flags = flags
            v = O.View(24, 24, 0)
            for f in range(nf):
                img, ok = O.render_frame(v, geoms[f], sc, f, seed=3, nthreads=8)
            out.append(img)
        assert np.array_equal(out[0], out[1])
        assert out[0].sum() > 0


def test_pairwise_mis_unbiased(oracle_lib):
    """Pairwise MIS weights sum to one over the techniques at every y, so the estimator stays
    unbiased with k = 3 reused domains (and differs from the balance heuristic per seed)."""
    O = oracle_lib
    sc = _box(1)
    sc.params.n_spatial = 3
    sc.params.flags = scenes.FLAG_PAIRWISE_MIS
    gz, rel, z = _unbiased(O, sc, 1)
    assert abs(gz) < 3.5, (gz, rel)
    assert abs(rel) < 0.03, (gz, rel)
    assert np.max(np.abs(z)) < 4.5, z
    g = O.Geom(sc, 0)
    a = O.render_frame(O.View(32, 32, 0), g, sc, 0, seed=5, nthreads=8)[0]
    sc.params.flags = 0
    b = O.render_frame(O.View(32, 32, 0), g, sc, 0, seed=5, nthreads=8)[0]
    assert not np.array_equal(a, b)


@pytest.mark.parametrize("spatial", [0, 2])
def test_transient_bin_reuse_unbiased(oracle_lib, spatial):
    """Bin reuse (Sec. 4.5's extra reuse axis): each bin's reservoir also reuses the same pixel's
    neighbouring bins, shifted by one bin width; absent bins (outside the histogram) take no part in
    the MIS.  The histogram stays unbiased per bin."""
    O = oracle_lib
    sc = scenes.box_icosphere(W=16, H=16, frames=2)
    sc.params.n_spatial, sc.params.radius, sc.params.temporal = spatial, 4, 1
    sc.params.flags = scenes.FLAG_BIN_REUSE
    sc.bins = (4.4, 0.1, 16)
    gz, rel, z = _unbiased(O, sc, 2, nseeds=128, nbatches=32, spp=64, B=16)
    assert abs(gz) < 3.5, (gz, rel)
    assert abs(rel) < 0.03
    assert np.max(np.abs(z)) < 4.5, z
