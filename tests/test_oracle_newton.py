"""Pins of the path-length-aware shift (Sec. 4.2-4.3) in the oracle.

* grad / Hessian of L(xi) = |p1 - p(xi)| + |p2 - p(xi)| against central finite differences
  (the closed forms of Sec. 4.3 "Gradient and Hessian Evaluation", Q = 0 on a flat triangle);
* Newton reaches |L(y') - L_target| < 1e-6 L (invariant);
* delta = 0 on an already-valid path takes 0 iterations and returns the identity;
* the shift Jacobian det(dF/dxi) / det(dF/dxi') (implicit differentiation) against central
  finite differences of the solved map xi -> xi';
* reversibility of the average-gradient gauge: solving back from xi' with -delta returns xi and
  the two determinants multiply to 1;
* the printed sign of the 0.5 H R (xi' - xi) term in the second row of dF/dxi' disagrees with
  the finite differences while the derivative of the stated F agrees: differentiating
  (R m)^T (xi' - xi) with R^T = -R gives R m - 0.5 H(xi') R (xi' - xi), so the printed + is taken
  as a sign slip and the derivative is used.
"""
import numpy as np
import pytest


def _frame(v0, v1, v2):
    e1, e2 = v1 - v0, v2 - v0
    t = e1 / np.linalg.norm(e1)
    n = np.cross(e1, e2)
    n /= np.linalg.norm(n)
    b = np.cross(n, t)
    return dict(o=v0, t=t, b=b)


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    v0 = rng.normal(size=3) * 0.2
    v1 = v0 + np.array([1.0, 0.1, 0.05])
    v2 = v0 + np.array([0.2, 0.9, -0.1])
    fr = _frame(v0, v1, v2)
    p1x = v0 + np.array([0.4, 0.3, 2.0]) + rng.normal(size=3) * 0.1
    p2x = v0 + np.array([-1.0, 0.8, 1.5]) + rng.normal(size=3) * 0.1
    base = dict(p1=p1x, p2=p2x, **fr)
    off = dict(p1=p1x + np.array([0.08, -0.05, 0.02]), p2=p2x, **fr)
    xi = np.array([0.35, 0.25])
    return base, off, xi


def _L_np(path, xi):
    p = path["o"] + xi[0] * path["t"] + xi[1] * path["b"]
    return np.linalg.norm(path["p1"] - p) + np.linalg.norm(path["p2"] - p)


def test_length_gradient_hessian_fd(oracle_lib):
    O = oracle_lib
    base, _, xi = _setup(1)
    L, g, h = O.length_derivs(base["p1"], base["p2"], base["o"], base["t"], base["b"], xi)
    assert L == pytest.approx(_L_np(base, xi), rel=1e-14)
    H = np.array([[h[0], h[1]], [h[1], h[2]]])
    eps = 1e-5
    for i in range(2):
        e = np.zeros(2)
        e[i] = eps
        Lp = O.length_derivs(base["p1"], base["p2"], base["o"], base["t"], base["b"], xi + e)
        Lm = O.length_derivs(base["p1"], base["p2"], base["o"], base["t"], base["b"], xi - e)
        assert g[i] == pytest.approx((Lp[0] - Lm[0]) / (2 * eps), rel=1e-7, abs=1e-9)
        assert H[:, i] == pytest.approx((Lp[1] - Lm[1]) / (2 * eps), rel=1e-6, abs=1e-8)


def test_newton_invariant_and_identity(oracle_lib):
    O = oracle_lib
    base, off, xi = _setup(2)
    delta = 0.01
    ok, xp, det, it, F = O.newton(base, off, xi, delta, tol_stop=1e-13, tol_succ=1e-9)
    assert ok and 1 <= it <= 5
    target = _L_np(base, xi) + delta
    assert abs(_L_np(off, xp) - target) < 1e-6 * target
    assert abs(F[0]) < 1e-9 and abs(F[1]) < 1e-9
    # delta = 0 on the same path: zero iterations, identity, unit determinant
    ok, xp, det, it, F = O.newton(base, base, xi, 0.0, tol_stop=1e-12, tol_succ=1e-9)
    assert ok and it == 0
    assert np.allclose(xp, xi, atol=0) and det == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("seed,delta", [(3, 0.02), (4, -0.03), (5, 0.0), (6, 0.05)])
def test_shift_jacobian_fd_and_reversibility(oracle_lib, seed, delta):
    O = oracle_lib
    base, off, xi = _setup(seed)
    ok, xp, det, it, F = O.newton(base, off, xi, delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
    assert ok
    # finite differences of the solved map (delta held fixed, the base vertex moves)
    h = 1e-5
    Jfd = np.zeros((2, 2))
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        okp, xpp, *_ = O.newton(base, off, xi + e, delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
        okm, xpm, *_ = O.newton(base, off, xi - e, delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
        assert okp and okm
        Jfd[:, i] = (xpp - xpm) / (2 * h)
    assert abs(np.linalg.det(Jfd)) == pytest.approx(det, rel=2e-5)
    # reversibility: from the offset path back to the base path with -delta
    ok2, xb, det2, it2, F2 = O.newton(off, base, xp, -delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
    assert ok2
    assert np.allclose(xb, xi, atol=1e-9)
    assert det * det2 == pytest.approx(1.0, rel=1e-8)


def test_printed_sign_of_gauge_row_disagrees_with_fd(oracle_lib):
    """Reading c1: evaluate both signs of the 0.5 H(xi') R (xi' - xi) term of row 2 of dF/dxi'
    at the converged solution; only the derivative of the stated F matches the FD Jacobian."""
    O = oracle_lib
    base, off, xi = _setup(8)
    delta = 0.06
    ok, xp, det, it, F = O.newton(base, off, xi, delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
    assert ok
    _, gx, hx = O.length_derivs(base["p1"], base["p2"], base["o"], base["t"], base["b"], xi)
    _, gy, hy = O.length_derivs(off["p1"], off["p2"], off["o"], off["t"], off["b"], xp)
    Hx = np.array([[hx[0], hx[1]], [hx[1], hx[2]]])
    Hy = np.array([[hy[0], hy[1]], [hy[1], hy[2]]])
    R = np.array([[0.0, -1.0], [1.0, 0.0]])
    m = 0.5 * (gx + gy)
    d = xp - xi
    Bm = np.array([-gx, -(R @ m + 0.5 * Hx @ R @ d)])
    A_derived = np.array([gy, R @ m - 0.5 * Hy @ R @ d])
    A_printed = np.array([gy, R @ m + 0.5 * Hy @ R @ d])
    det_derived = abs(np.linalg.det(Bm) / np.linalg.det(A_derived))
    det_printed = abs(np.linalg.det(Bm) / np.linalg.det(A_printed))
    assert det == pytest.approx(det_derived, rel=1e-10)
    h = 1e-5
    Jfd = np.zeros((2, 2))
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        _, xpp, *_ = O.newton(base, off, xi + e, delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
        _, xpm, *_ = O.newton(base, off, xi - e, delta, max_iter=20, tol_stop=1e-14, tol_succ=1e-10)
        Jfd[:, i] = (xpp - xpm) / (2 * h)
    fd = abs(np.linalg.det(Jfd))
    assert det_derived == pytest.approx(fd, rel=2e-5)
    assert abs(det_printed - fd) > 1e-3 * fd


@pytest.mark.parametrize("gauge", ["axis_t", "axis_b", "start"])
def test_comparison_gauges_jacobian_fd(oracle_lib, gauge):
    """The comparison gauges of Sec. 4.3 (fixed axis G(xi) = a^T xi, start-point gradient): the
    implicit-function determinant of each matches central differences of its solved map."""
    O = oracle_lib
    base, off, xi = _setup(9)
    delta = 0.03
    kw = dict(max_iter=30, tol_stop=1e-14, tol_succ=1e-10, gauge=gauge)
    ok, xp, det, it, F = O.newton(base, off, xi, delta, **kw)
    assert ok and abs(F[0]) < 1e-10 and abs(F[1]) < 1e-10
    h = 1e-5
    Jfd = np.zeros((2, 2))
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        Jfd[:, i] = (O.newton(base, off, xi + e, delta, **kw)[1] - O.newton(base, off, xi - e, delta, **kw)[1]) / (2 * h)
    assert abs(np.linalg.det(Jfd)) == pytest.approx(det, rel=2e-5)
    if gauge == "axis_t":
        assert xp[1] == pytest.approx(xi[1], abs=1e-12)
    if gauge == "axis_b":
        assert xp[0] == pytest.approx(xi[0], abs=1e-12)


def test_axis_gauges_reversible_start_gradient_is_not(oracle_lib):
    """Sec. 4.3: a fixed axis and the average gradient are reversible (solving back with -delta
    returns xi, the determinants multiply to 1); moving along the start point's gradient alone is
    not, unless the gradients at both ends are parallel."""
    O = oracle_lib
    base, _, xi = _setup(10)
    delta = 0.15
    kw = dict(max_iter=40, tol_stop=1e-15, tol_succ=1e-10)
    for gauge in ("average", "axis_t", "axis_b", "start"):
        ok, xp, det, *_ = O.newton(base, base, xi, delta, gauge=gauge, **kw)
        assert ok, gauge
        ok2, xb, det2, *_ = O.newton(base, base, xp, -delta, gauge=gauge, **kw)
        assert ok2, gauge
        err = float(np.abs(xb - xi).max())
        if gauge == "start":
            assert err > 1e-4, err
        else:
            assert err < 1e-9 and det * det2 == pytest.approx(1.0, rel=1e-8), (gauge, err)
