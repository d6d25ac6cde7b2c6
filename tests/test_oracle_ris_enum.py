"""Exhaustive-enumeration pins of the resampling steps of Sec. 3.2 (RIS; GRIS with the generalized
balance heuristic, and pairwise MIS) on the oracle's own primitives: ris_accept (one step of the
streaming selection), ris_W (the contribution weight W = sum w / p_hat(y)) and gris_mis (the MIS
weight of a merge candidate).  Every initial-candidate stream and every reuse merge of the
oracle's pipeline calls these routines.

On a finite sample space every expectation is a finite sum.  All tuples of up to 6 candidates are
enumerated, and for each tuple every accept / reject pattern of the streaming selection, each
step's acceptance region being measured on the routine itself by bisection in u.  That gives the
exact distribution of the selected sample and of its W, which is checked against:
* the selection probabilities w_i / sum_j w_j of every tuple;
* E[g(Y) W_Y] = sum over {x : p_hat(x) > 0} of g(x), for g = p_hat and for another integrand
  (unbiased RIS with w = (1/N) p_hat / p);
* for GRIS merges of 2 and 3 domains with their own pmfs, targets, candidate counts and
  confidences (each input a reservoir of that domain's RIS, identity shifts): the MIS weights of
  one y summing to 1, and E[g(Y) W_Y] = sum_x g(x) exactly, for both heuristics.
A contribution weight off by the 1/N factor, or a heuristic whose denominator drops the canonical
domain, misses these sums (checked as controls)."""
import itertools

import numpy as np
import pytest

import oracle as O

TOL = 1e-12


def _threshold(S_before, w):
    """sup{u in [0, 1) : ris_accept(S_before, w, u) accepts}, by bisection on the routine."""
    assert O.ris_accept(S_before, w, 0.0)[0]
    if O.ris_accept(S_before, w, np.nextafter(1.0, 0.0))[0]:
        return 1.0
    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if O.ris_accept(S_before, w, mid)[0]:
            lo = mid
        else:
            hi = mid
    # the routine is monotone in u: accepted below the threshold, rejected above it
    for u in np.linspace(0.0, 1.0, 17)[:-1]:
        assert O.ris_accept(S_before, w, u)[0] == (u <= lo), (u, lo)
    return 0.5 * (lo + hi)


def selection(ws):
    """Exact distribution {index or None: probability} of the oracle's streaming selection over the
    weights ws, and the final running sum."""
    idx = [i for i, w in enumerate(ws) if w > 0]
    thr, S = [], 0.0
    for i in idx:
        thr.append(_threshold(S, ws[i]))
        S = O.ris_accept(S, ws[i], 0.5)[1]
    dist = {}
    for pat in itertools.product((True, False), repeat=len(idx)):
        prob = 1.0
        u = np.full(len(ws), 0.5)
        for k, (i, acc) in enumerate(zip(idx, pat)):
            prob *= thr[k] if acc else 1.0 - thr[k]
            u[i] = 0.5 * thr[k] if acc else 0.5 * (1.0 + thr[k])
        if prob == 0.0:
            continue
        sel, S_out = O.stream_select(ws, u)
        assert S_out == S
        key = sel if sel >= 0 else None
        dist[key] = dist.get(key, 0.0) + prob
    return dist, S


def ris_outcomes(p, phat, N, w_scale=1.0):
    """Distribution of one domain's RIS reservoir after N candidates drawn from the pmf p with
    target phat: {(y, W): probability}, y None for an empty reservoir.  w = (1/N) phat / p
    (times w_scale, for the controls)."""
    out = {}
    for tup in itertools.product(range(len(p)), repeat=N):
        pt = float(np.prod([p[x] for x in tup]))
        ws = [w_scale * phat[x] / p[x] / N for x in tup]
        dist, S = selection(ws)
        for i, q in dist.items():
            key = (None, 0.0) if i is None else (tup[i], O.ris_W(S, phat[tup[i]]))
            out[key] = out.get(key, 0.0) + pt * q
    return out


P0 = np.array([0.5, 0.2, 0.3])
PHAT0 = np.array([0.7, 1.3, 0.0])      # f * 1[tau in gate]: the third point is outside the gate
G2 = np.array([2.0, -1.0, 5.0])


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_ris_selection_probabilities_and_expectation_exact(N):
    E_phat = E_g = total = 0.0
    for tup in itertools.product(range(3), repeat=N):
        pt = float(np.prod([P0[x] for x in tup]))
        total += pt
        ws = [PHAT0[x] / P0[x] / N for x in tup]
        dist, S = selection(ws)
        if S > 0:
            for i, w in enumerate(ws):
                assert abs(dist.get(i, 0.0) - w / S) < TOL, (tup, i)
            assert None not in dist
        else:
            assert dist == {None: 1.0}
        for i, q in dist.items():
            if i is None:
                continue
            y = tup[i]
            W = O.ris_W(S, PHAT0[y])
            E_phat += pt * q * PHAT0[y] * W
            E_g += pt * q * G2[y] * W
    assert abs(total - 1.0) < TOL
    assert abs(E_phat - PHAT0.sum()) < TOL
    assert abs(E_g - G2[PHAT0 > 0].sum()) < TOL


def test_ris_control_without_one_over_N_is_biased():
    out = ris_outcomes(P0, PHAT0, 3, w_scale=3.0)
    E = sum(q * PHAT0[y] * W for (y, W), q in out.items() if y is not None)
    assert abs(E - PHAT0.sum()) > 1.0


DOMAINS = [
    # (pmf, target, candidates N = confidence M)
    (np.array([0.5, 0.2, 0.3]), np.array([0.7, 1.3, 0.0]), 2),
    (np.array([0.25, 0.25, 0.5]), np.array([0.4, 0.0, 2.0]), 1),
    (np.array([0.6, 0.3, 0.1]), np.array([1.1, 0.9, 0.3]), 2),
]


def merge_expectation(doms, g, pairwise, mis=None):
    """E[g(Y) W_Y] of a GRIS merge into domain 0 of the domains' RIS reservoirs (identity shifts,
    Jacobian 1): w_s = m_s(y_s) phat_0(y_s) W_s, selection by the streaming routine, W = ris_W."""
    M = [float(N) for _, _, N in doms]
    mis = mis or (lambda T, s: O.gris_mis(M, T, s, pairwise))
    outs = [list(ris_outcomes(p, ph, N).items()) for p, ph, N in doms]
    E = 0.0
    for combo in itertools.product(*outs):
        pc = float(np.prod([q for _, q in combo]))
        ws, ys = [], []
        for s, ((y, W), _) in enumerate(combo):
            w = 0.0
            if y is not None and doms[0][1][y] > 0:
                T = [ph[y] for _, ph, _ in doms]
                w = mis(T, s) * doms[0][1][y] * W
            ws.append(w)
            ys.append(y)
        dist, S = selection(ws)
        if S > 0:
            for s, w in enumerate(ws):
                assert abs(dist.get(s, 0.0) - w / S) < TOL
        for s, q in dist.items():
            if s is not None:
                E += pc * q * g[ys[s]] * O.ris_W(S, doms[0][1][ys[s]])
    return E


@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("pairwise", [False, True])
def test_gris_merge_expectation_exact(n, pairwise):
    doms = DOMAINS[:n]
    M = [float(N) for _, _, N in doms]
    # the MIS weights of any y over the domains that can produce it sum to 1
    for y in range(3):
        if doms[0][1][y] > 0:
            T = [ph[y] for _, ph, _ in doms]
            tot = sum(O.gris_mis(M, T, s, pairwise) for s in range(n) if T[s] > 0)
            assert abs(tot - 1.0) < TOL, (y, tot)
    g = np.where(doms[0][1] > 0, G2, 0.0)      # integrands supported where the canonical target is
    assert abs(merge_expectation(doms, doms[0][1], pairwise) - doms[0][1].sum()) < TOL
    assert abs(merge_expectation(doms, g, pairwise) - g.sum()) < TOL


def test_gris_control_without_canonical_term_is_biased():
    doms = DOMAINS[:3]

    def no_conf(T, s):
        den = sum(T)
        return T[s] / den if den > 0 else 0.0
    M = [float(N) for _, _, N in doms]
    # a heuristic without the confidences differs from the oracle's, but is still a partition of
    # unity (so unbiased): it is no control.  The control that must fail drops the canonical term.
    T = [ph[0] for _, ph, _ in doms]
    assert abs(no_conf(T, 0) - O.gris_mis(M, T, 0, False)) > 1e-3

    def no_canonical(T, s):
        den = sum(M[j] * T[j] for j in range(1, len(T)))
        return M[s] * T[s] / den if den > 0 else 0.0
    E = merge_expectation(doms, doms[0][1], False, mis=no_canonical)
    assert abs(E - doms[0][1].sum()) > 1e-3
