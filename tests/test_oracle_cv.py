"""Pins for the oracle's control-variate query (Section 'Control variates', equation
CVEstimator, in estimator-value form out_j = L_j - beta t_j C_{j+1} + beta C_j).

The control variate h = f * L~_i has known integral I_h = L~_{o\\e}.  Here the
integrand is a cos^32 lobe over the hemisphere, whose integral has the closed
form 2*pi/33; the table is filled through ordinary inserts so that the next
vertices' cells hold the lobe at Gauss-Legendre nodes and the vertex's own cell
holds 2*pi/33.  With the quadrature weights carried in the throughput t, the
mean of t * C_next equals I_h up to fixed-point rounding, so the mean of the CV
estimator must equal the mean of the plain estimator."""

import math

import numpy as np
import pytest

from helpers import stack, vertex

K = 17  # Gauss-Legendre nodes: exact for polynomials of degree <= 33 >= 32
SCALE = np.array([1.0, 0.5, 2.0])  # different per channel to catch channel mix-ups
I_H = 2.0 * math.pi / 33.0  # integral of cos^32 over the hemisphere


def _nodes():
    x, w = np.polynomial.legendre.leggauss(K)
    return (x + 1.0) / 2.0, w / 2.0  # on [0, 1]


def _next_pos(k):
    return ((k + 0.5) / 16.0, 0.25 / 16.0, 0.25 / 16.0)


SELF_POS = (0.5, 0.9, 0.9)


def _filled_oracle(oracle_mod, beta):
    mu, _ = _nodes()
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2, beta=beta)
    recs = [vertex(_next_pos(k), L=tuple(mu[k] ** 32 * SCALE)) for k in range(K)]
    recs.append(vertex(SELF_POS, L=tuple(I_H * SCALE)))
    o.insert(stack(recs))
    o.update()
    return o


def _paths(k_of_path, L0, t0):
    P = len(k_of_path)
    v = np.empty((2 * P, 16), dtype=np.float32)
    for p, k in enumerate(k_of_path):
        v[p] = vertex(SELF_POS, L=tuple(L0[p]), t=tuple(t0[p]))
        v[P + p] = vertex(_next_pos(k), L=(0.25, 0.5, 0.75), t=(0.3, 0.3, 0.3))
    return v


@pytest.mark.parametrize("beta", [1.0, 0.5])
def test_cv_mean_equals_plain_mean_quadrature(oracle_mod, beta):
    mu, wq = _nodes()
    assert abs(2.0 * math.pi * float(np.sum(wq * mu ** 32)) - I_H) < 1e-14  # the quadrature is exact
    o = _filled_oracle(oracle_mod, beta)
    rng = np.random.default_rng(5)
    ks = list(range(K))
    t0 = np.outer(2.0 * math.pi * wq * K, np.ones(3))
    L0 = rng.lognormal(0.0, 1.0, size=(K, 3))
    v = _paths(ks, L0, t0)
    out = o.query_cv(v, K, 2)
    plain = v[:K, 12:15].astype(np.float64)
    diff = out[:K].mean(axis=0) - plain.mean(axis=0)
    # fixed-point rounding of the stored lobe values (2^-25 each) and of float32 t bounds the gap
    assert np.all(np.abs(diff) < 1e-6), diff
    # the last vertex of every path carries no control variate
    assert np.array_equal(out[K:], v[K:, 12:15].astype(np.float64))
    # a sign or index error in either beta term would move the mean by O(beta * I_h)
    assert beta * I_H * SCALE.min() > 1e-2


def test_cv_mean_statistical_and_variance_reduction(oracle_mod):
    mu, wq = _nodes()
    o = _filled_oracle(oracle_mod, 1.0)
    rng = np.random.default_rng(9)
    N = 20000
    ks = rng.integers(0, K, size=N)
    # node k chosen uniformly (p = 1/K); the plain estimator integrates
    # g = lobe * (1 + 0.2 (u - 0.5)) * scale, which is correlated with h
    L0 = np.outer(2.0 * math.pi * wq[ks] * K * (mu[ks] ** 32) * (1.0 + 0.2 * (rng.random(N) - 0.5)),
                  SCALE)
    t0 = np.outer(2.0 * math.pi * wq[ks] * K, np.ones(3))
    v = _paths(ks, L0, t0)
    out = o.query_cv(v, N, 2)[:N]
    plain = v[:N, 12:15].astype(np.float64)
    sigma = np.std(out - plain, axis=0)
    diff = np.abs(out.mean(axis=0) - plain.mean(axis=0))
    assert np.all(diff <= 4.0 * sigma / math.sqrt(N) + 1e-6), (diff, sigma)
    # the control variate removes most of the variance of this correlated integrand
    assert np.all(np.var(out, axis=0) < 0.1 * np.var(plain, axis=0))


def test_cv_depth_limit_absent_cells_and_single_vertex_paths(oracle_mod):
    o = _filled_oracle(oracle_mod, 1.0)
    t0 = np.full((3, 3), 2.0)
    L0 = np.array([[1.0, 2.0, 3.0]] * 3)
    v = _paths([0, 1, 2], L0, t0)
    # next vertex of path 2 moved to an empty cell: C_next = 0
    v[3 + 2, 0:3] = (0.9, 0.1, 0.1)
    out = o.query_cv(v, 3, 2)
    key_self = oracle_mod.vertex_key(o.cfg, v[0])
    rec = o.export()
    C0 = rec[rec["key"] == key_self][0]["L"]
    np.testing.assert_allclose(out[2], L0[2] + C0, rtol=1e-15)
    # cv_max_depth = 0 switches the control variate off everywhere
    o0 = oracle_mod.Oracle(pos_bits=4, dir_bits=2, cv_max_depth=0)
    o0.import_records(rec)
    assert np.array_equal(o0.query_cv(v, 3, 2), v[:, 12:15].astype(np.float64))
    # paths of depth 1 have no successor
    assert np.array_equal(o.query_cv(v[:3], 3, 1), v[:3, 12:15].astype(np.float64))


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0])
def test_biased_estimator_mean_matches_closed_form(oracle_mod, gamma):
    """BiasedEstimator: mean(gamma (L - t C_next) + C) = gamma mean(L) + (1 - gamma) I_h,
    with I_h = 2 pi / 33 from the cos^32 quadrature."""
    _, wq = _nodes()
    o = _filled_oracle(oracle_mod, 1.0)
    rng = np.random.default_rng(6)
    t0 = np.outer(2.0 * math.pi * wq * K, np.ones(3))
    L0 = rng.lognormal(0.0, 1.0, size=(K, 3))
    v = _paths(list(range(K)), L0, t0)
    out = o.query_biased(v, K, 2, gamma, 0, 1)
    plain = v[:K, 12:15].astype(np.float64)
    want = gamma * plain.mean(axis=0) + (1.0 - gamma) * I_H * SCALE
    assert np.all(np.abs(out[:K].mean(axis=0) - want) < 1e-6)
    assert np.array_equal(out[K:], v[K:, 12:15].astype(np.float64))


def test_biased_estimator_gamma_zero_returns_the_approximant(oracle_mod):
    o = _filled_oracle(oracle_mod, 1.0)
    v = _paths([0, 3, 5], np.full((3, 3), 7.0), np.full((3, 3), 2.0))
    out = o.query_biased(v, 3, 2, 0.0, 0, 1)
    np.testing.assert_array_equal(out[:3], o.lookup(v)[:3])
    # outside [j_begin, j_end) the plain estimate passes through
    assert np.array_equal(o.query_biased(v, 3, 2, 0.0, 1, 2), v[:, 12:15].astype(np.float64))
    # gamma = 1 is the control-variate estimator with beta = 1
    np.testing.assert_allclose(o.query_biased(v, 3, 2, 1.0), o.query_cv(v, 3, 2), rtol=1e-15)


def test_biased_estimator_vertex_range_on_three_vertex_paths(oracle_mod):
    """Only vertices j_begin <= j < j_end (with a successor) get the estimator."""
    o = _filled_oracle(oracle_mod, 1.0)
    P, D = 4, 3
    v = np.empty((P * D, 16), dtype=np.float32)
    for p in range(P):
        v[p] = vertex(SELF_POS, L=(1.0, 2.0, 3.0), t=(0.5, 0.5, 0.5))
        v[P + p] = vertex(_next_pos(p), L=(4.0, 5.0, 6.0), t=(0.25, 0.25, 0.25))
        v[2 * P + p] = vertex(_next_pos(p + 5), L=(7.0, 8.0, 9.0), t=(0.1, 0.1, 0.1))
    C = o.lookup(v)
    L = v[:, 12:15].astype(np.float64)
    t = v[:, [7, 11, 15]].astype(np.float64)
    for jb, je in [(0, 1), (1, 2), (0, 2), (1, 1), (0, 3)]:
        out = o.query_biased(v, P, D, 0.25, jb, je)
        for j in range(D):
            rows = slice(j * P, (j + 1) * P)
            if jb <= j < je and j + 1 < D:
                want = 0.25 * (L[rows] - t[rows] * C[(j + 1) * P:(j + 2) * P]) + C[rows]
                np.testing.assert_allclose(out[rows], want, rtol=1e-15)
            else:
                assert np.array_equal(out[rows], L[rows]), (jb, je, j)
