"""The POISSON work function oracle (Sec. 6.3.2) against what mathematics fixes.

Pins: e^-mu against the C library's exp; Algorithm Q on hand-worked uniform
sequences (closed forms); the uniforms' distribution; the deviates' mean,
variance and histogram against the Poisson pmf on the paper's 750x750 test
image of 24.3 and at other means.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle

GAMMA = 0x9E3779B97F4A7C15
M64 = 2**64 - 1


def test_exp_neg_matches_libm():
    assert oracle.exp_neg(0.0) == 1.0
    for mu in np.concatenate([np.linspace(0, 700, 7001), [1e-12, 1e-6, 0.3465, 0.3466, 24.3, 699.999]]):
        a, b = oracle.exp_neg(float(mu)), math.exp(-float(mu))
        assert abs(a - b) <= 5e-14 * b, mu


def test_stream_value_arithmetic():
    """The C stream's 64-bit arithmetic against Python integers (a cross-check of the build, not a pin)."""
    def mix13(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    for s, j in [(0, 0), (0, 1), (1, 0), (M64, 5), (123456789, 2**40), (0xDEADBEEF, 3)]:
        assert oracle.stream_value(s, j) == mix13((s + (j + 1) * GAMMA) & M64)


def test_uniforms_are_uniform():
    from scipy import stats
    v = np.array([oracle.stream_value(7, j) >> 11 for j in range(200_000)], dtype=np.float64) * 2.0**-53
    assert v.min() >= 0.0 and v.max() < 1.0
    assert stats.kstest(v, "uniform").pvalue > 1e-6
    # successive pairs: no linear correlation
    assert abs(np.corrcoef(v[:-1], v[1:])[0, 1]) < 0.01


def test_algorithm_q_hand_cases():
    e1 = math.exp(-1.0)
    # mu = 1, e^-1 = 0.368: 0.5 >= it, 0.25 < it -> one factor
    assert oracle.algorithm_q(1.0, [0.5, 0.5]) == 1
    assert oracle.algorithm_q(1.0, [0.3]) == 0
    assert oracle.algorithm_q(1.0, [e1 + 1e-9, 0.999]) >= 1
    # constant uniforms u: the deviate is max{c : u^c >= e^-mu} = floor(mu / -ln u)
    for mu, u in [(2.0, 0.9), (5.0, 0.5), (24.3, 0.9), (0.7, 0.6)]:
        expect = math.floor(mu / -math.log(u))
        assert oracle.algorithm_q(mu, [u] * 400) == expect, (mu, u)
    # no mean, no draws
    for mu in (0.0, -3.0, float("nan")):
        assert oracle.algorithm_q(mu, []) == 0
    # needs more uniforms than given
    assert oracle.algorithm_q(5.0, [0.99] * 3) == -1


def _chi2_poisson(x, mu):
    from scipy import stats
    x = x.astype(np.int64).ravel()
    lo, hi = int(stats.poisson.ppf(1e-6, mu)), int(stats.poisson.ppf(1 - 1e-6, mu))
    edges = np.arange(lo, hi + 2)
    obs = np.array([(x < lo).sum()] + [np.sum(x == k) for k in edges[:-1]] + [(x > hi).sum()], dtype=float)
    p = np.concatenate([[stats.poisson.cdf(lo - 1, mu)], stats.poisson.pmf(edges[:-1], mu),
                        [stats.poisson.sf(hi, mu)]])
    exp = p * x.size
    # merge bins until every expected count is >= 5
    o2, e2, ao, ae = [], [], 0.0, 0.0
    for o, e in zip(obs, exp):
        ao, ae = ao + o, ae + e
        if ae >= 5:
            o2.append(ao), e2.append(ae)
            ao = ae = 0.0
    o2[-1] += ao
    e2[-1] += ae
    return stats.chisquare(o2, e2).pvalue


@pytest.mark.parametrize("mu,shape", [(24.3, (750, 750)), (0.7, (300, 300)), (300.0, (200, 200))])
def test_deviates_follow_the_poisson_law(mu, shape):
    """The paper's test image (750x750, every pixel 24.3) and two other means."""
    img = np.full(shape, mu, np.float32)
    out = oracle.poisson(img, seed=2010)
    assert np.array_equal(out, np.round(out)) and out.min() >= 0
    n = out.size
    m = float(np.float32(mu))
    assert abs(out.mean() - m) < 6 * math.sqrt(m / n)
    assert abs(out.var() - m) < 6 * m * math.sqrt(2.0 / n) + 6 * math.sqrt(m / n)
    assert _chi2_poisson(out, m) > 1e-4


def test_seeds_and_edge_values():
    img = np.full((64, 64), 24.3, np.float32)
    a, b, c = oracle.poisson(img, 1), oracle.poisson(img, 1), oracle.poisson(img, 2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    special = np.array([[0.0, -5.0, np.nan, 1e-30, 1e6, 700.0]], np.float32)
    out = oracle.poisson(special, 3)
    assert out[0, 0] == 0 and out[0, 1] == 0 and out[0, 2] == 0
    assert out[0, 3] == 0  # P(X > 0) = 1e-30
    assert abs(out[0, 4] - 700) < 150 and abs(out[0, 5] - 700) < 150  # mu above 700 is taken as 700
