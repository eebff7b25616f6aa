"""Pins of the POISSON work function oracle (Sec. 6.3.2), usable with any build of ``poisson.cpp``.

Each pin takes a ``PoissonLib`` and raises on a mismatch with what mathematics fixes: e^-mu against
the C library's exp; Algorithm Q on hand-worked uniform sequences (closed forms); the generator's
stream against published SplitMix64 outputs; the deviates' mean,
variance and histogram against the Poisson pmf on the paper's 750x750 test image of 24.3 and at other
means; the seed, edge-value and cap rules.
"""

from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np


class PoissonLib:
    """The oracle's POISSON functions bound to one compiled library."""

    def __init__(self, path):
        lib = ctypes.CDLL(path)
        lib.oracle_exp_neg.restype = ctypes.c_double
        lib.oracle_exp_neg.argtypes = [ctypes.c_double]
        lib.oracle_stream_value.restype = ctypes.c_uint64
        lib.oracle_stream_value.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_algorithm_q.restype = ctypes.c_int
        lib.oracle_algorithm_q.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_poisson.restype = ctypes.c_int
        lib.oracle_poisson.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_void_p]
        self.lib = lib

    def exp_neg(self, mu):
        return float(self.lib.oracle_exp_neg(float(mu)))

    def stream_value(self, s, j):
        return int(self.lib.oracle_stream_value(s & (2**64 - 1), j & (2**64 - 1)))

    def algorithm_q(self, mu, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        return int(self.lib.oracle_algorithm_q(float(mu), u.ctypes.data, int(u.size)))

    def poisson(self, img, seed):
        a = np.ascontiguousarray(img, dtype=np.float32)
        out = np.empty_like(a)
        h, w = a.shape
        if self.lib.oracle_poisson(a.ctypes.data, w, h, seed & (2**64 - 1), out.ctypes.data) != 0:
            raise ValueError("oracle_poisson rejected its arguments")
        return out


def pin_stream_published_outputs(P):
    """The counter-based stream is SplitMix64: value(s, j) is the (j+1)-th output of the sequential
    generator started at state s, which the published reference outputs fix (tests/golden/splitmix64.json)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.json")
    with open(path) as f:
        seqs = json.load(f)["sequences"]
    for seed, outs in seqs.items():
        for j, v in enumerate(outs):
            assert P.stream_value(int(seed), j) == int(v, 0), (seed, j)


def pin_exp_neg(P):
    assert P.exp_neg(0.0) == 1.0
    for mu in np.concatenate([np.linspace(0, 700, 7001), [1e-12, 1e-6, 0.3465, 0.3466, 24.3, 699.999]]):
        a, b = P.exp_neg(float(mu)), math.exp(-float(mu))
        assert abs(a - b) <= 5e-14 * b, mu


def pin_algorithm_q_hand_cases(P):
    # mu = 1, e^-1 = 0.368: 0.5 >= it, 0.25 < it -> one factor
    assert P.algorithm_q(1.0, [0.5, 0.5]) == 1
    assert P.algorithm_q(1.0, [0.3]) == 0
    # a product equal to e^-mu still counts (the comparison is >=)
    assert P.algorithm_q(1.0, [P.exp_neg(1.0), 0.1]) == 1
    # constant uniforms u: the deviate is max{c : u^c >= e^-mu} = floor(mu / -ln u)
    for mu, u in [(2.0, 0.9), (5.0, 0.5), (24.3, 0.9), (0.7, 0.6)]:
        assert P.algorithm_q(mu, [u] * 400) == math.floor(mu / -math.log(u)), (mu, u)
    # no mean, no draws
    for mu in (0.0, -3.0, float("nan")):
        assert P.algorithm_q(mu, []) == 0
    # needs more uniforms than given
    assert P.algorithm_q(5.0, [0.99] * 3) == -1


def _chi2_poisson(x, mu):
    from scipy import stats
    x = x.astype(np.int64).ravel()
    lo, hi = int(stats.poisson.ppf(1e-6, mu)), int(stats.poisson.ppf(1 - 1e-6, mu))
    edges = np.arange(lo, hi + 2)
    obs = np.array([(x < lo).sum()] + [np.sum(x == k) for k in edges[:-1]] + [(x > hi).sum()], dtype=float)
    p = np.concatenate([[stats.poisson.cdf(lo - 1, mu)], stats.poisson.pmf(edges[:-1], mu),
                        [stats.poisson.sf(hi, mu)]])
    exp = p * x.size
    o2, e2, ao, ae = [], [], 0.0, 0.0  # merge bins until every expected count is >= 5
    for o, e in zip(obs, exp):
        ao, ae = ao + o, ae + e
        if ae >= 5:
            o2.append(ao)
            e2.append(ae)
            ao = ae = 0.0
    o2[-1] += ao
    e2[-1] += ae
    return stats.chisquare(o2, e2).pvalue


def pin_poisson_law(P, mu=24.3, shape=(750, 750)):
    """The paper's test image (750x750, every pixel 24.3) by default."""
    out = P.poisson(np.full(shape, mu, np.float32), 2010)
    assert np.array_equal(out, np.round(out)) and out.min() >= 0
    n = out.size
    m = float(np.float32(mu))
    assert abs(out.mean() - m) < 6 * math.sqrt(m / n)
    assert abs(out.var() - m) < 6 * m * math.sqrt(2.0 / n) + 6 * math.sqrt(m / n)
    assert _chi2_poisson(out, m) > 1e-4


def pin_seeds_and_edges(P):
    img = np.full((64, 64), 24.3, np.float32)
    a, b, c = P.poisson(img, 1), P.poisson(img, 1), P.poisson(img, 2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    out = P.poisson(np.array([[0.0, -5.0, np.nan, 1e-30, 1e6, 700.0]], np.float32), 3)
    assert out[0, 0] == 0 and out[0, 1] == 0 and out[0, 2] == 0
    assert out[0, 3] == 0  # P(X > 0) = 1e-30
    assert abs(out[0, 4] - 700) < 150 and abs(out[0, 5] - 700) < 150  # mu above 700 is taken as 700


ALL_PINS = [pin_stream_published_outputs, pin_exp_neg, pin_algorithm_q_hand_cases, pin_poisson_law,
            pin_seeds_and_edges]
