"""The order-statistic and rounding facts behind the CUDA path's exact pruning, checked on CPU.

The CUDA path skips work only where a bound proves that the skipped value cannot decide a flag
(the end-to-end GPU tests then find the results bit-identical to the oracle). The bounds rest on:
  * a 5x5 median is at least the smallest of its five column medians: at most two values of a
    column lie below that column's median, so at most 10 of the 25 lie below the smallest one;
  * a 7x7 median lies between the smallest and the largest of its seven column medians (at most
    21 of the 49 values on either side), which brackets med7 in the candidate test;
  * the median of five values, four of them shared with the neighbouring window, is the fifth
    value clamped between the middle two of the four (the sliding column median);
  * the screen S+ > t, evaluated in float32 as L+^2 > k (gain max(m, 0) + rn^2) with
    k = 4 t^2 (1 - 1e-4) / gain^2, never rejects a pixel whose float32 S = L+ / (2N) exceeds t,
    for any m at most the 5x5 median (N from the floored median, the oracle's order of operations).
These are facts of order statistics and of IEEE float32 arithmetic; the checks draw random windows
(with ties) and random pixels at the threshold, and run the four-plus-one identity exhaustively.
"""

import itertools

import numpy as np

F = np.float32


def _col_medians(win):
    return np.sort(win, axis=0)[win.shape[0] // 2]


def test_column_medians_bound_the_window_median():
    rng = np.random.default_rng(1)
    for trial in range(4000):
        for n in (5, 7):
            win = (rng.integers(0, 4, size=(n, n)).astype(np.float32) if trial % 2
                   else rng.normal(size=(n, n)).astype(np.float32))
            med = np.sort(win, axis=None)[n * n // 2]
            cm = _col_medians(win)
            assert cm.min() <= med <= cm.max(), (n, win)


def test_sliding_column_median_identity():
    """median(a, b, c, d, e) = min(max(a, c1), c2) with c1 <= c2 the middle two of (b, c, d, e),
    taken as max(min(b, c), min(d, e)) and min(max(b, c), max(d, e)); exhaustive on 0..4."""
    for a, b, c, d, e in itertools.product(range(5), repeat=5):
        u = max(min(b, c), min(d, e))
        v = min(max(b, c), max(d, e))
        c1, c2 = min(u, v), max(u, v)
        assert min(max(a, c1), c2) == sorted((a, b, c, d, e))[2]


def _fma32(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def test_screen_never_rejects_a_pixel_above_the_threshold():
    rng = np.random.default_rng(2)
    n = 200_000
    gain = rng.uniform(1.0, 7.0, n).astype(F)
    rn = np.where(rng.random(n) < 0.1, 0.0, rng.uniform(0.0, 10.0, n)).astype(F)
    m5 = np.where(rng.random(n) < 0.1, rng.uniform(-50.0, 0.0, n), rng.uniform(0.0, 5000.0, n)).astype(F)
    t = np.choose(rng.integers(0, 3, n), [np.full(n, 4.5), np.full(n, 2.25), rng.uniform(0.3, 12.0, n)]).astype(F)
    rejected_above = 0
    for i in range(n):
        g, r, m, th = gain[i], rn[i], m5[i], t[i]
        rn2 = F(r * r)
        mf = m if m > 0 else F(1e-4)                  # the floored median of the noise model
        N = F(F(np.sqrt(F(F(g * mf) + rn2))) / g)       # sqrt(gain m5 + rn^2) / gain
        lp = F(th * F(2) * N * F(1 + rng.uniform(-3e-6, 3e-6)))  # L+ with S at t within a few ulp
        S = F(lp / F(F(2) * N))
        g2 = F(g * g)
        k = F(F(F(F(F(4) * th) * th) * F(0.9999)) / g2)
        den = _fma32(g, max(m, F(0)), rn2)              # m = m5 itself: the largest lower bound
        hot = F(lp * lp) > F(k * den)
        if S > th and not hot:
            rejected_above += 1
    assert rejected_above == 0


def test_objlim_statistic_is_monotone_in_med7():
    """R = S' / max((m3 - med7) / N, 0.01) in float32 (the oracle's order) does not decrease as med7
    grows, for S' > 0 and N > 0: every step is a monotone IEEE operation. So the values of R at the
    smallest and the largest column median of the 7x7 window bracket R at the true med7."""
    rng = np.random.default_rng(3)
    n = 200_000
    m3 = rng.uniform(-100, 5000, n).astype(F)
    N = rng.uniform(0.5, 40, n).astype(F)
    sp = rng.uniform(1e-3, 500, n).astype(F)
    a = (m3 + rng.normal(0, 30, n)).astype(F)
    b = (a + np.abs(rng.normal(0, 30, n)) * (rng.random(n) < 0.9)).astype(F)  # b >= a, some equal

    def R(med7):
        f = (m3 - med7).astype(F)
        fn = np.maximum((f / N).astype(F), F(0.01))
        return (sp / fn).astype(F)

    assert np.all(b >= a)
    assert np.all(R(a) <= R(b))
