"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError
when the oracle is wrong. ``test_oracle_pins.py`` runs them on the oracle;
``test_oracle_mutants.py`` runs them on copies with planted mistakes and
requires that every mistake fails at least one pin.

What pins what:
  * medians         -- rank counting on tiny frames (no sorting), with ties;
  * L+ (stage a)    -- the literal definition (2x block replication, 3x3
                       Laplacian, clip, 2x2 mean) built here; analytic planes
                       and quadratics;
  * replacement (e) -- brute-force sorted lists per flagged pixel;
  * whole iteration -- the closed form of a hot pixel on a flat sky, of a
                       hot pixel with a weaker neighbour, of a plateau, and of
                       stripes (the med3 -> med7 chain); strict thresholds at
                       binary-exact statistics;
                       physics checks (noise-only field, hot pixel, FWHM-2
                       star); invariants (monotone mask, untouched unflagged
                       pixels, transpose/flip equivariance, fixed point);
                       the dependency radius (mask <= 6 = the paper's BORDER,
                       image <= 8 per iteration) and crops with 8*niter context;
  * fragile map     -- the closed form of a hot pixel whose statistic sits at a
                       stated relative distance from each threshold (inside and
                       outside the 1e-4 tolerance; interior and corner cone).
"""

from __future__ import annotations

import json
import math
import os

import numpy as np

import synth
from oracle import Params

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        return json.load(f)


def _clamped_window(a, x, y, r):
    h, w = a.shape
    return [a[min(max(y + dy, 0), h - 1), min(max(x + dx, 0), w - 1)]
            for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def _sizes():
    out = [(1, 1), (1, 9), (9, 1), (2, 3), (3, 2), (5, 5), (7, 4), (4, 7), (9, 9), (8, 6)]
    return out


# ----------------------------------------------------------------------------- medians
def pin_median_rank(orc):
    """The median filter output v satisfies #(<v) <= n//2 < #(<=v) in every clamped window."""
    rng = np.random.default_rng(11)
    for (w, h) in _sizes():
        for kind in ("ties", "floats"):
            a = (rng.integers(0, 4, size=(h, w)).astype(np.float64) if kind == "ties"
                 else rng.normal(size=(h, w)))
            for r in (1, 2, 3):
                out = orc.median_filter(a, r)
                n = (2 * r + 1) ** 2
                for y in range(h):
                    for x in range(w):
                        win = np.array(_clamped_window(a, x, y, r))
                        v = out[y, x]
                        lt, le = int(np.sum(win < v)), int(np.sum(win <= v))
                        assert lt <= n // 2 < le, (w, h, r, x, y, kind)
                        assert v in win


# ----------------------------------------------------------------------------- L+
def _lplus_literal(J):
    """2x block replication, clamped 3x3 Laplacian [[0,-1,0],[-1,4,-1],[0,-1,0]], clip <0, 2x2 mean."""
    B = np.repeat(np.repeat(J, 2, axis=0), 2, axis=1)
    P = np.pad(B, 1, mode="edge")
    lap = 4 * P[1:-1, 1:-1] - P[:-2, 1:-1] - P[2:, 1:-1] - P[1:-1, :-2] - P[1:-1, 2:]
    lap = np.maximum(lap, 0)
    h, w = J.shape
    return lap.reshape(h, 2, w, 2).mean(axis=(1, 3))


def pin_lplus_literal(orc):
    rng = np.random.default_rng(5)
    for (w, h) in _sizes() + [(17, 13)]:
        Ji = rng.integers(-50, 50, size=(h, w)).astype(np.float64)  # integer-valued: exact in fp64
        assert np.array_equal(orc.lplus(Ji), _lplus_literal(Ji)), (w, h)
        Jf = rng.normal(10, 3, size=(h, w))
        np.testing.assert_allclose(orc.lplus(Jf), _lplus_literal(Jf), rtol=1e-12, atol=1e-12)


def pin_lplus_plane(orc):
    """Interior of a plane gx*x + gy*y: L+ = max(|gx|, |gy|) / 2."""
    yy, xx = np.mgrid[0:12, 0:15].astype(np.float64)
    for gx, gy in [(3.0, 1.0), (-2.0, 0.5), (0.25, -4.0), (1.5, 1.5), (0.0, 0.0), (-1.0, -3.0)]:
        out = orc.lplus(gx * xx + gy * yy)
        assert np.all(out[1:-1, 1:-1] == max(abs(gx), abs(gy)) / 2), (gx, gy)


def pin_lplus_quadratic(orc):
    """Interior of a*x^2 (a > 0): only the west difference a(2x-1) is positive, so
    L+ = a(2x-1)/2; a*y^2 likewise along y; for -a*x^2 only the east difference a(2x+1)
    is positive, so L+ = a(2x+1)/2."""
    yy, xx = np.mgrid[0:10, 0:11].astype(np.float64)
    for a in (1.0, 3.0, 0.5):
        assert np.array_equal(orc.lplus(a * xx ** 2)[1:-1, 1:-1], (a * (2 * xx - 1) / 2)[1:-1, 1:-1])
        assert np.array_equal(orc.lplus(a * yy ** 2)[1:-1, 1:-1], (a * (2 * yy - 1) / 2)[1:-1, 1:-1])
        assert np.array_equal(orc.lplus(-a * xx ** 2)[1:-1, 1:-1], (a * (2 * xx + 1) / 2)[1:-1, 1:-1])
    # integer-coefficient quadratics with cross terms against the literal definition (exact)
    for (a, b, c, d, e) in [(1, 2, -1, 3, -2), (-2, 1, 1, 0, 5), (0, 3, 0, -1, 1)]:
        Q = a * xx ** 2 + b * xx * yy + c * yy ** 2 + d * xx + e * yy
        assert np.array_equal(orc.lplus(Q), _lplus_literal(Q))


# ----------------------------------------------------------------------------- replacement
def _replace_brute(J, M):
    h, w = J.shape
    out = J.copy()
    none_left = 0
    for y in range(h):
        for x in range(w):
            if not M[y, x]:
                continue
            vals, allv = [], []
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    yy, xx = min(max(y + dy, 0), h - 1), min(max(x + dx, 0), w - 1)
                    allv.append(J[yy, xx])
                    if not M[yy, xx]:
                        vals.append(J[yy, xx])
            if vals:
                out[y, x] = sorted(vals)[(len(vals) + 1) // 2 - 1]
            else:
                m5 = sorted(allv)[12]
                out[y, x] = m5 if m5 > 0 else np.float32(1e-4)
                none_left += 1
    return out, none_left


def pin_replace_bruteforce(orc):
    rng = np.random.default_rng(7)
    for (w, h) in _sizes() + [(13, 7)]:
        for dens in (0.05, 0.3, 0.7, 1.0):
            J = rng.integers(1, 6, size=(h, w)).astype(np.float32) * np.float32(1.25)
            M = (rng.random((h, w)) < dens).astype(np.uint8)
            for prec in ("f64", "f32"):
                out, c = orc.replace(J, M, prec)
                exp, ce = _replace_brute(J, M)
                assert np.array_equal(out, exp), (w, h, dens, prec)
                assert c == ce


# ----------------------------------------------------------------------------- closed form
def pin_hot_pixel_closed_form(orc):
    """Flat sky b with one pixel b+A in the middle, no noise; every map in closed form.

    m5 = m3 = b everywhere (one outlier per window); N = sqrt(gain*max'(b) + rn^2)/gain with
    max'(b) = b if b > 0 else 1e-4 (the floor); L+ = 2A at p (all four differences are A)
    and 0 elsewhere; S = S' = A/N at p; F = 0 so R = S'/0.01; only p is flagged; I_1(p) = b.
    """
    P = Params(gain=7.0, readnoise=5.0, sigclip=4.5, sigfrac=0.5, objlim=1.0)
    A = 50.0
    for b in (20.0, 0.0, -10.0):
        J = np.full((15, 17), b, np.float32)
        py, px = 7, 8
        J[py, px] = b + A
        r = orc.iterate(J, None, P, maps=True)
        m5f = b if b > 0 else 1e-4
        N = math.sqrt(7.0 * m5f + 25.0) / 7.0
        m = r.maps
        assert np.all(m["m3"] == b) and np.all(m["m5"] == m5f)
        np.testing.assert_allclose(m["noise"], N, rtol=1e-15)
        lp = np.zeros_like(m["lplus"])
        lp[py, px] = 2 * A
        assert np.array_equal(m["lplus"], lp)
        s = np.zeros_like(lp)
        s[py, px] = A / N
        np.testing.assert_allclose(m["s"], s, rtol=1e-15, atol=0)
        np.testing.assert_allclose(m["sprime"], s, rtol=1e-15, atol=0)
        assert np.all(m["f"] == 0)
        rr = np.zeros_like(lp)
        rr[py, px] = (A / N) / 0.01
        np.testing.assert_allclose(m["r"], rr, rtol=1e-14, atol=0)
        only = np.zeros(J.shape, np.uint8)
        only[py, px] = 1
        for name in ("cand", "g1", "g2"):
            assert np.array_equal(m[name].astype(np.uint8), only), name
        assert np.array_equal(r.Mk, only) and r.n_new == 1
        rest = np.ones(J.shape, bool)
        rest[py, px] = False
        assert r.Ik[py, px] == np.float32(b) and np.array_equal(r.Ik[rest], J[rest])
    # below the limit, A/N <= sigclip, nothing is flagged
    b = 20.0
    N = math.sqrt(7.0 * b + 25.0) / 7.0
    J2 = np.full((15, 17), b, np.float32)
    J2[7, 8] = b + np.float32(4.4 * N)
    assert orc.iterate(J2, None, P).Mk.sum() == 0


def pin_grown_neighbour_closed_form(orc):
    """Hot pixel p = b+A with its east neighbour q = b+d (A > 2d), no noise.

    At q the differences are dN = dS = dE = d and dW = d - A < -d, so L+(q) = (2d + 2d)/4 = d
    and S'(q) = d/(2N) (med5(S) = 0, m5 = m3 = b). With d/(2N) = 3 (between sigfrac*sigclip =
    2.25 and sigclip = 4.5) q is not a candidate and fails the first growth, but the second
    growth from p flags it: M_1 = {p, q}. With d/(2N) = 2 nothing but p is flagged.
    """
    P = Params()
    b, A = 20.0, 400.0
    N = math.sqrt(7.0 * b + 25.0) / 7.0
    for sq, expect_q in ((3.0, 1), (2.0, 0)):
        d = np.float32(2 * N * sq)
        J = np.full((15, 17), b, np.float32)
        J[7, 8] = b + A
        J[7, 9] = b + d
        r = orc.iterate(J, None, P, maps=True)
        d = float(J[7, 9]) - b  # the stored (float32-rounded) excess
        np.testing.assert_allclose(r.maps["lplus"][7, 9], d, rtol=1e-14)
        np.testing.assert_allclose(r.maps["sprime"][7, 9], d / (2 * N), rtol=1e-14)
        assert r.maps["cand"][7, 9] == 0 and r.maps["g1"][7, 9] == 0
        exp = np.zeros(J.shape, np.uint8)
        exp[7, 8] = 1
        exp[7, 9] = expect_q
        assert np.array_equal(r.Mk, exp)


def pin_block_closed_form(orc):
    """A 3x5 plateau b+c (c = 40 N_b) on a flat sky, no noise; the two growth steps in closed form.

    m5 = b+c on the block's middle column (15 of 25 elevated) and b elsewhere, so N = N_b except
    N' = sqrt(gain(b+c) + rn^2)/gain there. m3 = b+c on the block minus its corners (>= 5 of 9
    elevated); med7(m3) = b everywhere (<= 11 of 49 elevated), so F = c on those pixels and 0 at
    the corners. L+ = c at the corners, c/2 on the other perimeter pixels, 0 inside and outside;
    med5(S) = 0 on the perimeter. Hence S' = c/(2N) = 20 at the corners (R = 2000: candidates),
    c/(4N) = 10 on the short sides and next to the corners (R = 1/4: first growth only), and
    c/(4N') ~ 4.9 at the middle of the long sides, which the second growth alone reaches.
    M_1 = the 12 perimeter pixels.
    """
    P = Params()
    b = 20.0
    N = math.sqrt(7.0 * b + 25.0) / 7.0
    c = np.float32(40.0 * N)
    J = np.full((17, 19), b, np.float32)
    y0, x0 = 7, 7
    J[y0:y0 + 3, x0:x0 + 5] = b + c
    cc = float(J[y0, x0]) - b
    N2 = math.sqrt(7.0 * (b + cc) + 25.0) / 7.0
    r = orc.iterate(J, None, P, maps=True)
    m = r.maps
    per = np.zeros(J.shape, bool)
    per[y0:y0 + 3, x0:x0 + 5] = True
    per[y0 + 1, x0 + 1:x0 + 4] = False
    corners = np.zeros(J.shape, bool)
    for (yy, xx) in [(y0, x0), (y0, x0 + 4), (y0 + 2, x0), (y0 + 2, x0 + 4)]:
        corners[yy, xx] = True
    mid = np.zeros(J.shape, bool)
    mid[y0, x0 + 2] = mid[y0 + 2, x0 + 2] = True
    side = per & ~corners & ~mid
    midcol = np.zeros(J.shape, bool)
    midcol[y0:y0 + 3, x0 + 2] = True
    np.testing.assert_allclose(m["noise"][~midcol], N, rtol=1e-15)
    np.testing.assert_allclose(m["noise"][midcol], N2, rtol=1e-15)
    np.testing.assert_allclose(m["lplus"][corners], cc, rtol=1e-15)
    np.testing.assert_allclose(m["lplus"][side | mid], cc / 2, rtol=1e-15)
    assert np.all(m["lplus"][~per] == 0)
    np.testing.assert_allclose(m["sprime"][corners], cc / (2 * N), rtol=1e-14)
    np.testing.assert_allclose(m["sprime"][side], cc / (4 * N), rtol=1e-14)
    np.testing.assert_allclose(m["sprime"][mid], cc / (4 * N2), rtol=1e-14)
    assert np.all(m["f"][corners] == 0)
    np.testing.assert_allclose(m["f"][side | mid], cc, rtol=1e-15)
    assert np.array_equal(m["cand"].astype(bool), corners)
    assert np.array_equal(m["g1"].astype(bool), corners | side)
    assert np.array_equal(r.Mk.astype(bool), per)


def pin_strict_thresholds(orc):
    """Every threshold comparison is strict: a statistic equal to its threshold does not pass.

    With gain 1, read noise 0 and a flat sky b = 16, N = sqrt(16)/1 = 4 exactly, so the closed
    forms above give exact binary values. A hot pixel b+A has S' = 2A/(2N) = A/4 and F = 0, so
    R = S'/0.01: A = 18 puts S' at 4.5 = sigclip, A = 20 puts R at 500 (S' = 5). A hot pixel
    p = b+400 with its east neighbour q = b+d has S'(q) = d/(2N) = d/8 (the dN, dS, dE terms of
    L+(q) are d, dW = d-400): d = 36 puts S'(q) at sigclip, d = 18 at sigfrac*sigclip = 2.25.
    Each case is run at the threshold (the statistic must fail) and at the next float32 below it
    (it must pass), in both precisions.
    """
    b = 16.0
    below = lambda v: float(np.nextafter(np.float32(v), np.float32(0)))  # noqa: E731
    p, q = (7, 8), (7, 9)
    only_p = np.zeros((15, 17), np.uint8)
    only_p[p] = 1
    p_and_q = only_p.copy()
    p_and_q[q] = 1
    for prec in ("f64", "f32"):
        def run(A, d, **kw):
            J = np.full((15, 17), b, np.float32)
            J[p] = b + A
            if d:
                J[q] = b + d
            return orc.iterate(J, None, Params(gain=1.0, readnoise=0.0, **kw), precision=prec, maps=True)
        # S' = sigclip at a lone hot pixel: no candidate
        r = run(18.0, 0.0)
        assert r.maps["sprime"][p] == 4.5 and r.Mk.sum() == 0 and r.maps["cand"].sum() == 0, prec
        assert np.array_equal(run(18.0, 0.0, sigclip=below(4.5)).Mk, only_p), prec
        # R = objlim at a lone hot pixel with S' = 5 > sigclip: no candidate
        r = run(20.0, 0.0, objlim=500.0)
        assert r.maps["r"][p] == 500.0 and r.Mk.sum() == 0, prec
        assert np.array_equal(run(20.0, 0.0, objlim=below(500.0)).Mk, only_p), prec
        # S'(q) = sigclip next to a candidate: q is outside the first growth
        r = run(400.0, 36.0)
        assert r.maps["sprime"][q] == 4.5 and r.maps["cand"][p] == 1, prec
        assert r.maps["g1"][q] == 0 and r.maps["g1"][p] == 1, prec
        assert run(400.0, 36.0, sigclip=below(4.5)).maps["g1"][q] == 1, prec
        # S'(q) = sigfrac*sigclip next to a grown pixel: q is outside M_1
        r = run(400.0, 18.0)
        assert r.maps["sprime"][q] == 2.25 and np.array_equal(r.Mk, only_p), prec
        assert np.array_equal(run(400.0, 18.0, sigfrac=below(0.5)).Mk, p_and_q), prec


def pin_fine_structure_stripes(orc):
    """Vertical stripes J = b + A [x even], no noise: med3 and the med3 -> med7 chain in closed form.

    A 3x3 window centred on an even column holds 3 raised values of 9, one centred on an odd
    column 6, so med3 inverts the stripes: m3 = b + A [x odd] (columns 1 .. w-2, whose windows
    reach no clamped column). A 7x7 window of m3 centred on an even column spans four odd columns
    (28 raised values of 49), one centred on an odd column three (21), so med7(m3) = b + A [x even]
    and F = m3 - med7(m3) = +A on odd and -A on even columns (columns 4 .. w-5). The 7x7 median of
    J itself would be b + A [x odd] there, giving F = 0. Rows are identical, so the vertical clamp
    changes nothing.
    """
    b, A = 20.0, 64.0
    w, h = 23, 12
    x = np.arange(w)
    J = np.tile(np.where(x % 2 == 0, b + A, b).astype(np.float32), (h, 1))
    for prec in ("f64", "f32"):
        m = orc.iterate(J, None, Params(), precision=prec, maps=True).maps
        m3 = np.where(x % 2 == 1, b + A, b)
        assert np.array_equal(m["m3"][:, 1:w - 1], np.tile(m3[1:w - 1], (h, 1))), prec
        f = np.where(x % 2 == 1, A, -A)
        assert np.array_equal(m["f"][:, 4:w - 4], np.tile(f[4:w - 4], (h, 1))), prec


# ----------------------------------------------------------------------------- physics
def pin_flat_field_empty(orc):
    """Flat fields. Noiseless: nothing flagged, output identical. Noise-only (Poisson sky 100 e-,
    read noise 5 e-, gain 7): at sigclip 4.5 every flag is a positive single-pixel excursion of
    more than 4 noise sigmas above the local 5x5 median and the flagged fraction stays below
    2e-4; at sigclip 8 an 800x800 noise field is empty."""
    P = Params()
    b = np.full((40, 50), 14.25, np.float32)
    r = orc.clean(b, P, 4)
    assert r.mask.sum() == 0 and np.array_equal(r.clean, b)
    img = synth.flat(256, 256, seed=0, sky=100.0, gain=7.0, readnoise=5.0)
    it = orc.iterate(img, None, P, maps=True)
    ys, xs = np.nonzero(it.Mk)
    assert it.Mk.mean() < 2e-4
    for y, x in zip(ys, xs):
        assert img[y, x] - it.maps["m5"][y, x] > 4.0 * it.maps["noise"][y, x]
    big = synth.flat(800, 800, seed=0, sky=100.0, gain=7.0, readnoise=5.0)
    assert orc.clean(big, Params(sigclip=8.0), 4).mask.sum() == 0


def pin_hot_pixel_noisy(orc):
    """A single high-amplitude hot pixel on a noisy flat field is flagged; any other flag is a
    grown neighbour (within 2 px, S' above sigfrac*sigclip); I_1(p) is the lower median of the
    unflagged pixels of its 5x5 window, and nothing is flagged without the hot pixel."""
    P = Params()
    img = synth.flat(64, 64, seed=4, sky=100.0, gain=7.0, readnoise=5.0)
    assert orc.iterate(img, None, P).Mk.sum() == 0
    py, px = 30, 37
    img[py, px] += np.float32(5000.0 / 7.0)
    r = orc.iterate(img, None, P, maps=True)
    assert r.Mk[py, px] == 1
    for (y, x) in np.argwhere(r.Mk):
        assert max(abs(y - py), abs(x - px)) <= 2 and r.maps["sprime"][y, x] > 0.5 * 4.5
    nb = [img[py + dy, px + dx] for dy in range(-2, 3) for dx in range(-2, 3)
          if not r.Mk[py + dy, px + dx]]
    assert r.Ik[py, px] == sorted(nb)[(len(nb) + 1) // 2 - 1]


def gaussian_star(n, flux, fwhm, sky, cx=None, cy=None):
    """Pixel-integrated circular Gaussian (erf differences) on a flat sky, in electrons."""
    cx = n / 2 if cx is None else cx
    cy = n / 2 if cy is None else cy
    s = fwhm / 2.3548200450309493
    k = 1 / (math.sqrt(2) * s)
    fx = np.array([0.5 * (math.erf((x + 1 - cx) * k) - math.erf((x - cx) * k)) for x in range(n)])
    fy = np.array([0.5 * (math.erf((y + 1 - cy) * k) - math.erf((y - cy) * k)) for y in range(n)])
    return sky + flux * np.outer(fy, fx)


def star_margin(orc, form):
    """Largest objlim statistic R over pixels with S' > sigclip for a bright FWHM-2 star."""
    e = gaussian_star(31, 1e6, 2.0, 100.0)
    img = (e / 7.0).astype(np.float32)
    r = orc.iterate(img, None, Params(objlim_form=form), maps=True)
    sel = r.maps["sprime"] > 4.5
    return (float(r.maps["r"][sel].max()) if sel.any() else 0.0), r


def pin_star_not_flagged(orc):
    """A bright (1e6 e-) FWHM-2 px star is not flagged with the script-form statistic, with and
    without noise; the article form L+/F would flag its core (the reason for the script form)."""
    rmax, r = star_margin(orc, 0)
    assert r.Mk.sum() == 0 and rmax < 1.0
    rmax_a, ra = star_margin(orc, 1)
    assert ra.Mk.sum() > 0 and rmax_a > 1.0
    rng = np.random.default_rng(9)
    e = gaussian_star(31, 1e6, 2.0, 100.0, cx=15.3, cy=15.7)
    img = ((rng.poisson(e) + rng.normal(0, 5, e.shape)) / 7.0).astype(np.float32)
    assert orc.clean(img, Params(), 4).mask.sum() == 0


# ----------------------------------------------------------------------------- invariants
def _scene(w=96, h=80, seed=2):
    return synth.frame(w, h, seed=seed, sky=100.0, nstars=6, ncr=40)


def pin_invariants(orc):
    img = _scene()
    P = Params()
    J, M = img, np.zeros(img.shape, np.uint8)
    for _ in range(4):
        r = orc.iterate(J, M, P)
        assert np.all(r.Mk >= M)                                  # monotone flags
        assert np.array_equal(r.Ik[r.Mk == 0], img[r.Mk == 0])     # unflagged pixels keep I0
        assert r.n_new == int(r.Mk.sum()) - int(M.sum())          # the count of new flags
        J, M = r.Ik, r.Mk
    full = orc.clean(img, P, 4, fragile=True)
    assert np.array_equal(full.mask, M) and np.array_equal(full.clean, J)
    for f, finv in [(lambda a: a.T, lambda a: a.T), (lambda a: a[:, ::-1], lambda a: a[:, ::-1]),
                    (lambda a: a[::-1, :], lambda a: a[::-1, :])]:
        t = orc.clean(np.ascontiguousarray(f(img)), P, 4)
        tm, tc = finv(t.mask), finv(t.clean)
        ok = full.fragile == 0
        assert np.array_equal(tm[ok], full.mask[ok])
        agree = (tm == full.mask)
        assert np.array_equal(tc[agree], full.clean[agree])


def pin_fixed_point(orc):
    """Once an iteration adds no flag and no pixel lost all unflagged neighbours, the state is fixed."""
    img = _scene(seed=7)
    P = Params()
    J, M = img, None
    for _ in range(12):
        r = orc.iterate(J, M, P)
        J, M = r.Ik, r.Mk
        if r.n_new == 0 and r.n_none_left == 0:
            break
    assert r.n_new == 0 and r.n_none_left == 0
    again = orc.iterate(J, M, P)
    assert np.array_equal(again.Ik, J) and np.array_equal(again.Mk, M)


def pin_dependency_radius(orc):
    """Changing one input pixel changes M_1 only within Chebyshev distance 6 (the paper's
    BORDER) and I_1 only within distance 8."""
    border = paper_constants()["BORDER"]["value"]
    img = _scene(64, 64, seed=8)
    P = Params()
    base = orc.iterate(img, None, P)
    rng = np.random.default_rng(3)
    for _ in range(60):
        q = (int(rng.integers(0, 64)), int(rng.integers(0, 64)))
        J = img.copy()
        J[q] = np.float32(J[q] + rng.choice([-1, 1]) * rng.uniform(5, 800))
        r = orc.iterate(J, None, P)
        for a, b, lim in ((r.Mk, base.Mk, border), (r.Ik, base.Ik, border + 2)):
            d = np.argwhere(a != b)
            if len(d):
                assert np.max(np.maximum(abs(d[:, 0] - q[0]), abs(d[:, 1] - q[1]))) <= lim


def pin_crop_context(orc):
    """A crop processed with 8*niter pixels of context equals the full frame on the crop."""
    img = _scene(128, 112, seed=10)
    P = Params()
    niter = 2
    full = orc.clean(img, P, niter)
    ctx = 8 * niter
    for (y0, x0, hh, ww) in [(0, 0, 40, 50), (30, 40, 40, 30), (70, 90, 42, 38), (50, 0, 20, 128)]:
        ya, xa = max(0, y0 - ctx), max(0, x0 - ctx)
        yb, xb = min(img.shape[0], y0 + hh + ctx), min(img.shape[1], x0 + ww + ctx)
        c = orc.clean(np.ascontiguousarray(img[ya:yb, xa:xb]), P, niter)
        sl = (slice(y0 - ya, y0 - ya + hh), slice(x0 - xa, x0 - xa + ww))
        assert np.array_equal(c.mask[sl], full.mask[y0:y0 + hh, x0:x0 + ww])
        assert np.array_equal(c.clean[sl], full.clean[y0:y0 + hh, x0:x0 + ww])


# ----------------------------------------------------------------------------- fragile map
def _cone(shape, py, px):
    """The clamped 5x5 box around (py, px): the pixels whose growth can reach from p."""
    h, w = shape
    c = np.zeros(shape, np.uint8)
    c[max(py - 2, 0):min(py + 3, h), max(px - 2, 0):min(px + 3, w)] = 1
    return c


def pin_fragile_closed_form(orc):
    """The fragile map of a hot pixel on a flat sky, no noise, in closed form.

    From the closed form of pin_hot_pixel_closed_form, S'(p) = kA/N and R(p) = S'(p)/0.01 at the
    hot pixel p, and S' = 0 everywhere else; k = 1 in the interior, where all four differences
    are A, and k = 1/2 at a frame corner, where the two clamped differences vanish (L+ = A;
    med5(S) stays 0, p filling 9 of the 25 clamped window places). Choosing A puts one statistic
    at a stated relative
    distance d from its threshold: S' = sigclip (1 + d), S' = sigfrac sigclip (1 + d), or, with
    S' = 9 > sigclip, R = objlim (1 + d) by setting objlim = 900 (1 + d). A statistic within 1e-4
    (relative) of its threshold marks the clamped 5x5 box around it, so the fragile map is
    exactly that box for |d| = 5e-5 (either side) and empty for |d| = 1.5e-4. The corner position
    of p checks the clamp of the box. R near objlim marks nothing where S' is clearly below sigclip
    (S' = 3 or 1), since no candidate can form there.
    """
    b = 20.0
    N = math.sqrt(7.0 * b + 25.0) / 7.0
    shape = (15, 17)
    for (py, px), kappa in (((7, 8), 1.0), ((0, 0), 0.5)):
        for d, inside in ((5e-5, True), (-5e-5, True), (1.5e-4, False), (-1.5e-4, False)):
            cases = (("sigclip", Params(), 4.5 * (1 + d)),
                     ("sigfrac", Params(), 0.5 * 4.5 * (1 + d)),
                     ("objlim", Params(objlim=900.0 * (1 + d)), 9.0))
            for name, P, s_target in cases:
                J = np.full(shape, b, np.float32)
                J[py, px] = np.float32(b + s_target * N / kappa)
                r = orc.iterate(J, None, P, maps=True, fragile=True)
                got_sp = r.maps["sprime"][py, px]
                assert abs(got_sp / s_target - 1) < 1e-6, (name, got_sp, s_target)
                exp = _cone(shape, py, px) if inside else np.zeros(shape, np.uint8)
                assert np.array_equal(r.fragile, exp), (name, d, (py, px), int(r.fragile.sum()))
    # R within the tolerance of objlim where S' is clearly below sigclip (between the two growth
    # thresholds, or below both) decides nothing: no pixel is fragile
    for s_target in (3.0, 1.0):
        J = np.full(shape, b, np.float32)
        J[7, 8] = np.float32(b + s_target * N)
        r = orc.iterate(J, None, Params(objlim=100.0 * s_target * (1 + 5e-5)), maps=True, fragile=True)
        assert abs(r.maps["r"][7, 8] / (100.0 * s_target) - 1) < 1e-6
        assert r.fragile.sum() == 0 and r.Mk.sum() == 0, s_target
    # the end-to-end fragile map is the union over the iterations
    J = np.full(shape, b, np.float32)
    J[7, 8] = np.float32(b + 4.5 * (1 + 5e-5) * N)
    assert np.array_equal(orc.clean(J, Params(), 2, fragile=True).fragile, _cone(shape, 7, 8))


def pin_precisions_agree(orc):
    """The FP32 run of the same steps agrees with FP64 except on fragile pixels."""
    img = _scene(seed=12)
    P = Params()
    a = orc.clean(img, P, 4, fragile=True)
    b = orc.clean(img, P, 4, precision="f32")
    ok = a.fragile == 0
    assert np.array_equal(a.mask[ok], b.mask[ok])
    agree = a.mask == b.mask
    np.testing.assert_allclose(a.clean[agree], b.clean[agree], rtol=1e-5)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
