"""The synthetic frame generator follows its stated recipe.

Every input of the tests and the benchmark comes from ``synth`` (the paper's
WFPC2 frame is not available), so its generative model is checked here
against the recipe: electrons = Poisson(sky + stars) + cosmic-ray deposits +
Normal(0, read noise), divided by the gain; stars are pixel-integrated
Gaussians of FWHM uniform in [1.5, 2.5] px and total flux log-uniform in
[1e3, 1e6] e-; cosmic rays deposit an amplitude log-uniform in [1e2, 1e4] e-
once on every pixel of a track, 20 % of them a single pixel, the rest straight
tracks of length uniform in [1, 10] px. Each check is statistical with a fixed
seed and a wide margin.
"""

import numpy as np
import pytest

import synth

stats = pytest.importorskip("scipy.stats")


def test_same_seed_same_bytes_other_index_other_frame():
    a = synth.frame(300, 200, seed=4, index=2)
    assert np.array_equal(a, synth.frame(300, 200, seed=4, index=2))
    assert not np.array_equal(a, synth.frame(300, 200, seed=4, index=3))
    assert not np.array_equal(a, synth.frame(300, 200, seed=5, index=2))


@pytest.mark.parametrize("sky", [3.0, 100.0, 300.0])  # both Poisson samplers (inversion below 10)
def test_sky_is_poisson_in_electrons(sky):
    """With no read noise, gain * DN is an integer count whose histogram is Poisson(sky)."""
    gain = 7.0
    img = synth.flat(512, 512, seed=1, sky=sky, gain=gain, readnoise=0.0)
    e = img.astype(np.float64) * gain
    k = np.rint(e)
    assert np.max(np.abs(e - k)) < 1e-3 * max(1.0, k.max())  # DN = counts / gain, stored in float32
    n = k.size
    assert abs(k.mean() - sky) < 5 * np.sqrt(sky / n)
    assert abs(k.var() / sky - 1) < 0.03
    lo, hi = int(max(0, sky - 4 * np.sqrt(sky))), int(sky + 4 * np.sqrt(sky)) + 1
    kk = np.arange(lo, hi)  # each count in [lo, hi) on its own, both tails pooled
    ki = k.astype(np.int64)
    obs = np.array([np.sum(ki < lo)] + [np.sum(ki == v) for v in kk] + [np.sum(ki >= hi)])
    exp = np.array([stats.poisson.cdf(lo - 1, sky)] + list(stats.poisson.pmf(kk, sky)) +
                   [stats.poisson.sf(hi - 1, sky)]) * n
    assert obs.sum() == n
    keep = exp > 20
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


def test_read_noise_adds_its_variance():
    gain, sky, rn = 2.5, 100.0, 8.0
    e = synth.flat(512, 512, seed=2, sky=sky, gain=gain, readnoise=rn).astype(np.float64) * gain
    assert abs(e.mean() - sky) < 5 * np.sqrt((sky + rn * rn) / e.size)
    assert abs(e.var() / (sky + rn * rn) - 1) < 0.03


def _cosmic_only(n, ncr, seed, index=0):
    img, truth = synth.frame(n, n, seed=seed, index=index, sky=0.0, gain=1.0, readnoise=0.0, nstars=0,
                             ncr=ncr, truth=True)
    return img.astype(np.float64), truth


def test_cosmic_ray_amplitudes_and_shapes():
    """On an empty, noiseless frame only the deposits remain: the truth mask is exactly the non-zero
    pixels, every deposit is at least 100 e-, and the pixels of one track share its amplitude, whose
    log10 is uniform on [2, 4]. A fifth of the tracks (and a few short ones) are one pixel; no track
    spans more than 11 pixels along an axis."""
    vals, exts, singles = [], [], 0
    for index in range(4):
        e, truth = _cosmic_only(1024, 300, seed=7, index=index)
        assert np.array_equal(truth.astype(bool), e > 0)
        v = e[e > 0]
        assert v.min() >= 100.0 * (1 - 1e-6)
        # tracks seldom touch at this density: group pixels by their (shared) amplitude
        uniq, inv, cnt = np.unique(v, return_inverse=True, return_counts=True)
        ys, xs = np.nonzero(e > 0)
        for j, u in enumerate(uniq):
            if u > 1e4 * (1 + 1e-6):  # two tracks crossed: a sum, not an amplitude
                continue
            sel = inv == j
            exts.append(max(np.ptp(xs[sel]), np.ptp(ys[sel])) + 1)
            singles += cnt[j] == 1
            vals.append(u)
    vals = np.array(vals)
    assert len(vals) > 0.97 * 4 * 300
    p = stats.kstest(np.log10(vals), "uniform", args=(2.0, 2.0)).pvalue
    assert p > 1e-4, p
    frac = singles / len(vals)
    assert 0.2 <= frac <= 0.32, frac  # 20 % single hits plus short tracks within one pixel
    assert max(exts) <= 11


def test_star_fluxes_and_widths():
    """One star per noiseless frame with no sky: its electrons sum to a Poisson draw of its flux,
    whose log10 is uniform on [3, 6], and its second moment is that of a Gaussian of FWHM in
    [1.5, 2.5] px integrated over pixels (sigma^2 + 1/12 per axis)."""
    fluxes, var_ok = [], 0
    n = 64
    for index in range(300):
        img = synth.frame(n, n, seed=11, index=index, sky=0.0, gain=1.0, readnoise=0.0, nstars=1, ncr=0)
        e = img.astype(np.float64)
        tot = e.sum()
        if tot == 0:
            continue
        yy, xx = np.mgrid[0:n, 0:n]
        cx, cy = (e * xx).sum() / tot, (e * yy).sum() / tot
        if not (8 < cx < n - 8 and 8 < cy < n - 8):
            continue  # the star's wings are cut by the frame edge
        fluxes.append(tot)
        if tot > 2e4:  # enough electrons for a tight second moment
            vx = (e * (xx - cx) ** 2).sum() / tot
            vy = (e * (yy - cy) ** 2).sum() / tot
            lo = (1.5 / 2.35482) ** 2 + 1 / 12
            hi = (2.5 / 2.35482) ** 2 + 1 / 12
            var_ok += int(0.9 * lo < vx < 1.1 * hi and 0.9 * lo < vy < 1.1 * hi)
            assert 0.8 * lo < vx < 1.2 * hi and 0.8 * lo < vy < 1.2 * hi, (index, vx, vy)
    fluxes = np.array(fluxes)
    assert len(fluxes) > 150
    assert fluxes.min() > 1e3 * 0.85 and fluxes.max() < 1e6 * 1.01
    p = stats.kstest(np.log10(fluxes), "uniform", args=(3.0, 3.0)).pvalue
    assert p > 1e-4, p
    assert var_ok > 0


def test_workload_recipes():
    """The five workloads: sizes, counts and the per-frame gain and read-noise ranges of the batch."""
    from synth import workloads as wl
    b = wl.batch_64()
    assert len(b) == 64
    sizes = [(r["w"], r["h"]) for r in b]
    for s in wl.BATCH_SIZES:
        assert sizes.count(s) == 16
    assert sum(r["w"] * r["h"] for r in b) == 429_670_400
    for r in b:
        assert 1.0 <= r["gain"] <= 7.0 and 3.0 <= r["readnoise"] <= 10.0
        assert r["sky"] == (300.0 if r["w"] * r["h"] >= 4096 * 4096 else 100.0)
        assert r["nstars"] == round(200 / 640000 * r["w"] * r["h"])
        assert r["ncr"] == round(1500 / 640000 * r["w"] * r["h"])
    s = wl.single_800()
    assert (s["w"], s["h"], s["nstars"], s["ncr"], s["sky"], s["gain"], s["readnoise"]) == \
        (800, 800, 200, 1500, 100.0, 7.0, 5.0)
    s = wl.single_4096()
    assert (s["w"], s["nstars"], s["ncr"], s["sky"]) == (4096, 5000, 40000, 300.0)
    s = wl.mosaic_16384()
    assert (s["w"], s["h"], s["nstars"], s["ncr"]) == (16384, 16384, 200000, 600000)
    t, rec = wl.serving_stream(4000, 500.0)
    gaps = np.diff(t)
    assert abs(gaps.mean() * 500.0 - 1) < 0.06 and abs(gaps.std() / gaps.mean() - 1) < 0.08  # exponential
    counts = [sum((r["w"], r["h"]) == s for r in rec) for s in wl.BATCH_SIZES]
    assert min(counts) > 900 and max(counts) < 1100  # sizes uniform over the four


def test_frames_do_not_depend_on_the_thread_count():
    """Each row of the noise pass draws from its own stream, so a frame is the same bytes whatever the
    number of OpenMP threads (the GPU tests and the oracle's may run on hosts with different cores)."""
    import hashlib
    import os
    import subprocess
    import sys
    code = ("import hashlib, synth; "
            "print(hashlib.sha256(synth.frame(517, 333, seed=9, index=4).tobytes()).hexdigest())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    digests = set()
    for threads in ("1", "3", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                             check=True)
        digests.add(out.stdout.strip())
    digests.add(hashlib.sha256(synth.frame(517, 333, seed=9, index=4).tobytes()).hexdigest())
    assert len(digests) == 1
