"""The benchmark workloads, as frame recipes for ``synth.frame``.

Each recipe is a dict: w, h, sky, gain, readnoise, nstars, ncr, seed, index.
The cleaning parameters of every workload are sigclip=4.5, sigfrac=0.5,
objlim=1.0, niter=4.
"""

from __future__ import annotations

import numpy as np

from . import CR_DENSITY, STAR_DENSITY, frame

CLEAN_PARAMS = dict(sigclip=4.5, sigfrac=0.5, objlim=1.0, niter=4)

BATCH_SIZES = [(800, 800), (1024, 1024), (2048, 4096), (4096, 4096)]  # (w, h)


def _recipe(w, h, *, sky, gain, readnoise, nstars, ncr, seed, index):
    return dict(w=w, h=h, sky=sky, gain=gain, readnoise=readnoise, nstars=nstars, ncr=ncr,
                seed=seed, index=index)


def single_800(seed: int = 0):
    """800x800, sky 100 e-, gain 7, read noise 5 e-, 200 stars, 1500 cosmic rays."""
    return _recipe(800, 800, sky=100.0, gain=7.0, readnoise=5.0, nstars=200, ncr=1500,
                   seed=seed, index=0)


def single_4096(seed: int = 0):
    """4096x4096, sky 300 e-, gain 7, read noise 5 e-, 5000 stars, 40000 cosmic rays."""
    return _recipe(4096, 4096, sky=300.0, gain=7.0, readnoise=5.0, nstars=5000, ncr=40000,
                   seed=seed, index=0)


def mosaic_16384(seed: int = 0):
    """16384x16384 (1 GiB), sky 300 e-, gain 7, read noise 5 e-, 2e5 stars, 6e5 cosmic rays."""
    return _recipe(16384, 16384, sky=300.0, gain=7.0, readnoise=5.0, nstars=200000, ncr=600000,
                   seed=seed, index=0)


def _scaled(w, h, gain, readnoise, seed, index):
    sky = 300.0 if w * h >= 4096 * 4096 else 100.0
    return _recipe(w, h, sky=sky, gain=gain, readnoise=readnoise,
                   nstars=int(round(STAR_DENSITY * w * h)), ncr=int(round(CR_DENSITY * w * h)),
                   seed=seed, index=index)


def batch_64(seed: int = 0, sizes=None, per_size: int = 16):
    """64 uneven frames: 16 each of 800^2, 1024^2, 2048x4096, 4096^2.

    Per-frame gain uniform in [1, 7] e-/DN and read noise uniform in [3, 10] e-.
    Star and cosmic-ray counts scale with area at the 800x800 densities; sky is
    100 e- below 4096^2 pixels and 300 e- from there on.
    """
    sizes = BATCH_SIZES if sizes is None else sizes
    rng = np.random.default_rng([seed, 3])
    out = []
    for (w, h) in sizes:
        for _ in range(per_size):
            gain = float(np.float32(rng.uniform(1.0, 7.0)))
            rn = float(np.float32(rng.uniform(3.0, 10.0)))
            out.append(_scaled(w, h, gain, rn, seed, len(out)))
    return out


def serving_stream(n_frames: int, rate_hz: float, seed: int = 0):
    """Poisson arrivals at ``rate_hz``; sizes uniform over the batch sizes.

    Returns (arrival_times_s, recipes).
    """
    rng = np.random.default_rng([seed, 5, int(rate_hz)])
    gaps = rng.exponential(1.0 / rate_hz, size=n_frames)
    t = np.cumsum(gaps) - gaps[0]
    recipes = []
    for i in range(n_frames):
        w, h = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        gain = float(np.float32(rng.uniform(1.0, 7.0)))
        rn = float(np.float32(rng.uniform(3.0, 10.0)))
        recipes.append(_scaled(w, h, gain, rn, seed, 1000 + i))
    return t, recipes


def make(recipe, truth: bool = False):
    """Generate the frame of a recipe (float32 DN, shape (h, w))."""
    r = recipe
    return frame(r["w"], r["h"], seed=r["seed"], index=r["index"], sky=r["sky"], gain=r["gain"],
                 readnoise=r["readnoise"], nstars=r["nstars"], ncr=r["ncr"], truth=truth)
