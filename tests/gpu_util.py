"""Shared helpers of the GPU tests: device transfer, GPU runs and the parity checks.

Tolerances (GPU float32 against the FP64 oracle):

* Intermediate maps agree within 1e-5 relative, with an absolute floor of 1e-5
  times the magnitude of the operands that produced the value *at that pixel*
  (``map_floors``). A value that cancels (L+ from differences of the pixel
  values, S' = S - med5(S), F = m3 - med7(m3)) can be far smaller than its
  operands, and its float32 rounding is a fraction of the operands, not of the
  result. The floors carry the operands' scale through the formulas: L+ from
  the pixel and its four neighbours; S = L+/(2N); S' from S and med5(S), whose
  error is that of some S in the 5x5 window; F from m3 and med7(m3); R = S'/Fn
  from the errors of S' and of Fn = max(F/N, 0.01).
* Masks are identical except on the oracle's fragile pixels (a decision
  statistic within 1e-4 relative of its threshold, in the growth cone).
* Cleaned pixels agree within 1e-5 relative wherever the masks agree over the
  pixel's 5x5 window: a replaced value is the median of its window's unflagged
  pixels, so a flag that differs anywhere in the window changes which values
  are taken.

Against the FP32 oracle (the same steps in the kernel's precision) everything
is bit-identical.
"""

from __future__ import annotations

import numpy as np
import torch

import oracle
from oracle import Params

RTOL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def gpu_clean(cl, img):
    out, mask = cl.clean(dev(img))
    cl.sync()
    return host(out), host(mask)


def _clamped_shift(a, dy, dx):
    """a[clamp(y + dy), clamp(x + dx)] for every (y, x)."""
    h, w = a.shape
    ys = np.clip(np.arange(h) + dy, 0, h - 1)
    xs = np.clip(np.arange(w) + dx, 0, w - 1)
    return a[np.ix_(ys, xs)]


def _window_max(a, r):
    """Largest value of the clamped (2r+1)^2 window around every pixel."""
    out = np.full(a.shape, -np.inf)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            out = np.maximum(out, _clamped_shift(a, dy, dx))
    return out


def map_floors(J, ref_maps):
    """Absolute tolerance floor of every map at every pixel: RTOL times the magnitude of the values
    the map's formula combines there (module docstring). J is the iteration's input frame, ref_maps
    the FP64 oracle's maps of that iteration."""
    J = np.abs(np.asarray(J, dtype=np.float64))
    m = {k: np.asarray(v, dtype=np.float64) for k, v in ref_maps.items()}
    jmag = J.copy()
    for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        jmag = np.maximum(jmag, _clamped_shift(J, dy, dx))
    lp_floor = RTOL * 4.0 * jmag                                    # four differences per term
    s_floor = lp_floor / (2.0 * m["noise"]) + RTOL * np.abs(m["s"])
    smed = m["s"] - m["sprime"]
    sp_floor = RTOL * (np.abs(m["s"]) + np.abs(smed)) + s_floor + _window_max(s_floor, 2)
    m37 = m["m3"] - m["f"]
    f_floor = RTOL * (np.abs(m["m3"]) + np.abs(m37))
    fn = np.maximum(m["f"] / m["noise"], 0.01)
    r_floor = (sp_floor + np.abs(m["r"]) * f_floor / m["noise"]) / fn
    zero = np.zeros_like(J)
    return {"m5": zero, "lplus": lp_floor, "noise": zero, "s": s_floor, "sprime": sp_floor, "m3": zero,
            "f": f_floor, "r": r_floor}


def assert_map_close(got, ref, name, floor=0.0):
    """got within RTOL relative of ref, or within `floor` (per pixel, map_floors) absolute."""
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    bad = ~np.isclose(got, ref, rtol=RTOL, atol=0.0, equal_nan=True)
    bad &= ~(np.abs(got - ref) <= floor)
    assert not bad.any(), f"map {name}: {int(bad.sum())} values differ, first {np.argwhere(bad)[:5]}"


def dilate(mask, r):
    """Clamped (2r+1)^2 dilation of a 0/1 map."""
    a = np.asarray(mask, dtype=bool)
    out = np.zeros_like(a)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            out |= _clamped_shift(a, dy, dx)
    return out


def compare_f64(clean, mask, ref_clean, ref_mask, fragile, what=""):
    """The FP64 contract: mask flips only on fragile pixels, cleaned values within RTOL wherever the
    masks agree over the 5x5 window. Returns (flips, fragile pixels)."""
    flips = mask != ref_mask
    ok = fragile == 0
    off = flips & ok
    assert not off.any(), f"{what}: {int(off.sum())} mask flips off fragile pixels, first {np.argwhere(off)[:5]}"
    agree = ~dilate(flips, 2)
    np.testing.assert_allclose(clean[agree], ref_clean[agree], rtol=RTOL, atol=0, err_msg=what)
    return int(flips.sum()), int((~ok).sum())


def assert_clean_matches_f64(clean, mask, ref: "oracle.CleanResult", what=""):
    return compare_f64(clean, mask, ref.clean, ref.mask, ref.fragile, what)


def params_of(cl_kwargs):
    return Params(gain=cl_kwargs.get("gain", 7.0), readnoise=cl_kwargs.get("readnoise", 5.0),
                  sigclip=cl_kwargs.get("sigclip", 4.5), sigfrac=cl_kwargs.get("sigfrac", 0.5),
                  objlim=cl_kwargs.get("objlim", 1.0), objlim_form=cl_kwargs.get("objlim_form", 0))


def crop_with_context(img, y0, x0, hh, ww, ctx):
    """Crop plus `ctx` pixels of context (clipped at the frame); returns (crop, slice of the window)."""
    H, W = img.shape
    ya, xa = max(0, y0 - ctx), max(0, x0 - ctx)
    yb, xb = min(H, y0 + hh + ctx), min(W, x0 + ww + ctx)
    return (np.ascontiguousarray(img[ya:yb, xa:xb]),
            (slice(y0 - ya, y0 - ya + hh), slice(x0 - xa, x0 - xa + ww)))
