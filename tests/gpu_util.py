"""Shared helpers of the GPU tests: device transfer, GPU runs and the parity checks.

Tolerances (GPU float32 vs the FP64 oracle): intermediate maps within 1e-5
relative (with an absolute floor of 1e-5 times the map's scale, for values
that cancel to ~0); masks identical except on the oracle's fragile pixels
(a decision statistic within 1e-4 relative of its threshold in the growth
cone); cleaned pixels within 1e-5 relative where the masks agree. Against the
FP32 oracle (the same steps in the kernel's precision) everything is
bit-identical.
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


def assert_map_close(got, ref, name):
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    scale = max(1.0, float(np.max(np.abs(ref[np.isfinite(ref)]))) if np.isfinite(ref).any() else 1.0)
    bad = ~np.isclose(got, ref, rtol=RTOL, atol=RTOL * scale, equal_nan=True)
    assert not bad.any(), f"map {name}: {int(bad.sum())} values differ, first {np.argwhere(bad)[:5]}"


def assert_clean_matches_f64(clean, mask, ref: "oracle.CleanResult", what=""):
    ok = ref.fragile == 0
    flips = int((mask != ref.mask).sum())
    assert np.array_equal(mask[ok], ref.mask[ok]), f"{what}: mask differs off fragile pixels"
    agree = mask == ref.mask
    np.testing.assert_allclose(clean[agree], ref.clean[agree], rtol=RTOL, err_msg=what)
    return flips, int((~ok).sum())


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
