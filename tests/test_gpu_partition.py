"""crb_clean_rects on the GPU: the paper's segmentation cleaned rectangle by rectangle, then assembled.

With a context of 8 * niter pixels every rectangle's cleaned interior equals the whole-frame clean's,
so the assembled frame must be bit-identical to crb_clean's, for the 2-D cuts crb_partition picks,
the 1-D slices, a prime count and the 16384x16384 mosaic in four quadrants.
"""

import ctypes

import numpy as np
import pytest

import synth
from synth import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1008_2192_gb300._lib as L  # noqa: E402
from paper_1008_2192_gb300 import Cleaner, partition  # noqa: E402


@pytest.mark.parametrize("w,h,n,cols,niter", [(2048, 1536, 6, 0, 4), (1000, 613, 7, 0, 4), (800, 800, 8, 1, 3),
                                              (333, 257, 1, 0, 2), (64, 640, 4, 0, 1)])
def test_rects_equal_whole_frame(w, h, n, cols, niter):
    img = torch.from_numpy(synth.frame(w, h, seed=w + h)).cuda()
    c = Cleaner(niter=niter)
    ref_out, ref_mask = c.clean(img)
    c.sync()
    ncols, nrows, rects = partition.plan(w, h, n, 8 * niter, cols=cols)
    assert ncols * nrows == n
    out = torch.full_like(img, float("nan"))
    mask = torch.full(img.shape, 7, dtype=torch.uint8, device="cuda")
    c.clean_rects_into(img, rects, out, mask)
    c.sync()
    assert ref_mask.sum().item() > 0
    assert torch.equal(mask, ref_mask) and torch.equal(out, ref_out)


def test_mosaic_in_four_quadrants():
    """The 16384x16384 mosaic (1 GiB) as the paper's 2x2 segmentation with a 32-pixel context."""
    rec = workloads.mosaic_16384()
    img = torch.from_numpy(workloads.make(rec)).cuda()
    c = Cleaner(gain=rec["gain"], readnoise=rec["readnoise"], niter=4)
    ref_out, ref_mask = c.clean(img)
    cols, rows, rects = partition.plan(16384, 16384, 4, 32)
    assert (cols, rows) == (2, 2)
    out, mask = c.clean_rects(img, rects)
    c.sync()
    assert torch.equal(mask, ref_mask) and torch.equal(out, ref_out)


def test_invalid_rectangles_rejected():
    img = torch.from_numpy(synth.frame(100, 80, seed=1)).cuda()
    out = torch.empty_like(img)
    mask = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    c = Cleaner(niter=2)
    lib = L.load()
    bad = [partition.Rect(10, 10, 20, 20, 12, 10, 20, 20),   # context does not contain the interior
           partition.Rect(90, 70, 10, 10, 80, 60, 30, 20),   # context beyond the frame
           partition.Rect(0, 0, 0, 5, 0, 0, 5, 5)]           # empty interior
    for r in bad:
        rc = lib.crb_clean_rects(c.handle, ctypes.c_void_p(img.data_ptr()), 100, 80, 1, partition.to_c([r]),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr()), None)
        assert rc == L.CRB_EINVAL, r
    ok = partition.plan(100, 80, 2, 16)[2]
    rc = lib.crb_clean_rects(c.handle, ctypes.c_void_p(img.data_ptr()), 100, 80, 2, partition.to_c(ok),
                             ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(mask.data_ptr()), None)
    assert rc == L.CRB_EALIAS
