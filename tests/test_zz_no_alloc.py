"""The allocation-free entry point crb_clean_noalloc against crb_clean.

crb_clean_noalloc serves callers that cannot allocate device memory while they
run (fixed memory plans, latency-bound loops, device memory owned by another
allocator): its scratch is a fixed array inside the library. This file is
collected last so that a run stopping at the first failure has run every other
test first; it passes alone in a fresh process and after the other tests.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1008_2192_gb300._lib as L  # noqa: E402
from paper_1008_2192_gb300 import Cleaner  # noqa: E402

PARAMS = (7.0, 5.0, 4.5, 0.5, 1.0)


def _call(img, out, mask, niter):
    h, w = img.shape
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.load().crb_clean_noalloc(*PARAMS, niter, ctypes.c_void_p(img.data_ptr()), w, h,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr()), s)


@pytest.mark.parametrize("niter", [0, 1, 3, 4])
def test_noalloc_equals_crb_clean_two_calls_in_a_row(niter):
    """Two consecutive calls (different frames and sizes) each equal crb_clean exactly; niter 0 (copy
    and clear), 1 (the image scratch unused), odd (the buffers alternate to the other side) and 4. The
    second call changes neither torch's allocations nor the device's free memory."""
    cl = Cleaner(*PARAMS, niter=niter)
    for i, (w, h) in enumerate([(800, 800), (1000, 613)]):
        img = torch.from_numpy(synth.frame(w, h, seed=21, index=i)).cuda()
        ref_out, ref_mask = cl.clean(img)
        cl.sync()
        out = torch.full_like(img, -1.0)
        mask = torch.full(img.shape, 7, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        rc = _call(img, out, mask, niter)
        assert rc == L.CRB_OK, L.load().crb_last_error()
        torch.cuda.synchronize()
        if i == 1:  # the first call may load the library's device code and commit its scratch
            assert (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]) == before
        if niter > 0:
            assert ref_mask.sum().item() > 0
        assert torch.equal(mask, ref_mask), f"call {i + 1}: mask"
        assert torch.equal(out, ref_out), f"call {i + 1}: cleaned frame"
    cl.close()


def test_noalloc_rejects_frames_beyond_its_scratch():
    """Sizes beyond the fixed scratch and niter beyond its counters are refused before any work; the
    buffers passed are real and large enough, so no check relies on another to stay in bounds."""
    lib = L.load()
    for (w, h) in ((16385, 1), (2049, 2049)):  # a side above 16384; more than 4,194,304 pixels
        img = torch.zeros((h, w), dtype=torch.float32, device="cuda")
        out = torch.empty_like(img)
        mask = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
        assert _call(img, out, mask, 4) == L.CRB_EINVAL
        assert b"exceeds the fixed scratch" in lib.crb_last_error()
    img = torch.from_numpy(synth.frame(8, 8, seed=1)).cuda()
    out = torch.empty_like(img)
    mask = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    assert _call(img, out, mask, 65) == L.CRB_EINVAL
    assert _call(img, img, mask, 2) == L.CRB_EALIAS
