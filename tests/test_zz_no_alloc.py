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


def _noalloc(img, niter=4):
    h, w = img.shape
    out = torch.empty_like(img)
    mask = torch.empty(img.shape, dtype=torch.uint8, device=img.device)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.load().crb_clean_noalloc(*PARAMS, niter, ctypes.c_void_p(img.data_ptr()), w, h,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr()), s)
    assert rc == L.CRB_OK, L.load().crb_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy(), mask.cpu().numpy()


def test_noalloc_equals_crb_clean_two_calls_in_a_row():
    """Two consecutive calls (different frames and sizes) each equal crb_clean exactly."""
    cl = Cleaner(*PARAMS, niter=4)
    for i, (w, h) in enumerate([(800, 800), (1000, 613)]):
        img = torch.from_numpy(synth.frame(w, h, seed=21, index=i)).cuda()
        ref_out, ref_mask = cl.clean(img)
        cl.sync()
        out, mask = _noalloc(img)
        assert mask.sum() > 0
        assert np.array_equal(mask, ref_mask.cpu().numpy()), f"call {i + 1}: mask"
        assert np.array_equal(out, ref_out.cpu().numpy()), f"call {i + 1}: cleaned frame"
    cl.close()


def test_noalloc_rejects_frames_beyond_its_scratch():
    big = torch.empty((1, 1), dtype=torch.float32, device="cuda")
    lib = L.load()
    p = ctypes.c_void_p(big.data_ptr())
    rc = lib.crb_clean_noalloc(*PARAMS, 4, p, 4096, 4096, ctypes.c_void_p(big.data_ptr() + 64),
                               ctypes.c_void_p(big.data_ptr() + 128), None)
    assert rc == L.CRB_EINVAL
    assert b"exceeds the fixed scratch" in lib.crb_last_error()
    rc = lib.crb_clean_noalloc(*PARAMS, 65, p, 8, 8, ctypes.c_void_p(big.data_ptr() + 64),
                               ctypes.c_void_p(big.data_ptr() + 512), None)
    assert rc == L.CRB_EINVAL
