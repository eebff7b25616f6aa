"""The POISSON work function on the GPU (C ABI) against the CPU oracle: bit-identical deviates."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1008_2192_gb300 as pkg  # noqa: E402
import paper_1008_2192_gb300._lib as L  # noqa: E402


def gpu_poisson(img, seed):
    out = pkg.poisson(dev(img), seed)
    torch.cuda.synchronize()
    return host(out)


@pytest.mark.parametrize("seed", [0, 2010, 2**64 - 1])
def test_paper_test_image(seed):
    """750x750, every pixel 24.3 (the paper's POISSON test image)."""
    img = np.full((750, 750), 24.3, np.float32)
    assert np.array_equal(gpu_poisson(img, seed), oracle.poisson(img, seed))


@pytest.mark.parametrize("w,h", [(1, 1), (17, 1), (1, 33), (100, 77), (1024, 3), (257, 129)])
def test_ragged_sizes_on_frame_values(w, h):
    """Means from a synthetic frame (sky, stars, cosmic rays: 0 .. far above the 700 cap)."""
    img = synth.frame(w, h, seed=w * 7 + h, sky=100.0, nstars=max(1, w * h // 500), ncr=max(1, w * h // 300))
    assert np.array_equal(gpu_poisson(img, 99), oracle.poisson(img, 99))


def test_special_values():
    row = np.array([0.0, -0.0, -5.0, np.nan, np.inf, -np.inf, 1e-30, 1e-8, 0.5, 699.9, 700.0, 700.5, 1e6,
                    3.4e38], np.float32)
    img = np.tile(row, (40, 1))
    assert np.array_equal(gpu_poisson(img, 5), oracle.poisson(img, 5))


def test_batch_equals_single_and_many_frames():
    """Frames with their own seeds in one call (more than one launch of 256 frames) equal single calls."""
    rng = np.random.default_rng(4)
    sizes = [(int(rng.integers(1, 40)), int(rng.integers(1, 40))) for _ in range(300)] + [(640, 480)]
    imgs = [rng.uniform(0, 60, size=(h, w)).astype(np.float32) for (w, h) in sizes]
    seeds = [int(rng.integers(0, 2**63)) for _ in sizes]
    outs = [torch.empty((h, w), dtype=torch.float32, device="cuda") for (w, h) in sizes]
    pkg.poisson_batch_into([dev(a) for a in imgs], outs, seeds)
    torch.cuda.synchronize()
    for a, o, s in zip(imgs, outs, seeds):
        assert np.array_equal(host(o), oracle.poisson(a, s))


def test_in_place():
    img = np.full((300, 200), 24.3, np.float32)
    t = dev(img)
    pkg.poisson_into(t, t, 11)
    torch.cuda.synchronize()
    assert np.array_equal(host(t), oracle.poisson(img, 11))


def test_invalid_arguments():
    import ctypes
    lib = L.load()
    t = dev(np.zeros((4, 4), np.float32))
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.crb_poisson(None, 4, 4, 0, p, None) == L.CRB_EINVAL
    assert lib.crb_poisson(p, 0, 4, 0, p, None) == L.CRB_EINVAL
    assert lib.crb_poisson(p, 4, -1, 0, p, None) == L.CRB_EINVAL
    assert lib.crb_poisson_batch(-1, None, None, None, None, None, None) == L.CRB_EINVAL
    assert lib.crb_poisson_batch(0, None, None, None, None, None, None) == L.CRB_OK
