"""Convenience wrapper over the C ABI for torch CUDA tensors.

Torch provides device memory and streams; every step of the cleaning runs in
the library's CUDA kernels.
"""

from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_img(t, name="img"):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2
            and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous 2-D float32 CUDA tensor")


def _check_out(t, like, dtype, name):
    """An output the library writes w*h elements into: a contiguous CUDA tensor of `dtype` with the
    shape of `like` on its device (the C ABI cannot see a device buffer's size)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and t.shape == like.shape and t.device == like.device):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor of shape {tuple(like.shape)} "
                         f"on {like.device}")


def _check_lengths(n, **arrays):
    for name, a in arrays.items():
        if a is not None and len(a) != n:
            raise ValueError(f"{name} has {len(a)} entries for {n} frames")


# crb_options.pipeline: "auto" picks by the pixels of each call (queue from 6 Mpix on)
PIPELINES = {"auto": 0, "tile": 1, "queue": 2}


class Cleaner:
    """One cleaning context (crb_create_ex). Not thread-safe; use one per thread."""

    def __init__(self, gain=7.0, readnoise=5.0, sigclip=4.5, sigfrac=0.5, objlim=1.0, niter=4, *,
                 objlim_form=0, early_exit=False, tile_shape=0, use_graphs=False, profile=False,
                 fusion=True, pipeline="auto", autotune=False, fuse2=False):
        lib = _lib.load()
        opt = _lib.crb_options(int(objlim_form), int(bool(early_exit)), int(tile_shape), int(bool(use_graphs)),
                               int(bool(profile)), int(not fusion), PIPELINES[pipeline], int(bool(autotune)),
                               int(bool(fuse2)))
        h = lib.crb_create_ex(gain, readnoise, sigclip, sigfrac, objlim, int(niter), ctypes.byref(opt))
        if not h:
            raise ValueError("crb_create_ex: " + lib.crb_last_error().decode())
        self._h = ctypes.c_void_p(h)
        self.niter = int(niter)
        self.gain, self.readnoise = float(gain), float(readnoise)

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().crb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    @property
    def handle(self):
        return self._h

    def clean_into(self, img, out_clean, out_mask, stream=None):
        _check_img(img)
        _check_out(out_clean, img, torch.float32, "out_clean")
        _check_out(out_mask, img, torch.uint8, "out_mask")
        h, w = img.shape
        rc = _lib.load().crb_clean(self._h, _ptr(img), w, h, _ptr(out_clean), _ptr(out_mask), _stream(stream))
        check(rc, "crb_clean")

    def clean(self, img, stream=None):
        """Returns (cleaned float32 frame, uint8 mask) as new CUDA tensors."""
        _check_img(img)
        out = torch.empty_like(img)
        mask = torch.empty(img.shape, dtype=torch.uint8, device=img.device)
        self.clean_into(img, out, mask, stream)
        return out, mask

    def clean_batch_into(self, imgs, outs, masks, gains=None, readnoises=None, stream=None):
        n = len(imgs)
        _check_lengths(n, outs=outs, masks=masks, gains=gains, readnoises=readnoises)
        for t, o, m in zip(imgs, outs, masks):
            _check_img(t)
            _check_out(o, t, torch.float32, "each out")
            _check_out(m, t, torch.uint8, "each mask")
        P = ctypes.c_void_p * n
        I = ctypes.c_int * n
        F = ctypes.c_float * n
        a_img = P(*[t.data_ptr() for t in imgs])
        a_out = P(*[t.data_ptr() for t in outs])
        a_msk = P(*[t.data_ptr() for t in masks])
        a_w = I(*[t.shape[1] for t in imgs])
        a_h = I(*[t.shape[0] for t in imgs])
        a_g = F(*gains) if gains is not None else None
        a_r = F(*readnoises) if readnoises is not None else None
        rc = _lib.load().crb_clean_batch(self._h, n, a_img, a_w, a_h, a_g, a_r, a_out, a_msk, _stream(stream))
        check(rc, "crb_clean_batch")

    def clean_batch_host_into(self, imgs, outs, masks, gains=None, readnoises=None, stream=None):
        """crb_clean_batch_host: frames, outputs and masks are CPU tensors (pinned memory lets the copies
        overlap the work); the outputs are valid once `stream` (default: the current stream) is synchronised."""
        n = len(imgs)
        _check_lengths(n, outs=outs, masks=masks, gains=gains, readnoises=readnoises)
        for t, o, m in zip(imgs, outs, masks):
            if t.device.type != "cpu" or o.device.type != "cpu" or m.device.type != "cpu":
                raise ValueError("clean_batch_host_into takes CPU tensors")
            if t.dtype != torch.float32 or o.dtype != torch.float32 or m.dtype != torch.uint8:
                raise ValueError("frames and outputs float32, masks uint8")
            if (t.dim() != 2 or not t.is_contiguous() or not o.is_contiguous() or not m.is_contiguous()
                or o.shape != t.shape or m.shape != t.shape):
                raise ValueError("contiguous 2-D frames with outputs of the same shape")
        P = ctypes.c_void_p * n
        I = ctypes.c_int * n
        F = ctypes.c_float * n
        a_img = P(*[t.data_ptr() for t in imgs])
        a_out = P(*[t.data_ptr() for t in outs])
        a_msk = P(*[t.data_ptr() for t in masks])
        a_w = I(*[t.shape[1] for t in imgs])
        a_h = I(*[t.shape[0] for t in imgs])
        a_g = F(*gains) if gains is not None else None
        a_r = F(*readnoises) if readnoises is not None else None
        rc = _lib.load().crb_clean_batch_host(self._h, n, a_img, a_w, a_h, a_g, a_r, a_out, a_msk,
                                              _stream(stream))
        check(rc, "crb_clean_batch_host")

    def clean_rects_into(self, img, rects, out_clean, out_mask, stream=None):
        """crb_clean_rects: each rectangle (partition.Rect) cleaned as its context region, its interior
        written into out_clean / out_mask."""
        from .partition import to_c
        _check_img(img)
        _check_out(out_clean, img, torch.float32, "out_clean")
        _check_out(out_mask, img, torch.uint8, "out_mask")
        h, w = img.shape
        arr = to_c(rects)
        rc = _lib.load().crb_clean_rects(self._h, _ptr(img), w, h, len(rects), arr, _ptr(out_clean),
                                         _ptr(out_mask), _stream(stream))
        check(rc, "crb_clean_rects")

    def clean_rects(self, img, rects, stream=None):
        """crb_clean_rects into new tensors (pixels outside every interior are left unset)."""
        out = torch.empty_like(img)
        mask = torch.empty(img.shape, dtype=torch.uint8, device=img.device)
        self.clean_rects_into(img, rects, out, mask, stream)
        return out, mask

    def clean_batch(self, imgs, gains=None, readnoises=None, stream=None):
        outs = [torch.empty_like(t) for t in imgs]
        masks = [torch.empty(t.shape, dtype=torch.uint8, device=t.device) for t in imgs]
        self.clean_batch_into(imgs, outs, masks, gains, readnoises, stream)
        return outs, masks

    def iterate(self, J, Mprev=None, maps=False, stream=None):
        """One iteration from (J, Mprev). Returns (I_k, M_k, maps dict or None)."""
        _check_img(J, "J")
        if Mprev is not None:
            _check_out(Mprev, J, torch.uint8, "Mprev")
        h, w = J.shape
        outJ = torch.empty_like(J)
        outM = torch.empty(J.shape, dtype=torch.uint8, device=J.device)
        mp = torch.empty((_lib.NUM_MAPS, h, w), dtype=torch.float32, device=J.device) if maps else None
        rc = _lib.load().crb_iterate(self._h, _ptr(J), _ptr(Mprev) if Mprev is not None else None, w, h,
                                     _ptr(outJ), _ptr(outM), _ptr(mp) if maps else None, _stream(stream))
        check(rc, "crb_iterate")
        md = {n: mp[i] for i, n in enumerate(_lib.MAP_NAMES)} if maps else None
        return outJ, outM, md

    def sync(self, stream=None):
        check(_lib.load().crb_sync_status(self._h, _stream(stream)), "crb_sync_status")

    def last_counts(self):
        """[(new flags, flagged pixels with no unflagged neighbour)] per iteration of the last call."""
        buf = (ctypes.c_longlong * (2 * max(self.niter, 1)))()
        k = _lib.load().crb_last_counts(self._h, buf, max(self.niter, 1))
        if k < 0:
            raise RuntimeError("crb_last_counts failed")
        return [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(k)]

    def last_work(self):
        """Per iteration of the last call: positions given (S, S', med3, candidate test, full 7x7 median of
        the test, bound test)."""
        buf = (ctypes.c_longlong * (6 * max(self.niter, 1)))()
        k = _lib.load().crb_last_work(self._h, buf, max(self.niter, 1))
        if k < 0:
            raise RuntimeError("crb_last_work failed")
        return [tuple(int(buf[6 * i + j]) for j in range(6)) for i in range(k)]

    QUEUE_KERNELS = ("bound", "need", "s", "sprime", "m3need", "m3", "cand_test", "rep_compute", "bound_sparse",
                     "rq", "rep_write", "d2", "cand_full", "grow", "mask", "seg_list", "d2_seg", "need_seg",
                     "m3need_seg", "m3need_first", "grow_first")

    def tuned_config(self):
        """Launch configuration of the last call: ({kernel: blocks per SM}, first segment-list iteration,
        pipeline "tile" or "queue")."""
        n = len(self.QUEUE_KERNELS)
        occ = (ctypes.c_int * n)()
        sf, pl = ctypes.c_int(), ctypes.c_int()
        k = _lib.load().crb_tuned_config(self._h, occ, n, ctypes.byref(sf), ctypes.byref(pl))
        if k < 0:
            check(k, "crb_tuned_config")
        return dict(zip(self.QUEUE_KERNELS, list(occ)[:k])), sf.value, {1: "tile", 2: "queue"}.get(pl.value)

    def last_launches(self):
        """Kernel launches the last call enqueued."""
        return int(_lib.load().crb_last_launches(self._h))

    def profile_read(self, reset=True):
        """(detect ms, detect launches, replace ms, replace launches) since the last reset."""
        dm, rm = ctypes.c_double(), ctypes.c_double()
        dn, rn = ctypes.c_int(), ctypes.c_int()
        check(_lib.load().crb_profile_read(self._h, ctypes.byref(dm), ctypes.byref(dn), ctypes.byref(rm),
                                           ctypes.byref(rn), int(reset)), "crb_profile_read")
        return dm.value, dn.value, rm.value, rn.value

    PROFILE_KINDS = ("bound", "need", "s", "sprime", "m3need", "m3", "cand", "grow", "reserved", "tile_detect",
                     "replace", "mask", "tile_replace", "work")

    def profile_kernels(self, reset=True):
        """{kind: (ms, timed brackets)} since the last reset (crb_profile_kernels)."""
        n = len(self.PROFILE_KINDS)
        ms = (ctypes.c_double * n)()
        br = (ctypes.c_int * n)()
        k = _lib.load().crb_profile_kernels(self._h, ms, br, n, int(reset))
        if k < 0:
            check(k, "crb_profile_kernels")
        return {self.PROFILE_KINDS[i]: (ms[i], br[i]) for i in range(k)}


def fadd_peak(stream=None):
    """Measured FP32 adds per second."""
    a = ctypes.c_double()
    check(_lib.load().crb_fadd_peak(ctypes.byref(a), _stream(stream)), "crb_fadd_peak")
    return a.value


def alu_peak(stream=None):
    """Measured FP32 min/max operations per second: (2-input form, 3-input form)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(_lib.load().crb_alu_peak(ctypes.byref(a), ctypes.byref(b), _stream(stream)), "crb_alu_peak")
    return a.value, b.value


def poisson_into(img, out, seed, stream=None):
    """The POISSON work function (crb_poisson): out[p] = a Poisson deviate of mean img[p]."""
    _check_img(img)
    _check_img(out, "out")
    if out.shape != img.shape:
        raise ValueError("out must have the shape of img")
    h, w = img.shape
    check(_lib.load().crb_poisson(_ptr(img), w, h, ctypes.c_uint64(seed & (2**64 - 1)), _ptr(out),
                                  _stream(stream)), "crb_poisson")
    return out


def poisson(img, seed, stream=None):
    """The POISSON work function into a new tensor."""
    return poisson_into(img, torch.empty_like(img), seed, stream)


def poisson_batch_into(imgs, outs, seeds, stream=None):
    """crb_poisson_batch: frame i with seed seeds[i] into outs[i]."""
    n = len(imgs)
    if len(outs) != n or len(seeds) != n:
        raise ValueError("imgs, outs and seeds must have the same length")
    for a, o in zip(imgs, outs):
        _check_img(a)
        _check_img(o, "out")
        if o.shape != a.shape:
            raise ValueError("each out must have the shape of its img")
    P = ctypes.c_void_p * n
    I = ctypes.c_int * n
    rc = _lib.load().crb_poisson_batch(
        n, P(*[a.data_ptr() for a in imgs]), I(*[a.shape[1] for a in imgs]), I(*[a.shape[0] for a in imgs]),
        (ctypes.c_uint64 * n)(*[s & (2**64 - 1) for s in seeds]), P(*[o.data_ptr() for o in outs]), _stream(stream))
    check(rc, "crb_poisson_batch")
    return outs


class Server:
    """Continuous-batching server (crb_server_*): submit device frames, poll finished tags."""

    def __init__(self, gain=7.0, readnoise=5.0, sigclip=4.5, sigfrac=0.5, objlim=1.0, niter=4, *,
                 budget_bytes=64 << 30, max_inflight=2, max_batch=64, objlim_form=0, tile_shape=0, fuse2=False):
        lib = _lib.load()
        opt = _lib.crb_options(int(objlim_form), 0, int(tile_shape), 0, 0, 0, 0, 0, int(bool(fuse2)))
        h = lib.crb_server_create(gain, readnoise, sigclip, sigfrac, objlim, int(niter), ctypes.byref(opt),
                                  int(budget_bytes), int(max_inflight), int(max_batch))
        if not h:
            raise ValueError("crb_server_create: " + lib.crb_last_error().decode())
        self._h = ctypes.c_void_p(h)
        self._keep = {}  # tag -> tensors kept alive until done

    def submit(self, img, out, mask, tag, gain, readnoise):
        """Queues a frame; returns False when the memory budget refuses it (CRB_EBUSY)."""
        _check_img(img)
        _check_out(out, img, torch.float32, "out")
        _check_out(mask, img, torch.uint8, "mask")
        h, w = img.shape
        rc = _lib.load().crb_server_submit(self._h, _ptr(img), w, h, float(gain), float(readnoise), _ptr(out),
                                           _ptr(mask), int(tag))
        if rc == _lib.CRB_EBUSY:
            return False
        check(rc, "crb_server_submit")
        self._keep[int(tag)] = (img, out, mask)
        return True

    def poll(self, max_n=256, block_ms=0):
        """[(tag, latency seconds, status)] of frames finished since the last poll."""
        tags = (ctypes.c_uint64 * max_n)()
        lat = (ctypes.c_double * max_n)()
        st = (ctypes.c_int * max_n)()
        n = _lib.load().crb_server_poll(self._h, tags, lat, st, max_n, int(block_ms))
        if n < 0:
            raise RuntimeError("crb_server_poll failed")
        out = []
        for i in range(n):
            self._keep.pop(int(tags[i]), None)
            out.append((int(tags[i]), float(lat[i]), int(st[i])))
        return out

    def stats(self):
        buf = (ctypes.c_longlong * 10)()
        _lib.load().crb_server_stats(self._h, buf, 10)
        keys = ("submitted", "done", "waves", "max_wave", "rejected", "resident_bytes", "peak_resident_bytes",
                "queued", "max_enqueue_us", "max_submit_wait_us")
        return dict(zip(keys, (int(v) for v in buf)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().crb_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
