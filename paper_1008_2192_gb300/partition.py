"""The paper's 2-D image segmentation across ranks (Sec. 6.2, Sec. 6.3.1).

``plan`` calls crb_partition (C ABI): a frame cut into cols x rows rectangles
of nearly equal area, each with a context margin. Each rank cleans its
``share`` of them (``Cleaner.clean_rects`` on its own GPU) and ``gather``
sends the cleaned interiors to rank 0, which writes them into the frame: the
director's round of receives. Messages are point-to-point (torch.distributed
send/recv: gloo for CPU tensors, NCCL for CUDA tensors); the ranks cleaning
rectangles never exchange anything, as the paper's actors do not.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib


@dataclass(frozen=True)
class Rect:
    """Interior (x0, y0, w, h) and context region (cx0, cy0, cw, ch) of one rectangle."""
    x0: int
    y0: int
    w: int
    h: int
    cx0: int
    cy0: int
    cw: int
    ch: int

    def interior_of_crop(self):
        """(rows, cols) slices of the interior within a result of the context region."""
        return (slice(self.y0 - self.cy0, self.y0 - self.cy0 + self.h),
                slice(self.x0 - self.cx0, self.x0 - self.cx0 + self.w))

    def interior(self):
        """(rows, cols) slices of the interior within the frame."""
        return slice(self.y0, self.y0 + self.h), slice(self.x0, self.x0 + self.w)

    def context(self):
        """(rows, cols) slices of the context region within the frame."""
        return slice(self.cy0, self.cy0 + self.ch), slice(self.cx0, self.cx0 + self.cw)


def plan(w, h, nparts, context, cols=0):
    """crb_partition: (cols, rows, [Rect] row by row). cols=0 picks the cut closest to square."""
    lib = _lib.load()
    nc, nr = ctypes.c_int(), ctypes.c_int()
    n = lib.crb_partition(int(w), int(h), int(nparts), int(cols), int(context), None, 0, ctypes.byref(nc),
                          ctypes.byref(nr))
    if n < 0:
        raise ValueError("crb_partition: " + lib.crb_last_error().decode())
    arr = (_lib.crb_rect * n)()
    lib.crb_partition(int(w), int(h), int(nparts), int(cols), int(context), arr, n, None, None)
    rects = [Rect(r.x0, r.y0, r.w, r.h, r.cx0, r.cy0, r.cw, r.ch) for r in arr]
    return nc.value, nr.value, rects


def to_c(rects):
    """The rectangles as a crb_rect array for the C ABI."""
    arr = (_lib.crb_rect * len(rects))()
    for a, r in zip(arr, rects):
        a.x0, a.y0, a.w, a.h, a.cx0, a.cy0, a.cw, a.ch = r.x0, r.y0, r.w, r.h, r.cx0, r.cy0, r.cw, r.ch
    return arr


def share(n, rank, world):
    """Indices of the rectangles rank `rank` of `world` cleans (round robin over the plan)."""
    return [i for i in range(n) if i % world == rank]


def gather(rects, mine, out_clean, out_mask, rank, world, group=None):
    """Sends this rank's cleaned interiors to rank 0, which writes every interior into its frame.

    mine: {index: (clean interior, mask interior)} of this rank's rectangles (torch tensors shaped like
    the interior; CPU for gloo, CUDA for NCCL). out_clean / out_mask: the frame on rank 0 (ignored
    elsewhere). Rectangles go in plan order, each from its owner (``share``) to rank 0.
    """
    import torch
    import torch.distributed as dist

    for i, r in enumerate(rects):
        owner = i % world
        ys, xs = r.interior()
        if rank == 0:
            if owner == 0:
                c, m = mine[i]
            else:
                c = torch.empty((r.h, r.w), dtype=out_clean.dtype, device=out_clean.device)
                m = torch.empty((r.h, r.w), dtype=out_mask.dtype, device=out_mask.device)
                dist.recv(c, src=owner, group=group)
                dist.recv(m, src=owner, group=group)
            out_clean[ys, xs] = c
            out_mask[ys, xs] = m
        elif owner == rank:
            c, m = mine[i]
            dist.send(c.contiguous(), dst=0, group=group)
            dist.send(m.contiguous(), dst=0, group=group)
