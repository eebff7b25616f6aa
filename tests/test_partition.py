"""The paper's 2-D image segmentation (crb_partition, host code) and the multi-rank gather.

crb_partition needs no GPU, so its checks run on the CPU against the segmentations the paper
describes (tests/golden/paper_partition.json). The multi-rank path (each rank cleans its share of
the rectangles, rank 0 assembles the interiors) runs as two gloo ranks on the CPU, with the oracle
cleaning each rectangle's context region in place of a rank's GPU: the assembled frame must equal
the whole-frame clean bit for bit, which the 8 * niter context guarantees.
"""

from __future__ import annotations

import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "paper_partition.json")

from paper_1008_2192_gb300 import partition  # noqa: E402


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_paper_six_by_six():
    g = _golden()["six_by_six_750"]
    cols, rows, rects = partition.plan(g["w"], g["h"], g["nparts"], g["border"])
    assert (cols, rows) == (g["cols"], g["rows"])
    inner = [r for r in rects if r.x0 > 0 and r.y0 > 0 and r.x0 + r.w < g["w"] and r.y0 + r.h < g["h"]]
    assert len(inner) == 16 and all(r.w == r.h == g["interior_side"] for r in rects)
    assert all(r.cw == r.ch == g["subimage_side"] for r in inner)
    r = inner[0]
    assert round(100 * (r.cw * r.ch - r.w * r.h) / (r.w * r.h), 1) == g["edge_ratio_percent"]


def test_paper_one_by_36():
    g = _golden()["one_by_36_750"]
    cols, rows, rects = partition.plan(g["w"], g["h"], g["nparts"], g["border"], cols=1)
    assert (cols, rows) == (g["cols"], g["rows"])
    slices = [r for r in rects if r.h == g["slice_rows"] and 0 < r.y0 and r.y0 + r.h < g["h"]]
    assert len(slices) > 20 and all(r.cw * r.ch == g["subimage_pixels"] for r in slices)
    assert round(100 * 2 * g["border"] / g["slice_rows"], 1) == g["edge_ratio_percent"]


def test_paper_two_by_four_and_primes():
    gd = _golden()
    g = gd["two_by_four_800"]
    assert partition.plan(g["w"], g["h"], g["nparts"], 6)[:2] == (g["cols"], g["rows"])
    g = gd["one_by_37"]
    assert partition.plan(g["w"], g["h"], g["nparts"], 6)[:2] == (g["cols"], g["rows"])
    g = gd["primes_one_by_n"]
    for n in g["nparts"]:
        assert partition.plan(g["w"], g["h"], n, 6)[:2] == (1, n), n


@pytest.mark.parametrize("w,h,n,ctx", [(1, 1, 1, 0), (17, 5, 4, 3), (100, 77, 6, 16), (64, 640, 8, 32),
                                       (333, 129, 12, 8), (5, 40, 8, 2), (100, 77, 6, 2**31 - 1)])
def test_rectangles_tile_the_frame(w, h, n, ctx):
    """Interiors tile the frame exactly once; contexts are the interiors widened by ctx, clipped."""
    cols, rows, rects = partition.plan(w, h, n, ctx)
    assert cols * rows == n == len(rects)
    cover = np.zeros((h, w), np.int32)
    for r in rects:
        cover[r.interior()] += 1
        assert (r.cx0, r.cy0) == (max(r.x0 - ctx, 0), max(r.y0 - ctx, 0))
        assert (r.cx0 + r.cw, r.cy0 + r.ch) == (min(r.x0 + r.w + ctx, w), min(r.y0 + r.h + ctx, h))
    assert (cover == 1).all()
    widths = {r.w for r in rects}
    heights = {r.h for r in rects}
    assert max(widths) - min(widths) <= 1 and max(heights) - min(heights) <= 1  # nearly equal area


def test_invalid_plans_rejected():
    for args in [(0, 5, 1, 0), (5, 5, 0, 0), (5, 5, 2, -1), (3, 3, 16, 0)]:
        with pytest.raises(ValueError):
            partition.plan(*args)
    with pytest.raises(ValueError):
        partition.plan(10, 10, 6, 0, cols=4)  # 4 does not divide 6


# ---------------------------------------------------------------------------------------- two ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1008_2192_gb300 import partition as part
    oracle.set_threads(2)
    niter = 2
    img = synth.frame(160, 120, seed=9, sky=100.0, nstars=10, ncr=120)
    P = oracle.Params()
    cols, rows, rects = part.plan(160, 120, 6, 8 * niter)
    mine = {}
    for i in part.share(len(rects), rank, world):  # this rank's actors
        r = rects[i]
        res = oracle.clean(np.ascontiguousarray(img[r.context()]), P, niter, precision="f32")
        sl = r.interior_of_crop()
        mine[i] = (torch.from_numpy(np.ascontiguousarray(res.clean[sl])),
                   torch.from_numpy(np.ascontiguousarray(res.mask[sl])))
    out = torch.full((120, 160), float("nan"), dtype=torch.float32)
    mask = torch.full((120, 160), 7, dtype=torch.uint8)
    part.gather(rects, mine, out, mask, rank, world)
    ok = None
    if rank == 0:
        whole = oracle.clean(img, P, niter, precision="f32")
        ok = bool(np.array_equal(out.numpy(), whole.clean) and np.array_equal(mask.numpy(), whole.mask)
                  and whole.mask.sum() > 0)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, sorted(mine), ok))


def test_two_ranks_assemble_the_whole_frame_clean():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == [0, 2, 4] and out[1][1] == [1, 3, 5]  # round robin over the 3 x 2 plan
    assert out[0][2] is True
