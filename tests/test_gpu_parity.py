"""GPU (CUDA library, through the C ABI) against the CPU oracle on seeded synthetic frames."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from synth import workloads
from gpu_util import (assert_clean_matches_f64, assert_map_close, compare_f64, crop_with_context, dev,
                      gpu_clean, host, map_floors, params_of)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1008_2192_gb300 import Cleaner  # noqa: E402

# sizes spanning several tiles with ragged tails, degenerate strips and odd widths
SIZES = [(1, 1), (1, 17), (17, 1), (2, 2), (7, 13), (13, 7), (31, 33), (64, 32), (65, 33), (100, 77),
         (129, 70), (200, 150)]


def scene(w, h, seed=0):
    n = w * h
    return synth.frame(w, h, seed=seed, sky=100.0, nstars=max(1, n // 2000),
                       ncr=max(1, int(n * synth.CR_DENSITY * 3)))


@pytest.fixture(scope="module", params=["queue", "auto"])
def cl(request):
    """The queue pipeline, and the default choice by call size (the tile pipeline below 6 Mpix)."""
    c = Cleaner(niter=4, pipeline=request.param)
    yield c
    c.close()


@pytest.mark.parametrize("w,h", SIZES)
def test_stage_maps_match_oracle(w, h):
    """One iteration with every intermediate map exported: bit-identical to the FP32 oracle,
    within tolerance of the FP64 oracle."""
    cl1 = Cleaner(niter=1)
    img = scene(w, h, seed=w * 1000 + h)
    J, M, maps = cl1.iterate(dev(img), None, maps=True)
    cl1.sync()
    J, M = host(J), host(M)
    gm = {k: host(v) for k, v in maps.items()}
    P = params_of({})
    r32 = oracle.iterate(img, None, P, precision="f32", maps=True)
    r64 = oracle.iterate(img, None, P, precision="f64", maps=True, fragile=True)
    lazy = ("f", "r")  # computed only where S' > sigclip
    both = (gm["sprime"] > 4.5) & (r32.maps["sprime"] > 4.5)
    for name in oracle.MAP_NAMES:
        g, o = gm[name], r32.maps[name]
        if name in lazy:
            assert np.array_equal(g[both], o[both]), name
        else:
            assert np.array_equal(g, o.astype(np.float32)), name
    assert np.array_equal(M, r32.Mk) and np.array_equal(J, r32.Ik)
    floors = map_floors(img, r64.maps)
    for name in ("m5", "lplus", "noise", "s", "sprime", "m3"):
        assert_map_close(gm[name], r64.maps[name], name, floors[name])
    both64 = (gm["sprime"] > 4.5) & (r64.maps["sprime"] > 4.5)
    for name in lazy:
        assert_map_close(gm[name][both64], r64.maps[name][both64], name, floors[name][both64])
    ok = r64.fragile == 0
    assert np.array_equal(M[ok], r64.Mk[ok])


def test_lockstep_iterations(cl):
    """Each GPU iteration fed the oracle's state (J, M_{k-1}) reproduces the oracle's next state."""
    img = workloads.make(workloads.single_800())
    P = params_of({})
    c1 = Cleaner(niter=1)
    J, M = img, np.zeros(img.shape, np.uint8)
    for k in range(4):
        r = oracle.iterate(J, M, P, precision="f32")
        gJ, gM, _ = c1.iterate(dev(J), dev(M))
        c1.sync()
        assert np.array_equal(host(gM), r.Mk), f"iteration {k + 1} mask"
        assert np.array_equal(host(gJ), r.Ik), f"iteration {k + 1} image"
        assert c1.last_counts()[0] == (r.n_new, r.n_none_left)
        J, M = r.Ik, r.Mk


def test_end_to_end_800(cl):
    """The 800x800 workload, niter=4, end to end: exact vs FP32 oracle, tolerance vs FP64."""
    img = workloads.make(workloads.single_800())
    out, mask = gpu_clean(cl, img)
    P = params_of({})
    r32 = oracle.clean(img, P, 4, precision="f32")
    assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean)
    counts = cl.last_counts()
    assert [c[0] for c in counts] == r32.n_new and [c[1] for c in counts] == r32.n_none_left
    r64 = oracle.clean(img, P, 4, fragile=True)
    flips, nfragile = assert_clean_matches_f64(out, mask, r64, "800x800")
    print(f"800x800: mask flips vs FP64 {flips}, fragile pixels {nfragile}, flagged {int(mask.sum())}")


PATHS = [dict(pipeline="queue"), dict(pipeline="tile", fusion=True), dict(pipeline="tile", fusion=False),
         dict(pipeline="tile", fuse2=True)]
PATH_IDS = ["queue", "tile-fused", "tile-two-launch", "tile-two-iterations"]


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("w,h", SIZES)
@pytest.mark.parametrize("niter", [1, 2, 3, 4])
def test_clean_sizes(w, h, niter, path):
    img = scene(w, h, seed=7 * w + h)
    c = Cleaner(niter=niter, **path)
    out, mask = gpu_clean(c, img)
    r32 = oracle.clean(img, params_of({}), niter, precision="f32")
    assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean)


def test_flags_across_strip_and_word_edges():
    """Cosmic-ray hits planted on both sides of the edges of 32-px words and of the column kernels'
    strips (32 words = 1024 px wide, 16 rows high), at the frame's borders and in a ragged last strip
    in both directions: the queue pipeline is bit-identical to the FP32 oracle at every niter, and
    the hits are flagged."""
    w, h = 2080, 50
    img = scene(w, h, seed=5)
    rng = np.random.default_rng(11)
    xs = [0, 1, 31, 32, 1022, 1023, 1024, 1025, 2046, 2047, 2048, 2079]
    ys = [0, 1, 15, 16, 31, 32, 47, 48, 49]
    for x in xs:
        for y in ys:
            img[y, x] += np.float32(rng.uniform(500.0, 3000.0))
    for niter in (1, 2, 4):
        out, mask = gpu_clean(Cleaner(niter=niter, pipeline="queue"), img)
        r32 = oracle.clean(img, params_of({}), niter, precision="f32")
        assert mask[np.ix_(ys, xs)].mean() > 0.5
        assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean), niter


def test_niter_zero_copies():
    img = scene(50, 40)
    c = Cleaner(niter=0)
    out, mask = gpu_clean(c, img)
    assert np.array_equal(out, img) and not mask.any()


@pytest.mark.parametrize("pipeline", ["queue", "tile"])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("pset", [dict(), dict(gain=1.5, readnoise=9.0, sigclip=5.0, sigfrac=0.3, objlim=4.0),
                                  dict(sigclip=3.0, sigfrac=1.6, objlim=0.5)])
def test_parameters_and_objlim_forms(form, pset, pipeline):
    img = scene(160, 120, seed=3)
    kw = dict(pset, objlim_form=form)
    c = Cleaner(niter=4, pipeline=pipeline, **kw)
    out, mask = gpu_clean(c, img)
    r32 = oracle.clean(img, params_of(kw), 4, precision="f32")
    assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean)


@pytest.mark.parametrize("fusion", [True, False], ids=["fused", "two-launch"])
@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5])
def test_tile_shapes_agree(shape, fusion):
    img = scene(300, 230, seed=11)
    ref = oracle.clean(img, params_of({}), 4, precision="f32")
    c = Cleaner(niter=4, tile_shape=shape, fusion=fusion, pipeline="tile")
    out, mask = gpu_clean(c, img)
    assert np.array_equal(mask, ref.mask) and np.array_equal(out, ref.clean)


def test_batch_equals_single(cl):
    """Uneven frames with per-frame gain/read noise in one batched call equal per-frame calls."""
    rng = np.random.default_rng(1)
    sizes = [(800, 800), (97, 211), (1024, 64), (1, 5), (333, 333), (64, 1)]
    imgs = [synth.frame(w, h, seed=5, index=i) for i, (w, h) in enumerate(sizes)]
    gains = [float(np.float32(rng.uniform(1, 7))) for _ in sizes]
    rns = [float(np.float32(rng.uniform(3, 10))) for _ in sizes]
    outs, masks = cl.clean_batch([dev(a) for a in imgs], gains, rns)
    cl.sync()
    for i, a in enumerate(imgs):
        ci = Cleaner(gain=gains[i], readnoise=rns[i], niter=4, pipeline="queue")
        o, m = gpu_clean(ci, a)
        assert np.array_equal(host(outs[i]), o) and np.array_equal(host(masks[i]), m), i
        if a.size <= 400_000:
            r32 = oracle.clean(a, params_of(dict(gain=gains[i], readnoise=rns[i])), 4, precision="f32")
            assert np.array_equal(m, r32.mask) and np.array_equal(o, r32.clean)


def test_repeated_calls_deterministic(cl):
    img = scene(257, 129, seed=2)
    a = gpu_clean(cl, img)
    b = gpu_clean(cl, img)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_alias_and_invalid_sizes_rejected(cl):
    import paper_1008_2192_gb300._lib as L
    t = dev(scene(40, 30))
    with pytest.raises(L.CrbError) as e:
        cl.clean_into(t, t, torch.empty((30, 40), dtype=torch.uint8, device="cuda"))
    assert e.value.status == L.CRB_EALIAS
    lib = L.load()
    import ctypes
    o = torch.empty_like(t)
    m = torch.empty(t.shape, dtype=torch.uint8, device="cuda")
    for (w, h) in ((0, 30), (40, 0), (-1, 30)):
        rc = lib.crb_clean(cl.handle, ctypes.c_void_p(t.data_ptr()), w, h, ctypes.c_void_p(o.data_ptr()),
                           ctypes.c_void_p(m.data_ptr()), None)
        assert rc == L.CRB_EINVAL
    rc = lib.crb_clean(cl.handle, ctypes.c_void_p(t.data_ptr()), 40, 30, None, ctypes.c_void_p(m.data_ptr()), None)
    assert rc == L.CRB_EINVAL


def _check_crops(img, out, mask, niter, crops, P, what=""):
    """Oracle on crops with 8*niter context (exact by the dependency radius) vs the GPU full frame:
    bit-identical to the FP32 oracle; against FP64, mask flips only on fragile pixels and cleaned
    values within tolerance. Returns (flips, fragile pixels) summed over the crops."""
    ctx = 8 * niter
    flips = fragile = 0
    for (y0, x0, hh, ww) in crops:
        c, sl = crop_with_context(img, y0, x0, hh, ww, ctx)
        go, gm = out[y0:y0 + hh, x0:x0 + ww], mask[y0:y0 + hh, x0:x0 + ww]
        r = oracle.clean(c, P, niter, precision="f32")
        assert np.array_equal(r.mask[sl], gm), (y0, x0)
        assert np.array_equal(r.clean[sl], go), (y0, x0)
        r64 = oracle.clean(c, P, niter, fragile=True)
        a, b = compare_f64(go, gm, r64.clean[sl], r64.mask[sl], r64.fragile[sl], f"{what} crop {(y0, x0)}")
        flips += a
        fragile += b
    print(f"{what}: {len(crops)} crops, mask flips vs FP64 {flips}, fragile pixels {fragile}")
    return flips, fragile


def test_4096_sampled_crops():
    """The 4096x4096 workload: the full GPU run against the oracle on 256x256 crops."""
    rec = workloads.single_4096()
    img = workloads.make(rec)
    c = Cleaner(gain=rec["gain"], readnoise=rec["readnoise"], niter=4)
    out, mask = gpu_clean(c, img)
    rng = np.random.default_rng(0)
    crops = [(0, 0, 256, 256), (0, 3840, 256, 256), (3840, 0, 256, 256), (3840, 3840, 256, 256)]
    crops += [(int(rng.integers(0, 3840)), int(rng.integers(0, 3840)), 256, 256) for _ in range(6)]
    _check_crops(img, out, mask, 4, crops, params_of(rec), "4096x4096")


def test_mosaic_16384_sampled_crops():
    """The 16384x16384 mosaic (1 GiB) in one call; 512x512 crops: corners, edge midpoints, random."""
    rec = workloads.mosaic_16384()
    img = workloads.make(rec)
    c = Cleaner(gain=rec["gain"], readnoise=rec["readnoise"], niter=4)
    out, mask = gpu_clean(c, img)
    S, n = 16384, 512
    crops = [(0, 0), (0, S - n), (S - n, 0), (S - n, S - n), (0, S // 2), (S // 2, 0), (S - n, S // 2),
             (S // 2, S - n)]
    rng = np.random.default_rng(4)
    crops += [(int(rng.integers(0, S - n)), int(rng.integers(0, S - n))) for _ in range(8)]
    _check_crops(img, out, mask, 4, [(y, x, n, n) for (y, x) in crops], params_of(rec), "16384x16384")


def test_batch_size_classes_f64():
    """One frame of each size class of the 64-frame batch (800^2, 1024^2, 2048x4096, 4096^2), with its
    per-frame gain and read noise, cleaned in one batched call: 256x256 crops (corners and random
    ones) against the FP32 oracle (bit-identical) and the FP64 oracle (flips only on fragile pixels)."""
    recs = [workloads.batch_64()[i] for i in (0, 16, 32, 48)]
    imgs = [workloads.make(r) for r in recs]
    c = Cleaner(niter=4)
    outs, masks = c.clean_batch([dev(a) for a in imgs], [r["gain"] for r in recs], [r["readnoise"] for r in recs])
    c.sync()
    rng = np.random.default_rng(6)
    for rec, img, o, m in zip(recs, imgs, outs, masks):
        H, W = img.shape
        n = 256
        crops = [(0, 0, n, n), (H - n, W - n, n, n)]
        crops += [(int(rng.integers(0, H - n)), int(rng.integers(0, W - n)), n, n) for _ in range(4)]
        _check_crops(img, host(o), host(m), 4, crops, params_of(rec), f"{W}x{H} gain {rec['gain']:.2f}")


@pytest.mark.parametrize("pipeline", ["queue", "tile"])
@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("shape", [0, -1])
def test_graphs_and_autotune(graphs, shape, pipeline):
    """Graph replay and autotuned tile shapes give the plain path's results, call after call."""
    c = Cleaner(niter=4, use_graphs=graphs, tile_shape=shape, pipeline=pipeline)
    for seed in range(3):
        img = scene(333, 251, seed=40 + seed)
        out, mask = gpu_clean(c, img)
        r32 = oracle.clean(img, params_of({}), 4, precision="f32")
        assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean), seed
    imgs = [scene(200, 150, seed=50 + i) for i in range(3)] + [scene(97, 400, seed=60)]
    for rep in range(2):
        outs, masks = c.clean_batch([dev(a) for a in imgs])
        c.sync()
        for a, o, m in zip(imgs, outs, masks):
            r32 = oracle.clean(a, params_of({}), 4, precision="f32")
            assert np.array_equal(host(m), r32.mask) and np.array_equal(host(o), r32.clean)


@pytest.mark.parametrize("niter", [1, 2, 4])
def test_launch_counts(niter):
    """crb_last_launches reports the kernels a call enqueues: 1 descriptor upload + 11 + 14 (niter - 1) + 1
    on the queue pipeline, plus the segment list of each iteration from the third on, and 1 upload +
    niter + 1 on the fused tile pipeline."""
    img = scene(120, 90, seed=9)
    cq = Cleaner(niter=niter, pipeline="queue")
    gpu_clean(cq, img)
    assert cq.last_launches() == 1 + 11 + 14 * (niter - 1) + max(0, niter - 2) + 1
    ct = Cleaner(niter=niter, pipeline="tile")
    gpu_clean(ct, img)
    assert ct.last_launches() == 1 + niter + 1
    ca = Cleaner(niter=niter)  # automatic: tiles for a frame this small
    gpu_clean(ca, img)
    assert ca.last_launches() == 1 + niter + 1


def test_auto_takes_the_queue_pipeline_for_large_calls():
    """From 6,000,000 pixels per call the automatic choice is the queue pipeline (57 launches at niter 4)."""
    img = synth.frame(2048, 3072, seed=3)
    ca = Cleaner(niter=4)
    out, mask = gpu_clean(ca, img)
    assert ca.last_launches() == 1 + 11 + 14 * 3 + 2 + 1
    ct = Cleaner(niter=4, pipeline="tile")
    o2, m2 = gpu_clean(ct, img)
    assert np.array_equal(out, o2) and np.array_equal(mask, m2)


@pytest.mark.parametrize("pipeline", ["queue", "auto"])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_batch_host_equals_device_batch(pinned, pipeline):
    """crb_clean_batch_host (host buffers, chunked copies overlapping the cleans) gives crb_clean_batch's
    results, call after call (the staging slots are reused)."""
    rng = np.random.default_rng(3)
    sizes = [(300, 200), (64, 1), (517, 333), (1, 40), (256, 256), (800, 600), (33, 97), (1024, 512), (90, 90)]
    c_dev = Cleaner(niter=4, pipeline=pipeline)
    c_host = Cleaner(niter=4, pipeline=pipeline)
    for rep in range(2):
        imgs = [synth.frame(w, h, seed=20 + rep, index=i) for i, (w, h) in enumerate(sizes)]
        gains = [float(np.float32(rng.uniform(1, 7))) for _ in sizes]
        rns = [float(np.float32(rng.uniform(3, 10))) for _ in sizes]
        outs, masks = c_dev.clean_batch([dev(a) for a in imgs], gains, rns)
        c_dev.sync()
        h_imgs = [torch.from_numpy(a) for a in imgs]
        h_outs = [torch.empty(a.shape, dtype=torch.float32) for a in imgs]
        h_masks = [torch.empty(a.shape, dtype=torch.uint8) for a in imgs]
        if pinned:
            h_imgs = [t.pin_memory() for t in h_imgs]
            h_outs = [t.pin_memory() for t in h_outs]
            h_masks = [t.pin_memory() for t in h_masks]
        c_host.clean_batch_host_into(h_imgs, h_outs, h_masks, gains, rns)
        torch.cuda.synchronize()
        for i in range(len(sizes)):
            assert np.array_equal(h_outs[i].numpy(), host(outs[i])), (rep, i)
            assert np.array_equal(h_masks[i].numpy(), host(masks[i])), (rep, i)


@pytest.mark.parametrize("graphs", [False, True])
def test_queue_autotune(graphs):
    """The queue-pipeline autotuner (occupancies, segment-list start, queue or tile) changes no result:
    call after call (the first tunes, the later ones reuse the choice, replayed from a graph or not),
    on a single 2048x3072 frame and on an uneven batch, the outputs stay bit-identical to the FP32
    oracle; the reported configuration is a valid one."""
    c = Cleaner(niter=4, autotune=True, use_graphs=graphs)
    img = synth.frame(2048, 3072, seed=13)
    r32 = oracle.clean(img, params_of({}), 4, precision="f32")
    for rep in range(3):
        out, mask = gpu_clean(c, img)
        assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean), rep
    occ, seg_from, pipeline = c.tuned_config()
    assert pipeline in ("tile", "queue") and 2 <= seg_from <= 5
    if pipeline == "queue":
        assert all(v >= 1 for v in occ.values()), occ
    print(f"2048x3072: {pipeline}, segment lists from iteration {seg_from}, blocks per SM {occ}")
    sizes = [(800, 800), (1024, 1024), (2048, 1024), (97, 211), (3000, 2500)]
    imgs = [synth.frame(w, h, seed=31, index=i) for i, (w, h) in enumerate(sizes)]
    refs = [oracle.clean(a, params_of({}), 4, precision="f32") for a in imgs[:4]]
    plain = Cleaner(niter=4, pipeline="queue")
    p_outs, p_masks = plain.clean_batch([dev(a) for a in imgs])
    plain.sync()
    for rep in range(2):
        outs, masks = c.clean_batch([dev(a) for a in imgs])
        c.sync()
        for i in range(len(imgs)):
            assert torch.equal(outs[i], p_outs[i]) and torch.equal(masks[i], p_masks[i]), (rep, i)
            if i < 4:
                assert np.array_equal(host(masks[i]), refs[i].mask) and np.array_equal(host(outs[i]), refs[i].clean)
    assert c.tuned_config()[2] == "queue"  # 12.6 Mpix: the tile pipeline is slower


def test_bounded_wait_reports_timeout():
    """A device-side wait that runs out (on a barrier nothing completes, as a TMA wait would if its box
    never landed) records CRB_ETIMEOUT in the context's status without faulting; crb_sync_status reports
    it once, and the context keeps cleaning correctly."""
    import ctypes
    import paper_1008_2192_gb300._lib as L
    c = Cleaner(niter=2, pipeline="tile")
    lib = L.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.crb_selftest_wait_timeout(c.handle, 1000, s) == L.CRB_OK
    assert lib.crb_sync_status(c.handle, s) == L.CRB_ETIMEOUT
    assert b"bounded device-side wait" in lib.crb_last_error()
    assert lib.crb_sync_status(c.handle, s) == L.CRB_OK  # reported once
    img = scene(256, 200, seed=17)
    out, mask = gpu_clean(c, img)
    r32 = oracle.clean(img, params_of({}), 2, precision="f32")
    assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean)
    assert lib.crb_selftest_wait_timeout(c.handle, 0, s) == L.CRB_EINVAL



@pytest.mark.parametrize("niter", [3, 4, 5, 6])
def test_two_iteration_fusion(niter):
    """Iterations 2 and 3 in one launch (halo recompute over the widened tile): bit-identical to the FP32
    oracle on the 800x800 workload and on an uneven batch (frame edges, ragged tiles, widths off the
    16-byte boundary), with one launch fewer."""
    img = workloads.make(workloads.single_800())
    c = Cleaner(niter=niter, pipeline="tile", fuse2=True)
    out, mask = gpu_clean(c, img)
    r32 = oracle.clean(img, params_of({}), niter, precision="f32")
    assert np.array_equal(mask, r32.mask) and np.array_equal(out, r32.clean)
    assert [n for n, _ in c.last_counts()] == r32.n_new
    assert c.last_launches() == 1 + niter + 1 - 1
    sizes = [(333, 251), (64, 16), (65, 17), (200, 150), (1, 40), (97, 300)]
    imgs = [scene(w, h, seed=70 + i) for i, (w, h) in enumerate(sizes)]
    outs, masks = c.clean_batch([dev(a) for a in imgs])
    c.sync()
    for a, o, m in zip(imgs, outs, masks):
        r = oracle.clean(a, params_of({}), niter, precision="f32")
        assert np.array_equal(host(m), r.mask) and np.array_equal(host(o), r.clean), a.shape
