"""Serving: continuous batching gives each frame the same result as cleaning it alone."""

import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1008_2192_gb300 import Cleaner, Server  # noqa: E402


def _frames(n, seed=0):
    rng = np.random.default_rng(seed)
    sizes = [(256, 256), (512, 384), (800, 800), (1024, 200), (97, 311), (2048, 1024)]
    out = []
    for i in range(n):
        w, h = sizes[i % len(sizes)]
        g = float(np.float32(rng.uniform(1, 7)))
        r = float(np.float32(rng.uniform(3, 10)))
        img = synth.frame(w, h, seed=seed, index=i, sky=100.0, gain=g, readnoise=r)
        out.append((torch.from_numpy(img).cuda(), g, r))
    return out


def test_served_results_equal_solo():
    frames = _frames(24)
    srv = Server(niter=4, budget_bytes=2 << 30, max_inflight=2, max_batch=5)
    outs = {}
    rng = np.random.default_rng(3)
    for i, (img, g, r) in enumerate(frames):
        o = torch.empty_like(img)
        m = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
        assert srv.submit(img, o, m, tag=i, gain=g, readnoise=r)
        outs[i] = (o, m)
        if i % 6 == 5:  # bursts of six arrivals while earlier waves run
            time.sleep(float(rng.uniform(0, 0.002)))
    done = {}
    t0 = time.time()
    while len(done) < len(frames) and time.time() - t0 < 60:
        for tag, lat, st in srv.poll(block_ms=100):
            assert st == 0 and lat >= 0
            done[tag] = lat
    assert len(done) == len(frames)
    st = srv.stats()
    assert st["done"] == len(frames) and st["resident_bytes"] == 0 and st["queued"] == 0
    assert st["waves"] >= 2 and st["max_wave"] >= 2, st  # batches formed and overlapped
    for i, (img, g, r) in enumerate(frames):
        c = Cleaner(gain=g, readnoise=r, niter=4)
        ro, rm = c.clean(img)
        c.sync()
        o, m = outs[i]
        assert torch.equal(o, ro) and torch.equal(m, rm), i
    srv.close()


def test_budget_admission():
    img = torch.from_numpy(synth.frame(512, 512, seed=1)).cuda()
    o = torch.empty_like(img)
    m = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    import paper_1008_2192_gb300._lib as L
    per_frame = L.load().crb_server_frame_bytes(512, 512)
    assert per_frame >= 512 * 512 * (9 + 32)
    small = Server(niter=2, budget_bytes=per_frame - 1, max_inflight=1, max_batch=4)
    with pytest.raises(L.CrbError) as e:  # more than the whole budget: never admissible, not busy
        small.submit(img, o, m, tag=1, gain=7.0, readnoise=5.0)
    assert e.value.status == L.CRB_EINVAL
    assert b"more than the whole budget" in L.load().crb_last_error()
    assert small.stats()["rejected"] == 0 and small.stats()["submitted"] == 0
    small.close()
    one = Server(niter=2, budget_bytes=per_frame, max_inflight=1, max_batch=4)
    assert one.submit(img, o, m, tag=7, gain=7.0, readnoise=5.0)
    # refused as busy while tag 7 is resident (admitted only if tag 7 already finished)
    o2, m2 = torch.empty_like(img), torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    second = one.submit(img, o2, m2, tag=9, gain=7.0, readnoise=5.0)
    assert one.stats()["rejected"] == (0 if second else 1)
    want = {7, 9} if second else {7}
    got = {}
    t0 = time.time()
    while len(got) < len(want) and time.time() - t0 < 30:
        got.update({t: st for t, _, st in one.poll(block_ms=100)})
    assert got == {t: 0 for t in want}
    assert one.stats()["resident_bytes"] == 0
    assert one.submit(img, o, m, tag=8, gain=7.0, readnoise=5.0)  # budget released
    t0 = time.time()
    got = []
    while not got and time.time() - t0 < 30:
        got = one.poll(block_ms=100)
    one.close()


def test_submit_not_held_up_by_a_wave_enqueue():
    """The worker enqueues a wave without holding the server's lock: while it enqueues the first wave of a
    fresh slot (which grows the slot's workspace and staging buffers, milliseconds of host work), further
    submissions return at once. The server records its longest wave enqueue and the longest time a
    submission waited for the lock."""
    big = torch.from_numpy(synth.frame(4096, 4096, seed=2)).cuda()
    small = torch.from_numpy(synth.frame(64, 64, seed=3)).cuda()
    srv = Server(niter=4, budget_bytes=8 << 30, max_inflight=1, max_batch=64)
    bufs = [(torch.empty_like(big), torch.empty(big.shape, dtype=torch.uint8, device="cuda"))]
    bufs += [(torch.empty_like(small), torch.empty(small.shape, dtype=torch.uint8, device="cuda"))
             for _ in range(400)]
    torch.cuda.synchronize()
    assert srv.submit(big, *bufs[0], tag=0, gain=7.0, readnoise=5.0)
    tag, t0 = 1, time.perf_counter()
    while time.perf_counter() - t0 < 0.2 and tag < len(bufs):  # submissions while the first wave is enqueued
        assert srv.submit(small, *bufs[tag], tag=tag, gain=7.0, readnoise=5.0)
        tag += 1
    done = set()
    t0 = time.time()
    while len(done) < tag and time.time() - t0 < 60:
        for t, lat, st in srv.poll(block_ms=100):
            assert st == 0
            done.add(t)
    assert len(done) == tag
    st = srv.stats()
    print(f"longest wave enqueue {st['max_enqueue_us']} us, longest submit wait {st['max_submit_wait_us']} us, "
          f"{tag} submissions, {st['waves']} waves")
    assert st["max_enqueue_us"] > 0
    if st["max_enqueue_us"] > 2000:  # a window in which a held lock would have shown
        assert st["max_submit_wait_us"] < st["max_enqueue_us"] / 4
    srv.close()
