"""Host-side serving logic without a GPU: the memory arena's admission
policy and the camera stand-in's arrivals and injected faults."""
import random
import time

import pytest

from paper_2211_00645_gb300.serve import Camera, DeviceArena, PinnedRing, percentile


def test_arena_first_fit_and_coalesce():
    a = DeviceArena(4096, align=256)
    x = a.alloc(1000)          # 1024
    y = a.alloc(256)
    z = a.alloc(2000)          # 2048
    assert (x, y, z) == (0, 1024, 1280)
    assert a.alloc(1024) is None          # 768 left
    a.free(y)
    assert a.alloc(800) is None           # 256-byte hole + 768 tail, neither fits 1024
    a.free(x)
    assert a.alloc(1200) == 0             # hole coalesced to 1280
    a.free(0)
    a.free(z)
    assert a.in_use == 0 and a.alloc(4096) == 0


def test_arena_never_exceeds_budget_random():
    rng = random.Random(3)
    a = DeviceArena(1 << 20, align=256)
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.45:
            a.free(live.pop(rng.randrange(len(live))))
        else:
            off = a.alloc(rng.randint(1, 200_000))
            if off is not None:
                live.append(off)
        assert a.in_use <= a.budget
        spans = sorted((o, a._used[o]) for o in a._used)
        for (o1, s1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2                      # no overlap
    for off in live:
        a.free(off)
    assert a._free == [(0, a.budget)]


def _ring(nbytes):
    return PinnedRing(nbytes, pin=False, fill=lambda out, seed: out.fill(seed & 0xFF))


def test_ring_wraps_in_order_and_respects_refs():
    r = _ring(4096)
    a = r.acquire(1000)                # [0, 1024)
    b = r.acquire(2000, refs=2)        # [1024, 3072)
    c = r.acquire(900)                 # [3072, 3968)
    assert (a, b, c) == (0, 1024, 3072)
    with pytest.raises(TimeoutError):
        r.acquire(300, timeout=0.01)   # 128 left at the end, nothing before the tail
    r.release(b)                       # one of two refs: tail still at a
    r.release(a)                       # tail -> b (still referenced)
    with pytest.raises(TimeoutError):
        r.acquire(1100, timeout=0.01)  # [0, 1024) free but 1100 > 1024
    assert r.acquire(1000) == 0        # wraps before the tail
    r.release(b)                       # tail -> c
    with pytest.raises(TimeoutError):
        r.acquire(2100, timeout=0.01)  # only [1024, 3072) between head and tail
    d = r.acquire(2048)
    assert d == 1024 and r.in_use() == 4096
    for off in (c, 0, d):
        r.release(off)
    assert r.in_use() == 0 and r.acquire(4096) == 0
    with pytest.raises(ValueError):
        r.acquire(5000)
    with pytest.raises(KeyError):
        r.release(12345)


def test_ring_backpressure_blocks_until_release():
    import threading
    r = _ring(2048)
    a = r.acquire(2048)
    got = []
    t = threading.Thread(target=lambda: got.append(r.acquire(1024, timeout=10)))
    t.start()
    time.sleep(0.05)
    assert not got and r.stalls == 1
    r.release(a)
    t.join(timeout=10)
    assert got == [0]


def test_ring_view_shares_host_bytes():
    import torch
    r = PinnedRing(1 << 16, pin=False, seed=5)
    off = r.acquire(2 * 4 * 8 * 16)
    v = r.view(off, (4, 8, 16))
    assert v.dtype == torch.uint16 and tuple(v.shape) == (4, 8, 16)
    assert int(v.view(torch.int16).ne(0).sum()) > 0      # filled with stack tiles


class _Sink:
    def __init__(self, ring):
        self.got = []
        self.ring = ring

    def submit(self, req):
        self.got.append(req)
        req.release_host()


def test_camera_faults_and_rate():
    shapes = [(10, 8, 8, 2), (20, 8, 8, 2)]
    ring = _ring(1 << 14)
    sink = _Sink(ring)
    cam = Camera(sink, ring, shapes, n=40, rate=2000.0, seed=1, drop={3, 7}, duplicate={5}, delay_s={9: 0.01})
    cam.start()
    cam.join(timeout=30)
    assert not cam.is_alive() and cam.error is None
    assert len(sink.got) == cam.expected() == 40 - 2 + 1
    assert [q.rid for q in sink.got] == list(range(len(sink.got)))
    dup = [q for q in sink.got if q.ring_off == sink.got[5].ring_off and q.host is not None]
    assert ring.in_use() == 0
    arrivals = [q.t_arrival for q in sink.got]
    span = max(arrivals) - min(arrivals)
    assert 0.005 < span < 5.0
    assert dup


def test_camera_stall_counts_as_lag():
    """Arrival times are the scheduled ones, not the publication times, so a
    slow consumer's delay before publication counts as latency."""
    shapes = [(10, 8, 8, 2)]
    ring = _ring(2 * 10 * 8 * 16)
    got = []

    class Slow:
        def submit(self, req):
            got.append(req)
            time.sleep(0.02)
            req.release_host()

    cam = Camera(Slow(), ring, shapes, n=5, rate=None)
    cam.start()
    cam.join(timeout=30)
    assert len(got) == 5 and cam.error is None
    assert all(q.t_arrival == got[0].t_arrival for q in got)   # all scheduled at t0


def test_percentile_helper():
    assert percentile([], 50) is None
    assert percentile([1.0, 2.0, 3.0], 50) == 2.0


def test_camera_streams_frames_before_completion():
    """With a frame rate and streaming on, a request is published with its
    first frames, well before its stack is complete; its ready-frame count
    only grows, in whole chunks, and reaches nscan at the arrival time."""
    import threading
    shapes = [(40, 8, 8, 2), (24, 8, 8, 1)]
    ring = _ring(1 << 16)
    got, seen = [], []

    class Rec:
        def submit(self, req):
            got.append((time.perf_counter(), req.frames_ready, req))

    cam = Camera(Rec(), ring, shapes, n=6, rate=50.0, seed=2, fps=2000.0, stream_frames=True, chunk_frames=8)
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            for _, _, r in list(got):
                seen.append((r.rid, r.nscan, r.frames_ready))
            time.sleep(0.0002)

    w = threading.Thread(target=watch)
    w.start()
    cam.start()
    cam.join(timeout=30)
    stop.set()
    w.join()
    assert cam.error is None and len(got) == 6
    for t_sub, fr0, r in got:
        assert fr0 == 0 and t_sub < r.t_arrival - 0.5 * r.nscan / 2000.0
        assert r.frames_ready == r.nscan
        r.release_host()
    last = {}
    for rid, nscan, f in seen:
        assert f >= last.get(rid, 0)
        last[rid] = f
        assert f == nscan or f % 8 == 0
    assert max(last.values()) > 0 and ring.in_use() == 0


def test_camera_frame_rate_without_streaming_submits_complete_stacks():
    shapes = [(30, 8, 8, 2)]
    ring = _ring(1 << 16)
    got = []

    class Rec:
        def submit(self, req):
            got.append((time.perf_counter(), req.frames_ready, req))
            req.release_host()

    cam = Camera(Rec(), ring, shapes, n=4, rate=100.0, seed=3, fps=3000.0)
    cam.start()
    cam.join(timeout=30)
    assert cam.error is None and len(got) == 4
    for t_sub, fr, r in got:
        assert fr == r.nscan and t_sub >= r.t_arrival
