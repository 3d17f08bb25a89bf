"""Live-view serving loop: stacks written into a pinned ring, admitted by a
device-memory budget, batched into persistent launches while earlier ticks
copy in and out.  Every served request must equal the plain
one-request-at-a-time path on the same host bytes bit for bit, the arena must
stay inside its budget, and host-side faults (dropped, duplicated and late
frames, an oversize stack) must not disturb the other requests."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEOM = (35.0, 0.3, 0.1)
SHAPES = [(50, 64, 128, 2), (100, 128, 256, 2), (50, 256, 128, 1), (150, 64, 512, 2), (40, 72, 136, 3)]


@pytest.fixture(scope="module")
def ring(lib):
    from paper_2211_00645_gb300.serve import PinnedRing
    return PinnedRing(64 << 20, seed=7)


def _check_results(reqs):
    """Re-serves each distinct (ring range, shape) on the plain path: the
    ring's bytes are written once, so they still hold what was served."""
    from paper_2211_00645_gb300.serve import PlainServer, PlanCache, Request
    plain = PlainServer(PlanCache(*GEOM), result_bytes=64 << 20)
    ref = {}
    for req in reqs:
        key = (req.host.data_ptr(), tuple(req.host.shape), req.channels, req.geometry)
        if key not in ref:
            plain._serve(Request(req.rid, req.nscan, req.nrows, req.ncols, req.channels, req.host,
                                 geometry=req.geometry))
            ref[key] = plain.done[-1].results
        want = ref[key]
        assert len(req.results) == len(want) == req.channels
        for got, w in zip(req.results, want):
            assert torch.equal(got["zmip"], w["zmip"]), f"request {req.rid} zmip"
            assert torch.equal(got["ymip"], w["ymip"]), f"request {req.rid} ymip"


def _run(ring, n, budget, rate=None, **cam):
    from paper_2211_00645_gb300.serve import Camera, LiveViewServer, PlanCache
    srv = LiveViewServer(PlanCache(*GEOM), budget, max_items=16, max_units=1 << 16, result_bytes=64 << 20)
    camera = Camera(srv, ring, SHAPES, n, rate, seed=3, **cam)
    camera.start()
    srv.run(camera.expected(), timeout_s=120)
    camera.join(timeout=30)
    assert camera.error is None
    torch.cuda.synchronize()
    assert ring.in_use() == 0
    return srv, camera


def test_saturated_batches_equal_plain_path(ring):
    srv, cam = _run(ring, 30, budget=256 << 20)
    assert len(srv.done) == 30 and not srv.rejected
    assert max(srv.batch_sizes) > 1                      # continuous batching happened
    assert srv.peak_in_use <= srv.arena.budget
    assert srv.arena.in_use == 0 and not srv.resident
    _check_results(srv.done)


def test_tight_budget_waits_for_memory(ring):
    from paper_2211_00645_gb300.serve import PlanCache, request_bytes
    pc = PlanCache(*GEOM)
    big = max(request_bytes(pc.get(n, r, c), C) for (n, r, c, C) in SHAPES)
    srv, _ = _run(ring, 20, budget=big + big // 2)
    assert len(srv.done) == 20
    assert srv.peak_in_use <= srv.arena.budget
    _check_results(srv.done)


def test_small_ring_backpressure(lib):
    """A ring that holds about two stacks stalls the camera; every stack is
    still served correctly."""
    from paper_2211_00645_gb300.serve import PinnedRing
    small = PinnedRing(2 * 150 * 64 * 1024 * 2 + 4096, seed=9)
    srv, _ = _run(small, 20, budget=256 << 20)
    assert len(srv.done) == 20 and small.stalls > 0
    _check_results(srv.done)


def test_paced_arrivals_with_host_faults(ring):
    srv, cam = _run(ring, 25, budget=256 << 20, rate=400.0,
                    drop={2, 11}, duplicate={4, 20}, delay_s={6: 0.02, 7: 0.0})
    assert len(srv.done) == cam.expected() == 25
    assert sorted(r.rid for r in srv.done) == list(range(25))
    _check_results(srv.done)
    assert all(r.latency_ms > 0 for r in srv.done)


def test_oversize_request_is_rejected_others_served(ring):
    from paper_2211_00645_gb300.serve import LiveViewServer, PlanCache, Request, request_bytes
    pc = PlanCache(*GEOM)
    big = max(request_bytes(pc.get(n, r, c), C) for (n, r, c, C) in SHAPES)
    srv = LiveViewServer(pc, big + 4096, max_items=16, max_units=1 << 16, result_bytes=64 << 20)
    huge = Request(99, 400, 512, 512, 2, torch.empty((400, 512, 1024), dtype=torch.uint16))
    srv.submit(huge)
    reqs = []
    for i, (n, r, c, C) in enumerate(SHAPES):
        off = ring.acquire(2 * n * r * c * C, timeout=5)
        reqs.append(Request(i, n, r, c, C, ring.view(off, (n, r, c * C)), ring=ring, ring_off=off))
        srv.submit(reqs[-1])
    srv.run(len(SHAPES) + 1, timeout_s=60)
    torch.cuda.synchronize()
    assert [r.rid for r in srv.rejected] == [99] and "budget" in huge.error
    assert len(srv.done) == len(SHAPES) and ring.in_use() == 0
    _check_results(srv.done)


def test_results_released_back_to_the_arena(ring):
    """Without keep_results the pinned read-back space is reused: a small
    result arena serves many more requests than it holds at once."""
    from paper_2211_00645_gb300.serve import Camera, LiveViewServer, PlanCache, result_bytes
    pc = PlanCache(*GEOM)
    most = max(result_bytes(pc.get(n, r, c), C) for (n, r, c, C) in SHAPES)
    srv = LiveViewServer(pc, 256 << 20, max_items=16, max_units=1 << 16, keep_results=False,
                         result_bytes=2 * most + 4096)
    cam = Camera(srv, ring, SHAPES, 30, None, seed=4)
    cam.start()
    srv.run(cam.expected(), timeout_s=120)
    cam.join(timeout=30)
    torch.cuda.synchronize()
    assert len(srv.done) == 30 and srv.results.in_use == 0
    assert all(r.results is None for r in srv.done)


def test_cancel_queued_request(ring):
    """A request still waiting for memory can be withdrawn; the others are
    served and its ring range is returned."""
    from paper_2211_00645_gb300.serve import LiveViewServer, PlanCache, Request, request_bytes
    pc = PlanCache(*GEOM)
    big = max(request_bytes(pc.get(n, r, c), C) for (n, r, c, C) in SHAPES)
    srv = LiveViewServer(pc, big + 4096, max_items=16, max_units=1 << 16, result_bytes=64 << 20)
    reqs = []
    for i, (n, r, c, C) in enumerate(SHAPES + SHAPES[:2]):      # about 55 MB: fits the 64 MB ring
        off = ring.acquire(2 * n * r * c * C, timeout=5)
        reqs.append(Request(i, n, r, c, C, ring.view(off, (n, r, c * C)), ring=ring, ring_off=off))
        srv.submit(reqs[-1])
    srv._admit()                      # the budget holds about one request: the rest queue
    assert srv.waiting, "expected queued requests"
    victim = srv.waiting[-1].rid
    assert srv.cancel(victim) and not srv.cancel(victim) and not srv.cancel(12345)
    srv.run(len(reqs), timeout_s=60)
    torch.cuda.synchronize()
    assert [r.rid for r in srv.cancelled] == [victim]
    assert len(srv.done) == len(reqs) - 1 and ring.in_use() == 0
    _check_results(srv.done)


def test_plain_server_run_loop(ring):
    """The plain path's own run loop with a camera: every request served,
    results equal to the batched server's on the same bytes."""
    from paper_2211_00645_gb300.serve import Camera, PlainServer, PlanCache
    srv = PlainServer(PlanCache(*GEOM), result_bytes=64 << 20)
    cam = Camera(srv, ring, SHAPES, 12, 500.0, seed=8)
    cam.start()
    srv.run(cam.expected(), timeout_s=120)
    cam.join(timeout=30)
    assert cam.error is None and len(srv.done) == 12 and ring.in_use() == 0
    _check_results(srv.done)


@pytest.mark.parametrize("new_geom", [(45.0, 0.2, 0.115),   # fast kernels
                                      (35.0, 0.05, 0.1)])   # pixel > step: the general kernel
def test_geometry_change_while_serving(ring, new_geom):
    """New deskew parameters mid-stream: requests admitted before keep
    theirs, later ones use the new plans (batches may mix both, and items of
    the fast and the general kernel), and every result equals the plain path
    with the geometry it was served with."""
    from paper_2211_00645_gb300.serve import LiveViewServer, PlanCache, Request
    srv = LiveViewServer(PlanCache(*GEOM), 256 << 20, max_items=16, max_units=1 << 16, result_bytes=64 << 20)
    reqs = []

    def submit(i, shape):
        n, r, c, C = shape
        off = ring.acquire(2 * n * r * c * C, timeout=5)
        reqs.append(Request(i, n, r, c, C, ring.view(off, (n, r, c * C)), ring=ring, ring_off=off))
        srv.submit(reqs[-1])

    for i, shp in enumerate(SHAPES):
        submit(i, shp)
    for _ in range(20000):                        # admit the first five until their copies land
        srv.step()
        if all(r.ring is None for r in reqs):     # ring ranges returned
            break
    assert all(r.ring is None for r in reqs)
    srv.set_geometry(*new_geom)
    for i, shp in enumerate(SHAPES):
        submit(10 + i, shp)
    srv.run(len(reqs), timeout_s=60)
    torch.cuda.synchronize()
    assert len(srv.done) == len(reqs) and ring.in_use() == 0
    geos = {r.rid: r.geometry for r in srv.done}
    assert all(geos[i] == GEOM for i in range(5))
    assert all(geos[10 + i] == new_geom for i in range(5))
    _check_results(srv.done)


def test_streamed_frames_equal_plain_path(ring):
    """Frames copied to the device as the camera writes them (the projection
    runs once the stack is complete): every result equals the plain path,
    and requests were admitted while their stacks were still being
    acquired."""
    srv, cam = _run(ring, 24, budget=256 << 20, rate=300.0, fps=20000.0, stream_frames=True, chunk_frames=8,
                    drop={5}, duplicate={9})
    assert len(srv.done) == cam.expected() == 24
    assert sum(r.t_admit < r.t_arrival for r in srv.done) >= len(srv.done) // 2
    assert all(r.t_done > r.t_arrival for r in srv.done)
    _check_results(srv.done)
