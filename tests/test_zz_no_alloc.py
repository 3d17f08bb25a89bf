"""Allocation-free batched live view (``opm_batch_project_static``).

Collected last on purpose: it must give the same results whether or not
other tests ran before it in the process.  Two calls in a row are each
compared with the allocating batch path; repeated calls must leave the
device's free memory unchanged, and oversize requests must be refused."""
import numpy as np
import pytest

import opm_synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _items(lib, seed):
    items = []
    for i, shape in enumerate([(64, 128, 128, 30.0, 0.4, 0.115), (33, 50, 264, 45.0, 0.2, 0.115)]):
        n, r, c = shape[:3]
        R = opm_synth.raw_stack(opm_synth.StackConfig("s", n, r, c, *shape[3:], n_blobs=10, sigma=(1.0, 3.0),
                                                      amp=(200.0, 4000.0), seed=seed + i))
        plan = lib.Plan(*shape)
        items.append({"plan": plan, "raw": to_dev(R, torch),
                      "zmip": torch.full((plan.ny, plan.nx), -1.0, device="cuda"),
                      "ymip": torch.full((plan.nz, plan.nx), -1.0, device="cuda")})
    # two channels side by side in one frame stack: strided ROIs
    R2 = opm_synth.raw_stack(opm_synth.StackConfig("c", 40, 70, 272, 35.0, 0.3, 0.1, n_blobs=10, sigma=(1.0, 3.0),
                                                   amp=(200.0, 4000.0), seed=seed + 7))
    raw2 = to_dev(R2, torch)
    plan = lib.Plan(40, 70, 136, 35.0, 0.3, 0.1)
    for c in range(2):
        items.append({"plan": plan, "raw": raw2[:, :, 136 * c:], "row_pitch": 272, "plane_pitch": 70 * 272,
                      "zmip": torch.full((plan.ny, plan.nx), -1.0, device="cuda"),
                      "ymip": torch.full((plan.nz, plan.nx), -1.0, device="cuda") if c == 0 else None})
    return items


def _reference(lib, items):
    ref = [{"zmip": None if it["zmip"] is None else torch.full_like(it["zmip"], -2.0),
            "ymip": None if it["ymip"] is None else torch.full_like(it["ymip"], -2.0)} for it in items]
    b = lib.Batch(max_items=8)
    b.set([dict(it, zmip=r["zmip"], ymip=r["ymip"]) for it, r in zip(items, ref)])
    b.run()
    torch.cuda.synchronize()
    b.check()
    b.close()
    return ref


def _equal(items, ref):
    for it, r in zip(items, ref):
        for k in ("zmip", "ymip"):
            if it[k] is not None:
                assert torch.equal(it[k], r[k]), k


def test_two_calls_in_a_row_match_batch_path(lib):
    first, second = _items(lib, 100), _items(lib, 200)
    ref1, ref2 = _reference(lib, first), _reference(lib, second)
    lib.batch_project_static(first, check=True)
    lib.batch_project_static(second, check=True)        # rewrites the same static work list
    torch.cuda.synchronize()
    _equal(first, ref1)
    _equal(second, ref2)
    # and back to back on one stream without a check in between
    for it in first + second:
        for k in ("zmip", "ymip"):
            if it[k] is not None:
                it[k].fill_(-3.0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lib.batch_project_static(first, kchunk=32, ctas_per_sm=2, stream=s)
        lib.batch_project_static(second, stream=s)
    s.synchronize()
    _equal(first, ref1)
    _equal(second, ref2)


def test_no_device_memory_is_allocated(lib):
    items = _items(lib, 300)
    lib.batch_project_static(items, check=True)         # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for kc in (0, 16, 128):
        lib.batch_project_static(items, kchunk=kc)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_limits_are_enforced(lib):
    items = _items(lib, 400)
    with pytest.raises(lib.OpmError) as e:
        lib.batch_project_static(items * 17)             # 68 items > 64
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED and "limit of 64" in str(e.value)
    big = lib.Plan(400, 1024, 2048, 35.0, 0.3, 0.1)
    raw = torch.zeros(big.raw_shape, dtype=torch.uint16, device="cuda")
    z = torch.empty((big.ny, big.nx), device="cuda")
    with pytest.raises(lib.OpmError) as e:
        lib.batch_project_static([{"plan": big, "raw": raw, "zmip": z}] * 8, kchunk=16)
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED and "work units" in str(e.value)
    # a refused call launches nothing and leaves the next call correct
    ref = _reference(lib, items)
    lib.batch_project_static(items, check=True)
    _equal(items, ref)
    assert np.isfinite(items[0]["zmip"].cpu().numpy()).all()


def test_capture_is_refused(lib):
    """The call copies a process-wide host image with a pageable copy, which a
    graph cannot record: on a capturing stream it refuses and launches
    nothing, and the stream stays usable."""
    items = _items(lib, 500)
    ref = _reference(lib, items)
    lib.batch_project_static(items, check=True)          # set-up happens outside the capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(lib.OpmError) as e:
                lib.batch_project_static(items, stream=s)
        finally:
            g.capture_end()
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED and "captured" in str(e.value)
    for it in items:
        for k in ("zmip", "ymip"):
            if it[k] is not None:
                it[k].fill_(-4.0)
    lib.batch_project_static(items, stream=s)
    s.synchronize()
    _equal(items, ref)


def test_threads_on_one_stream(lib):
    """Two host threads call it at once on one stream: the shared host image
    is built and copied under a lock, and the kernels run in stream order, so
    each thread's results equal the allocating path's."""
    import threading
    sets = [_items(lib, 600), _items(lib, 700)]
    refs = [_reference(lib, it) for it in sets]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    errors = []

    def worker(items):
        try:
            for _ in range(20):
                lib.batch_project_static(items, stream=s)
        except Exception as exc:  # reported below
            errors.append(exc)

    ts = [threading.Thread(target=worker, args=(it,)) for it in sets]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    s.synchronize()
    assert not errors, errors
    for items, ref in zip(sets, refs):
        _equal(items, ref)
