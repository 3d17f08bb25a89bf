"""Batched live view: one persistent launch over stacks, channels (strided
ROIs of a shared frame stack) and ROIs of uneven sizes.  Every item's result
must equal its stand-alone opm_project result (same arithmetic, max-combined)
and the oracle; CUDA-graph replay must equal eager launches."""
import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import TOL, assert_between, assert_close, check_argz, nearest_bounds, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _stack(shape, seed):
    n, r, c = shape[:3]
    cfg = opm_synth.StackConfig("b", n, r, c, *shape[3:], n_blobs=10, sigma=(1.0, 3.0), amp=(200.0, 4000.0),
                                seed=seed)
    return opm_synth.raw_stack(cfg)


def _mixed(lib, seed=0):
    """Items: two stacks of different shapes and a 2-channel frame stack."""
    items, refs = [], []
    for i, shape in enumerate([(64, 128, 128, 30.0, 0.4, 0.115), (33, 50, 264, 45.0, 0.2, 0.115)]):
        R = _stack(shape, 10 + i + seed)
        plan = lib.Plan(*shape)
        raw = to_dev(R, torch)
        items.append({"plan": plan, "raw": raw,
                      "zmip": torch.full((plan.ny, plan.nx), -1.0, device="cuda"),
                      "ymip": torch.full((plan.nz, plan.nx), -1.0, device="cuda")})
        refs.append((shape, R))
    # two colour channels side by side in one camera frame: [n][r][2 * 136]
    ch = (40, 70, 136, 35.0, 0.3, 0.1)
    R2 = _stack((40, 70, 272, 35.0, 0.3, 0.1), 20 + seed)
    raw2 = to_dev(R2, torch)
    plan = lib.Plan(*ch)
    for c in range(2):
        items.append({"plan": plan, "raw": raw2[:, :, 136 * c:], "row_pitch": 272, "plane_pitch": 70 * 272,
                      "zmip": torch.full((plan.ny, plan.nx), -1.0, device="cuda") if c == 0 else None,
                      "ymip": torch.full((plan.nz, plan.nx), -1.0, device="cuda")})
        refs.append((ch, np.ascontiguousarray(R2[:, :, 136 * c:136 * (c + 1)])))
    return items, refs


def test_batch_matches_single_and_oracle(lib):
    items, refs = _mixed(lib)
    b = lib.Batch(max_items=8)
    b.set(items)
    info = b.info()
    assert info["items"] == 4 and info["units"] > 0
    b.run()
    torch.cuda.synchronize()
    b.check()
    for it, (shape, R) in zip(items, refs):
        plan = it["plan"]
        single = lib.project(plan, to_dev(R, torch), zmip=True, ymip=True)
        zref, _, yref, _ = O.project(R.astype(np.float64), O.geometry(*shape))
        if it["zmip"] is not None:
            assert torch.equal(it["zmip"], single["zmip"])
            assert_close(it["zmip"].cpu().numpy(), zref, what="batch zmip")
        assert torch.equal(it["ymip"], single["ymip"])
        assert_close(it["ymip"].cpu().numpy(), yref, what="batch ymip")


@pytest.mark.parametrize("kchunk,ctas", [(16, 1), (64, 2), (256, 4), (1000, 3)])
def test_batch_tunables_do_not_change_results(lib, kchunk, ctas):
    items, _ = _mixed(lib)
    b = lib.Batch(max_items=8)
    b.set(items, kchunk=0)
    b.run()
    ref = [(it["zmip"].clone() if it["zmip"] is not None else None, it["ymip"].clone()) for it in items]
    b.set(items, kchunk=kchunk)
    b.run(ctas_per_sm=ctas)
    torch.cuda.synchronize()
    for it, (z, y) in zip(items, ref):
        if z is not None:
            assert torch.equal(it["zmip"], z)
        assert torch.equal(it["ymip"], y)


def test_batch_graph_replay_equals_eager(lib):
    items, _ = _mixed(lib)
    b = lib.Batch(max_items=8)
    b.set(items)
    b.upload()
    b.launch()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        b.launch(stream=s)  # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            b.launch(stream=s)
    torch.cuda.synchronize()
    # new data with the same shapes in the same raw buffers (item 2's raw is
    # the whole two-channel frame stack), then replay
    items2, refs2 = _mixed(lib, seed=5)
    for i in range(3):
        items[i]["raw"].copy_(items2[i]["raw"])
    graph.replay()
    torch.cuda.synchronize()
    replayed = [(it["zmip"].clone() if it["zmip"] is not None else None, it["ymip"].clone()) for it in items]
    b.launch()
    torch.cuda.synchronize()
    for it, (z, y) in zip(items, replayed):
        if z is not None:
            assert torch.equal(it["zmip"], z)
        assert torch.equal(it["ymip"], y)
    single = lib.project(items[0]["plan"], items2[0]["raw"], zmip=True)
    assert torch.equal(replayed[0][0], single["zmip"])


def test_batch_rejects_bad_items(lib):
    b = lib.Batch(max_items=2, max_units=8)
    deep = lib.Plan(400, 20, 64, 35.0, 0.005, 0.1)            # 31 * pixel/step > 256 planes per slab
    raw = torch.zeros(deep.raw_shape, dtype=torch.uint16, device="cuda")
    with pytest.raises(lib.OpmError) as e:
        b.set([{"plan": deep, "raw": raw, "zmip": torch.empty((deep.ny, deep.nx), device="cuda")}])
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED
    plan = lib.Plan(64, 128, 128, 30.0, 0.4, 0.115)
    raw = torch.zeros(plan.raw_shape, dtype=torch.uint16, device="cuda")
    z = torch.empty((plan.ny, plan.nx), device="cuda")
    with pytest.raises(lib.OpmError) as e:
        b.set([{"plan": plan, "raw": raw, "zmip": z}])        # more units than max_units
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED
    with pytest.raises(lib.OpmError) as e:
        b.set([{"plan": plan, "raw": raw, "zmip": z, "row_pitch": 100}])   # pitch < ncols
    assert e.value.status == lib.OPM_ERR_INVALID_ARG
    with pytest.raises(lib.OpmError) as e:
        b.set([{"plan": plan, "raw": raw, "zmip": z}] * 3)    # more items than max_items
    assert e.value.status == lib.OPM_ERR_INVALID_ARG


def test_graph_launch_serves_any_content_of_one_slab_depth(lib):
    """One captured graph replays for batches of different item and unit
    counts (the counts are read from the device work list)."""
    b = lib.Batch(max_items=8)
    items_a, _ = _mixed(lib)
    b.set(items_a[:2])
    b.run(graph=True)
    torch.cuda.synchronize()
    b.check()
    first = b.info()
    assert first["graph_captures"] == 1
    got_a = [(it["zmip"].clone(), it["ymip"].clone()) for it in items_a[:2]]
    items_b, _ = _mixed(lib, seed=3)
    b.set(items_b)
    b.upload()
    b.launch_graph()
    torch.cuda.synchronize()
    b.check()
    second = b.info()
    assert second["units"] != first["units"]
    expect = 1 if second["smem_bytes"] == first["smem_bytes"] else 2
    assert second["graph_captures"] == expect
    got_b = [(None if it["zmip"] is None else it["zmip"].clone(), it["ymip"].clone()) for it in items_b]
    for it in items_a[:2] + items_b:
        for k in ("zmip", "ymip"):
            if it[k] is not None:
                it[k].fill_(-5.0)
    e = lib.Batch(max_items=8)
    e.set(items_a[:2])
    e.run()
    e.set(items_b)
    e.run()
    torch.cuda.synchronize()
    for it, (z, y) in zip(items_a[:2] + items_b, got_a + got_b):
        if z is not None:
            assert torch.equal(it["zmip"], z)
        assert torch.equal(it["ymip"], y)


def test_graph_launch_with_an_empty_batch(lib):
    b = lib.Batch(max_items=2)
    b.set([])
    b.run(graph=True)
    torch.cuda.synchronize()
    b.check()
    assert b.info()["units"] == 0


# Items the fast kernels do not take: pixel > step, ny < 32, and z-sum /
# arg-max outputs of a fast-eligible plan, beside a fast item.
GENERAL = [(16, 20, 64, 35.0, 0.05, 0.1),     # pixel > step
           (40, 70, 264, 35.0, 0.05, 0.1),    # pixel > step, ragged x tile
           (6, 10, 136, 35.0, 0.3, 0.1),      # ny = 28
           (4, 16, 264, 45.0, 0.2, 0.115)]    # ny = 19
KEYS = ("zmip", "ymip", "zsum", "argz")


def _general(lib, seed=0):
    items, refs = [], []

    def add(shape, keys, s):
        R = _stack(shape, s)
        plan = lib.Plan(*shape)
        it = {"plan": plan, "raw": to_dev(R, torch)}
        for k in keys:
            rows = plan.nz if k == "ymip" else plan.ny
            dt = torch.int32 if k == "argz" else torch.float32
            it[k] = torch.full((rows, plan.nx), -7, dtype=dt, device="cuda")
        items.append(it)
        refs.append((shape, R))

    for i, shape in enumerate(GENERAL):
        add(shape, KEYS if i % 2 == 0 else ("zmip", "ymip"), 40 + i + seed)
    add((64, 128, 128, 30.0, 0.4, 0.115), ("zsum", "argz", "ymip"), 50 + seed)   # fast plan, general kernel
    add((33, 50, 264, 45.0, 0.2, 0.115), ("zmip", "ymip"), 51 + seed)            # fast kernels
    return items, refs


def _outs(items):
    return [{k: it[k].clone() for k in KEYS if it.get(k) is not None} for it in items]


def test_general_items_match_single_and_oracle(lib):
    items, refs = _general(lib)
    b = lib.Batch(max_items=8)
    b.set(items)
    assert b.info()["units"] > 0
    b.run()
    torch.cuda.synchronize()
    b.check()
    for it, (shape, R) in zip(items, refs):
        keys = [k for k in KEYS if it.get(k) is not None]
        single = lib.project(it["plan"], to_dev(R, torch), **{k: k in keys for k in KEYS})
        for k in keys:
            assert torch.equal(it[k], single[k]), (shape, k)
        g = O.geometry(*shape)
        Rf = R.astype(np.float64)
        zmip, zsum, ymip, _ = O.project(Rf, g)
        ref = {"zmip": zmip, "zsum": zsum, "ymip": ymip}
        for k in keys:
            if k != "argz":
                assert_close(it[k].cpu().numpy(), ref[k], what=f"batch {k} {shape}")
        if "argz" in keys:
            check_argz(it["argz"].cpu().numpy(), O.deskew(Rf, g), zmip, TOL * max(np.max(np.abs(zmip)), 1e-30))


@pytest.mark.parametrize("kchunk,ctas", [(16, 1), (1000, 3)])
def test_general_items_graph_static_and_tunables(lib, kchunk, ctas):
    """Graph replay, the allocation-free call and other tunables give the
    eager launch's results bit for bit; a new graph is captured when the
    kinds of items change, and the earlier one stays cached."""
    items, _ = _general(lib, seed=1)
    b = lib.Batch(max_items=8)
    b.set(items)
    b.run()
    torch.cuda.synchronize()
    want = _outs(items)
    b.set(items, kchunk=kchunk)
    b.run(ctas_per_sm=ctas, graph=True)
    torch.cuda.synchronize()
    b.check()
    assert b.info()["graph_captures"] == 1
    for it, w in zip(items, want):
        for k, v in w.items():
            assert torch.equal(it[k], v), k
    fast_only = items[-1:]
    b.set(fast_only)
    b.run(ctas_per_sm=ctas, graph=True)
    b.set(items)
    b.run(ctas_per_sm=ctas, graph=True)
    torch.cuda.synchronize()
    b.check()
    assert b.info()["graph_captures"] == 2
    for it, w in zip(items, want):
        for k, v in w.items():
            assert torch.equal(it[k], v), k
    for it in items:
        for k in KEYS:
            if it.get(k) is not None:
                it[k].fill_(-3)
    lib.batch_project_static(items, kchunk=kchunk, ctas_per_sm=ctas, check=True)
    for it, w in zip(items, want):
        for k, v in w.items():
            assert torch.equal(it[k], v), k


def test_general_and_fast_items_nearest(lib):
    """NEAREST plans in one batch: general items (pixel > step, ny < 32, z-sum)
    and a fast item equal their stand-alone calls bit for bit, and lie within
    the oracle's bounds at half-plane ties."""
    shapes = [((16, 20, 64, 35.0, 0.05, 0.1), ("zmip", "ymip", "zsum")),
              ((6, 10, 136, 35.0, 0.3, 0.1), ("zmip", "ymip")),
              ((64, 128, 128, 30.0, 0.4, 0.115), ("zmip", "ymip"))]
    items, refs = [], []
    for i, (shape, keys) in enumerate(shapes):
        R = _stack(shape, 80 + i)
        plan = lib.Plan(*shape, interp=lib.OPM_INTERP_NEAREST)
        it = {"plan": plan, "raw": to_dev(R, torch)}
        for k in keys:
            it[k] = torch.full((plan.nz if k == "ymip" else plan.ny, plan.nx), -7.0, device="cuda")
        items.append(it)
        refs.append((shape, R, keys))
    b = lib.Batch(max_items=4)
    b.set(items)
    b.run()
    torch.cuda.synchronize()
    b.check()
    for it, (shape, R, keys) in zip(items, refs):
        single = lib.project(it["plan"], to_dev(R, torch), **{k: k in keys for k in KEYS})
        for k in keys:
            assert torch.equal(it[k], single[k]), (shape, k)
        g = O.geometry(*shape)
        lo, hi = nearest_bounds(R, g, O)
        assert_between(it["zmip"].cpu().numpy(), lo.max(0), hi.max(0), what=f"zmip nearest {shape}")
        assert_between(it["ymip"].cpu().numpy(), lo.max(1), hi.max(1), what=f"ymip nearest {shape}")
        if "zsum" in keys:
            assert_between(it["zsum"].cpu().numpy(), lo.sum(0), hi.sum(0), what=f"zsum nearest {shape}")


@pytest.mark.parametrize("width", [2048, 512, 128])
def test_batch_default_units_follow_the_plan_rule(lib, width):
    """kchunk 0: the batch cuts its fast items' units by the single-stack
    plan's rule (largest of 256 .. 16 rows giving 1.1 units per CTA list), so
    a batch of one stack holds exactly the plan's own units."""
    plan = lib.Plan(200, 512, width, 35.0, 0.3, 0.1)
    raw = torch.zeros(plan.raw_shape, dtype=torch.uint16, device="cuda")
    z = torch.empty((plan.ny, plan.nx), device="cuda")
    y = torch.empty((plan.nz, plan.nx), device="cuda")
    nunits, nlists, rows = lib.opm_plan_schedule(plan)
    assert nunits > 0 and nlists > 0 and rows in (16, 32, 64, 128, 256)
    b = lib.Batch(max_items=1)
    b.set([{"plan": plan, "raw": raw, "zmip": z, "ymip": y}])
    assert b.info()["units"] == nunits
    b.close()
