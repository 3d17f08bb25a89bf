"""Autotuner and kernel shapes on the GPU: every kernel shape gives the same
results bit for bit, the graph cache keeps one graph per launch shape, the
chosen candidate is one of those timed, and the batch's results do not
depend on it."""
import pytest

import opm_synth
from gpu_util import to_dev
from test_gpu_batch import _mixed

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEO = (35.0, 0.3, 0.1)   # pixel/step = 1/3: a periodic family


def _periodic_items(lib):
    """Stacks of one periodic family (several shapes, a ragged x tile, two
    channels of one frame stack) and one item with z-sum and arg-max."""
    items = []
    for i, (n, r, c) in enumerate([(60, 96, 256), (40, 70, 264), (100, 128, 128)]):
        R = opm_synth.raw_stack(opm_synth.StackConfig("t", n, r, c, *GEO, n_blobs=10, sigma=(1.0, 3.0),
                                                      amp=(200.0, 4000.0), seed=60 + i))
        plan = lib.Plan(n, r, c, *GEO)
        it = {"plan": plan, "raw": to_dev(R, torch),
              "zmip": torch.full((plan.ny, plan.nx), -1.0, device="cuda"),
              "ymip": torch.full((plan.nz, plan.nx), -1.0, device="cuda")}
        if i == 2:
            it["zsum"] = torch.full((plan.ny, plan.nx), -1.0, device="cuda")
            it["argz"] = torch.full((plan.ny, plan.nx), -1, dtype=torch.int32, device="cuda")
        items.append(it)
    R2 = opm_synth.raw_stack(opm_synth.StackConfig("t", 50, 64, 272, *GEO, n_blobs=10, sigma=(1.0, 3.0),
                                                   amp=(200.0, 4000.0), seed=70))
    raw2 = to_dev(R2, torch)
    plan = lib.Plan(50, 64, 136, *GEO)
    for ch in range(2):
        items.append({"plan": plan, "raw": raw2[:, :, 136 * ch:], "row_pitch": 272, "plane_pitch": 64 * 272,
                      "zmip": torch.full((plan.ny, plan.nx), -1.0, device="cuda"),
                      "ymip": torch.full((plan.nz, plan.nx), -1.0, device="cuda")})
    return items


def _outs(items):
    keys = ("zmip", "ymip", "zsum", "argz")
    return [{k: it[k].clone() for k in keys if it.get(k) is not None} for it in items]


def test_every_shape_gives_identical_results(lib):
    items = _periodic_items(lib)
    b = lib.Batch(max_items=8)
    b.set(items)
    b.run()
    torch.cuda.synchronize()
    b.check()
    assert b.info()["shape"] == lib.OPM_SHAPE_PER_J32X2
    want = _outs(items)
    single = lib.project(items[0]["plan"], items[0]["raw"], zmip=True, ymip=True)
    assert torch.equal(want[0]["zmip"], single["zmip"]) and torch.equal(want[0]["ymip"], single["ymip"])
    shapes = [lib.OPM_SHAPE_PER_J32X2, lib.OPM_SHAPE_PER_J16X2, lib.OPM_SHAPE_FAST_J8X4, lib.OPM_SHAPE_GEN_J8X4]
    for graph in (False, True):
        for sh in shapes:
            for kchunk, ctas in ((32, 2), (128, 4)):
                for it in items:
                    for v in it.values():
                        if torch.is_tensor(v) and v.dtype in (torch.float32, torch.int32):
                            v.fill_(-9)
                b.set(items, kchunk, sh)
                assert b.info()["shape"] == sh
                b.run(ctas, graph=graph)
                torch.cuda.synchronize()
                b.check()
                for it, w in zip(items, want):
                    for k, v in w.items():
                        assert torch.equal(it[k], v), (lib.SHAPE_NAMES[sh], kchunk, ctas, graph, k)
    # one graph per launch shape: 3 fast-kernel shapes x 2 grids, plus the
    # general shape whose grid is 2 CTAs per SM for both; the cache keeps
    # the 4 most recently used, so replaying one of those captures nothing
    n = b.info()["graph_captures"]
    assert n == 7
    b.set(items, 128, lib.OPM_SHAPE_GEN_J8X4)
    b.run(4, graph=True)
    b.set(items, 128, lib.OPM_SHAPE_FAST_J8X4)
    b.run(4, graph=True)
    torch.cuda.synchronize()
    assert b.info()["graph_captures"] == n


def test_periodic_shape_falls_back_without_a_common_family(lib):
    items, _ = _mixed(lib)    # two families: periodic 1/3 and a plain fast plan
    b = lib.Batch(max_items=8)
    b.set(items, 64, lib.OPM_SHAPE_PER_J16X2)
    assert b.info()["shape"] == lib.OPM_SHAPE_FAST_J8X4


def test_tuner_choice_keeps_results(lib, tmp_path):
    from paper_2211_00645_gb300.tune import Tuner, candidates, shapes_for
    items = _periodic_items(lib)
    b = lib.Batch(max_items=8)
    b.set(items)
    b.run()
    torch.cuda.synchronize()
    want = _outs(items)
    t = Tuner(str(tmp_path / "t.json"))
    shapes = shapes_for(items)
    assert shapes == (lib.OPM_SHAPE_PER_J32X2, lib.OPM_SHAPE_PER_J16X2, lib.OPM_SHAPE_FAST_J8X4,
                      lib.OPM_SHAPE_GEN_J8X4)
    e = t.tune(items, kchunks=(16, 64, 256), ctas=(2, 4), reps=2)
    assert len(e["candidates"]) == len(candidates((16, 64, 256), (2, 4), shapes))
    assert all(v > 0 for v in e["candidates"].values())
    sh, k, c = t.best(items, torch.cuda.get_device_properties(0).multi_processor_count)
    assert lib.SHAPE_NAMES[sh] == e["shape"]
    b.set(items, k, sh)
    b.run(c)
    torch.cuda.synchronize()
    b.check()
    for it, w in zip(items, want):
        for key, v in w.items():
            assert torch.equal(it[key], v), key
