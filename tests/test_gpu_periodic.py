"""The periodic live-view kernel: plans whose pixel/step is a compiled ratio
p/q (1/3, 1/2) step through their staged planes in one of q patterns per
32-column tile row and run straight-line code per pattern.  It must reproduce the FP64 oracle within the
bound, the fast kernel (same plan made with OPM_NO_PERIODIC=1) bit for bit,
the maxima of the deskewed volume bit for bit, and the batched path."""
import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import assert_close, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (nscan, nrows, ncols, theta, step, pixel), pixel/step = 1/3
PER_SHAPES = [
    (40, 70, 264, 35.0, 0.3, 0.1),     # ragged x tile (264 = 2 x 128 + 8), ny % 32 != 0
    (64, 128, 128, 30.0, 0.3, 0.1),
    (33, 50, 200, 60.0, 0.45, 0.15),   # exact cos 1/2
    (50, 33, 136, 45.0, 0.3, 0.1),     # odd row count: the last stage's second row is padding
    (20, 3, 256, 35.0, 0.3, 0.1),      # three camera rows
    (200, 64, 512, 35.0, 0.3, 0.1),    # the live-view geometry, fewer rows and columns
]


def _stack(shape, seed):
    n, r, c = shape[:3]
    return opm_synth.raw_stack(opm_synth.StackConfig("p", n, r, c, *shape[3:], n_blobs=14, sigma=(1.0, 3.0),
                                                     amp=(200.0, 5000.0), seed=seed))


def _fast_plan(lib, monkeypatch, shape, interp=0):
    monkeypatch.setenv("OPM_NO_PERIODIC", "1")
    try:
        return lib.Plan(*shape, interp=interp)
    finally:
        monkeypatch.delenv("OPM_NO_PERIODIC")


@pytest.mark.parametrize("shape", PER_SHAPES)
def test_periodic_matches_oracle_and_fast_kernel(lib, monkeypatch, shape):
    R = _stack(shape, seed=11)
    plan = lib.Plan(*shape)
    assert lib.opm_plan_path(plan) == (lib.OPM_PATH_PERIODIC, 1, 3)
    fast = _fast_plan(lib, monkeypatch, shape)
    assert lib.opm_plan_path(fast)[0] == lib.OPM_PATH_FAST
    raw = to_dev(R, torch)
    a = lib.project(plan, raw, zmip=True, ymip=True)
    b = lib.project(fast, raw, zmip=True, ymip=True)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    assert torch.equal(a["zmip"], b["zmip"]) and torch.equal(a["ymip"], b["ymip"])
    g = O.geometry(*shape)
    zmip, _, ymip, _ = O.project(R.astype(np.float64), g)
    assert_close(a["zmip"].cpu().numpy(), zmip, what="zmip")
    assert_close(a["ymip"].cpu().numpy(), ymip, what="ymip")
    # one output at a time takes the same kernel
    z_only = lib.project(plan, raw, zmip=True)
    y_only = lib.project(plan, raw, zmip=False, ymip=True)
    torch.cuda.synchronize()
    assert torch.equal(z_only["zmip"], a["zmip"]) and torch.equal(y_only["ymip"], a["ymip"])


@pytest.mark.parametrize("shape", [PER_SHAPES[0], PER_SHAPES[2]])
def test_periodic_nearest_matches_fast_kernel(lib, monkeypatch, shape):
    R = _stack(shape, seed=12)
    plan = lib.Plan(*shape, interp=1)
    assert lib.opm_plan_path(plan)[0] == lib.OPM_PATH_PERIODIC
    fast = _fast_plan(lib, monkeypatch, shape, interp=1)
    raw = to_dev(R, torch)
    a = lib.project(plan, raw, zmip=True, ymip=True)
    b = lib.project(fast, raw, zmip=True, ymip=True)
    torch.cuda.synchronize()
    assert torch.equal(a["zmip"], b["zmip"]) and torch.equal(a["ymip"], b["ymip"])


@pytest.mark.parametrize("shape", [PER_SHAPES[0], PER_SHAPES[3]])
def test_periodic_equals_volume_maxima(lib, shape):
    """The projections are exactly the maxima of the deskewed FP32 volume."""
    R = _stack(shape, seed=13)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    vol = lib.deskew(plan, raw)
    out = lib.project(plan, raw, zmip=True, ymip=True)
    torch.cuda.synchronize()
    assert torch.equal(out["zmip"], vol.amax(dim=0))
    assert torch.equal(out["ymip"], vol.amax(dim=1))


def test_periodic_batch_and_mixed_batch(lib):
    """A batch of periodic items (two stacks and a two-channel frame stack as
    strided ROIs) runs the periodic batch kernel; a batch that also holds a
    fast-kernel plan runs the fast one.  Both equal the stand-alone calls."""
    shapes = [PER_SHAPES[0], PER_SHAPES[3]]
    stacks = [to_dev(_stack(s, seed=20 + i), torch) for i, s in enumerate(shapes)]
    plans = [lib.Plan(*s) for s in shapes]
    two = to_dev(_stack((40, 70, 528, 35.0, 0.3, 0.1), seed=30), torch)
    cplan = lib.Plan(40, 70, 264, 35.0, 0.3, 0.1)
    other = lib.Plan(64, 128, 128, 30.0, 0.4, 0.115)
    assert lib.opm_plan_path(other)[0] == lib.OPM_PATH_FAST
    oraw = to_dev(_stack((64, 128, 128, 30.0, 0.4, 0.115), seed=40), torch)

    def items(with_other):
        it = [{"plan": p, "raw": r, "zmip": torch.full((p.ny, p.nx), -1.0, device="cuda"),
               "ymip": torch.full((p.nz, p.nx), -1.0, device="cuda")} for p, r in zip(plans, stacks)]
        for c in range(2):
            it.append({"plan": cplan, "raw": two[:, :, 264 * c:], "row_pitch": 528, "plane_pitch": 70 * 528,
                       "zmip": torch.full((cplan.ny, cplan.nx), -1.0, device="cuda"),
                       "ymip": torch.full((cplan.nz, cplan.nx), -1.0, device="cuda")})
        if with_other:
            it.append({"plan": other, "raw": oraw, "zmip": torch.full((other.ny, other.nx), -1.0, device="cuda"),
                       "ymip": torch.full((other.nz, other.nx), -1.0, device="cuda")})
        return it

    for with_other in (False, True):
        its = items(with_other)
        b = lib.Batch(max_items=8)
        b.set(its)
        b.run(graph=True)
        torch.cuda.synchronize()
        b.check()
        for it in its:
            raw = it["raw"] if "row_pitch" not in it else it["raw"][:, :, :264].contiguous()
            ref = lib.project(it["plan"], raw, zmip=True, ymip=True)
            torch.cuda.synchronize()
            assert torch.equal(it["zmip"], ref["zmip"]) and torch.equal(it["ymip"], ref["ymip"])
        b.close()


# the other compiled family: pixel/step = 1/2
FAMILY_SHAPES = [
    ((100, 96, 264, 35.0, 0.2, 0.1), (1, 2)),    # ragged x tile
    ((64, 128, 256, 30.0, 0.4, 0.2), (1, 2)),
    ((41, 33, 128, 60.0, 0.25, 0.125), (1, 2)),  # exact cos 1/2, odd row count
]


@pytest.mark.parametrize("shape,pq", FAMILY_SHAPES)
def test_other_families_match_oracle_fast_kernel_and_batch(lib, monkeypatch, shape, pq):
    R = _stack(shape, seed=13)
    plan = lib.Plan(*shape)
    assert lib.opm_plan_path(plan) == (lib.OPM_PATH_PERIODIC, *pq)
    fast = _fast_plan(lib, monkeypatch, shape)
    assert lib.opm_plan_path(fast)[0] == lib.OPM_PATH_FAST
    raw = to_dev(R, torch)
    a = lib.project(plan, raw, zmip=True, ymip=True)
    b = lib.project(fast, raw, zmip=True, ymip=True)
    bt = lib.Batch(max_items=1)
    item = {"plan": plan, "raw": raw, "zmip": torch.empty_like(a["zmip"]), "ymip": torch.empty_like(a["ymip"])}
    bt.set([item], 64, lib.OPM_SHAPE_PER_J16X2)       # 16-column runs fall back to 32 outside 1/3
    assert bt.info()["shape"] == lib.OPM_SHAPE_PER_J32X2
    bt.run()
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    bt.check()
    assert torch.equal(a["zmip"], b["zmip"]) and torch.equal(a["ymip"], b["ymip"])
    assert torch.equal(item["zmip"], a["zmip"]) and torch.equal(item["ymip"], a["ymip"])
    g = O.geometry(*shape)
    zmip, _, ymip, _ = O.project(R.astype(np.float64), g)
    assert_close(a["zmip"].cpu().numpy(), zmip, what="zmip")
    assert_close(a["ymip"].cpu().numpy(), ymip, what="ymip")
