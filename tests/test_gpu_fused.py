"""Volume and live view in one call (opm_deskew_mip): the FP32 and uint16
volumes and the z-MIP / y-MIP equal the separate opm_deskew /
opm_deskew_dual / opm_project calls bit for bit, in both of its modes: the
live view beside the volume on the plan's side stream (default) and the
single fused kernel (plans created with OPM_ONE_PASS_FUSED=1)."""
import os

import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import assert_close, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(64, 128, 128, 30.0, 0.4, 0.115),     # fused
          (33, 50, 264, 45.0, 0.2, 0.115),      # fused, partial x-tile and last j-tile
          (40, 70, 136, 35.0, 0.3, 0.1),        # fused, nx not a multiple of 128
          (16, 20, 64, 35.0, 0.05, 0.1),        # pixel > step: separate kernels
          (12, 9, 30, 90.0, 0.1, 0.1)]          # rows of 60 bytes: separate kernels


MODES = ["beside", "fused"]


def _plan(lib, shape, mode):
    if mode == "fused":
        os.environ["OPM_ONE_PASS_FUSED"] = "1"
    try:
        return lib.Plan(*shape)
    finally:
        os.environ.pop("OPM_ONE_PASS_FUSED", None)


def _stack(shape, seed=4):
    return opm_synth.raw_stack(opm_synth.StackConfig("f", *shape, n_blobs=8, sigma=(1.0, 3.0),
                                                     amp=(200.0, 4000.0), seed=seed))


def _fused(lib, plan, raw, f32=True, u16=True, z=True, y=True):
    vf = torch.full(plan.vol_shape, -7.0, device="cuda") if f32 else None
    vh = torch.full(plan.vol_shape, 7, dtype=torch.int16, device="cuda").view(torch.uint16) if u16 else None
    zm = torch.full((plan.ny, plan.nx), -7.0, device="cuda") if z else None
    ym = torch.full((plan.nz, plan.nx), -7.0, device="cuda") if y else None
    lib.opm_deskew_mip(plan, raw, vf, vh, zm, ym)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    return vf, vh, zm, ym


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_equals_separate_calls(lib, shape, mode):
    R = _stack(shape)
    plan = _plan(lib, shape, mode)
    raw = to_dev(R, torch)
    vf, vh, zm, ym = _fused(lib, plan, raw)
    ref_f = lib.deskew(plan, raw)
    ref_h = lib.deskew(plan, raw, out_dtype=torch.uint16)
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    torch.cuda.synchronize()
    assert torch.equal(vf, ref_f)
    assert torch.equal(vh.view(torch.int16), ref_h.view(torch.int16))
    assert torch.equal(zm, ref["zmip"]) and torch.equal(ym, ref["ymip"])
    g = O.geometry(*shape)
    V = O.deskew(R.astype(np.float64), g)
    assert_close(vf.cpu().numpy(), V, what="fused volume")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("outs", [(True, False, True, False), (False, True, False, True), (True, False, False, False)])
def test_fused_output_subsets(lib, outs, mode):
    shape = SHAPES[0]
    R = _stack(shape, seed=9)
    plan = _plan(lib, shape, mode)
    raw = to_dev(R, torch)
    vf, vh, zm, ym = _fused(lib, plan, raw, *outs)
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    if vf is not None:
        assert torch.equal(vf, lib.deskew(plan, raw))
    if vh is not None:
        assert torch.equal(vh.view(torch.int16), lib.deskew(plan, raw, out_dtype=torch.uint16).view(torch.int16))
    if zm is not None:
        assert torch.equal(zm, ref["zmip"])
    if ym is not None:
        assert torch.equal(ym, ref["ymip"])


@pytest.mark.parametrize("mode", MODES)
def test_fused_liveview_full_size(lib, mode):
    c = opm_synth.CONFIGS["liveview_200x512x2048"]
    R = opm_synth.tiled_stack((c.nscan, c.nrows, c.ncols), seed=2)
    plan = _plan(lib, (c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel), mode)
    raw = to_dev(R, torch)
    vf, _, zm, ym = _fused(lib, plan, raw, u16=False)
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    assert torch.equal(zm, ref["zmip"]) and torch.equal(ym, ref["ymip"])
    assert torch.equal(vf, lib.deskew(plan, raw))
    assert torch.equal(vf.max(dim=0).values, zm)


@pytest.mark.parametrize("mode", MODES)
def test_fused_f32_input(lib, mode):
    """FP32 raw input: the volumes and projections equal the separate calls."""
    shape = SHAPES[2]
    R = _stack(shape, seed=11).astype(np.float32)
    plan = _plan(lib, shape, mode)
    raw = to_dev(R, torch)
    vf, vh, zm, ym = _fused(lib, plan, raw)
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    torch.cuda.synchronize()
    assert torch.equal(vf, lib.deskew(plan, raw))
    assert torch.equal(vh.view(torch.int16), lib.deskew(plan, raw, out_dtype=torch.uint16).view(torch.int16))
    assert torch.equal(zm, ref["zmip"]) and torch.equal(ym, ref["ymip"])


def test_fused_argument_checks(lib):
    plan = lib.Plan(*SHAPES[0])
    raw = torch.zeros(plan.raw_shape, dtype=torch.uint16, device="cuda")
    with pytest.raises(lib.OpmError) as e:
        lib.opm_deskew_mip(plan, raw, None, None, torch.empty((plan.ny, plan.nx), device="cuda"), None)
    assert e.value.status == lib.OPM_ERR_INVALID_ARG


def test_beside_joins_the_callers_stream(lib):
    """Work queued on the caller's stream after the call sees the finished
    live view (the side stream is joined back), on a non-default stream,
    call after call."""
    shape = (120, 256, 512, 35.0, 0.3, 0.1)
    R = opm_synth.tiled_stack(shape[:3], seed=5)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    ref_v = lib.deskew(plan, raw)
    vf = torch.empty(plan.vol_shape, device="cuda")
    zm = torch.empty((plan.ny, plan.nx), device="cuda")
    ym = torch.empty((plan.nz, plan.nx), device="cuda")
    s = torch.cuda.Stream()
    lib.opm_deskew_mip(plan, raw, vf, None, zm, ym, s)      # first call loads the modules
    s.synchronize()
    copies = []
    with torch.cuda.stream(s):
        for _ in range(4):
            zm.fill_(-1.0)
            ym.fill_(-1.0)
            lib.opm_deskew_mip(plan, raw, vf, None, zm, ym, s)
            copies.append((zm.clone(), ym.clone()))
    s.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lib.opm_deskew_mip(plan, raw, vf, None, zm, ym, s)
    s.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "opm_deskew_mip allocated device memory"
    for z, y in copies:
        assert torch.equal(z, ref["zmip"]) and torch.equal(y, ref["ymip"])
    assert torch.equal(vf, ref_v)
    lib.opm_plan_check(plan)


def test_beside_in_a_cuda_graph(lib):
    """The fork onto the side stream and the join back are capturable: a
    graph of the call replays to the same outputs."""
    shape = SHAPES[0]
    R = _stack(shape, seed=6)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    vf = torch.empty(plan.vol_shape, device="cuda")
    zm = torch.empty((plan.ny, plan.nx), device="cuda")
    ym = torch.empty((plan.nz, plan.nx), device="cuda")
    s = torch.cuda.Stream()
    lib.opm_deskew_mip(plan, raw, vf, None, zm, ym, s)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        lib.opm_deskew_mip(plan, raw, vf, None, zm, ym, s)
    zm.zero_()
    ym.zero_()
    vf.zero_()
    graph.replay()
    torch.cuda.synchronize()
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    assert torch.equal(zm, ref["zmip"]) and torch.equal(ym, ref["ymip"])
    assert torch.equal(vf, lib.deskew(plan, raw))
