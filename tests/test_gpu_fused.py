"""Volume and live view in one pass (opm_deskew_mip): the FP32 and uint16
volumes and the z-MIP / y-MIP equal the separate opm_deskew /
opm_deskew_dual / opm_project calls bit for bit, on plans the fused kernel
takes and on plans that fall back to the separate kernels."""
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


@pytest.mark.parametrize("shape", SHAPES)
def test_fused_equals_separate_calls(lib, shape):
    R = _stack(shape)
    plan = lib.Plan(*shape)
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


@pytest.mark.parametrize("outs", [(True, False, True, False), (False, True, False, True), (True, False, False, False)])
def test_fused_output_subsets(lib, outs):
    shape = SHAPES[0]
    R = _stack(shape, seed=9)
    plan = lib.Plan(*shape)
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


def test_fused_liveview_full_size(lib):
    c = opm_synth.CONFIGS["liveview_200x512x2048"]
    R = opm_synth.tiled_stack((c.nscan, c.nrows, c.ncols), seed=2)
    plan = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    raw = to_dev(R, torch)
    vf, _, zm, ym = _fused(lib, plan, raw, u16=False)
    ref = lib.project(plan, raw, zmip=True, ymip=True)
    assert torch.equal(zm, ref["zmip"]) and torch.equal(ym, ref["ymip"])
    assert torch.equal(vf, lib.deskew(plan, raw))
    assert torch.equal(vf.max(dim=0).values, zm)


def test_fused_argument_checks(lib):
    plan = lib.Plan(*SHAPES[0])
    raw = torch.zeros(plan.raw_shape, dtype=torch.uint16, device="cuda")
    with pytest.raises(lib.OpmError) as e:
        lib.opm_deskew_mip(plan, raw, None, None, torch.empty((plan.ny, plan.nx), device="cuda"), None)
    assert e.value.status == lib.OPM_ERR_INVALID_ARG
