"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, validates arguments and answers shape queries without a
GPU (plans made without a device refuse compute calls)."""
import ctypes
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def opm():
    from paper_2211_00645_gb300 import build as b
    b.build()
    import paper_2211_00645_gb300 as m
    m.load()
    return m


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "opm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:opm_status|const char\s*\*|int)\s+(opm_\w+)\s*\(", src, re.M)))


def test_header_symbols_exported(opm):
    syms = _header_symbols()
    assert len(syms) >= 10
    lib = ctypes.CDLL(opm.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(opm.exported_symbols()) == syms


def test_version(opm):
    assert opm.load().opm_version() >= 100


@pytest.mark.parametrize("name", ["oracle_64x128x128", "liveview_200x512x2048",
                                  "large_1000x1024x2048", "diff_128x256x256"])
def test_plan_shape_matches_oracle(opm, name):
    import opm_synth
    c = opm_synth.CONFIGS[name]
    p = opm.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    g = O.geometry(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    assert (p.nz, p.ny, p.nx, p.J0) == (g.nz, g.ny, g.nx, g.J0)


@pytest.mark.parametrize("args", [
    (64, 128, 128, 30.0, 0.4, 0.115, 1),
    (7, 5, 3, 90.0, 0.125, 0.125, 0),
    (6, 3, 2, 35.0, 0.05, 0.1, 0),
    (2, 1, 1, 60.0, 0.2, 0.1, 1),
    (3, 2, 3, 12.5, 0.37, 0.11, 0),
])
def test_plan_shape_small(opm, args):
    p = opm.Plan(*args)
    g = O.geometry(*args[:6])
    assert (p.nz, p.ny, p.nx, p.J0) == (g.nz, g.ny, g.nx, g.J0)


@pytest.mark.parametrize("bad", [
    (1, 4, 4, 30.0, 0.4, 0.1, 0),      # nscan < 2
    (4, 0, 4, 30.0, 0.4, 0.1, 0),      # nrows < 1
    (4, 4, 0, 30.0, 0.4, 0.1, 0),      # ncols < 1
    (4, 4, 4, 0.0, 0.4, 0.1, 0),       # theta = 0
    (4, 4, 4, 90.5, 0.4, 0.1, 0),      # theta > 90
    (4, 4, 4, -30.0, 0.4, 0.1, 0),
    (4, 4, 4, float("nan"), 0.4, 0.1, 0),
    (4, 4, 4, 30.0, 0.0, 0.1, 0),      # step = 0
    (4, 4, 4, 30.0, 0.4, -0.1, 0),     # pixel < 0
    (4, 4, 4, 30.0, float("inf"), 0.1, 0),
    (4, 4, 4, 30.0, 0.4, 0.1, 2),      # interp
])
def test_plan_create_rejects(opm, bad):
    with pytest.raises(opm.OpmError) as e:
        opm.Plan(*bad)
    assert e.value.status == opm.OPM_ERR_INVALID_ARG


def test_plan_create_too_large(opm):
    with pytest.raises(opm.OpmError) as e:
        opm.Plan(1 << 20, 1 << 20, 1 << 20, 30.0, 0.4, 0.1)
    assert e.value.status == opm.OPM_ERR_UNSUPPORTED


def test_null_arguments(opm):
    lib = opm.load()
    assert lib.opm_plan_create(4, 4, 4, 30.0, 0.4, 0.1, 0, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_plan_shape(None, None, None, None, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_plan_destroy(None) == opm.OPM_OK
    assert lib.opm_deskew(None, None, 0, None, 1, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_project(None, None, 0, None, None, None, None, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_skew_adjoint(None, None, None, 1, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_mip_backward(None, None, None, None, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_plan_check(None) == opm.OPM_ERR_INVALID_ARG
    assert b"NULL" in lib.opm_last_error()


def test_host_only_plan_refuses_compute(opm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only behaviour needs a machine without a CUDA device")
    p = opm.Plan(8, 6, 16, 30.0, 0.4, 0.115)
    lib = opm.load()
    dummy = ctypes.c_void_p(16)
    st = lib.opm_project(p.handle, dummy, opm.OPM_U16, dummy, None, None, None, None)
    assert st == opm.OPM_ERR_CUDA
    assert b"without a CUDA device" in lib.opm_last_error()
    assert lib.opm_plan_check(p.handle) == opm.OPM_OK


def test_shape_arguments_optional(opm):
    p = opm.Plan(8, 6, 16, 30.0, 0.4, 0.115)
    nz = ctypes.c_int64()
    assert opm.load().opm_plan_shape(p.handle, ctypes.byref(nz), None, None, None) == opm.OPM_OK
    assert nz.value == 6


def test_plan_path_classification(opm):
    """Which live-view kernel a plan takes is decided on the host: pixel/step
    = 1/3 or 1/2 plans take the periodic kernel, other pixel <= step plans
    the fast one, pixel > step plans the general one."""
    cases = [((200, 512, 2048, 35.0, 0.3, 0.1), (opm.OPM_PATH_PERIODIC, 1, 3)),
             ((33, 50, 200, 60.0, 0.45, 0.15), (opm.OPM_PATH_PERIODIC, 1, 3)),
             ((64, 128, 128, 30.0, 0.4, 0.115), (opm.OPM_PATH_FAST, 0, 0)),
             ((100, 96, 264, 35.0, 0.2, 0.1), (opm.OPM_PATH_PERIODIC, 1, 2)),
             ((100, 96, 264, 35.0, 0.15, 0.1), (opm.OPM_PATH_FAST, 0, 0)),
             ((16, 20, 64, 35.0, 0.05, 0.1), (opm.OPM_PATH_GENERAL, 0, 0))]
    for shape, want in cases:
        plan = opm.Plan(*shape)
        assert opm.opm_plan_path(plan) == want, shape
        plan.close()


def test_plan_schedule_without_device(opm):
    """A plan made with no CUDA device has no live-view schedule: units,
    lists and rows per unit all read 0 (compute calls refuse such a plan)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only behaviour needs a machine without a CUDA device")
    plan = opm.Plan(200, 512, 2048, 35.0, 0.3, 0.1)
    assert opm.opm_plan_schedule(plan) == (0, 0, 0)
    plan.close()


def test_sheet_check_without_device(opm):
    """With no usable CUDA device the sheet view's error-word check reports
    OPM_ERR_CUDA rather than failing silently or crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only behaviour needs a machine without a CUDA device")
    with pytest.raises(opm.OpmError) as e:
        opm.opm_sheet_check()
    assert e.value.status == opm.OPM_ERR_CUDA


def test_sliding_and_combine_argument_checks(opm):
    """opm_max_combine and opm_sliding_push refuse bad arguments before any
    device work: NULL arrays, a negative length, a NULL plan, a frame index
    outside [0, nscan)."""
    lib = opm.load()
    p = ctypes.c_void_p(16)
    assert lib.opm_max_combine(None, p, p, 4, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_max_combine(p, p, p, -1, None) == opm.OPM_ERR_INVALID_ARG
    assert lib.opm_sliding_push(None, p, 0, p, p, p, None) == opm.OPM_ERR_INVALID_ARG
    import torch
    if not torch.cuda.is_available():
        plan = opm.Plan(8, 6, 16, 30.0, 0.4, 0.115)
        # a plan made without a device refuses before looking at the arguments
        assert lib.opm_sliding_push(plan.handle, p, 0, p, p, p, None) == opm.OPM_ERR_CUDA
        plan.close()
