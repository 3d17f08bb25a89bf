"""The paper's sheet-frame live view (remap + maximum, Fig. 2c-d) and the
shear-warp warp (Fig. 3) against the FP64 oracle."""
import math

import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import TOL, assert_close, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _stack(n, r, c, seed=6):
    cfg = opm_synth.StackConfig("s", n, r, c, 35.0, 0.3, 0.1, n_blobs=8, sigma=(1.0, 3.0), amp=(200.0, 4000.0),
                                seed=seed)
    return opm_synth.raw_stack(cfg)


@pytest.mark.parametrize("shape", [(40, 64, 128), (17, 33, 70), (5, 9, 3)])
@pytest.mark.parametrize("shear", [0.0, 1.0, 0.37, 2.4574561328, 7.5])
def test_sheet_project_u16(lib, shape, shear):
    R = _stack(*shape)
    out = lib.opm_sheet_project(to_dev(R, torch), shear)
    torch.cuda.synchronize()
    ref = O.sheet_project(R.astype(np.float64), shear)
    assert out.shape == ref.shape
    assert_close(out.cpu().numpy(), ref, what=f"sheet shear={shear}")
    if shear == math.floor(shear):                        # integer shifts: exact
        assert np.array_equal(out.cpu().numpy(), ref.astype(np.float32))


@pytest.mark.parametrize("shape", [(120, 64, 136), (75, 40, 256), (60, 100, 128), (51, 33, 384)])
@pytest.mark.parametrize("shear", [0.0, 1.0, 0.37, 2.4574561328, 7.5])
def test_sheet_project_tma_path(lib, shape, shear):
    """uint16 stacks the TMA kernel takes (rows of 8k columns, >= 128 columns,
    >= 33 rows): a ragged last 128-column tile, output rows that are not a
    multiple of the 32-row tile, several 50-frame chunks per tile, and frames
    whose rows miss a tile.  Integer shears are exact; no ring wait gives up."""
    R = _stack(*shape, seed=9)
    out = lib.opm_sheet_project(to_dev(R, torch), shear)
    torch.cuda.synchronize()
    lib.opm_sheet_check()
    ref = O.sheet_project(R.astype(np.float64), shear)
    assert out.shape == ref.shape
    assert_close(out.cpu().numpy(), ref, what=f"sheet tma {shape} shear={shear}")
    if shear == math.floor(shear):
        assert np.array_equal(out.cpu().numpy(), ref.astype(np.float32))


def test_sheet_tma_and_plain_kernels_agree(lib):
    """The same frames through the TMA kernel (136 columns) and the plain one
    (a 130-column copy, not a multiple of 8): identical bits on the shared
    columns."""
    R = _stack(90, 48, 136, seed=4)
    shear = 2.4574561328
    a = lib.opm_sheet_project(to_dev(R, torch), shear)
    b = lib.opm_sheet_project(to_dev(np.ascontiguousarray(R[:, :, :130]), torch), shear)
    torch.cuda.synchronize()
    lib.opm_sheet_check()
    assert torch.equal(a[:, :130], b)


def test_sheet_project_f32_signed(lib):
    R = opm_synth.gaussian((12, 20, 36), 4, np.float32)
    out = lib.opm_sheet_project(to_dev(R, torch), 1.3)
    torch.cuda.synchronize()
    assert_close(out.cpu().numpy(), O.sheet_project(R.astype(np.float64), 1.3), what="sheet f32")


def test_sheet_liveview_size(lib):
    c = opm_synth.CONFIGS["liveview_200x512x2048"]
    R = opm_synth.tiled_stack((c.nscan, c.nrows, c.ncols), seed=2)
    shear = c.step * O.cos_deg(c.theta_deg) / c.pixel
    out = lib.opm_sheet_project(to_dev(R, torch), shear)
    torch.cuda.synchronize()
    assert out.shape == (1002, 2048)
    xs = np.array([0, 1, 777, 2047])
    ref = O.sheet_project(R[:, :, xs].astype(np.float64), shear)
    assert_close(out.cpu().numpy()[:, xs], ref, what="sheet live-view columns")


@pytest.mark.parametrize("a,b,rows", [(1.0, 0.0, 50), (1.0, 3.0, 50), (0.6, -4.25, 90), (1.7, 10.5, 30)])
def test_warp_rows(lib, a, b, rows):
    P = np.abs(opm_synth.gaussian((50, 68), 9, np.float32)) * 10
    out = lib.opm_warp_rows(to_dev(P, torch), rows, a, b)
    torch.cuda.synchronize()
    ref = O.warp_rows(P.astype(np.float64), rows, a, b)
    assert_close(out.cpu().numpy(), ref, what=f"warp a={a} b={b}")


def test_shear_warp_view(lib):
    """A reduced shear then a warp: the same two steps through the library
    and through the oracle."""
    R = _stack(30, 40, 64)
    s = 0.5 * 2.4574561328
    P = lib.opm_sheet_project(to_dev(R, torch), s)
    W = lib.opm_warp_rows(P, P.shape[0], 0.8, 2.0)
    torch.cuda.synchronize()
    ref = O.warp_rows(O.sheet_project(R.astype(np.float64), s), P.shape[0], 0.8, 2.0)
    assert_close(W.cpu().numpy(), ref, what="shear-warp")


def test_sheet_arguments(lib):
    raw = torch.zeros((4, 5, 8), dtype=torch.uint16, device="cuda")
    assert lib.opm_sheet_rows(4, 5, 1.5) == 5 + 5
    with pytest.raises(lib.OpmError) as e:
        lib.opm_sheet_rows(4, 5, -1.0)
    assert e.value.status == lib.OPM_ERR_INVALID_ARG
    bad = torch.empty((3, 8), device="cuda")
    with pytest.raises(ValueError):
        lib.opm_sheet_project(raw, 1.5, out=bad)
