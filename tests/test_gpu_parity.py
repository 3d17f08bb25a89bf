"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
identical seeded inputs.  Bound: max |gpu - oracle| <= 1e-4 * max |oracle| per
FP32 output array, rounded uint16 outputs within 1 LSB, argmax pointing at a
maximal voxel (and at the oracle's first one wherever the maximum is clear).
"""
import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import TOL, assert_between, assert_close, check_argz, nearest_bounds, rel_err, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (nscan, nrows, ncols, theta, step, pixel): tiles, ragged tails, exact-cos
# angles, step < pixel, odd column counts (no TMA), single row/column.
SHAPES = [
    (64, 128, 128, 30.0, 0.4, 0.115),     # the oracle-sized workload
    (40, 70, 264, 35.0, 0.3, 0.1),        # ragged x tile (264 = 256 + 8), ny % 32 != 0
    (33, 50, 200, 45.0, 0.2, 0.115),
    (12, 30, 40, 90.0, 0.125, 0.125),     # pure transpose
    (10, 24, 48, 60.0, 0.125, 0.125),     # weights in {0, 1/2}
    (16, 20, 64, 35.0, 0.05, 0.1),        # step < pixel: two planes per column step
    (9, 17, 37, 30.0, 0.4, 0.115),        # odd column count: plain kernels
    (2, 1, 1, 90.0, 0.2, 0.1),
    (2, 3, 9, 30.0, 0.4, 0.115),
    (5, 1, 8, 20.0, 0.7, 0.1),
]


def _stack(shape, seed=3, blobs=12):
    n, r, c = shape[:3]
    cfg = opm_synth.StackConfig("t", n, r, c, *shape[3:], n_blobs=blobs, sigma=(1.0, 3.0),
                                amp=(200.0, 4000.0), seed=seed)
    return opm_synth.raw_stack(cfg)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("interp", [0, 1])
def test_deskew_u16_to_f32(lib, shape, interp):
    R = _stack(shape)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape, interp=interp)
    vol = lib.deskew(plan, to_dev(R, torch))
    torch.cuda.synchronize()
    if interp == O.NEAREST:
        lo, hi = nearest_bounds(R, g, O)
        assert_between(vol.cpu().numpy(), lo, hi, what=f"deskew nearest {shape}")
    else:
        V = O.deskew(R.astype(np.float64), g, interp)
        assert_close(vol.cpu().numpy(), V, what=f"deskew {shape}")
    lib.opm_plan_check(plan)


@pytest.mark.parametrize("shape", SHAPES[:6])
def test_deskew_u16_rounded(lib, shape):
    R = _stack(shape)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    vol = lib.deskew(plan, to_dev(R, torch), out_dtype=torch.uint16)
    torch.cuda.synchronize()
    ref = O.to_u16(O.deskew(R.astype(np.float64), g)).astype(np.int64)
    got = vol.cpu().to(torch.int32).numpy().astype(np.int64)
    assert np.max(np.abs(got - ref)) <= 1


@pytest.mark.parametrize("shape", SHAPES[:7])
def test_deskew_f32_signed(lib, shape):
    x = opm_synth.gaussian(shape[:3], 5, np.float32)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    vol = lib.deskew(plan, to_dev(x, torch))
    torch.cuda.synchronize()
    assert_close(vol.cpu().numpy(), O.deskew(x.astype(np.float64), g), what="deskew f32")


@pytest.mark.parametrize("shape", [SHAPES[1], SHAPES[5], SHAPES[6]])
def test_deskew_f64(lib, shape):
    x = opm_synth.gaussian(shape[:3], 6, np.float64)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    vol = lib.deskew(plan, to_dev(x, torch))
    torch.cuda.synchronize()
    # weights carry the FP32 fraction of the split tables (~6e-8)
    assert_close(vol.cpu().numpy(), O.deskew(x, g), tol=1e-6, what="deskew f64")


def test_theta60_bitwise(lib):
    """Weights are exactly 0 or 1/2: the FP32 result equals the oracle rounded to FP32."""
    shape = (10, 24, 48, 60.0, 0.125, 0.125)
    R = _stack(shape)
    plan = lib.Plan(*shape)
    vol = lib.deskew(plan, to_dev(R, torch)).cpu().numpy()
    ref = O.deskew(R.astype(np.float64), O.geometry(*shape)).astype(np.float32)
    assert np.array_equal(vol, ref)


def test_bright_voxel_position(lib):
    shape = (64, 128, 16, 30.0, 0.4, 0.115)
    R = opm_synth.bright_voxel(shape[:3], 20, 70, 5, 1000.0, np.float64).astype(np.uint16)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    vol = lib.deskew(plan, to_dev(R, torch)).cpu().numpy()
    nzk, nzj, nzx = np.nonzero(vol)
    assert set(nzk) == {70} and set(nzx) == {5}
    jstar = g.J0 + (20 * g.step + 70 * g.pixel * g.c) / g.pixel
    assert abs(int(np.argmax(vol[70, :, 5])) - round(jstar)) <= 1


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("interp", [0, 1])
def test_project_u16_all_outputs(lib, shape, interp):
    R = _stack(shape)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape, interp=interp)
    out = lib.project(plan, to_dev(R, torch), zmip=True, zsum=True, ymip=True, argz=True)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    Rf = R.astype(np.float64)
    if interp == O.NEAREST:
        lo, hi = nearest_bounds(R, g, O)
        assert_between(out["zmip"].cpu().numpy(), lo.max(0), hi.max(0), what="zmip nearest")
        assert_between(out["zsum"].cpu().numpy(), lo.sum(0), hi.sum(0), what="zsum nearest")
        assert_between(out["ymip"].cpu().numpy(), lo.max(1), hi.max(1), what="ymip nearest")
        a = out["argz"].cpu().numpy().astype(np.int64)
        picked = np.take_along_axis(hi, a[None], axis=0)[0]
        assert np.all(picked >= lo.max(0) - TOL * max(np.max(hi), 1e-30))
        return
    zmip, zsum, ymip, argz = O.project(Rf, g, interp)
    assert_close(out["zmip"].cpu().numpy(), zmip, what="zmip")
    assert_close(out["zsum"].cpu().numpy(), zsum, what="zsum")
    assert_close(out["ymip"].cpu().numpy(), ymip, what="ymip")
    V = O.deskew(Rf, g, interp)
    check_argz(out["argz"].cpu().numpy(), V, zmip, TOL * max(np.max(np.abs(zmip)), 1e-30))


@pytest.mark.parametrize("shape", SHAPES)
def test_project_u16_fast_path(lib, shape):
    """z-MIP and y-MIP only: the two-row, chunked variant."""
    R = _stack(shape, seed=4)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    for want in ({"zmip": True, "ymip": True}, {"zmip": True}, {"ymip": True, "zmip": False}):
        out = lib.project(plan, raw, **want)
        torch.cuda.synchronize()
        zmip, _, ymip, _ = O.project(R.astype(np.float64), g)
        if "zmip" in out:
            assert_close(out["zmip"].cpu().numpy(), zmip, what=f"zmip {want}")
        if "ymip" in out:
            assert_close(out["ymip"].cpu().numpy(), ymip, what=f"ymip {want}")
    lib.opm_plan_check(plan)


@pytest.mark.parametrize("shape", SHAPES[:7])
def test_project_f32_signed(lib, shape):
    """Negative inputs: zero-padded voxels must still take part in the maxima."""
    x = opm_synth.gaussian(shape[:3], 8, np.float32) - 2.0
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    out = lib.project(plan, to_dev(x, torch), zmip=True, zsum=True, ymip=True, argz=True)
    torch.cuda.synchronize()
    xf = x.astype(np.float64)
    zmip, zsum, ymip, argz = O.project(xf, g)
    assert_close(out["zmip"].cpu().numpy(), zmip, what="zmip f32")
    assert_close(out["zsum"].cpu().numpy(), zsum, what="zsum f32")
    assert_close(out["ymip"].cpu().numpy(), ymip, what="ymip f32")
    V = O.deskew(xf, g)
    check_argz(out["argz"].cpu().numpy(), V, zmip, TOL * np.max(np.abs(zmip)))


def test_project_matches_reduced_deskew_bitwise(lib):
    """The fused projections reduce exactly the FP32 voxels opm_deskew writes."""
    shape = SHAPES[1]
    R = _stack(shape)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    vol = lib.deskew(plan, raw)
    fast = lib.project(plan, raw, zmip=True, ymip=True)
    full = lib.project(plan, raw, zmip=True, ymip=True, argz=True)
    torch.cuda.synchronize()
    zref = vol.max(dim=0).values
    yref = vol.max(dim=1).values
    assert torch.equal(fast["zmip"], zref) and torch.equal(fast["ymip"], yref)
    assert torch.equal(full["zmip"], zref) and torch.equal(full["ymip"], yref)


def test_plain_kernels_match_tma(lib, monkeypatch):
    """OPM_FORCE_GENERIC selects the plain kernels; both paths agree."""
    shape = SHAPES[1]
    R = _stack(shape)
    raw = to_dev(R, torch)
    tma = lib.project(lib.Plan(*shape), raw, zmip=True, zsum=True, ymip=True, argz=True)
    monkeypatch.setenv("OPM_FORCE_GENERIC", "1")
    plain_plan = lib.Plan(*shape)
    monkeypatch.delenv("OPM_FORCE_GENERIC")
    plain = lib.project(plain_plan, raw, zmip=True, zsum=True, ymip=True, argz=True)
    torch.cuda.synchronize()
    for k in ("zmip", "ymip"):
        assert torch.equal(tma[k], plain[k]), k
    assert rel_err(tma["zsum"].cpu().numpy(), plain["zsum"].cpu().numpy()) < 1e-6
    assert torch.equal(tma["argz"], plain["argz"])


@pytest.mark.parametrize("shape", SHAPES[:7])
def test_adjoint_f32(lib, shape):
    g = O.geometry(*shape)
    y = opm_synth.gaussian((g.nz, g.ny, g.nx), 9, np.float32)
    plan = lib.Plan(*shape)
    G = lib.skew_adjoint(plan, to_dev(y, torch))
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    assert_close(G.cpu().numpy(), O.skew_adjoint(y.astype(np.float64), g), what="adjoint")


@pytest.mark.parametrize("shape", [(19, 6, 7, 30.0, 0.4, 0.115), (9, 5, 7, 35.0, 0.05, 0.1),
                                   (12, 4, 9, 20.0, 0.7, 0.1)])
@pytest.mark.parametrize("interp", [0, 1])
def test_adjoint_f32_explicit_transpose(lib, shape, interp):
    """Tiny plans, LINEAR and NEAREST, ragged plane groups and columns: the
    adjoint against the transpose of the oracle's entry-by-entry matrix, and
    no device error flag raised."""
    g = O.geometry(*shape)
    y = opm_synth.gaussian((g.nz, g.ny, g.nx), 12, np.float32)
    plan = lib.Plan(*shape, interp=interp)
    G = lib.skew_adjoint(plan, to_dev(y, torch))
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    A = O.explicit_matrix(g, interp)
    ref = (A.T @ y.astype(np.float64).ravel()).reshape(g.nscan, g.nrows, g.ncols)
    assert_close(G.cpu().numpy(), ref, what=f"adjoint vs explicit transpose {shape} interp {interp}")


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[5], SHAPES[6]])
def test_adjoint_f64(lib, shape):
    g = O.geometry(*shape)
    y = opm_synth.gaussian((g.nz, g.ny, g.nx), 10, np.float64)
    plan = lib.Plan(*shape)
    G = lib.skew_adjoint(plan, to_dev(y, torch))
    torch.cuda.synchronize()
    assert_close(G.cpu().numpy(), O.skew_adjoint(y, g), tol=1e-6, what="adjoint f64")


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[2], SHAPES[5]])
def test_dot_test_fp32(lib, shape):
    """<A x, y> = <x, A^T y> to 1e-6 relative with the FP32 kernels."""
    g = O.geometry(*shape)
    x = opm_synth.gaussian(shape[:3], 11, np.float32)
    y = opm_synth.gaussian((g.nz, g.ny, g.nx), 12, np.float32)
    plan = lib.Plan(*shape)
    Ax = lib.deskew(plan, to_dev(x, torch)).double()
    Aty = lib.skew_adjoint(plan, to_dev(y, torch)).double()
    lhs = float((Ax * to_dev(y, torch).double()).sum())
    rhs = float((to_dev(x, torch).double() * Aty).sum())
    scale = float(Ax.norm() * to_dev(y, torch).double().norm())
    assert abs(lhs - rhs) <= 1e-6 * scale
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1], SHAPES[6]])
def test_mip_backward(lib, shape):
    g = O.geometry(*shape)
    x = opm_synth.gaussian(shape[:3], 13, np.float32)   # continuous: no ties
    gz = opm_synth.gaussian((g.ny, g.nx), 14, np.float32)
    plan = lib.Plan(*shape)
    out = lib.project(plan, to_dev(x, torch), zmip=True, argz=True)
    torch.cuda.synchronize()
    zmip, _, _, argz = O.project(x.astype(np.float64), g)
    a_gpu = out["argz"].cpu().numpy()
    agree = a_gpu == argz
    assert agree.mean() > 0.999
    G = lib.mip_backward(plan, to_dev(gz, torch), to_dev(argz.astype(np.int32), torch))
    torch.cuda.synchronize()
    assert_close(G.cpu().numpy(), O.mip_backward(gz.astype(np.float64), argz, g), what="mip backward")


@pytest.mark.parametrize("shape", [(24, 6, 203, 30.0, 0.4, 0.115), SHAPES[4], SHAPES[5], SHAPES[9]])
def test_mip_backward_collisions(lib, shape):
    """Arbitrary arg-max rows, out-of-range ones included: few rows make many
    columns j of one x feed the same raw sample.  The output buffer is
    misaligned and pre-filled with NaN, so every sample must be written."""
    g = O.geometry(*shape)
    rng = np.random.default_rng(21)
    gz = rng.standard_normal((g.ny, g.nx)).astype(np.float32)
    argz = rng.integers(-1, g.nz + 1, size=(g.ny, g.nx)).astype(np.int32)
    plan = lib.Plan(*shape)
    n = int(np.prod(plan.raw_shape))
    buf = torch.full((n + 1,), float("nan"), device="cuda")
    G = buf[1:].view(plan.raw_shape)
    lib.opm_mip_backward(plan, to_dev(gz, torch), to_dev(argz, torch), G)
    torch.cuda.synchronize()
    ref = O.mip_backward(gz.astype(np.float64), argz, g)
    got = G.cpu().numpy()
    assert np.isfinite(got).all()
    assert_close(got, ref, what=f"mip backward {shape}")


@pytest.mark.parametrize("shape,interp", [(SHAPES[0], 0), (SHAPES[4], 1), (SHAPES[5], 0),
                                          ((24, 6, 203, 30.0, 0.4, 0.115), 0)])
def test_mip_backward_is_the_adjoint_of_the_argmax_volume(lib, shape, interp):
    """The z-MIP backward equals the skew adjoint applied to the volume that
    holds g[j][x] at (argz[j][x], j, x) and zero elsewhere, bit for bit: both
    sum each raw sample's terms in ascending j with the same weights, and a
    zero term leaves a sum unchanged.  Arg-max rows are arbitrary (long runs
    of one row, out-of-range rows included) and g has signed zeros."""
    g = O.geometry(*shape)
    rng = np.random.default_rng(31)
    gz = rng.standard_normal((g.ny, g.nx)).astype(np.float32)
    gz[rng.random(gz.shape) < 0.05] = -0.0
    argz = rng.integers(-1, g.nz + 1, size=(g.ny, g.nx)).astype(np.int32)
    argz[:, :5] = 0
    plan = lib.Plan(*shape, interp=interp)
    G = lib.mip_backward(plan, to_dev(gz, torch), to_dev(argz, torch))
    vol = np.zeros((g.nz, g.ny, g.nx), np.float32)
    jj, xx = np.nonzero((argz >= 0) & (argz < g.nz))
    vol[argz[jj, xx], jj, xx] = gz[jj, xx]
    A = lib.skew_adjoint(plan, to_dev(vol, torch))
    torch.cuda.synchronize()
    assert torch.equal(G, A)


def test_non_default_stream_and_no_allocation(lib):
    shape = SHAPES[0]
    R = _stack(shape)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    zmip = torch.empty((plan.ny, plan.nx), device="cuda")
    ymip = torch.empty((plan.nz, plan.nx), device="cuda")
    vol = torch.empty(plan.vol_shape, device="cuda")
    s = torch.cuda.Stream()
    # warm-up: the first launch of each kernel loads its module
    lib.opm_project(plan, raw, zmip, None, ymip, None)
    lib.opm_deskew(plan, raw, vol)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with torch.cuda.stream(s):
        for _ in range(3):
            lib.opm_project(plan, raw, zmip, None, ymip, None, stream=s)
            lib.opm_deskew(plan, raw, vol, stream=s)
    s.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    zref, _, yref, _ = O.project(R.astype(np.float64), O.geometry(*shape))
    assert_close(zmip.cpu().numpy(), zref)
    assert_close(ymip.cpu().numpy(), yref)


def test_abi_errors_on_device(lib):
    plan = lib.Plan(8, 6, 16, 30.0, 0.4, 0.115)
    raw = torch.zeros(plan.raw_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.OpmError) as e:
        lib.project(plan, raw)
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED
    vol = torch.zeros(plan.vol_shape, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.OpmError) as e:
        lib.opm_deskew(plan, raw, vol)
    assert e.value.status == lib.OPM_ERR_UNSUPPORTED
    raw16 = torch.zeros(plan.raw_shape, dtype=torch.uint16, device="cuda")
    st = lib.load().opm_project(plan.handle, __import__("ctypes").c_void_p(raw16.data_ptr()), lib.OPM_U16,
                                None, None, None, None, None)
    assert st == lib.OPM_ERR_INVALID_ARG


@pytest.fixture(scope="module")
def liveview():
    c = opm_synth.CONFIGS["liveview_200x512x2048"]
    return c, opm_synth.raw_stack(c)


def test_liveview_full_size_sampled(lib, liveview):
    """200x512x2048 live-view stack in the bench's launch configuration:
    every z-MIP/y-MIP pixel of seeded sample columns and all tile edges."""
    c, R = liveview
    g = O.geometry(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    plan = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    raw = to_dev(R, torch)
    out = lib.project(plan, raw, zmip=True, ymip=True)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    zg = out["zmip"].cpu().numpy()
    yg = out["ymip"].cpu().numpy()
    rng = np.random.default_rng(2)
    xs = np.unique(np.concatenate([rng.integers(0, c.ncols, 24), [0, 255, 256, 1023, 1024, c.ncols - 1]]))
    Rs = R[:, :, xs].astype(np.float64)       # x columns are independent
    gs = O.geometry(c.nscan, c.nrows, len(xs), c.theta_deg, c.step, c.pixel)
    zmip, _, ymip, _ = O.project(Rs, gs)
    assert_close(zg[:, xs], zmip, what="zmip sampled")
    assert_close(yg[:, xs], ymip, what="ymip sampled")
    # every column: the fused projection equals a second path (plain kernels)
    vol = lib.deskew(plan, raw)
    torch.cuda.synchronize()
    assert torch.equal(vol.max(dim=0).values, out["zmip"])
    assert torch.equal(vol.max(dim=1).values, out["ymip"])
    del vol
    # full FP32 volume on sampled voxels
    ks = rng.integers(0, g.nz, 2000)
    js = rng.integers(0, g.ny, 2000)
    xv = rng.integers(0, g.nx, 2000)
    vol = lib.deskew(plan, raw)
    torch.cuda.synchronize()
    got = vol[torch.from_numpy(ks).cuda(), torch.from_numpy(js).cuda(), torch.from_numpy(xv).cuda()].cpu().numpy()
    ref = O.voxels(R, g, ks, js, xv)
    assert np.max(np.abs(got - ref)) <= TOL * float(np.max(np.abs(zmip)))


def test_liveview_full_size_every_column(lib, liveview):
    """The live view of the full 200 x 512 x 2048 stack (the bench's step,
    periodic kernel) against the oracle on every column, the oracle run over
    blocks of columns on all host cores."""
    from oracle_pool import project_columns
    c, R = liveview
    plan = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    assert lib.opm_plan_path(plan)[0] == lib.OPM_PATH_PERIODIC
    out = lib.project(plan, to_dev(R, torch), zmip=True, ymip=True)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    zmip, ymip = project_columns(R, c.theta_deg, c.step, c.pixel)
    assert_close(out["zmip"].cpu().numpy(), zmip, what="zmip, every column")
    assert_close(out["ymip"].cpu().numpy(), ymip, what="ymip, every column")


@pytest.mark.parametrize("width", [1024, 512, 256, 128])
def test_liveview_narrow_stack_schedule(lib, liveview, width):
    """The first `width` columns of the 200 x 512 x 2048 stack (an x-shard of
    it): the plan cuts its units short enough that every persistent CTA list
    still gets work (at least 1.1 units per list, or the 16-row floor), and
    the live view matches the oracle on every column."""
    from oracle_pool import project_columns
    c, R = liveview
    Rw = np.ascontiguousarray(R[:, :, :width])
    plan = lib.Plan(c.nscan, c.nrows, width, c.theta_deg, c.step, c.pixel)
    whole = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    nunits, nlists, rows = lib.opm_plan_schedule(plan)
    _, wlists, wrows = lib.opm_plan_schedule(whole)
    assert nlists == wlists > 0
    assert rows in (16, 32, 64, 128, 256) and rows <= wrows
    assert nunits >= 1.1 * nlists or rows == 16
    if nlists <= 756:                       # 832 units of 256 rows at full width
        assert wrows == 256
    out = lib.project(plan, to_dev(Rw, torch), zmip=True, ymip=True)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    zmip, ymip = project_columns(Rw, c.theta_deg, c.step, c.pixel)
    assert_close(out["zmip"].cpu().numpy(), zmip, what=f"zmip, width {width}")
    assert_close(out["ymip"].cpu().numpy(), ymip, what=f"ymip, width {width}")


def test_large_full_size_sampled(lib):
    """1000 x 1024 x 2048 uint16 stack (theta 45, step 0.2, pixel 0.115):
    FP32 and round-to-nearest uint16 volumes and the z-MIP at full size,
    against the oracle on sampled columns and voxels; the uint16 volume equals
    the rounded FP32 volume everywhere."""
    c = opm_synth.CONFIGS["large_1000x1024x2048"]
    R = opm_synth.tiled_stack((c.nscan, c.nrows, c.ncols), seed=c.seed)
    g = O.geometry(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    plan = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    raw = to_dev(R, torch)
    zmip = lib.project(plan, raw, zmip=True)["zmip"]
    vol = lib.deskew(plan, raw)                                    # FP32, 20.7 GB
    vol16 = lib.deskew(plan, raw, out_dtype=torch.uint16)          # 10.3 GB
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    rng = np.random.default_rng(3)
    xs = np.unique(np.concatenate([rng.integers(0, c.ncols, 6), [0, 127, 128, c.ncols - 1]]))
    Rs = R[:, :, xs].astype(np.float64)
    gs = O.geometry(c.nscan, c.nrows, len(xs), c.theta_deg, c.step, c.pixel)
    zref, _, _, _ = O.project(Rs, gs)
    assert_close(zmip.cpu().numpy()[:, xs], zref, what="large zmip sampled")
    ks = rng.integers(0, g.nz, 4000)
    js = rng.integers(0, g.ny, 4000)
    xv = rng.integers(0, g.nx, 4000)
    idx = (torch.from_numpy(ks).cuda(), torch.from_numpy(js).cuda(), torch.from_numpy(xv).cuda())
    ref = O.voxels(R, g, ks, js, xv)
    got = vol[idx].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL * float(np.max(np.abs(zref)))
    got16 = vol16.view(torch.int16)[idx].cpu().numpy().view(np.uint16).astype(np.int64)
    assert np.max(np.abs(got16 - O.to_u16(ref).astype(np.int64))) <= 1
    for k0 in range(0, g.nz, 64):                                  # whole volume, in slabs of rows
        r = torch.round(vol[k0:k0 + 64]).clamp_(0, 65535).to(torch.int32)
        assert torch.equal(r, vol16[k0:k0 + 64].view(torch.int16).to(torch.int32) & 0xFFFF)
    assert torch.equal(vol.max(dim=0).values, zmip)
    # both volumes in one pass: the same bytes as the two separate calls
    vol_b = torch.empty_like(vol)
    vol16_b = torch.empty_like(vol16)
    lib.opm_deskew_dual(plan, raw, vol_b, vol16_b)
    torch.cuda.synchronize()
    assert torch.equal(vol_b, vol)
    assert torch.equal(vol16_b.view(torch.int16), vol16.view(torch.int16))


@pytest.mark.parametrize("shape", [(16, 24, 32, 45.0, 0.2, 0.115), (33, 50, 264, 35.0, 0.3, 0.1)])
@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_deskew_dual_small(lib, shape, dtype):
    n, r, c = shape[:3]
    R = opm_synth.raw_stack(opm_synth.StackConfig("d", *shape, n_blobs=5, sigma=(1.0, 3.0), amp=(200.0, 4000.0),
                                                  seed=8))
    if dtype == "f32":
        R = R.astype(np.float32) - 300.0
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    f = torch.empty(plan.vol_shape, device="cuda")
    u = torch.empty(plan.vol_shape, dtype=torch.uint16, device="cuda")
    lib.opm_deskew_dual(plan, raw, f, u)
    torch.cuda.synchronize()
    assert torch.equal(f, lib.deskew(plan, raw))
    assert torch.equal(u.view(torch.int16), lib.deskew(plan, raw, out_dtype=torch.uint16).view(torch.int16))
    g = O.geometry(*shape)
    ref = O.deskew(R.astype(np.float64), g)
    assert_close(f.cpu().numpy(), ref, what="dual f32")
    got = u.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.int64)
    assert np.max(np.abs(got - O.to_u16(ref).astype(np.int64))) <= 1


TINY = [(2, 1, 1, 90.0, 0.1, 0.1), (2, 1, 9, 45.0, 0.2, 0.115), (3, 2, 5, 30.0, 0.4, 0.115),
        (2, 3, 7, 60.0, 0.1, 0.1), (4, 1, 3, 35.0, 0.05, 0.1), (5, 2, 2, 89.0, 0.3, 0.1)]


@pytest.mark.parametrize("shape", TINY)
def test_tiny_odd_shapes_every_kernel(lib, shape):
    """Two planes, one row, 1..9 columns, 90 degrees: every call against the
    oracle (degenerate extents and ragged vectors everywhere)."""
    g = O.geometry(*shape)
    R = (np.arange(np.prod(g.nscan * g.nrows * g.ncols)).reshape(g.nscan, g.nrows, g.ncols) * 37 % 1000 + 1
         ).astype(np.uint16)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    Rf = R.astype(np.float64)
    V = O.deskew(Rf, g)
    assert_close(lib.deskew(plan, raw).cpu().numpy(), V, what="tiny deskew")
    out = lib.project(plan, raw, zmip=True, zsum=True, ymip=True, argz=True)
    zmip, zsum, ymip, _ = O.project(Rf, g)
    assert_close(out["zmip"].cpu().numpy(), zmip, what="tiny zmip")
    assert_close(out["zsum"].cpu().numpy(), zsum, what="tiny zsum")
    assert_close(out["ymip"].cpu().numpy(), ymip, what="tiny ymip")
    f = lib.project(plan, raw, zmip=True, ymip=True)
    assert torch.equal(f["zmip"], out["zmip"]) and torch.equal(f["ymip"], out["ymip"])
    vf = torch.empty(plan.vol_shape, device="cuda")
    zm = torch.empty((plan.ny, plan.nx), device="cuda")
    ym = torch.empty((plan.nz, plan.nx), device="cuda")
    lib.opm_deskew_mip(plan, raw, vf, None, zm, ym)
    zs, ys = torch.empty_like(zm), torch.empty_like(ym)
    lib.opm_stream_begin(plan, zs, None, ys)
    for n in range(-1, g.nscan):
        lib.opm_stream_pair(plan, raw[n] if n >= 0 else None, raw[n + 1] if n + 1 < g.nscan else None, n, zs, None, ys)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    assert torch.equal(vf, lib.deskew(plan, raw))
    assert torch.equal(zm, f["zmip"]) and torch.equal(ym, f["ymip"])
    assert torch.equal(zs, f["zmip"]) and torch.equal(ys, f["ymip"])
    Y = opm_synth.gaussian(plan.vol_shape, 5, np.float32)
    G = lib.skew_adjoint(plan, to_dev(Y, torch))
    torch.cuda.synchronize()
    assert_close(G.cpu().numpy(), O.skew_adjoint(Y.astype(np.float64), g), what="tiny adjoint")


def test_one_plan_many_threads(lib):
    """A plan is immutable after creation: several host threads use it on
    their own streams at once and each gets the single-threaded result."""
    import threading
    shape = (64, 128, 128, 30.0, 0.4, 0.115)
    plan = lib.Plan(*shape)
    stacks = [to_dev(_stack(shape, seed=50 + i), torch) for i in range(4)]
    ref = [lib.project(plan, r, zmip=True, ymip=True) for r in stacks]
    vref = [lib.deskew(plan, r) for r in stacks]
    torch.cuda.synchronize()
    got = [None] * 4
    errors = []

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(5):
                    o = lib.project(plan, stacks[i], zmip=True, ymip=True, stream=s)
                    v = lib.deskew(plan, stacks[i], stream=s)
            s.synchronize()
            got[i] = (o, v)
        except Exception as e:  # surfaced below
            errors.append(e)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors
    lib.opm_plan_check(plan)
    for i in range(4):
        o, v = got[i]
        assert torch.equal(o["zmip"], ref[i]["zmip"]) and torch.equal(o["ymip"], ref[i]["ymip"])
        assert torch.equal(v, vref[i])
