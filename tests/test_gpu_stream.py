"""Plane-by-plane live view: the projections accumulated one scan-plane
pair at a time equal the whole-stack projection (z-MIP and y-MIP bit for
bit, z-sum to the FP32 tolerance), partial views equal the oracle's
projection of the voxels already determined, and the rolling / global
modes publish what they promise."""
import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import assert_between, assert_close, nearest_bounds, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(64, 128, 128, 30.0, 0.4, 0.115), (33, 50, 264, 45.0, 0.2, 0.115), (40, 70, 136, 35.0, 0.3, 0.1),
          (16, 20, 64, 35.0, 0.05, 0.1), (12, 9, 30, 90.0, 0.1, 0.1)]


def _stack(shape, seed=3):
    return opm_synth.raw_stack(opm_synth.StackConfig("s", *shape, n_blobs=8, sigma=(1.0, 3.0),
                                                     amp=(200.0, 4000.0), seed=seed))


def _accumulate(lib, plan, raw, order=None, zsum=True):
    z = torch.empty((plan.ny, plan.nx), device="cuda")
    s = torch.empty((plan.ny, plan.nx), device="cuda") if zsum else None
    y = torch.empty((plan.nz, plan.nx), device="cuda")
    lib.opm_stream_begin(plan, z, s, y)
    ns = list(range(-1, plan.nscan)) if order is None else order
    for n in ns:
        lo = raw[n] if n >= 0 else None
        hi = raw[n + 1] if n + 1 < plan.nscan else None
        lib.opm_stream_pair(plan, lo, hi, n, z, s, y)
    torch.cuda.synchronize()
    lib.opm_plan_check(plan)
    return z, s, y


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("interp", [0, 1])
def test_pairs_equal_whole_stack(lib, shape, interp):
    R = _stack(shape)
    plan = lib.Plan(*shape, interp=interp)
    raw = to_dev(R, torch)
    z, s, y = _accumulate(lib, plan, raw)
    full = lib.project(plan, raw, zmip=True, zsum=True, ymip=True)
    assert torch.equal(z, full["zmip"])
    assert torch.equal(y, full["ymip"])
    g = O.geometry(*shape)
    if interp == O.NEAREST:                 # either plane is correct at an exact tie
        lo, hi = nearest_bounds(R, g, O)
        assert_between(z.cpu().numpy(), lo.max(0), hi.max(0), what="stream zmip nearest")
        assert_between(s.cpu().numpy(), lo.sum(0), hi.sum(0), what="stream zsum nearest")
        assert_between(y.cpu().numpy(), lo.max(1), hi.max(1), what="stream ymip nearest")
        return
    zr, sr, yr, _ = O.project(R.astype(np.float64), g, interp)
    assert_close(z.cpu().numpy(), zr, what="stream zmip")
    assert_close(s.cpu().numpy(), sr, what="stream zsum")
    assert_close(y.cpu().numpy(), yr, what="stream ymip")


def test_pair_order_does_not_matter(lib):
    shape = SHAPES[0]
    R = _stack(shape, seed=5)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    z0, _, y0 = _accumulate(lib, plan, raw, zsum=False)
    order = list(np.random.default_rng(1).permutation(np.arange(-1, plan.nscan)))
    z1, _, y1 = _accumulate(lib, plan, raw, order=order, zsum=False)
    assert torch.equal(z0, z1) and torch.equal(y0, y1)


@pytest.mark.parametrize("m", [0, 1, 17, 40])
def test_partial_view_is_the_projection_of_determined_voxels(lib, m):
    """After frames 0..m-1 the view holds exactly the voxels whose lower
    plane is at most m - 2 (both interpolation planes received)."""
    shape = SHAPES[2]
    R = _stack(shape, seed=7)
    g = O.geometry(*shape)
    plan = lib.Plan(*shape)
    raw = to_dev(R, torch)
    z, _, y = _accumulate(lib, plan, raw, order=list(range(-1, m - 1)), zsum=False)
    V = O.deskew(R.astype(np.float64), g)                       # [nz, ny, nx]
    kk, jj = np.meshgrid(np.arange(g.nz), np.arange(g.ny), indexing="ij")
    n0 = np.floor(O.plane_coord(g, jj, kk)).astype(np.int64)     # [nz, ny]
    Vm = np.where((n0 <= m - 2)[:, :, None], V, 0.0)
    assert_close(z.cpu().numpy(), Vm.max(axis=0), what=f"partial zmip m={m}")
    assert_close(y.cpu().numpy(), Vm.max(axis=1), what=f"partial ymip m={m}")


def test_rolling_and_global_modes(lib):
    from paper_2211_00645_gb300.rolling import RollingView
    shape = SHAPES[0]
    plan = lib.Plan(*shape)
    stacks = [_stack(shape, seed=s) for s in (11, 12)]
    roll = RollingView(plan, mode="rolling", zsum=True)
    glob = RollingView(plan, mode="global")
    for R in stacks:
        host = torch.from_numpy(R.view(np.int16)).view(torch.uint16)
        for n in range(plan.nscan):
            r = roll.push(host[n])
            gv = glob.push(host[n])
            assert r is not None and r["frames"] == n + 1
            assert (gv is not None) == (n == plan.nscan - 1)
        torch.cuda.synchronize()
        full = lib.project(plan, to_dev(R, torch), zmip=True, ymip=True)
        assert r["complete"] and gv["complete"]
        assert torch.equal(r["zmip"], full["zmip"]) and torch.equal(r["ymip"], full["ymip"])
        assert torch.equal(gv["zmip"], full["zmip"]) and torch.equal(gv["ymip"], full["ymip"])
    assert roll.stacks == glob.stacks == 2


def test_stream_argument_checks(lib):
    shape = SHAPES[0]
    plan = lib.Plan(*shape)
    raw = torch.zeros(plan.raw_shape, dtype=torch.uint16, device="cuda")
    z = torch.empty((plan.ny, plan.nx), device="cuda")
    for lo, hi, n in [(None, raw[0], 0), (raw[0], raw[1], -1), (raw[0], raw[1], plan.nscan - 1),
                      (raw[0], None, 3), (None, raw[0], -2), (raw[0], None, plan.nscan)]:
        with pytest.raises(lib.OpmError) as e:
            lib.opm_stream_pair(plan, lo, hi, n, z, None, None)
        assert e.value.status == lib.OPM_ERR_INVALID_ARG
    with pytest.raises(lib.OpmError):
        lib.opm_stream_begin(plan, None, None, None)


def test_sliding_mode_spans_a_full_stack(lib):
    """Sliding mode: after frames 0..m-1 of the second stack, the view is the
    projection of (second stack's frames 0..m-1, first stack's m..N-1)."""
    from paper_2211_00645_gb300.rolling import RollingView
    shape = SHAPES[2]
    plan = lib.Plan(*shape)
    A, B = _stack(shape, seed=21), _stack(shape, seed=22)
    view = RollingView(plan, mode="sliding")
    ha = torch.from_numpy(A.view(np.int16)).view(torch.uint16)
    hb = torch.from_numpy(B.view(np.int16)).view(torch.uint16)
    for n in range(plan.nscan):
        out = view.push(ha[n])
    assert out["complete"] and out["stacks"] == 1
    torch.cuda.synchronize()
    full_a = lib.project(plan, to_dev(A, torch), zmip=True, ymip=True)
    assert torch.equal(out["zmip"], full_a["zmip"]) and torch.equal(out["ymip"], full_a["ymip"])
    m = 17
    for n in range(m):
        out = view.push(hb[n])
    torch.cuda.synchronize()
    mixed = np.concatenate([B[:m], A[m:]], axis=0)
    ref = lib.project(plan, to_dev(mixed, torch), zmip=True, ymip=True)
    assert out["frames"] == m and not out["complete"]
    assert torch.equal(out["zmip"], ref["zmip"]) and torch.equal(out["ymip"], ref["ymip"])
    zr, _, yr, _ = O.project(mixed.astype(np.float64), O.geometry(*shape))
    assert_close(out["zmip"].cpu().numpy(), zr, what="sliding zmip")


@pytest.mark.parametrize("shape", [(12, 40, 72, 35.0, 0.3, 0.1), (2, 30, 64, 35.0, 0.3, 0.1),
                                   (9, 20, 64, 35.0, 0.05, 0.1), (7, 9, 30, 90.0, 0.1, 0.1)])
def test_sliding_view_every_push_over_three_stacks(lib, shape):
    """Sliding mode (running maximum + the previous stack's suffix maxima +
    the mixed pair): after every push of three stacks, starting from the
    all-zero stack, the view equals opm_project of the stack buffer it spans
    (newest frames 0..m, the previous stack's m+1..N-1) bit for bit."""
    from paper_2211_00645_gb300.rolling import RollingView
    plan = lib.Plan(*shape)
    N = plan.nscan
    stacks = [_stack(shape, seed=40 + i) for i in range(3)]
    view = RollingView(plan, mode="sliding")
    buf = np.zeros_like(stacks[0])
    for si, S in enumerate(stacks):
        hs = torch.from_numpy(S.view(np.int16)).view(torch.uint16)
        for m in range(N):
            out = view.push(hs[m])
            buf[m] = S[m]
            torch.cuda.synchronize()
            ref = lib.project(plan, to_dev(buf, torch), zmip=True, ymip=True)
            assert out["complete"] == (m == N - 1)
            assert torch.equal(out["zmip"], ref["zmip"]), (si, m, "zmip")
            assert torch.equal(out["ymip"], ref["ymip"]), (si, m, "ymip")
        assert out["stacks"] == si + 1
    lib.opm_plan_check(plan)


def test_max_combine(lib):
    """opm_max_combine: elementwise maximum, in place or into a third array,
    on aligned (vector) and unaligned / ragged (scalar) arrays, with signed
    values and infinities."""
    g = torch.Generator(device="cuda").manual_seed(5)
    for n, off in ((4096, 0), (1001, 0), (4096, 1)):
        a = torch.randn(n + off, device="cuda", generator=g)[off:]
        b = torch.randn(n + off, device="cuda", generator=g)[off:]
        a[::7] = -float("inf")
        out = torch.empty(n, device="cuda")
        lib.opm_max_combine(out, a, b)
        torch.cuda.synchronize()
        assert torch.equal(out, torch.maximum(a, b))
        a2 = a.clone()
        lib.opm_max_combine(a2, a2, b)
        torch.cuda.synchronize()
        assert torch.equal(a2, torch.maximum(a, b))
