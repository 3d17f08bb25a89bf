"""Differentiation through the library: autograd Functions, FP64 gradient
checks, finite differences of the z-MIP backward and a gradient-descent
reconstruction (the adjoint as the forward model of an acquisition)."""
import numpy as np
import pytest

import opm_synth
import oracle as O
from gpu_util import assert_close, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FD_SHAPE = (16, 24, 32, 30.0, 0.4, 0.115)     # the finite-difference case (ny = 79)


@pytest.fixture(scope="module")
def ag(lib):
    from paper_2211_00645_gb300 import autograd
    return autograd


def test_gradcheck_deskew_fp64(lib, ag):
    plan = lib.Plan(*FD_SHAPE)
    assert plan.ny == 79
    x = torch.from_numpy(opm_synth.gaussian(plan.raw_shape, 21)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: ag.deskew(t, plan), (x,), eps=1e-6, atol=1e-7, rtol=1e-6,
                                    fast_mode=True)


def test_gradcheck_skew_fp64(lib, ag):
    plan = lib.Plan(*FD_SHAPE)
    v = torch.from_numpy(opm_synth.gaussian(plan.vol_shape, 22)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: ag.skew(t, plan), (v,), eps=1e-6, atol=1e-7, rtol=1e-6,
                                    fast_mode=True)


def test_deskew_backward_matches_oracle_adjoint(lib, ag):
    plan = lib.Plan(*FD_SHAPE)
    g = O.geometry(*FD_SHAPE)
    x = torch.from_numpy(opm_synth.gaussian(plan.raw_shape, 23, np.float32)).cuda().requires_grad_(True)
    y = opm_synth.gaussian(plan.vol_shape, 24, np.float32)
    loss = (ag.deskew(x, plan) * to_dev(y, torch)).sum()
    loss.backward()
    assert_close(x.grad.cpu().numpy(), O.skew_adjoint(y.astype(np.float64), g), what="dL/draw")


def test_zmip_backward_finite_differences(lib, ag):
    """sum(g * zmip(R)) differentiated by central differences in FP64 (oracle)
    against ProjectFn.backward on a tie-free Gaussian stack."""
    shape = (6, 5, 8, 30.0, 0.4, 0.115)
    plan = lib.Plan(*shape)
    g = O.geometry(*shape)
    R = opm_synth.gaussian(plan.raw_shape, 25, np.float32)
    gz = opm_synth.gaussian((plan.ny, plan.nx), 26, np.float32)
    x = to_dev(R, torch).requires_grad_(True)
    (ag.zmip(x, plan) * to_dev(gz, torch)).sum().backward()
    Rd = R.astype(np.float64)
    h = 1e-5
    fd = np.empty_like(Rd)
    for idx in np.ndindex(Rd.shape):
        Rp = Rd.copy(); Rp[idx] += h
        Rm = Rd.copy(); Rm[idx] -= h
        fd[idx] = (np.sum(gz * O.project(Rp, g)[0]) - np.sum(gz * O.project(Rm, g)[0])) / (2 * h)
    assert_close(x.grad.cpu().numpy(), fd, tol=1e-4, what="zmip backward vs FD")


def test_dot_test_diff_config(lib):
    """128 x 256 x 256 differentiable stack: <A x, y> = <x, A^T y> to 1e-6 relative."""
    c = opm_synth.CONFIGS["diff_128x256x256"]
    plan = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    assert plan.ny == 670
    x = to_dev(opm_synth.gaussian(plan.raw_shape, 31, np.float32), torch)
    y = to_dev(opm_synth.gaussian(plan.vol_shape, 32, np.float32), torch)
    Ax = lib.deskew(plan, x).double()
    Aty = lib.skew_adjoint(plan, y).double()
    lhs = float((Ax * y.double()).sum())
    rhs = float((x.double() * Aty).sum())
    assert abs(lhs - rhs) <= 1e-6 * float(Ax.norm() * y.double().norm())


def _ground_truth_volume(plan, n_blobs=300, seed=4):
    """Seeded blobs on the output grid (k, j, x)."""
    cfg = opm_synth.StackConfig("gt", plan.nz, plan.ny, plan.nx, 30.0, 0.4, 0.115, n_blobs=n_blobs,
                                sigma=(1.5, 4.0), amp=(200.0, 1000.0), background=0.0, seed=seed)
    vol = np.zeros((plan.nz, plan.ny, plan.nx), dtype=np.float32)
    centres, sig, amp = opm_synth.blob_params(cfg)
    kk, jj, xx = [np.arange(n, dtype=np.float32) for n in (plan.nz, plan.ny, plan.nx)]
    for (ck, cj, cx), s, a in zip(centres, sig, amp):
        r = int(np.ceil(4 * s))
        k0, k1 = max(0, int(ck) - r), min(plan.nz, int(ck) + r + 1)
        j0, j1 = max(0, int(cj) - r), min(plan.ny, int(cj) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(plan.nx, int(cx) + r + 1)
        gk = np.exp(-(kk[k0:k1] - ck) ** 2 / (2 * s * s))
        gj = np.exp(-(jj[j0:j1] - cj) ** 2 / (2 * s * s))
        gx = np.exp(-(xx[x0:x1] - cx) ** 2 / (2 * s * s))
        vol[k0:k1, j0:j1, x0:x1] += a * gk[:, None, None] * gj[None, :, None] * gx[None, None, :]
    return vol


def test_gradient_descent_reconstruction(lib, ag):
    """GT volume -> A^T -> scaled to a 1000-count peak -> Poisson -> 100 GD steps
    on 0.5 ||A^T x - y||^2 with eta = 1/L: the loss never increases and the
    volume moves towards the ground truth."""
    c = opm_synth.CONFIGS["diff_128x256x256"]
    plan = lib.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    gt = torch.from_numpy(_ground_truth_volume(plan)).cuda()
    clean = ag.skew(gt, plan)
    scale = 1000.0 / float(clean.max())
    gt = gt * scale
    clean = clean * scale
    gen = torch.Generator(device="cuda").manual_seed(4)
    measured = torch.poisson(clean.clamp_min(0), generator=gen)
    L = ag.power_iteration(plan, iters=20)
    assert L > 0
    x, losses = ag.reconstruct(plan, measured, iters=100, eta=1.0 / L, lipschitz=L)
    torch.cuda.synchronize()
    losses = np.array(losses)
    assert np.all(np.diff(losses) <= 1e-6 * losses[0])       # monotone for eta <= 1/L
    assert losses[-1] < 0.05 * losses[0]
    err0 = float(gt.norm())
    err = float((x - gt).norm())
    assert err < 0.8 * err0


def test_reconstruction_checkpoint_resume(lib, ag, tmp_path):
    """An interrupted run resumed from its checkpoint ends on exactly the
    iterate (and losses) of an uninterrupted run."""
    plan = lib.Plan(32, 40, 48, 30.0, 0.4, 0.115)
    gen = torch.Generator(device="cuda").manual_seed(2)
    measured = torch.rand(plan.raw_shape, generator=gen, device="cuda") * 100
    L = ag.power_iteration(plan, iters=10)
    x_full, l_full = ag.reconstruct(plan, measured, iters=25, eta=1.0 / L, lipschitz=L)
    ck = str(tmp_path / "gd.pt")
    ag.reconstruct(plan, measured, iters=20, eta=1.0 / L, lipschitz=L, checkpoint=ck, every=10)   # "interrupted"
    x_res, l_res = ag.reconstruct(plan, measured, iters=25, checkpoint=ck, every=10)                # resumed
    torch.cuda.synchronize()
    assert torch.equal(x_res, x_full)
    assert l_res == l_full
    state = torch.load(ck)
    assert state["iters"] == 25 and len(state["losses"]) == 25
