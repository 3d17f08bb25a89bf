"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the explicit
interpolation matrix built entry by entry, closed forms (constant, affine and
single-voxel inputs), special angles where the deskew reduces to a transpose,
the grid extents, finite differences, and the Fig. 2 claim that deskewing
restores the true cross-section of an object.
"""
import math

import numpy as np
import pytest

import opm_synth
import oracle as O

# (nscan, nrows, ncols, theta, step, pixel): rho = pixel/step below and above 1,
# the exact-cos angles and generic ones.
TINY = [
    (5, 4, 3, 30.0, 0.4, 0.115),
    (4, 3, 2, 45.0, 0.2, 0.115),
    (3, 5, 2, 90.0, 0.3, 0.1),
    (4, 4, 2, 60.0, 0.1, 0.1),
    (6, 3, 2, 35.0, 0.05, 0.1),    # step < pixel: several planes per column
    (2, 1, 1, 90.0, 0.2, 0.1),
    (3, 2, 3, 12.5, 0.37, 0.11),
]


def _rand(shape, seed):
    return opm_synth.gaussian(shape, seed)


@pytest.mark.parametrize("p", TINY)
@pytest.mark.parametrize("interp", [O.LINEAR, O.NEAREST])
def test_gather_equals_explicit_matrix(p, interp):
    """Brute force: the row-wise gather equals A @ vec(R) entry for entry."""
    g = O.geometry(*p)
    A = O.explicit_matrix(g, interp)
    R = _rand(g.nscan * g.nrows * g.ncols, 11).reshape(g.nscan, g.nrows, g.ncols)
    V = O.deskew(R, g, interp)
    np.testing.assert_allclose(V.reshape(-1), A @ R.reshape(-1), rtol=0, atol=1e-12)
    # the per-voxel evaluator agrees with both
    k, j, x = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    np.testing.assert_allclose(O.voxels(R, g, k, j, x, interp), V, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", TINY)
def test_adjoint_is_transpose(p):
    g = O.geometry(*p)
    A = O.explicit_matrix(g)
    Y = _rand(g.nz * g.ny * g.nx, 12).reshape(g.nz, g.ny, g.nx)
    G = O.skew_adjoint(Y, g)
    np.testing.assert_allclose(G.reshape(-1), A.T @ Y.reshape(-1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("cfg", ["oracle_64x128x128", "diff_128x256x256"])
def test_dot_test_fp64(cfg):
    """<A x, y> = <x, A^T y> to 1e-12 relative on full-size shapes (one x-column band)."""
    c = opm_synth.CONFIGS[cfg]
    g = O.geometry(c.nscan, c.nrows, 8, c.theta_deg, c.step, c.pixel)
    x = _rand((g.nscan, g.nrows, g.ncols), 21)
    y = _rand((g.nz, g.ny, g.nx), 22)
    lhs = float(np.sum(O.deskew(x, g) * y))
    rhs = float(np.sum(x * O.skew_adjoint(y, g)))
    scale = np.linalg.norm(O.deskew(x, g)) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("p", TINY + [(64, 128, 4, 30.0, 0.4, 0.115), (200, 64, 3, 35.0, 0.3, 0.1)])
def test_constant_reproduced_on_covered_region(p):
    g = O.geometry(*p)
    R = np.full((g.nscan, g.nrows, g.ncols), 1234.0)
    V = O.deskew(R, g)
    cov = O.covered_mask(g)
    assert cov.any()
    np.testing.assert_allclose(V[cov], 1234.0, rtol=0, atol=1e-9)


def test_covered_mask_hand_counted():
    """The fully covered region {0 <= n_f <= nscan - 1}, counted by hand on
    geometries whose n_f is exact in binary: the constant and affine pins use
    this mask, so it must be neither too wide nor too narrow."""
    # theta 60 (cos = 1/2), step = pixel: n_f = j - k/2, J0 = 0, ny = ceil(3 + 1/2) = 4
    g = O.geometry(3, 2, 1, 60.0, 0.125, 0.125)
    assert (g.J0, g.ny) == (0, 4)
    want = np.array([[1, 1, 1, 0],    # n_f = 0, 1, 2, 3
                     [0, 1, 1, 0]],   # n_f = -1/2, 1/2, 3/2, 5/2
                    dtype=bool)
    assert np.array_equal(O.covered_mask(g), want)
    # step = 2 pixel: n_f = (j - 1)/2 - k/4, J0 = 1, ny = ceil(1 + 6 + 1) = 8
    g = O.geometry(3, 3, 1, 60.0, 0.25, 0.125)
    assert (g.J0, g.ny) == (1, 8)
    want = np.zeros((3, 8), dtype=bool)
    want[0, 1:6] = True               # (j - 1)/2 in [0, 2]
    want[1, 2:6] = True               # (j - 1)/2 - 1/4 in [0, 2]: j - 1 in [1/2, 9/2]
    want[2, 2:7] = True               # (j - 1)/2 - 1/2 in [0, 2]: j - 1 in [1, 5]
    assert np.array_equal(O.covered_mask(g), want)


@pytest.mark.parametrize("p", TINY + [(64, 128, 4, 30.0, 0.4, 0.115)])
def test_affine_ramp_reproduced(p):
    """R = a n + b r + c x + d  ->  V = a n_f + b k + c x + d where fully covered."""
    g = O.geometry(*p)
    a, b, cx, d = 3.5, -1.25, 0.75, 40.0
    n, r, x = np.meshgrid(np.arange(g.nscan), np.arange(g.nrows), np.arange(g.ncols), indexing="ij")
    R = a * n + b * r + cx * x + d
    V = O.deskew(R, g)
    k, j, xx = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    nf = ((j - g.J0) * g.pixel - k * g.pixel * g.c) / g.step
    expect = a * nf + b * k + cx * xx + d
    cov = np.broadcast_to(O.covered_mask(g)[:, :, None], V.shape)
    np.testing.assert_allclose(V[cov], expect[cov], rtol=0, atol=1e-9)


@pytest.mark.parametrize("p,vox", [
    ((64, 128, 16, 30.0, 0.4, 0.115), (20, 70, 5)),
    ((200, 64, 4, 35.0, 0.3, 0.1), (0, 63, 3)),
    ((50, 87, 4, 45.0, 0.2, 0.115), (49, 0, 0)),
    ((10, 10, 2, 35.0, 0.05, 0.1), (7, 4, 1)),
])
def test_bright_voxel_lands_at_eq1_position(p, vox):
    """One bright raw sample lands on row k = r0, column x0, at the y' of Eq. (1).

    In the lab frame the sample (n0, r0) sits at y = n0*step + r0*pixel*cos(theta):
    the per-plane offset along the sheet is step*cos(theta) (Eq. 1 with
    alpha = theta).  Its output column is j* = J0 + y / pixel; the tent puts
    weight 1 - |n_f - n0| on every column within one plane of it.
    """
    g = O.geometry(*p)
    n0, r0, x0 = vox
    R = opm_synth.bright_voxel((g.nscan, g.nrows, g.ncols), n0, r0, x0)
    V = O.deskew(R, g)
    nz_k, nz_j, nz_x = np.nonzero(V)
    assert set(nz_k) == {r0} and set(nz_x) == {x0}
    jstar = g.J0 + (n0 * g.step + r0 * g.pixel * g.c) / g.pixel
    for j in range(g.ny):
        nf = ((j - g.J0) * g.pixel - r0 * g.pixel * g.c) / g.step
        expect = max(0.0, 1.0 - abs(nf - n0))
        assert V[r0, j, x0] == pytest.approx(expect, abs=1e-12)
    jpk = int(np.argmax(V[r0, :, x0]))
    assert abs(jpk - round(jstar)) <= 1
    # mass: the column sum of the tent is 1/rho = step/pixel up to the sampling
    assert V.sum() == pytest.approx(g.step / g.pixel, rel=0.5)


@pytest.mark.parametrize("cfg,J0,ny", [
    ("oracle_64x128x128", 3, 336),
    ("liveview_200x512x2048", 2, 1021),
    ("large_1000x1024x2048", 1, 2464),
    ("diff_128x256x256", 3, 670),
])
def test_extent_closed_forms(cfg, J0, ny):
    c = opm_synth.CONFIGS[cfg]
    g = O.geometry(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    assert (g.J0, g.ny, g.nz, g.nx) == (J0, ny, c.nrows, c.ncols)


def test_extent_fd_case():
    g = O.geometry(16, 24, 32, 30.0, 0.4, 0.115)
    assert g.ny == 79


@pytest.mark.parametrize("p", TINY + [(64, 128, 1, 30.0, 0.4, 0.115), (9, 40, 1, 35.0, 0.05, 0.1)])
def test_extent_is_exactly_the_support(p):
    """Columns -1 and ny carry no weight; every raw sample reaches some voxel."""
    g = O.geometry(*p)
    for k in range(g.nz):
        for jj in (-1, g.ny):
            nf = ((jj - g.J0) * g.pixel - k * g.pixel * g.c) / g.step
            assert nf <= -1.0 + 1e-9 or nf >= g.nscan - 1e-9 * g.pixel / g.step
    # every raw sample of every row has a non-zero weight in some column, as
    # long as the output columns sample the planes closer than every 2 planes
    # (pixel/step < 2); coarser grids skip planes by construction
    j = np.arange(g.ny)
    for k in range(g.nz if g.pixel / g.step < 2 else 0):
        nf = ((j - g.J0) * g.pixel - k * g.pixel * g.c) / g.step
        for n in range(g.nscan):
            assert np.max(np.maximum(0, 1 - np.abs(nf - n))) > 0
    # column 0 is reached by row 0 and the last column by the last row
    assert ((0 - g.J0) * g.pixel) / g.step > -1.0
    nf_last = ((g.ny - 1 - g.J0) * g.pixel - (g.nz - 1) * g.pixel * g.c) / g.step
    assert nf_last < g.nscan


def test_theta90_step_equals_pixel_is_transpose():
    # dyadic step and pixel so that n_f = j holds exactly in binary
    g = O.geometry(7, 5, 3, 90.0, 0.125, 0.125)
    assert g.J0 == 0 and g.ny == 7
    R = _rand((7, 5, 3), 31)
    V = O.deskew(R, g)
    np.testing.assert_array_equal(V, np.transpose(R, (1, 0, 2)))
    np.testing.assert_array_equal(O.deskew(R, g, 1), np.transpose(R, (1, 0, 2)))


def test_theta60_step_equals_pixel_half_weights():
    g = O.geometry(6, 5, 2, 60.0, 0.125, 0.125)
    A = O.explicit_matrix(g)
    assert set(np.unique(A)) <= {0.0, 0.5, 1.0}
    assert 0.5 in set(np.unique(A))


def test_cos_exact_special_angles():
    assert O.cos_deg(90.0) == 0.0 and O.cos_deg(60.0) == 0.5
    assert O.cos_deg(30.0) == pytest.approx(math.sqrt(3) / 2, rel=1e-15)


def test_hand_worked_example_theta90():
    """nscan=2, one row, one column, theta=90, step=2*pixel.

    rho = 1/2, J0 = ceil(2) - 1 = 1, ny = ceil(1 + 2*2) = 5 and
    n_f(j) = (j - 1) / 2 = -0.5, 0, 0.5, 1, 1.5.  With R = (10, 30):
    V = 0.5*10, 10, 0.5*(10+30), 30, 0.5*30 = 5, 10, 20, 30, 15.
    """
    g = O.geometry(2, 1, 1, 90.0, 0.2, 0.1)
    assert (g.J0, g.ny) == (1, 5)
    R = np.array([10.0, 30.0]).reshape(2, 1, 1)
    np.testing.assert_allclose(O.deskew(R, g)[0, :, 0], [5, 10, 20, 30, 15], atol=1e-12)
    # NEAREST: floor(n_f + 1/2) = 0, 0, 1, 1, 2  ->  10, 10, 30, 30, 0
    np.testing.assert_array_equal(O.deskew(R, g, 1)[0, :, 0], [10, 10, 30, 30, 0])


def test_hand_worked_example_theta60():
    """nscan=3, two rows, theta=60, step=pixel: row 1 is shifted by half a plane.

    J0 = 0, ny = ceil(0 + 3 + 0.5) = 4.  Row 0: n_f = j; row 1: n_f = j - 1/2.
    With R[:, 0] = (1, 2, 3) and R[:, 1] = (4, 6, 8):
    row 0 -> 1, 2, 3, 0;  row 1 -> 2, 5, 7, 4.
    """
    g = O.geometry(3, 2, 1, 60.0, 0.1, 0.1)
    assert (g.J0, g.ny) == (0, 4)
    R = np.zeros((3, 2, 1))
    R[:, 0, 0] = [1, 2, 3]
    R[:, 1, 0] = [4, 6, 8]
    V = O.deskew(R, g)
    np.testing.assert_allclose(V[0, :, 0], [1, 2, 3, 0], atol=1e-12)
    np.testing.assert_allclose(V[1, :, 0], [2, 5, 7, 4], atol=1e-12)
    zmip, zsum, ymip, argz = O.project(R, g)
    np.testing.assert_allclose(zmip[:, 0], [2, 5, 7, 4])
    np.testing.assert_allclose(zsum[:, 0], [3, 7, 10, 4])
    np.testing.assert_allclose(ymip[:, 0], [3, 7])
    np.testing.assert_array_equal(argz[:, 0], [1, 1, 1, 1])


@pytest.mark.parametrize("p", TINY + [(64, 128, 16, 30.0, 0.4, 0.115)])
@pytest.mark.parametrize("interp", [0, 1])
def test_projections_match_numpy_reductions(p, interp):
    g = O.geometry(*p)
    R = opm_synth.raw_stack(opm_synth.StackConfig(
        "t", g.nscan, g.nrows, g.ncols, g.theta_deg, g.step, g.pixel,
        n_blobs=3, sigma=(1.0, 2.0), amp=(100, 900), seed=5)).astype(np.float64)
    V = O.deskew(R, g, interp)
    zmip, zsum, ymip, argz = O.project(R, g, interp)
    np.testing.assert_array_equal(zmip, V.max(axis=0))
    np.testing.assert_allclose(zsum, V.sum(axis=0), rtol=1e-13, atol=1e-9)
    np.testing.assert_array_equal(ymip, V.max(axis=1))
    np.testing.assert_array_equal(argz, np.argmax(V, axis=0))


def test_argz_first_occurrence_on_ties():
    g = O.geometry(8, 6, 2, 90.0, 0.1, 0.1)   # every row sees the same planes
    R = np.ones((8, 6, 2)) * 7.0
    zmip, _, _, argz = O.project(R, g)
    assert np.all(zmip == 7.0) and np.all(argz == 0)


def test_negative_input_includes_zero_voxels():
    """Zero-padded voxels take part in the maximum (reading 8)."""
    g = O.geometry(4, 3, 2, 30.0, 0.4, 0.115)
    R = -1.0 - np.abs(_rand((4, 3, 2), 41))
    zmip, _, ymip, argz = O.project(R, g)
    V = O.deskew(R, g)
    assert np.all(zmip <= 0.0) and np.all(ymip <= 0.0)
    np.testing.assert_array_equal(zmip, V.max(axis=0))
    np.testing.assert_array_equal(argz, np.argmax(V, axis=0))


def test_mip_backward_matches_finite_differences():
    """d/dR sum(gz * zmip(R)) by central differences, tie-free Gaussian input."""
    g = O.geometry(5, 4, 3, 30.0, 0.4, 0.115)
    R = _rand((g.nscan, g.nrows, g.ncols), 51)
    gz = _rand((g.ny, g.nx), 52)
    zmip, _, _, argz = O.project(R, g)
    G = O.mip_backward(gz, argz, g)
    h = 1e-6
    fd = np.empty_like(R)
    for idx in np.ndindex(R.shape):
        Rp = R.copy(); Rp[idx] += h
        Rm = R.copy(); Rm[idx] -= h
        fd[idx] = (np.sum(gz * O.project(Rp, g)[0]) - np.sum(gz * O.project(Rm, g)[0])) / (2 * h)
    np.testing.assert_allclose(G, fd, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("shape", [(6, 4, 3, 30.0, 0.4, 0.115), (5, 3, 2, 35.0, 0.05, 0.1)])
def test_mip_backward_equals_masked_explicit_transpose(shape):
    """Any arg-max map, out-of-range rows included: the z-MIP backward is the
    transpose of the entry-by-entry matrix applied to g placed at (argz, j, x)
    (rows outside [0, nz) place nothing)."""
    g = O.geometry(*shape)
    rng = np.random.default_rng(71)
    gz = rng.standard_normal((g.ny, g.nx))
    argz = rng.integers(-1, g.nz + 1, size=(g.ny, g.nx))
    Y = np.zeros((g.nz, g.ny, g.nx))
    for j in range(g.ny):
        for x in range(g.nx):
            if 0 <= argz[j, x] < g.nz:
                Y[argz[j, x], j, x] = gz[j, x]
    A = O.explicit_matrix(g)
    ref = (A.T @ Y.ravel()).reshape(g.nscan, g.nrows, g.ncols)
    np.testing.assert_allclose(O.mip_backward(gz, argz, g), ref, rtol=1e-12, atol=1e-12)


def test_adjoint_matches_finite_differences():
    g = O.geometry(4, 3, 2, 35.0, 0.3, 0.1)
    R = _rand((g.nscan, g.nrows, g.ncols), 61)
    Y = _rand((g.nz, g.ny, g.nx), 62)
    G = O.skew_adjoint(Y, g)
    h = 1e-6
    for idx in np.ndindex(R.shape):
        Rp = R.copy(); Rp[idx] += h
        Rm = R.copy(); Rm[idx] -= h
        fd = (np.sum(Y * O.deskew(Rp, g)) - np.sum(Y * O.deskew(Rm, g))) / (2 * h)
        assert G[idx] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_u16_rounding_half_even_and_clamp():
    v = np.array([0.5, 1.5, 2.5, 3.49999, -3.0, 65535.4, 70000.0, 65534.5])
    np.testing.assert_array_equal(O.to_u16(v), [0, 2, 2, 3, 0, 65535, 65535, 65534])


def test_fig2_deskew_restores_round_cross_section():
    """Fig. 2b-c: the raw stack shows a tilted object sheared; deskewing restores it.

    A Gaussian ball is sampled at the lab positions of the raw samples
    (y = n*step + r*pixel*cos(theta), z = r*pixel*sin(theta)).  Read naively as
    (plane, row) the cross-section is sheared; after the deskew its second
    moments in physical units are isotropic with no y-z correlation.
    """
    theta, step, pixel = 35.0, 0.2, 0.1
    nscan, nrows = 120, 80
    c, s = O.cos_deg(theta), math.sin(math.radians(theta))
    y0, z0, sig = 0.5 * nscan * step + 0.5 * nrows * pixel * c, 0.5 * nrows * pixel * s, 0.6
    n = np.arange(nscan)[:, None]
    r = np.arange(nrows)[None, :]
    yy = n * step + r * pixel * c
    zz = r * pixel * s
    R = np.exp(-((yy - y0) ** 2 + (zz - z0) ** 2) / (2 * sig * sig))[:, :, None]
    g = O.geometry(nscan, nrows, 1, theta, step, pixel)
    V = O.deskew(R, g)[:, :, 0]                     # [k, j]

    def moments(img, dy, dz):
        w = img / img.sum()
        kk, jj = np.meshgrid(np.arange(img.shape[0]), np.arange(img.shape[1]), indexing="ij")
        Y, Z = jj * dy, kk * dz
        my, mz = (w * Y).sum(), (w * Z).sum()
        vy, vz = (w * (Y - my) ** 2).sum(), (w * (Z - mz) ** 2).sum()
        cyz = (w * (Y - my) * (Z - mz)).sum()
        return vy, vz, cyz / math.sqrt(vy * vz)

    vy, vz, corr = moments(V, pixel, pixel * s)
    assert vy == pytest.approx(sig ** 2, rel=0.1) and vz == pytest.approx(sig ** 2, rel=0.1)
    assert abs(corr) < 0.02
    # raw stack read naively (plane index as y, row as z) is sheared
    _, _, corr_raw = moments(R[:, :, 0].T, step, pixel * s)
    assert abs(corr_raw) > 0.3
