"""Plant plausible mistakes in the oracle and check that its pins catch each one.

Every mutant is applied by monkeypatching the oracle module on the CPU; the
checks below restate the pins of test_oracle_pins in a pass/fail form.
"""
import numpy as np
import pytest

import opm_synth
import oracle as O
from oracle import opm as M


def _pins_pass():
    """True when every pin below holds for the (possibly mutated) oracle."""
    ok = True
    for p in [(5, 4, 3, 30.0, 0.4, 0.115), (4, 3, 2, 45.0, 0.2, 0.115), (6, 3, 2, 35.0, 0.05, 0.1)]:
        g = O.geometry(*p)
        R = opm_synth.gaussian((g.nscan, g.nrows, g.ncols), 7)
        A = O.explicit_matrix(g)
        V = O.deskew(R, g)
        ok &= np.allclose(V.reshape(-1), A @ R.reshape(-1), atol=1e-12)
        Y = opm_synth.gaussian((g.nz, g.ny, g.nx), 8)
        ok &= np.allclose(O.skew_adjoint(Y, g).reshape(-1), A.T @ Y.reshape(-1), atol=1e-12)
        zmip, zsum, ymip, argz = O.project(R, g)
        ok &= np.array_equal(zmip, V.max(0)) and np.array_equal(argz, np.argmax(V, 0))
        ok &= np.allclose(zsum, V.sum(0)) and np.array_equal(ymip, V.max(1))
        # z-MIP backward: the transpose applied to g placed at (argz, j, x)
        gz = opm_synth.gaussian((g.ny, g.nx), 9)
        az = np.random.default_rng(10).integers(-1, g.nz + 1, size=(g.ny, g.nx))
        Yg = np.zeros((g.nz, g.ny, g.nx))
        jj, xx = np.nonzero((az >= 0) & (az < g.nz))
        Yg[az[jj, xx], jj, xx] = gz[jj, xx]
        ok &= np.allclose(O.mip_backward(gz, az, g).reshape(-1), A.T @ Yg.reshape(-1), atol=1e-12)
    # single bright voxel at its Eq. (1) column
    g = O.geometry(64, 128, 4, 30.0, 0.4, 0.115)
    R = opm_synth.bright_voxel((64, 128, 4), 20, 70, 2)
    V = O.deskew(R, g)
    jstar = g.J0 + (20 * g.step + 70 * g.pixel * g.c) / g.pixel
    ok &= abs(int(np.argmax(V[70, :, 2])) - round(jstar)) <= 1
    # ties resolve to the first k
    g = O.geometry(8, 6, 2, 90.0, 0.125, 0.125)
    ok &= bool(np.all(O.project(np.ones((8, 6, 2)), g)[3] == 0))
    # extent
    g = O.geometry(200, 512, 4, 35.0, 0.3, 0.1)
    ok &= (g.J0, g.ny) == (2, 1021)
    # fully covered region, counted by hand (n_f = j - k/2)
    g = O.geometry(3, 2, 1, 60.0, 0.125, 0.125)
    ok &= np.array_equal(O.covered_mask(g), np.array([[1, 1, 1, 0], [0, 1, 1, 0]], dtype=bool))
    return bool(ok)


def test_unmutated_oracle_passes():
    assert _pins_pass()


def _wrong_shear_sign(g, j, k):
    j = np.asarray(j, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    return ((j - g.J0) * g.pixel + k * g.pixel * g.c) / g.step


def _swapped_weights(R, g, k, interp=0):
    j = np.arange(g.ny)
    nf = M.plane_coord(g, j, k)
    n0f = np.floor(nf)
    w = (nf - n0f)[:, None]
    n0 = n0f.astype(np.int64)[:, None]
    xs = np.arange(g.nx)[None, :]
    return w * M._padded(R, n0, k, xs) + (1.0 - w) * M._padded(R, n0 + 1, k, xs)


def _clamped_padding(R, n, k, x):
    n = np.clip(np.asarray(n), 0, R.shape[0] - 1)
    return np.asarray(R[n, k, x], dtype=np.float64)


_real_geometry = M.geometry


def _j0_off_by_one(*a):
    g = _real_geometry(*a)
    return M.Geometry(g.nscan, g.nrows, g.ncols, g.theta_deg, g.step, g.pixel, g.c,
                      g.J0 + 1, g.nz, g.ny, g.nx)


def _last_occurrence_project(R, g, interp=0):
    V = np.stack([M.deskew_row(R, g, k, interp) for k in range(g.nz)])
    argz = (g.nz - 1 - np.argmax(V[::-1], axis=0)).astype(np.int32)
    return V.max(0), V.sum(0), V.max(1), argz


def _shifted_adjoint(V, g):
    G = np.empty((g.nscan, g.nrows, g.ncols))
    for k in range(g.nz):
        nf = M.plane_coord(g, np.arange(g.ny), k)
        n = np.arange(g.nscan, dtype=np.float64)
        G[:, k, :] = M.tent(nf[None, :] - n[:, None] - 1.0) @ V[k]
    return G


def _mip_backward_next_row(gz, argz, g):
    gz = np.asarray(gz, dtype=np.float64)
    G = np.empty((g.nscan, g.nrows, g.ncols))
    for k in range(g.nz):
        G[:, k, :] = M._tent_matrix(g, k) @ np.where(np.asarray(argz) + 1 == k, gz, 0.0)
    return G


def _covered_strict(g):
    nf = M.plane_coord(g, np.arange(g.ny)[None, :], np.arange(g.nz)[:, None])
    return (nf > 0.0) & (nf < g.nscan - 1)


def _covered_wide(g):
    nf = M.plane_coord(g, np.arange(g.ny)[None, :], np.arange(g.nz)[:, None])
    return (nf > -1.0) & (nf < g.nscan)


_real_mip_backward = M.mip_backward


def _mip_backward_clipped_rows(gz, argz, g):
    return _real_mip_backward(gz, np.clip(argz, 0, g.nz - 1), g)


@pytest.mark.parametrize("target,mutant", [
    ("plane_coord", _wrong_shear_sign),
    ("deskew_row", _swapped_weights),
    ("_padded", _clamped_padding),
    ("geometry", _j0_off_by_one),
    ("project", _last_occurrence_project),
    ("skew_adjoint", _shifted_adjoint),
    ("mip_backward", _mip_backward_next_row),
    ("mip_backward", _mip_backward_clipped_rows),
    ("covered_mask", _covered_strict),
    ("covered_mask", _covered_wide),
])
def test_pins_catch_mutant(monkeypatch, target, mutant):
    monkeypatch.setattr(M, target, mutant)
    monkeypatch.setattr(O, target, mutant, raising=False)
    assert not _pins_pass()
