"""Pins of the sheet-frame oracle (the paper's remap, Fig. 2c-d, and the
shear-warp view, Fig. 3) against facts fixed by the mathematics, plus
planted mistakes that the pins must catch."""
import math

import numpy as np
import pytest

import opm_synth
import oracle as O
from oracle import sheet as S


def _stack(n, r, c, seed=3):
    return np.abs(opm_synth.gaussian((n, r, c), seed)) * 100.0


def _pins_pass():
    ok = True
    R = _stack(6, 7, 3)
    # zero shear: the plain maximum over frames
    ok &= np.array_equal(O.sheet_project(R, 0.0), R.max(axis=0))
    # integer shear: frames placed on a zero canvas, exactly
    for s in (1.0, 2.0, 3.0):
        H = O.sheet_rows(6, 7, s)
        canvas = np.zeros((6, H, 3))
        for n in range(6):
            canvas[n, int(n * s):int(n * s) + 7] = R[n]
        ok &= np.array_equal(O.sheet_project(R, s), canvas.max(axis=0))
    # brute force: every remapped frame against explicit weights
    for s in (0.37, 1.5, 2.4567):
        for n in range(6):
            Sn = O.sheet_frame(R, s, n)
            for Y in range(Sn.shape[0]):
                ok &= np.allclose(Sn[Y], O.sheet_matrix_row(7, s, n, Y) @ R[n], atol=1e-12)
            # the tent keeps each frame's mass: sum over Y of S = sum over r of R
            ok &= np.allclose(Sn.sum(axis=0), R[n].sum(axis=0), atol=1e-9)
    # a bright sample lands at row n*s + r (Eq. 1 shift), split by the tent
    B = np.zeros((5, 9, 2))
    B[3, 4, 1] = 1.0
    s = 1.25
    P = O.sheet_project(B, s)
    pos = 3 * s + 4
    ok &= abs(P[int(math.floor(pos)), 1] - (1.0 - (pos - math.floor(pos)))) < 1e-12
    ok &= abs(P[int(math.floor(pos)) + 1, 1] - (pos - math.floor(pos))) < 1e-12
    ok &= abs(P.sum() - 1.0) < 1e-12
    # extent: the last sample of the last frame reaches the last row
    ok &= O.sheet_rows(200, 512, 0.3 * math.cos(math.radians(35.0)) / 0.1) == 512 + 490
    # warp: identity, integer shift, and exact on a ramp
    P = O.sheet_project(R, 1.5)
    ok &= np.array_equal(O.warp_rows(P, P.shape[0], 1.0, 0.0), P)
    W = O.warp_rows(P, P.shape[0], 1.0, 2.0)
    ok &= np.array_equal(W[:-2], P[2:]) and np.all(W[-2:] == 0)
    ramp = np.repeat(np.arange(40, dtype=np.float64)[:, None], 2, axis=1)
    W = O.warp_rows(ramp, 30, 0.75, 3.5)
    ok &= np.allclose(W[:, 0], 0.75 * np.arange(30) + 3.5, atol=1e-12)
    return bool(ok)


def test_sheet_pins():
    assert _pins_pass()


def test_sheet_shear_of_eq1():
    """s = step * cos(theta) / pixel: a frame's shift in rows is its scan
    distance times cos(theta), in pixels (Eq. 1)."""
    g = O.geometry(200, 512, 4, 35.0, 0.3, 0.1)
    s = g.step * g.c / g.pixel
    assert abs(s - 2.4574561328) < 1e-9
    assert O.sheet_rows(200, 512, s) == 1002


def test_sheet_rejects_negative_shear():
    with pytest.raises(ValueError):
        O.sheet_rows(4, 4, -0.5)


def _wrong_sign_frame(R, shear, n):
    nscan, nrows, _ = R.shape
    H = S.sheet_rows(nscan, nrows, shear)
    Y = np.arange(H, dtype=np.float64)
    r = Y + n * shear - (nscan - 1) * shear
    r0 = np.floor(r)
    w = r - r0
    r0 = r0.astype(np.int64)
    f = np.asarray(R[n], dtype=np.float64)
    take = lambda i: np.where(((i >= 0) & (i < nrows))[:, None], f[np.clip(i, 0, nrows - 1)], 0.0)
    return (1.0 - w)[:, None] * take(r0) + w[:, None] * take(r0 + 1)


def _swapped_weight_frame(R, shear, n):
    nscan, nrows, _ = R.shape
    H = S.sheet_rows(nscan, nrows, shear)
    r = np.arange(H, dtype=np.float64) - n * shear
    r0 = np.floor(r)
    w = r - r0
    r0 = r0.astype(np.int64)
    f = np.asarray(R[n], dtype=np.float64)
    take = lambda i: np.where(((i >= 0) & (i < nrows))[:, None], f[np.clip(i, 0, nrows - 1)], 0.0)
    return w[:, None] * take(r0) + (1.0 - w)[:, None] * take(r0 + 1)


def _short_extent(nscan, nrows, shear):
    return nrows + int(math.floor((nscan - 1) * shear))


def _warp_off_by_one(P, out_rows, a, b):
    return _real_warp(P, out_rows, a, b + 1.0)


_real_warp = S.warp_rows


@pytest.mark.parametrize("target,mutant", [
    ("sheet_frame", _wrong_sign_frame),
    ("sheet_frame", _swapped_weight_frame),
    ("sheet_rows", _short_extent),
    ("warp_rows", _warp_off_by_one),
])
def test_sheet_pins_catch_mutant(monkeypatch, target, mutant):
    monkeypatch.setattr(S, target, mutant)
    monkeypatch.setattr(O, target, mutant, raising=False)
    assert not _pins_pass()
