"""FP64 oracle of the paper's own live view: the sheet-frame remap and the
shear-warp change of viewing angle.

TEST INFRASTRUCTURE.  Never on the library's execution path.

* Section "Physical principles for the processing of lightsheet imaging
  data", Fig. 2c: every raw frame n is placed into a larger image, shifted
  along the camera-row axis by the accumulated lateral offset; with Eq. (1)
  the offset of frame n is ``n * step * cos(alpha)``, i.e. ``n * s`` rows for
  the shear factor ``s = step * cos(alpha) / pixel``.
* Fig. 2d: the widefield-like view is the brightest value across the
  shifted frames at each pixel.
* Fig. 3: reducing the shear factor below Eq. (1)'s value and then warping
  the projected image changes the viewing angle.

Readings where the paper is silent (also listed in the design notes):

S1. Sub-row shifts are resolved by linear interpolation between the two
    neighbouring camera rows (zero outside [0, nrows)), the same tent as the
    lab-frame deskew uses between planes:
    ``S[n, Y, x] = sum_r R[n, r, x] * t(Y - n*s - r)``.
S2. The remapped image has ``H = nrows + ceil((nscan - 1) * s - 1e-9)`` rows
    (``s >= 0``): exactly the rows any frame reaches.  The view is
    ``P[Y, x] = max_n S[n, Y, x]`` over all frames, zero samples included.
S3. The warp is a 1-D affine resample along the row axis,
    ``W[Y', x] = sum_Y P[Y, x] * t(a * Y' + b - Y)``, zero outside
    [0, H); ``a`` and ``b`` are given by the caller (Fig. 3's warp of the
    projected image).
"""
from __future__ import annotations

import math

import numpy as np

from .opm import tent


def sheet_rows(nscan: int, nrows: int, shear: float) -> int:
    """Rows of the remapped image (reading S2)."""
    if shear < 0:
        raise ValueError("shear must be >= 0")
    return nrows + int(math.ceil((nscan - 1) * shear - 1e-9))


def sheet_frame(R, shear: float, n: int):
    """S[n, :, :] of reading S1 for one frame: [H, ncols]."""
    nscan, nrows, _ = R.shape
    H = sheet_rows(nscan, nrows, shear)
    Y = np.arange(H, dtype=np.float64)
    r = Y - n * shear                       # source row of output row Y
    r0 = np.floor(r)
    w = r - r0
    r0 = r0.astype(np.int64)
    frame = np.asarray(R[n], dtype=np.float64)

    def row(i):
        inside = (i >= 0) & (i < nrows)
        vals = frame[np.where(inside, i, 0), :]
        return np.where(inside[:, None], vals, 0.0)

    return (1.0 - w)[:, None] * row(r0) + w[:, None] * row(r0 + 1)


def sheet_project(R, shear: float):
    """P[Y, x] = max_n S[n, Y, x] (readings S1, S2)."""
    R = np.asarray(R)
    P = None
    for n in range(R.shape[0]):
        S = sheet_frame(R, shear, n)
        P = S if P is None else np.maximum(P, S)
    return P


def sheet_matrix_row(nrows: int, shear: float, n: int, Y: int):
    """Weights t(Y - n*s - r) over r for one output row (brute force)."""
    return np.array([float(tent(Y - n * shear - r)) for r in range(nrows)])


def warp_rows(P, out_rows: int, a: float, b: float):
    """W[Y', x] = P at row a*Y' + b, linear between rows, zero outside (S3)."""
    P = np.asarray(P, dtype=np.float64)
    H = P.shape[0]
    y = a * np.arange(out_rows, dtype=np.float64) + b
    y0 = np.floor(y)
    w = y - y0
    y0 = y0.astype(np.int64)

    def row(i):
        inside = (i >= 0) & (i < H)
        vals = P[np.where(inside, i, 0), :]
        return np.where(inside[:, None], vals, 0.0)

    return (1.0 - w)[:, None] * row(y0) + w[:, None] * row(y0 + 1)
