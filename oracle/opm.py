"""Plain FP64 oracle of the oblique-plane deskew and its projections.

TEST INFRASTRUCTURE.  This module is the reference the CUDA library is
checked against; it is never on the library's execution path.  Everything is
computed in float64 with plain NumPy, in the order the definitions below state,
with no blocking, fusion or reordering.

What the method computes (Lamb, Ward & Kaminski, arXiv 2211.00645):

* Eq. (1): consecutive raw frames are laterally offset by ``l = z cos(alpha)``
  where ``z`` is the scan distance between frames and ``alpha`` the sheet
  angle.
* Section "Physical principles for the processing of lightsheet imaging
  data" and Fig. 2c: deskewing places every raw frame into a larger image,
  shifted by the accumulated offset, restoring the sample geometry.
* Fig. 2d and the same section: the widefield-like live view is the
  brightest value across the deskewed stack at each pixel.

Readings where the paper is silent (each also listed in the design notes):

1. Lab frame.  Raw sample ``(n, r, x)`` (scan plane, camera row, column) sits
   at ``y = n*step + r*pixel*cos(theta)``, ``z = r*pixel*sin(theta)``.  The
   projection of the per-plane shift on the sheet is ``step*cos(theta)``,
   i.e. Eq. (1) with alpha = theta.  The scan moves the sheet towards +y.
2. Output grid ``V[k, j, x]``: ``k = r`` exactly (no interpolation across
   camera rows), ``y'_j = (j - J0) * pixel`` (square pixels in the (y', x)
   view), ``x`` unchanged.
3. Plane coordinate ``n_f(j, k) = ((j - J0)*pixel - k*pixel*cos(theta)) / step``.
4. LINEAR: ``V = (1-w) R~[n0] + w R~[n0+1]`` with ``n0 = floor(n_f)``,
   ``w = n_f - n0`` and ``R~`` equal to ``R`` for ``0 <= n < nscan`` and 0
   elsewhere (a zero-padded tent; no hard coverage cut).
5. NEAREST: ``V = R~[floor(n_f + 1/2)]`` (ties go to the upper plane).
6. ``J0 = ceil(step/pixel) - 1`` and ``ny = ceil(X - 1e-9)`` with
   ``X = J0 + nscan*(step/pixel) + (nrows-1)*cos(theta)``: exactly the
   columns that can carry a non-zero weight.
7. ``cos`` is exact at 90 degrees (0) and at 60 degrees (1/2).
8. Projections run over the whole materialised grid, zero voxels included:
   ``zmip = max_k V``, ``zsum = sum_k V``, ``ymip = max_j V``, ``argz`` = the
   smallest k attaining the maximum.
9. uint16 output: round half to even, clamp to [0, 65535].
10. The adjoint is the exact transpose of the linear map,
    ``G[n, k, x] = sum_j V[k, j, x] * t(n_f(j, k) - n)`` with the tent
    ``t(u) = max(0, 1 - |u|)``; the z-MIP backward routes ``g[j, x]`` to
    the raw samples of the voxel ``(argz[j, x], j, x)`` with the same tents.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LINEAR = 0
NEAREST = 1


def cos_deg(theta_deg: float) -> float:
    """cos(theta) for theta in degrees, exact at 90 (0) and 60 (1/2)."""
    if theta_deg == 90.0:
        return 0.0
    if theta_deg == 60.0:
        return 0.5
    return math.cos(theta_deg * math.pi / 180.0)


@dataclass(frozen=True)
class Geometry:
    nscan: int
    nrows: int
    ncols: int
    theta_deg: float
    step: float
    pixel: float
    c: float      # cos(theta)
    J0: int       # leading output columns before plane 0 of row 0
    nz: int
    ny: int
    nx: int


def geometry(nscan, nrows, ncols, theta_deg, step, pixel) -> Geometry:
    """Output grid of the deskew (readings 2, 6, 7)."""
    if not (nscan >= 2 and nrows >= 1 and ncols >= 1):
        raise ValueError("need nscan >= 2, nrows >= 1, ncols >= 1")
    if not (0.0 < theta_deg <= 90.0):
        raise ValueError("theta must lie in (0, 90] degrees")
    if not (step > 0.0 and pixel > 0.0):
        raise ValueError("step and pixel must be positive")
    c = cos_deg(theta_deg)
    J0 = int(math.ceil(step / pixel)) - 1
    X = J0 + nscan * (step / pixel) + (nrows - 1) * c
    ny = int(math.ceil(X - 1e-9))
    return Geometry(int(nscan), int(nrows), int(ncols), float(theta_deg),
                    float(step), float(pixel), c, J0, int(nrows), ny, int(ncols))


def plane_coord(g: Geometry, j, k):
    """Fractional scan-plane coordinate n_f(j, k) of output column j, row k."""
    j = np.asarray(j, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    return ((j - g.J0) * g.pixel - k * g.pixel * g.c) / g.step


def tent(u):
    """Linear-interpolation kernel t(u) = max(0, 1 - |u|)."""
    return np.maximum(0.0, 1.0 - np.abs(u))


def _padded(R, n, k, x):
    """R~[n, k, x]: R inside [0, nscan), zero outside (reading 4)."""
    n = np.asarray(n)
    inside = (n >= 0) & (n < R.shape[0])
    nn = np.where(inside, n, 0)
    vals = np.asarray(R[nn, k, x], dtype=np.float64)
    return np.where(inside, vals, 0.0)


def voxels(R, g: Geometry, k, j, x, interp: int = LINEAR):
    """V[k, j, x] for arrays of indices (per-voxel evaluation)."""
    k = np.asarray(k, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    x = np.asarray(x, dtype=np.int64)
    nf = plane_coord(g, j, k)
    if interp == NEAREST:
        n = np.floor(nf + 0.5).astype(np.int64)
        return _padded(R, n, k, x)
    n0f = np.floor(nf)
    w = nf - n0f
    n0 = n0f.astype(np.int64)
    return (1.0 - w) * _padded(R, n0, k, x) + w * _padded(R, n0 + 1, k, x)


def deskew_row(R, g: Geometry, k: int, interp: int = LINEAR):
    """Output row V[k, :, :] (ny x nx) from camera row k of every plane."""
    j = np.arange(g.ny)
    nf = plane_coord(g, j, k)
    xs = np.arange(g.nx)
    if interp == NEAREST:
        n = np.floor(nf + 0.5).astype(np.int64)
        return _padded(R, n[:, None], k, xs[None, :])
    n0f = np.floor(nf)
    w = (nf - n0f)[:, None]
    n0 = n0f.astype(np.int64)[:, None]
    a = _padded(R, n0, k, xs[None, :])
    b = _padded(R, n0 + 1, k, xs[None, :])
    return (1.0 - w) * a + w * b


def deskew(R, g: Geometry, interp: int = LINEAR):
    """Full deskewed volume V[k, j, x] in float64."""
    _check_raw(R, g)
    V = np.empty((g.nz, g.ny, g.nx), dtype=np.float64)
    for k in range(g.nz):
        V[k] = deskew_row(R, g, k, interp)
    return V


def project(R, g: Geometry, interp: int = LINEAR):
    """(zmip, zsum, ymip, argz) of the deskewed volume, row by row.

    zmip/zsum/argz are [ny, nx]; ymip is [nz, nx].  The running maximum is
    replaced only on a strictly larger value, so argz keeps the first k.
    """
    _check_raw(R, g)
    zmip = np.full((g.ny, g.nx), -np.inf)
    zsum = np.zeros((g.ny, g.nx))
    argz = np.zeros((g.ny, g.nx), dtype=np.int32)
    ymip = np.empty((g.nz, g.nx))
    for k in range(g.nz):
        Vk = deskew_row(R, g, k, interp)
        better = Vk > zmip
        zmip = np.where(better, Vk, zmip)
        argz = np.where(better, np.int32(k), argz)
        zsum += Vk
        ymip[k] = Vk.max(axis=0)
    return zmip, zsum, ymip, argz


def _tent_matrix(g: Geometry, k: int):
    """T[n, j] = t(n_f(j, k) - n) for one camera row (nscan x ny)."""
    nf = plane_coord(g, np.arange(g.ny), k)
    n = np.arange(g.nscan, dtype=np.float64)
    return tent(nf[None, :] - n[:, None])


def skew_adjoint(V, g: Geometry):
    """G = A^T V: G[n, k, x] = sum_j V[k, j, x] t(n_f(j, k) - n) (LINEAR map)."""
    V = np.asarray(V, dtype=np.float64)
    if V.shape != (g.nz, g.ny, g.nx):
        raise ValueError(f"volume must be {(g.nz, g.ny, g.nx)}, got {V.shape}")
    G = np.empty((g.nscan, g.nrows, g.ncols))
    for k in range(g.nz):
        G[:, k, :] = _tent_matrix(g, k) @ V[k]
    return G


def mip_backward(gz, argz, g: Geometry):
    """Gradient of sum(gz * zmip) w.r.t. the raw stack (LINEAR map).

    G[n, k, x] = sum_j [argz[j, x] == k] gz[j, x] t(n_f(j, k) - n).
    """
    gz = np.asarray(gz, dtype=np.float64)
    argz = np.asarray(argz)
    G = np.empty((g.nscan, g.nrows, g.ncols))
    for k in range(g.nz):
        G[:, k, :] = _tent_matrix(g, k) @ np.where(argz == k, gz, 0.0)
    return G


def explicit_matrix(g: Geometry, interp: int = LINEAR):
    """Dense matrix A with vec(V) = A vec(R), built entry by entry (tiny shapes).

    Rows are (k, j, x) in C order, columns (n, r, x') in C order.
    """
    rows = g.nz * g.ny * g.nx
    cols = g.nscan * g.nrows * g.ncols
    if rows * cols > 4_000_000:
        raise ValueError("explicit_matrix is for tiny shapes only")
    A = np.zeros((rows, cols))
    for k in range(g.nz):
        for j in range(g.ny):
            nf = float(((j - g.J0) * g.pixel - k * g.pixel * g.c) / g.step)
            for n in range(g.nscan):
                if interp == NEAREST:
                    wgt = 1.0 if n == math.floor(nf + 0.5) else 0.0
                else:
                    wgt = max(0.0, 1.0 - abs(nf - n))
                if wgt == 0.0:
                    continue
                for x in range(g.nx):
                    A[(k * g.ny + j) * g.nx + x, (n * g.nrows + k) * g.ncols + x] = wgt
    return A


def to_u16(V):
    """uint16 volume: round half to even, clamp to [0, 65535] (reading 9)."""
    return np.clip(np.rint(np.asarray(V, dtype=np.float64)), 0, 65535).astype(np.uint16)


def covered_mask(g: Geometry):
    """[nz, ny] mask of the fully covered region 0 <= n_f <= nscan - 1."""
    k = np.arange(g.nz)[:, None]
    j = np.arange(g.ny)[None, :]
    nf = plane_coord(g, j, k)
    return (nf >= 0.0) & (nf <= g.nscan - 1)


def _check_raw(R, g: Geometry):
    if tuple(R.shape) != (g.nscan, g.nrows, g.ncols):
        raise ValueError(f"raw stack must be {(g.nscan, g.nrows, g.ncols)}, got {R.shape}")
