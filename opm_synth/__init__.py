"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no deskew arithmetic: it only draws camera stacks and test
vectors.  Both the FP64 oracle and the CUDA path consume the exact bytes it
returns, so a parity test compares the two implementations on identical data.

Stack model (stand-in for the paper's Vero-cell acquisitions, which are not
available): each raw sample ``R[n, r, x]`` (scan plane n, camera row r,
column x) is ``Poisson(lambda)`` with

    lambda = background + sum_b A_b * exp(-|(n, r, x) - c_b|^2 / (2 sigma_b^2))

with blob centres ``c_b`` uniform over the raw index volume, clipped to the
uint16 range.  Blob parameters come from ``PCG64(seed)``; the Poisson draw of
plane n uses its own stream ``PCG64(SeedSequence([seed, n]))`` so that a stack
can be produced plane by plane (the large configurations do not fit a dense
FP64 intensity volume in host memory) and still be bit-identical on every
machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "StackConfig",
    "CONFIGS",
    "blob_params",
    "raw_stack",
    "gaussian",
    "bright_voxel",
]


@dataclass(frozen=True)
class StackConfig:
    """Shape, geometry and content recipe of one named workload."""

    name: str
    nscan: int
    nrows: int
    ncols: int
    theta_deg: float
    step: float          # scan step between planes (um)
    pixel: float         # sample-plane pixel size (um)
    n_blobs: int
    sigma: tuple         # (lo, hi) uniform, lo == hi for a fixed width
    amp: tuple           # (lo, hi) uniform amplitude in counts
    background: float = 100.0
    seed: int = 0
    notes: str = field(default="", compare=False)

    @property
    def shape(self):
        return (self.nscan, self.nrows, self.ncols)

    @property
    def raw_bytes_u16(self) -> int:
        return 2 * self.nscan * self.nrows * self.ncols


# Workloads shaped like the paper's acquisitions (camera ROI x planes per stack,
# 30-45 degree sheets, 0.1-0.115 um pixels).  The pixel size of the
# differentiable case is not given with it and is taken equal to the first
# case's 0.115 um.
CONFIGS = {
    "oracle_64x128x128": StackConfig(
        "oracle_64x128x128", 64, 128, 128, 30.0, 0.4, 0.115,
        n_blobs=40, sigma=(2.0, 2.0), amp=(500.0, 3000.0), seed=1,
        notes="plain deskew, FP32 volume + z-MIP + z-sum"),
    "liveview_200x512x2048": StackConfig(
        "liveview_200x512x2048", 200, 512, 2048, 35.0, 0.3, 0.1,
        n_blobs=2000, sigma=(1.5, 4.0), amp=(200.0, 5000.0), seed=2,
        notes="fused deskew + z-MIP + y-MIP, plus a full FP32 volume"),
    "large_1000x1024x2048": StackConfig(
        "large_1000x1024x2048", 1000, 1024, 2048, 45.0, 0.2, 0.115,
        n_blobs=10000, sigma=(1.5, 4.0), amp=(200.0, 5000.0), seed=3,
        notes="FP32 + round-to-nearest uint16 volume + z-MIP"),
    "diff_128x256x256": StackConfig(
        "diff_128x256x256", 128, 256, 256, 30.0, 0.4, 0.115,
        n_blobs=300, sigma=(1.5, 4.0), amp=(200.0, 1000.0), seed=4,
        notes="FP32 forward + adjoint; Gaussian test vectors"),
}


def blob_params(cfg: StackConfig):
    """Blob centres (n, r, x), widths and amplitudes drawn from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(cfg.seed))
    nb = cfg.n_blobs
    centres = rng.uniform(0.0, 1.0, size=(nb, 3)) * np.array(
        [cfg.nscan, cfg.nrows, cfg.ncols], dtype=np.float64)
    sig = rng.uniform(cfg.sigma[0], cfg.sigma[1], size=nb) if cfg.sigma[1] > cfg.sigma[0] \
        else np.full(nb, float(cfg.sigma[0]))
    amp = rng.uniform(cfg.amp[0], cfg.amp[1], size=nb)
    return centres, sig, amp


def _plane_intensity(cfg, n, centres, sig, amp, reach):
    lam = np.full((cfg.nrows, cfg.ncols), cfg.background, dtype=np.float64)
    dn = n - centres[:, 0]
    hit = np.nonzero(np.abs(dn) <= reach)[0]
    for b in hit:
        s = sig[b]
        wn = np.exp(-dn[b] * dn[b] / (2.0 * s * s))
        r_lo = max(0, int(np.floor(centres[b, 1] - reach[b])))
        r_hi = min(cfg.nrows, int(np.ceil(centres[b, 1] + reach[b])) + 1)
        x_lo = max(0, int(np.floor(centres[b, 2] - reach[b])))
        x_hi = min(cfg.ncols, int(np.ceil(centres[b, 2] + reach[b])) + 1)
        if r_lo >= r_hi or x_lo >= x_hi:
            continue
        rr = np.arange(r_lo, r_hi, dtype=np.float64) - centres[b, 1]
        xx = np.arange(x_lo, x_hi, dtype=np.float64) - centres[b, 2]
        wr = np.exp(-rr * rr / (2.0 * s * s))
        wx = np.exp(-xx * xx / (2.0 * s * s))
        lam[r_lo:r_hi, x_lo:x_hi] += amp[b] * wn * np.outer(wr, wx)
    return lam


def raw_stack(cfg: StackConfig, out: np.ndarray | None = None,
              planes: tuple | None = None) -> np.ndarray:
    """uint16 stack ``[nscan, nrows, ncols]`` (or planes ``[lo, hi)`` of it).

    ``out`` may be a preallocated (e.g. pinned) uint16 buffer of the right
    shape, which is filled in place and returned.
    """
    lo, hi = (0, cfg.nscan) if planes is None else planes
    shape = (hi - lo, cfg.nrows, cfg.ncols)
    if out is None:
        out = np.empty(shape, dtype=np.uint16)
    elif out.shape != shape or out.dtype != np.uint16:
        raise ValueError(f"out must be uint16 {shape}, got {out.dtype} {out.shape}")
    centres, sig, amp = blob_params(cfg)
    reach = np.ceil(4.0 * sig)
    for n in range(lo, hi):
        lam = _plane_intensity(cfg, n, centres, sig, amp, reach)
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([cfg.seed, n])))
        counts = rng.poisson(lam)
        np.clip(counts, 0, 65535, out=counts)
        out[n - lo] = counts.astype(np.uint16)
    return out


def gaussian(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded N(0, 1) array (dot tests, gradient checks)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x6A75])))
    return rng.standard_normal(size=shape).astype(dtype)


def bright_voxel(shape, n0: int, r0: int, x0: int, value: float = 1.0,
                 dtype=np.float64) -> np.ndarray:
    """All-zero stack with one sample set to ``value``."""
    a = np.zeros(shape, dtype=dtype)
    a[n0, r0, x0] = value
    return a


def tiled_stack(shape, seed: int = 5) -> np.ndarray:
    """uint16 stack of any shape filled by repeating one Poisson+blob tile.

    Content stand-in for the serving workload, where stacks of up to several
    GB arrive continuously and only their shapes matter for the schedule.
    """
    tile = raw_stack(StackConfig("tile", 50, 128, 256, 35.0, 0.3, 0.1, n_blobs=12, sigma=(1.5, 4.0),
                                 amp=(200.0, 5000.0), seed=seed))
    reps = [-(-s // t) for s, t in zip(shape, tile.shape)]
    return np.ascontiguousarray(np.tile(tile, reps)[: shape[0], : shape[1], : shape[2]])


SERVE_ROWS = (256, 512, 1024)
SERVE_COLS = (512, 1024, 2048)


def serve_shapes(n: int, seed: int = 5, planes=(50, 400), channels: int = 2,
                 rows=SERVE_ROWS, cols=SERVE_COLS):
    """Seeded request shapes (nscan, nrows, ncols per channel, channels):
    rows and columns uniform over the given sets, planes uniform over the
    range in steps of 50, as in a live-imaging session of varying ROIs."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x5E7])))
    pl = np.arange(planes[0], planes[1] + 1, 50)
    return [(int(rng.choice(pl)), int(rng.choice(rows)), int(rng.choice(cols)), channels) for _ in range(n)]
