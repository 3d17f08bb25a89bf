"""Helpers of the GPU tests (no deskew arithmetic here)."""
import numpy as np

TOL = 1e-4  # max |gpu - oracle| <= TOL * max |oracle|, per output array


def rel_err(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    scale = max(float(np.max(np.abs(ref))), 1e-30) if ref.size else 1.0
    return float(np.max(np.abs(gpu - ref))) / scale if ref.size else 0.0


def assert_close(gpu, ref, tol=TOL, what=""):
    e = rel_err(gpu, ref)
    assert e <= tol, f"{what}: max rel err {e:.3e} > {tol:.1e}"


def to_dev(a, torch, dev="cuda"):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.astype(np.int32)).to(dev).to(torch.uint16)
    return torch.from_numpy(a).to(dev)


def check_argz(argz_gpu, V, zmip_ref, tol_abs):
    """argz must point at a voxel attaining the maximum within tol; where the
    maximum is separated from every other value by more than tol it must be
    the oracle's (smallest) k."""
    nz = V.shape[0]
    a = np.asarray(argz_gpu)
    assert a.min() >= 0 and a.max() < nz
    picked = np.take_along_axis(V, a[None].astype(np.int64), axis=0)[0]
    assert np.all(picked >= zmip_ref - tol_abs)
    srt = np.sort(V, axis=0)
    clear = (srt[-1] - srt[-2]) > 2 * tol_abs if nz > 1 else np.ones(srt.shape[1:], dtype=bool)
    first = np.argmax(V, axis=0)
    assert np.array_equal(a[clear], first[clear])


def nearest_bounds(R, g, O, eps=1e-6):
    """Per-voxel [min, max] of the NEAREST volume over both neighbouring
    planes wherever n_f lies within eps of a half-integer (at such a tie either
    plane is a correct nearest plane)."""
    k = np.arange(g.nz)[:, None]
    j = np.arange(g.ny)[None, :]
    nf = O.plane_coord(g, j, k)
    R = np.asarray(R, dtype=np.float64)

    def gather(n):
        inside = (n >= 0) & (n < g.nscan)
        kk = np.broadcast_to(k, n.shape)
        vals = R[np.where(inside, n, 0), kk, :]
        return np.where(inside[..., None], vals, 0.0)

    a = gather(np.floor(nf + 0.5 - eps).astype(np.int64))
    b = gather(np.floor(nf + 0.5 + eps).astype(np.int64))
    return np.minimum(a, b), np.maximum(a, b)


def assert_between(gpu, lo, hi, tol=TOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    slack = tol * max(float(np.max(np.abs(hi))), float(np.max(np.abs(lo))), 1e-30)
    assert np.all(gpu >= lo - slack) and np.all(gpu <= hi + slack), what
