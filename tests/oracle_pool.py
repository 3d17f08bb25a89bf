"""Test infrastructure: the oracle's z-MIP and y-MIP of a full-size stack,
computed over blocks of x-columns in spawned processes (output column x
reads raw column x only, Eq. 1, so the blocks are independent).  Processes
are started with spawn, never forked from a process that has used the GPU."""
import os

import numpy as np


def _block(job):
    import oracle as O
    R, geo = job
    z, _, y, _ = O.project(R.astype(np.float64), O.geometry(*geo))
    return z, y


def project_columns(R, theta_deg, step, pixel, procs=None):
    """(zmip, ymip) of the oracle for the uint16 stack R [nscan][nrows][ncols]."""
    import multiprocessing as mp
    nscan, nrows, ncols = R.shape
    n = procs or os.cpu_count() or 1
    blocks = [b for b in np.array_split(np.arange(ncols), n) if len(b)]
    jobs = [(np.ascontiguousarray(R[:, :, b[0]:b[-1] + 1]), (nscan, nrows, len(b), theta_deg, step, pixel))
            for b in blocks]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        out = pool.map(_block, jobs)
    return np.concatenate([o[0] for o in out], axis=1), np.concatenate([o[1] for o in out], axis=1)
