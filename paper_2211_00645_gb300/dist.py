"""Multi-process helpers.

The deskew path has no exchange step.  Stacks (or stack items of a batch)
are independent, and so are the x-columns of one stack: output column x of
the volume and of both projections reads raw column x only (Eq. 1 shears
along the scan and row axes).  Ranks therefore split either whole stacks
(``shard``) or the columns of one stack (``xshard``), compute with the same
kernels, and the projections of a column split are reassembled by plain
concatenation (``gather_x``); nothing is reduced.  The other collectives
are for measurement: a barrier around the timed region and the maximum time
over ranks.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of items [0, n_items) for one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a host scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def xshard(ncols: int, rank: int, world: int, align: int = 8) -> tuple:
    """Column range [x0, x1) of one rank's share of a stack's ncols columns:
    balanced in blocks of ``align`` columns (8 uint16 = 16 bytes, the TMA
    alignment of a row), contiguous, in rank order, covering every column
    once.  A rank may get an empty range when there are more ranks than
    blocks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    if ncols < 0 or align < 1:
        raise ValueError("bad ncols/align")
    blocks = (ncols + align - 1) // align
    r = shard(blocks, rank, world)
    return min(ncols, r.start * align), min(ncols, r.stop * align)


def project_xshard(plan_args, raw_cols, stream=None):
    """Live view (z-MIP, y-MIP) of one rank's columns: ``raw_cols`` is the
    rank's [nscan][nrows][x1 - x0] uint16 part of the stack on its device,
    ``plan_args`` = (theta_deg, step, pixel).  The plan of a column range
    has the stack's output grid (nz, ny, J0 do not depend on the columns),
    so the parts are columns x0 .. x1 - 1 of the whole stack's views.
    Returns (zmip [ny][w], ymip [nz][w]); empty parts for w = 0."""
    import torch

    from . import Plan, opm_project
    nscan, nrows, w = raw_cols.shape
    if w == 0:
        from . import opm_plan_shape
        plan = Plan(nscan, nrows, 1, *plan_args)
        nz, ny, _, _ = opm_plan_shape(plan)
        dev = raw_cols.device
        return (torch.empty((ny, 0), dtype=torch.float32, device=dev),
                torch.empty((nz, 0), dtype=torch.float32, device=dev))
    plan = Plan(nscan, nrows, w, *plan_args)
    z = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=raw_cols.device)
    y = torch.empty((plan.nz, plan.nx), dtype=torch.float32, device=raw_cols.device)
    opm_project(plan, raw_cols.contiguous(), z, None, y, None, stream)
    return z, y


def gather_x(part, ncols: int, world: int, align: int = 8):
    """Concatenation along the last axis of every rank's column part (the
    ranks' ``xshard`` ranges, in rank order) into the whole [..., ncols]
    array on every rank: an all-gather of the parts padded to the widest
    one.  Without a process group the part is returned unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or world == 1:
        return part
    widths = [xshard(ncols, r, world, align) for r in range(world)]
    wmax = max(b - a for a, b in widths)
    lead = part.shape[:-1]
    pad = torch.zeros(*lead, wmax, dtype=part.dtype, device=part.device)
    pad[..., :part.shape[-1]] = part
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad.contiguous())
    return torch.cat([b[..., :hi - lo] for b, (lo, hi) in zip(bufs, widths)], dim=-1)
