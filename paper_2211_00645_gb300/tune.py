"""Autotuner for the batched live view.

The batched launch has three knobs that change its speed but not its
results (bit for bit):

* the kernel shape (``OPM_SHAPE_*``): how a 32 x 128 output tile is split
  among warps and lanes.  ``per_j32x2`` and ``per_j16x2`` are the periodic
  kernel with 32 or 16 columns j per warp and 2 columns x per lane (plans
  whose pixel/step is a periodic family), ``fast_j8x4`` the fast kernel with
  8 columns j per warp, 4 columns x per lane and two rows per stage, and
  ``gen_j8x4`` the general kernel (one row per stage, a whole row band per
  unit);
* ``kchunk``: camera rows per work unit of the fast kernels (longer units
  stream more stages per ring fill but balance worse across CTAs);
* ``ctas_per_sm``: persistent CTAs per SM (1..4; the general kernel takes
  at most 2).

``Tuner.tune`` times every candidate the items allow on the caller's items
with CUDA events and keeps the fastest per workload signature;
``Tuner.best`` looks a signature up and returns (shape, kchunk,
ctas_per_sm).  Signatures depend on the geometry (theta, step and pixel,
which fix the slab depth, the plan family and so the kernels that apply),
the SM count and the order of magnitude of the raw bytes and of the item
count, so one tuning serves every batch of that class.  The table can be
kept in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

KCHUNKS = (16, 32, 64, 128, 256)
CTAS = (2, 3, 4)
from . import OPM_SHAPE_FAST_J8X4 as FAST_J8X4
from . import OPM_SHAPE_GEN_J8X4 as GEN_J8X4
from . import OPM_SHAPE_PER_J16X2 as PER_J16X2
from . import OPM_SHAPE_PER_J32X2 as PER_J32X2
from . import SHAPE_NAMES

SHAPE_IDS = {v: k for k, v in SHAPE_NAMES.items()}


def shapes_for(items, path_of: Optional[Callable] = None) -> Tuple[int, ...]:
    """Kernel shapes that apply to ``items``: the periodic ones when every
    item the fast kernels take shares one periodic family (16-column runs
    for the 1/3 family only), the fast one, and the general one (which takes
    any item)."""
    if path_of is None:
        from . import opm_plan_path as path_of
    fams = set()
    fast = False
    for it in items:
        if it.get("zsum") is not None or it.get("argz") is not None:
            continue
        path, p, q = path_of(it["plan"])
        if path == 2:
            fams.add((p, q))
            fast = True
        elif path == 1:
            fams.add(None)
            fast = True
    out = []
    if fast and len(fams) == 1 and None not in fams:
        out += [PER_J32X2]
        if fams == {(1, 3)}:        # 16-column runs are compiled for the 1/3 family only
            out += [PER_J16X2]
    return tuple(out + [FAST_J8X4, GEN_J8X4])


def candidates(kchunks: Iterable[int] = KCHUNKS, ctas: Iterable[int] = CTAS,
               shapes: Iterable[int] = (FAST_J8X4,)):
    """(shape, kchunk, ctas) triples: every kchunk x ctas for the fast
    kernels' shapes; for the general kernel, which ignores kchunk and runs at
    most 2 CTAs per SM, the first kchunk with each distinct CTA count."""
    kchunks, ctas = list(kchunks), list(ctas)
    out = []
    for sh in shapes:
        if sh == GEN_J8X4:
            out += [(sh, kchunks[0], c) for c in sorted({min(c, 2) for c in ctas})]
        else:
            out += [(sh, k, c) for k in kchunks for c in ctas]
    return out


def signature(items, sm_count: int) -> str:
    """Workload class of a list of batch items (dicts as for ``Batch.set``)."""
    plans = [it["plan"] for it in items]
    geo = sorted({f"{p.theta_deg:g}/{p.step:g}/{p.pixel:g}" for p in plans})
    raw = sum(p.nscan * p.nrows * p.ncols * 2 for p in plans)
    rb = int(math.log2(raw)) if raw > 0 else 0
    ib = int(math.log2(len(items))) if items else 0
    return f"sm{sm_count}:{','.join(geo)}:raw2^{rb}:items2^{ib}"


class Tuner:
    """Table of the fastest (shape, kchunk, ctas_per_sm) per workload signature."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.table: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def best(self, items, sm_count: int) -> Optional[Tuple[int, int, int]]:
        e = self.table.get(signature(items, sm_count))
        return (SHAPE_IDS[e["shape"]], e["kchunk"], e["ctas_per_sm"]) if e else None

    def save(self) -> None:
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def record(self, sig: str, timings: Dict[Tuple[int, int, int], float]) -> dict:
        """Stores the fastest of ``timings`` {(shape, kchunk, ctas): microseconds}
        (ties to the smallest triple)."""
        (sh, k, c), us = min(timings.items(), key=lambda kv: (kv[1], kv[0]))
        entry = {"shape": SHAPE_NAMES[sh], "kchunk": k, "ctas_per_sm": c, "us": round(us, 2),
                 "candidates": {f"{SHAPE_NAMES[s_]}/{kk}x{cc}": round(t, 2)
                                for (s_, kk, cc), t in sorted(timings.items())}}
        self.table[sig] = entry
        return entry

    def tune(self, items, kchunks: Sequence[int] = KCHUNKS, ctas: Sequence[int] = CTAS,
             shapes: Optional[Sequence[int]] = None, reps: int = 3, warmup: int = 1,
             timer: Optional[Callable[[int, int, int], float]] = None, sm_count: Optional[int] = None,
             force: bool = False) -> dict:
        """Times every candidate on ``items`` and records the fastest.

        ``shapes`` defaults to ``shapes_for(items)``.  ``timer(shape, kchunk,
        ctas) -> microseconds`` replaces the GPU timing (for tests of the
        table logic).  Outputs of ``items`` are overwritten."""
        if sm_count is None:
            import torch
            sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        sig = signature(items, sm_count)
        if not force and sig in self.table:
            return self.table[sig]
        if shapes is None:
            shapes = shapes_for(items)
        if timer is None:
            timer = _gpu_timer(items, reps, warmup)
        timings = {cand: float(timer(*cand)) for cand in candidates(kchunks, ctas, shapes)}
        entry = self.record(sig, timings)
        self.save()
        return entry


def _gpu_timer(items, reps: int, warmup: int):
    import torch

    from . import Batch
    b = Batch(max_items=max(1, len(items)), max_units=1 << 24)
    s = torch.cuda.current_stream()

    def run(shape: int, kchunk: int, ctas: int) -> float:
        b.set(items, kchunk, shape)
        b.upload(s)
        for _ in range(warmup):
            b.launch(ctas, s)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            b.launch(ctas, s)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    return run
