"""Autotuner for the batched live view.

The persistent batch kernel has two launch-shape knobs that change its speed
but not its results: ``kchunk`` (camera rows per work unit: longer units
stream more stages per ring fill but balance worse across CTAs) and
``ctas_per_sm`` (resident CTAs per SM, 1..4, against shared memory per
CTA).  ``Tuner.tune`` times every candidate on the caller's items with CUDA
events and keeps the fastest per workload signature; ``Tuner.best`` looks a
signature up.  Signatures depend on the geometry (theta, step and pixel,
which fix the slab depth and so the kernel's shared memory), the SM count
and the order of magnitude of the raw bytes and of the item count, so one
tuning serves every batch of that class.  The table can be kept in a JSON
file.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

KCHUNKS = (16, 32, 64, 128, 256)
CTAS = (2, 3, 4)


def signature(items, sm_count: int) -> str:
    """Workload class of a list of batch items (dicts as for ``Batch.set``)."""
    plans = [it["plan"] for it in items]
    geo = sorted({f"{p.theta_deg:g}/{p.step:g}/{p.pixel:g}" for p in plans})
    raw = sum(p.nscan * p.nrows * p.ncols * 2 for p in plans)
    rb = int(math.log2(raw)) if raw > 0 else 0
    ib = int(math.log2(len(items))) if items else 0
    return f"sm{sm_count}:{','.join(geo)}:raw2^{rb}:items2^{ib}"


class Tuner:
    """Table of the fastest (kchunk, ctas_per_sm) per workload signature."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.table: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def best(self, items, sm_count: int) -> Optional[Tuple[int, int]]:
        e = self.table.get(signature(items, sm_count))
        return (e["kchunk"], e["ctas_per_sm"]) if e else None

    def save(self) -> None:
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def record(self, sig: str, timings: Dict[Tuple[int, int], float]) -> dict:
        """Stores the fastest of ``timings`` {(kchunk, ctas): microseconds}."""
        (k, c), us = min(timings.items(), key=lambda kv: (kv[1], kv[0]))
        entry = {"kchunk": k, "ctas_per_sm": c, "us": round(us, 2),
                 "candidates": {f"{kk}x{cc}": round(t, 2) for (kk, cc), t in sorted(timings.items())}}
        self.table[sig] = entry
        return entry

    def tune(self, items, kchunks: Sequence[int] = KCHUNKS, ctas: Sequence[int] = CTAS, reps: int = 3,
             warmup: int = 1, timer: Optional[Callable[[int, int], float]] = None, sm_count: Optional[int] = None,
             force: bool = False) -> dict:
        """Times every (kchunk, ctas) on ``items`` and records the fastest.

        ``timer(kchunk, ctas) -> microseconds`` replaces the GPU timing (for
        tests of the table logic).  Outputs of ``items`` are overwritten."""
        if sm_count is None:
            import torch
            sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        sig = signature(items, sm_count)
        if not force and sig in self.table:
            return self.table[sig]
        if timer is None:
            timer = _gpu_timer(items, reps, warmup)
        timings = {(k, c): float(timer(k, c)) for k in kchunks for c in ctas}
        entry = self.record(sig, timings)
        self.save()
        return entry


def _gpu_timer(items, reps: int, warmup: int):
    import torch

    from . import Batch
    b = Batch(max_items=max(1, len(items)), max_units=1 << 24)
    s = torch.cuda.current_stream()

    def run(kchunk: int, ctas: int) -> float:
        b.set(items, kchunk)
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


def candidates(kchunks: Iterable[int] = KCHUNKS, ctas: Iterable[int] = CTAS):
    return [(k, c) for k in kchunks for c in ctas]
