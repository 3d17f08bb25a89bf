"""Live-view serving: camera stacks arrive, live views come back.

The paper refreshes its widefield-like view while the camera keeps
acquiring, and shows that the lag between acquisition and display grows
once processing is slower than the camera (Supp. Fig. 1).  This module serves
that loop on one GPU:

* a producer (camera stand-in) writes each stack into a pinned host ring
  buffer (``PinnedRing``) and publishes it at its arrival time; when the ring
  is full the camera stalls (back-pressure) and the stall counts as lag;
* the scheduler admits a request when its device footprint (raw stack plus
  outputs) fits a memory budget, copies it to the device on a copy stream and
  keeps it resident until its views are back on the host;
* every tick launches one persistent batched projection (``Batch``) over all
  admitted requests whose copies have landed, channels as strided ROIs of the
  stack, while later copies and the previous tick's read-back proceed on the
  copy stream (continuous batching: a request that arrives while a batch runs
  joins the next tick);
* a ring range is released as soon as its copy to the device has landed;
* latency is arrival -> projections in host memory, the paper's lag.

``PlainServer`` is the reference path: one request at a time, synchronous
copy in, one projection per channel, copy out.
"""
from __future__ import annotations

import bisect
import dataclasses
import threading
import time
from collections import deque
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np


# ------------------------------------------------------------------ arena
class DeviceArena:
    """First-fit allocator of byte ranges inside a budget.

    Pure bookkeeping over offsets; ``base`` (a device tensor) is optional so
    the policy can be exercised without a GPU.  Free ranges are coalesced.
    """

    def __init__(self, budget: int, align: int = 256, base=None):
        if budget <= 0:
            raise ValueError("budget must be positive")
        self.budget = int(budget)
        self.align = int(align)
        self.base = base
        self._free: List[Tuple[int, int]] = [(0, self.budget)]  # sorted (offset, size)
        self._used: Dict[int, int] = {}

    def _round(self, n: int) -> int:
        return (int(n) + self.align - 1) // self.align * self.align

    @property
    def in_use(self) -> int:
        return sum(self._used.values())

    def alloc(self, nbytes: int) -> Optional[int]:
        size = self._round(max(1, nbytes))
        for i, (off, sz) in enumerate(self._free):
            if sz >= size:
                if sz == size:
                    self._free.pop(i)
                else:
                    self._free[i] = (off + size, sz - size)
                self._used[off] = size
                return off
        return None

    def free(self, off: int) -> None:
        size = self._used.pop(off)
        i = bisect.bisect_left(self._free, (off, 0))
        self._free.insert(i, (off, size))
        # coalesce with neighbours
        if i + 1 < len(self._free) and self._free[i][0] + self._free[i][1] == self._free[i + 1][0]:
            o, s = self._free.pop(i + 1)
            self._free[i] = (self._free[i][0], self._free[i][1] + s)
        if i > 0 and self._free[i - 1][0] + self._free[i - 1][1] == self._free[i][0]:
            o, s = self._free.pop(i)
            self._free[i - 1] = (self._free[i - 1][0], self._free[i - 1][1] + s)

    def view(self, off: int, nbytes: int):
        """uint8 device view of an allocation (needs ``base``)."""
        return self.base[off:off + nbytes]


# ------------------------------------------------------------ pinned ring
class PinnedRing:
    """Byte ring of (pinned) host memory that camera stacks are written into.

    Ranges are taken at the head in arrival order and wrap to the start when
    the tail end is too short; a range is returned when every request that
    refers to it has released it, and the tail advances over returned ranges
    in order.  ``acquire`` blocks while the ring is full (back-pressure).

    The content is written once at construction (``fill(uint8_array, seed)``
    fills it in place; default: repeated Poisson+blob tiles), standing in
    for the camera's DMA into the ring: a stack published at an offset holds
    whatever frames the ring has there, which keeps acquisition itself free.
    """

    def __init__(self, nbytes: int, pin: bool = True, align: int = 256, fill=None, seed: int = 5):
        import torch
        self.nbytes = int(nbytes)
        self.align = int(align)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=pin)
        (fill or _tile_fill)(self.buf.numpy(), seed)
        self._entries: deque = deque()          # [offset, size, refs]
        self._cond = threading.Condition()
        self.stalls = 0
        self.peak = 0

    def _round(self, n: int) -> int:
        return (int(n) + self.align - 1) // self.align * self.align

    def _place(self, size: int) -> Optional[int]:
        if not self._entries:
            return 0 if size <= self.nbytes else None
        tail = self._entries[0][0]
        last_off, last_size, _ = self._entries[-1]
        head = last_off + last_size
        if last_off >= tail:                    # not wrapped: free space at the end, then before tail
            if head + size <= self.nbytes:
                return head
            return 0 if size <= tail else None
        return head if head + size <= tail else None

    def in_use(self) -> int:
        with self._cond:
            return sum(e[1] for e in self._entries)

    def acquire(self, nbytes: int, refs: int = 1, timeout: Optional[float] = None) -> int:
        size = self._round(max(1, nbytes))
        if size > self.nbytes:
            raise ValueError(f"stack of {nbytes} bytes exceeds the {self.nbytes}-byte ring")
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self._cond:
            stalled = False
            while True:
                off = self._place(size)
                if off is not None:
                    break
                if not stalled:
                    self.stalls += 1
                    stalled = True
                left = None if t_end is None else t_end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError("pinned ring full")
                self._cond.wait(left if left is not None else 1.0)
            self._entries.append([off, size, int(refs)])
            self.peak = max(self.peak, sum(e[1] for e in self._entries))
            return off

    def try_acquire(self, nbytes: int, refs: int = 1) -> Optional[int]:
        """``acquire`` that returns None at once instead of waiting (no stall
        is counted: the caller decides what a failed attempt means)."""
        size = self._round(max(1, nbytes))
        if size > self.nbytes:
            raise ValueError(f"stack of {nbytes} bytes exceeds the {self.nbytes}-byte ring")
        with self._cond:
            off = self._place(size)
            if off is None:
                return None
            self._entries.append([off, size, int(refs)])
            self.peak = max(self.peak, sum(e[1] for e in self._entries))
            return off

    def wait_release(self, timeout: float) -> None:
        """Sleeps until a range is returned or ``timeout`` seconds pass."""
        with self._cond:
            self._cond.wait(max(0.0, timeout))

    def release(self, off: int) -> None:
        with self._cond:
            for e in self._entries:
                if e[0] == off and e[2] > 0:
                    e[2] -= 1
                    break
            else:
                raise KeyError(f"no live ring range at {off}")
            while self._entries and self._entries[0][2] == 0:
                self._entries.popleft()
            self._cond.notify_all()

    def view(self, off: int, shape):
        """uint16 host tensor of ``shape`` at byte offset ``off``."""
        import torch
        n = int(np.prod(shape)) * 2
        return self.buf[off:off + n].view(torch.uint16).view(*shape)


def _tile_fill(out: np.ndarray, seed: int) -> None:
    """Fills ``out`` in place with repeats of one 50x128x256 stack tile."""
    import opm_synth
    tile = opm_synth.tiled_stack((50, 128, 256), seed=seed).view(np.uint8).ravel()
    k = min(tile.size, out.size)
    out[:k] = tile[:k]
    while k < out.size:                       # doubling copies
        m = min(k, out.size - k)
        out[k:k + m] = out[:m]
        k += m


# ---------------------------------------------------------------- requests
@dataclasses.dataclass
class Request:
    rid: int
    nscan: int
    nrows: int
    ncols: int            # per channel
    channels: int
    host: object          # pinned uint16 tensor [nscan][nrows][channels*ncols]
    t_arrival: float = 0.0
    t_done: float = 0.0
    dropped: bool = False
    error: Optional[str] = None
    results: Optional[list] = None   # per channel {"zmip", "ymip"} host tensors
    ring: Optional[PinnedRing] = None  # ring holding ``host``, released once copied
    ring_off: int = -1
    t_admit: float = 0.0     # copy to the device issued
    t_launch: float = 0.0    # projection launched
    res_arena: Optional["DeviceArena"] = None  # pinned arena holding ``results``
    res_off: int = -1
    geometry: Optional[Tuple[float, float, float]] = None  # (theta, step, pixel) it was served with
    # device clock of its copy in (perf_counter seconds): when the copy engine
    # started it (after any earlier copy on the stream) and when it landed
    t_h2d_start: float = 0.0
    t_h2d_end: float = 0.0
    # planes written by the camera so far (a stack is complete at nscan)
    frames_ready: int = -1

    def __post_init__(self):
        if self.frames_ready < 0:
            self.frames_ready = self.nscan

    def release_host(self) -> None:
        if self.ring is not None:
            ring, self.ring = self.ring, None
            ring.release(self.ring_off)

    def release_results(self) -> None:
        """Returns the pinned result buffers to the server (the views in
        ``results`` must not be used afterwards)."""
        if self.res_arena is not None:
            arena, self.res_arena = self.res_arena, None
            arena.free(self.res_off)
            self.results = None

    @property
    def shape(self):
        return (self.nscan, self.nrows, self.ncols)

    @property
    def latency_ms(self) -> float:
        return (self.t_done - self.t_arrival) * 1e3


def request_bytes(plan, channels: int) -> int:
    """Device footprint: raw frames of every channel plus z-MIP and y-MIP."""
    raw = 2 * plan.nscan * plan.nrows * plan.ncols * channels
    outs = 4 * (plan.ny * plan.nx + plan.nz * plan.nx) * channels
    return raw + outs + (1 + 2 * channels) * 256  # one 256-byte alignment gap per sub-buffer


def result_bytes(plan, channels: int) -> int:
    """Pinned host bytes of one request's views: z-MIP and y-MIP per channel."""
    per = ((4 * plan.ny * plan.nx + 255) // 256 + (4 * plan.nz * plan.nx + 255) // 256) * 256
    return per * channels


def result_views(arena: "DeviceArena", off: int, plan, channels: int, torch):
    """Per-channel {"zmip", "ymip"} float32 views of a pinned arena range."""
    out, pos = [], off
    for _ in range(channels):
        nz = 4 * plan.ny * plan.nx
        z = arena.view(pos, nz).view(torch.float32).view(plan.ny, plan.nx)
        pos += (nz + 255) // 256 * 256
        ny = 4 * plan.nz * plan.nx
        y = arena.view(pos, ny).view(torch.float32).view(plan.nz, plan.nx)
        pos += (ny + 255) // 256 * 256
        out.append({"zmip": z, "ymip": y})
    return out


def percentile(xs, q):
    if not xs:
        return None
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


class PlanCache:
    """One plan per stack shape for a fixed sheet angle, scan step and pixel."""

    def __init__(self, theta_deg: float, step: float, pixel: float):
        self.theta_deg, self.step, self.pixel = float(theta_deg), float(step), float(pixel)
        self._plans: Dict[Tuple[int, int, int], object] = {}

    def get(self, nscan: int, nrows: int, ncols: int):
        from . import Plan
        key = (int(nscan), int(nrows), int(ncols))
        if key not in self._plans:
            self._plans[key] = Plan(*key, self.theta_deg, self.step, self.pixel)
        return self._plans[key]

    @property
    def geometry(self) -> Tuple[float, float, float]:
        return (self.theta_deg, self.step, self.pixel)


class _Geometries:
    """The servers' current plan cache, switchable while serving (the paper
    lets the user change the deskew parameters during imaging).  Caches of
    earlier geometries are kept, so switching back re-creates no plan."""

    def __init__(self, plans: PlanCache):
        self.current = plans
        self._all = {plans.geometry: plans}

    def cache(self, theta_deg: float, step: float, pixel: float) -> PlanCache:
        key = (float(theta_deg), float(step), float(pixel))
        if key not in self._all:
            self._all[key] = PlanCache(*key)
        return self._all[key]

    def set(self, theta_deg: float, step: float, pixel: float) -> PlanCache:
        self.current = self.cache(theta_deg, step, pixel)
        return self.current


class _Resident:
    """A request admitted to the device: arena range, device views, events."""

    def __init__(self, req: Request, plan, off: int, arena: DeviceArena, torch):
        self.req, self.plan, self.off = req, plan, off
        C = req.channels
        nraw = 2 * plan.nscan * plan.nrows * plan.ncols * C
        pos = off
        self.raw = arena.view(pos, nraw).view(torch.uint16).view(plan.nscan, plan.nrows, plan.ncols * C)
        pos += (nraw + 255) // 256 * 256
        self.z, self.y = [], []
        for _ in range(C):
            nz = 4 * plan.ny * plan.nx
            self.z.append(arena.view(pos, nz).view(torch.float32).view(plan.ny, plan.nx))
            pos += (nz + 255) // 256 * 256
            ny = 4 * plan.nz * plan.nx
            self.y.append(arena.view(pos, ny).view(torch.float32).view(plan.nz, plan.nx))
            pos += (ny + 255) // 256 * 256
        self.h2d = None           # event after the latest copy in
        self.h2d_start = None     # event before the copy of the last planes
        self.copied = 0           # planes whose copy has been issued
        self.launched = False


class LiveViewServer:
    """Continuous-batching live-view server on one GPU (see module docstring)."""

    def __init__(self, plans: PlanCache, budget_bytes: int, max_items: int = 256, max_units: int = 1 << 22,
                 kchunk: int = 0, ctas_per_sm: int = 0, max_inflight: int = 2, keep_results: bool = True,
                 result_bytes: int = 1 << 30, shape: int = 0):
        import torch

        from . import Batch
        self.torch = torch
        self._geo = _Geometries(plans)
        self.arena = DeviceArena(budget_bytes, base=torch.empty(int(budget_bytes), dtype=torch.uint8, device="cuda"))
        # pinned destination of the read-back, allocated once
        self.results = DeviceArena(result_bytes, base=torch.empty(int(result_bytes), dtype=torch.uint8,
                                                                   pin_memory=True))
        self.h2d = torch.cuda.Stream()
        self.d2h = torch.cuda.Stream()
        self.comp = torch.cuda.Stream()
        self.batches = [Batch(max_items, max_units) for _ in range(max_inflight)]
        self.max_items = max_items
        self.kchunk, self.ctas, self.shape = kchunk, ctas_per_sm, shape  # shape: an OPM_SHAPE_* value
        self.max_inflight = max_inflight
        self.keep_results = keep_results
        self._lock = threading.Lock()
        self._arrivals: deque = deque()
        self.waiting: deque = deque()
        self.resident: List[_Resident] = []
        self.inflight: deque = deque()
        self.done: List[Request] = []
        self.rejected: List[Request] = []
        self.cancelled: List[Request] = []
        self.poll_s = 50e-6     # scheduler poll interval while the device is busy
        self.host_set_s = 0.0   # host time spent building work lists
        self.peak_in_use = 0
        self.ticks = 0
        self.batch_sizes: List[int] = []
        # a timed event on the copy stream and its host time: converts the
        # copies' device timestamps to the host clock of the latencies
        self._clock_ev = None
        self._clock_host = 0.0
        # copy scheduling: pieces of a stack and the bytes kept queued
        self.copy_piece = 64 << 20
        self.copy_backlog = 512 << 20
        self._h2d_q: deque = deque()   # (event after a copy, its bytes), oldest first
        self._h2d_inflight = 0

    @property
    def plans(self) -> PlanCache:
        return self._geo.current

    def set_geometry(self, theta_deg: float, step: float, pixel: float) -> None:
        """New deskew parameters for requests admitted from now on; those
        already admitted finish with theirs.  Batches may mix geometries."""
        with self._lock:
            self._geo.set(theta_deg, step, pixel)

    # producer side ------------------------------------------------------
    def submit(self, req: Request) -> None:
        with self._lock:
            self._arrivals.append(req)

    def cancel(self, rid: int) -> bool:
        """Withdraws a request that has not been admitted yet (still queued
        for memory): it is returned to the caller's ring and listed in
        ``cancelled``.  Admitted requests run to completion; returns False
        for those and for unknown ids."""
        with self._lock:
            for q in (self._arrivals, self.waiting):
                for req in q:
                    if req.rid == rid:
                        q.remove(req)
                        req.error = "cancelled"
                        req.t_done = time.perf_counter()
                        req.release_host()
                        self.cancelled.append(req)
                        return True
        return False

    # scheduler ----------------------------------------------------------
    def _admit(self) -> None:
        torch = self.torch
        with self._lock:                       # cancel() touches the same queues
            while self._arrivals:
                self.waiting.append(self._arrivals.popleft())
            while self.waiting:
                req = self.waiting[0]
                plan = self.plans.get(req.nscan, req.nrows, req.ncols)
                req.geometry = self.plans.geometry
                need = request_bytes(plan, req.channels)
                if need > self.arena.budget or result_bytes(plan, req.channels) > self.results.budget:
                    # can never fit: refuse, keep serving others
                    self.waiting.popleft()
                    req.error = (f"needs {need} device bytes (budget {self.arena.budget}) and "
                                 f"{result_bytes(plan, req.channels)} result bytes ({self.results.budget})")
                    req.t_done = time.perf_counter()
                    self.rejected.append(req)
                    req.release_host()
                    continue
                off = self.arena.alloc(need)
                if off is None:                # wait for memory (FIFO, no overtaking)
                    break
                self.waiting.popleft()
                r = _Resident(req, plan, off, self.arena, torch)
                if self._clock_ev is None:
                    self._calibrate_clock()
                req.t_admit = time.perf_counter()
                self.resident.append(r)
                self.peak_in_use = max(self.peak_in_use, self.arena.in_use)

    def _calibrate_clock(self) -> None:
        """Host time of a timed event on the copy stream.  The host reads its
        clock after the event completes, so each reading is late by the
        synchronisation delay; the smallest of a few readings is kept."""
        torch = self.torch
        self._clock_ev = torch.cuda.Event(enable_timing=True)
        self._clock_ev.record(self.h2d)
        self._clock_ev.synchronize()
        best = time.perf_counter()
        for _ in range(4):
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.h2d)
            ev.synchronize()
            best = min(best, time.perf_counter() - self._clock_ev.elapsed_time(ev) * 1e-3)
        self._clock_host = best

    def _copy_frames(self, r: "_Resident", max_bytes: int) -> int:
        """Issues the copy of the next planes the camera has written for this
        request, at most ``max_bytes`` (at least one plane); returns bytes."""
        torch = self.torch
        plane = 2 * r.plan.nrows * r.plan.ncols * r.req.channels
        a = r.copied
        b = min(r.req.frames_ready, r.plan.nscan, a + max(1, max_bytes // plane))
        if b <= a:
            return 0
        host = r.req.host.view(torch.int16)
        with torch.cuda.stream(self.h2d):
            if b == r.plan.nscan:
                r.h2d_start = torch.cuda.Event(enable_timing=True)
                r.h2d_start.record(self.h2d)
            r.raw.view(torch.int16)[a:b].copy_(host[a:b], non_blocking=True)
            r.h2d = torch.cuda.Event(enable_timing=True)
            r.h2d.record(self.h2d)
        r.copied = b
        nbytes = (b - a) * plane
        self._h2d_q.append((r.h2d, nbytes))
        return nbytes

    def _copy_more(self) -> None:
        """Copies frames that have arrived for admitted requests, in pieces
        of at most ``copy_piece`` bytes, keeping at most ``copy_backlog``
        bytes queued on the copy stream: complete stacks first (their
        latency is running), oldest first, then stacks still being
        acquired.  A stack that has just been completed thus waits for at
        most the backlog, not for other stacks' whole copies."""
        q = self._h2d_q
        while q and q[0][0].query():
            self._h2d_inflight -= q.popleft()[1]
        pend = [r for r in self.resident if r.copied < r.plan.nscan and r.req.frames_ready > r.copied]
        if not pend:
            return
        pend.sort(key=lambda r: (r.req.frames_ready < r.plan.nscan, r.req.t_arrival))
        while self._h2d_inflight < self.copy_backlog and pend:
            r = pend[0]
            n = self._copy_frames(r, self.copy_piece)
            self._h2d_inflight += n
            if r.copied >= min(r.req.frames_ready, r.plan.nscan):
                pend.pop(0)

    def _landed(self, r: "_Resident") -> bool:
        return r.copied == r.plan.nscan and r.h2d.query()

    def _launch_tick(self) -> bool:
        torch = self.torch
        if len(self.inflight) >= self.max_inflight:
            return False
        ready = []
        nitems = 0
        full = False
        for r in self.resident:
            if r.launched or not self._landed(r):
                continue
            r.req.release_host()                 # copy landed: the ring range is free
            if full or nitems + r.req.channels > self.max_items:
                full = True                      # keep arrival order: later requests wait too
                continue
            off = self.results.alloc(result_bytes(r.plan, r.req.channels))
            if off is None:                      # read-back space is busy: wait for a retire
                full = True
                continue
            r.req.res_arena, r.req.res_off = self.results, off
            ready.append(r)
            nitems += r.req.channels
        if not ready:
            return False
        b = self.batches[self.ticks % len(self.batches)]
        items = []
        for r in ready:
            C, n = r.req.channels, r.plan.ncols
            for c in range(C):
                items.append({"plan": r.plan, "raw": r.raw[:, :, c * n:], "row_pitch": C * n,
                              "plane_pitch": r.plan.nrows * C * n, "zmip": r.z[c], "ymip": r.y[c]})
        t_set = time.perf_counter()
        b.set(items, self.kchunk, self.shape)
        self.host_set_s += time.perf_counter() - t_set
        for r in ready:
            self.comp.wait_event(r.h2d)
            r.launched = True
        b.upload(self.comp)
        b.launch_graph(self.ctas, self.comp)
        ev_c = torch.cuda.Event()
        ev_c.record(self.comp)
        self.d2h.wait_event(ev_c)
        t = time.perf_counter()
        with torch.cuda.stream(self.d2h):
            for r in ready:
                res = result_views(self.results, r.req.res_off, r.plan, r.req.channels, torch)
                for c, h in enumerate(res):
                    h["zmip"].copy_(r.z[c], non_blocking=True)
                    h["ymip"].copy_(r.y[c], non_blocking=True)
                r.req.results = res
                r.req.t_launch = t
            ev_d = torch.cuda.Event()
            ev_d.record(self.d2h)
        self.inflight.append((ready, ev_d))
        self.ticks += 1
        self.batch_sizes.append(len(ready))
        return True

    def _retire(self, block: bool) -> bool:
        if not self.inflight:
            return False
        ready, ev_d = self.inflight[0]
        if block:
            ev_d.synchronize()
        elif not ev_d.query():
            return False
        t = time.perf_counter()
        self.inflight.popleft()
        for r in ready:
            r.req.t_done = t
            r.req.t_h2d_start = self._clock_host + self._clock_ev.elapsed_time(r.h2d_start) * 1e-3
            r.req.t_h2d_end = self._clock_host + self._clock_ev.elapsed_time(r.h2d) * 1e-3
            if not self.keep_results:
                r.req.release_results()
            self.arena.free(r.off)
            self.resident.remove(r)
            self.done.append(r.req)
        return True

    def step(self) -> None:
        """One scheduler pass: admit, launch a tick, retire finished ticks
        (each phase an NVTX range for timeline profilers)."""
        nvtx = self.torch.cuda.nvtx
        nvtx.range_push("opm.admit")
        self._admit()
        self._copy_more()
        nvtx.range_pop()
        nvtx.range_push("opm.launch_tick")
        launched = self._launch_tick()
        nvtx.range_pop()
        retired = self._retire(block=False)
        if not launched and not retired and (self.inflight or self.resident):
            # nothing to launch or retire yet: hand landed copies' ring ranges
            # back to the camera and poll again shortly (a blocking wait on
            # the oldest tick would hold them and stall the camera; a busy
            # loop would starve the camera thread)
            self._release_landed()
            time.sleep(self.poll_s)

    def _release_landed(self) -> None:
        for r in self.resident:
            if not r.launched and r.req.ring is not None and self._landed(r):
                r.req.release_host()

    def run(self, n_expected: int, timeout_s: float = 600.0, idle=None) -> None:
        """Serves until ``n_expected`` requests are done, rejected or cancelled."""
        t_end = time.perf_counter() + timeout_s
        while len(self.done) + len(self.rejected) + len(self.cancelled) < n_expected:
            if time.perf_counter() > t_end:
                raise TimeoutError(f"served {len(self.done)} of {n_expected} requests")
            self.step()
            if not self.inflight and not self.resident and not self.waiting:
                with self._lock:
                    empty = not self._arrivals
                if empty:
                    time.sleep(idle if idle is not None else 0.0002)


class PlainServer:
    """Reference path: one request at a time on one stream, synchronous copy
    in, one stand-alone projection per channel, copy out."""

    def __init__(self, plans: PlanCache, keep_results: bool = True, result_bytes: int = 1 << 30):
        import torch
        self.torch = torch
        self._geo = _Geometries(plans)
        self.keep_results = keep_results
        self.results = DeviceArena(result_bytes, base=torch.empty(int(result_bytes), dtype=torch.uint8,
                                                                  pin_memory=True))
        self._lock = threading.Lock()
        self._arrivals: deque = deque()
        self.done: List[Request] = []
        self.rejected: List[Request] = []
        self.cancelled: List[Request] = []   # kept for the common run() contract; the plain path has no queue

    @property
    def plans(self) -> PlanCache:
        return self._geo.current

    def set_geometry(self, theta_deg: float, step: float, pixel: float) -> None:
        with self._lock:
            self._geo.set(theta_deg, step, pixel)

    def submit(self, req: Request) -> None:
        with self._lock:
            self._arrivals.append(req)

    def _serve(self, req: Request) -> None:
        from . import opm_project
        torch = self.torch
        # a request that names its geometry is served with it, else the current one
        plans = self.plans if req.geometry is None else self._geo.cache(*req.geometry)
        plan = plans.get(req.nscan, req.nrows, req.ncols)
        req.geometry = plans.geometry
        off = self.results.alloc(result_bytes(plan, req.channels))
        if off is None:
            req.error = "result buffers exhausted (keep_results without release_results)"
            req.t_done = time.perf_counter()
            self.rejected.append(req)
            req.release_host()
            return
        req.t_admit = time.perf_counter()
        raw = torch.empty(req.host.shape, dtype=torch.uint16, device="cuda")
        raw.view(torch.int16).copy_(req.host.view(torch.int16))
        req.release_host()
        req.t_launch = time.perf_counter()
        res = result_views(self.results, off, plan, req.channels, torch)
        req.res_arena, req.res_off = self.results, off
        n = req.ncols
        for c in range(req.channels):
            ch = raw[:, :, c * n:(c + 1) * n].contiguous()
            z = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device="cuda")
            y = torch.empty((plan.nz, plan.nx), dtype=torch.float32, device="cuda")
            opm_project(plan, ch, z, None, y, None)
            res[c]["zmip"].copy_(z)
            res[c]["ymip"].copy_(y)
        req.results = res
        req.t_done = time.perf_counter()
        if not self.keep_results:
            req.release_results()
        self.done.append(req)

    def run(self, n_expected: int, timeout_s: float = 600.0, idle=None) -> None:
        """Serves until ``n_expected`` requests are done, rejected or cancelled."""
        t_end = time.perf_counter() + timeout_s
        while len(self.done) + len(self.rejected) + len(self.cancelled) < n_expected:
            if time.perf_counter() > t_end:
                raise TimeoutError(f"served {len(self.done)} of {n_expected} requests")
            with self._lock:
                req = self._arrivals.popleft() if self._arrivals else None
            if req is None:
                time.sleep(idle if idle is not None else 0.0002)
                continue
            self._serve(req)


class Camera(threading.Thread):
    """Camera stand-in: writes stacks into a pinned ring and publishes them.

    ``shapes`` lists request shapes (nscan, nrows, ncols per channel,
    channels); stack i takes ``shapes[order[i]]`` with a seeded order and is
    complete at a Poisson time (``rate`` stacks/s; None: all at once,
    saturating).  A request's arrival time is that completion time, so a
    stall on a full ring counts as lag.

    ``fps``: frames per second of the acquisition.  With it, stack i is
    acquired plane by plane over the nscan / fps seconds that end at its
    completion time: its ring range is taken when its first frame is due
    and ``frames_ready`` grows as its frames are written (in steps of
    ``chunk_frames``).  ``stream_frames`` submits the request with its first
    frames, so a server can copy frames while the stack is still being
    acquired (the paper builds the projection as each image is received);
    otherwise the request is submitted complete.  Without ``fps`` every
    stack is written at once at its completion time.

    Host-side fault injection for tests: ``drop`` (arrival indices never
    delivered), ``duplicate`` (delivered twice, sharing one ring range) and
    ``delay_s`` (extra delay per index).
    """

    def __init__(self, server, ring: PinnedRing, shapes, n: int, rate: Optional[float], seed: int = 0,
                 drop=(), duplicate=(), delay_s=None, ring_timeout: float = 120.0, fps: Optional[float] = None,
                 stream_frames: bool = False, chunk_frames: int = 8):
        super().__init__(daemon=True)
        self.server, self.ring, self.shapes, self.n, self.rate = server, ring, list(shapes), n, rate
        rng = np.random.default_rng(seed)
        self.order = rng.integers(0, len(self.shapes), n)
        gaps = rng.exponential(1.0 / rate, n) if rate else np.zeros(n)
        self.offsets = np.cumsum(gaps) - (gaps[0] if n else 0.0)
        self.fps = float(fps) if fps else None
        if self.fps:   # the first stack's first frame is due at the start
            lead = max(self.shapes[int(k)][0] for k in self.order) / self.fps if n else 0.0
            self.offsets = self.offsets + lead
        self.stream_frames = bool(stream_frames) and self.fps is not None
        self.chunk_frames = max(1, int(chunk_frames))
        self.drop, self.duplicate = set(drop), set(duplicate)
        self.delay_s = dict(delay_s or {})
        self.ring_timeout = ring_timeout
        self.delivered = 0
        self.error: Optional[BaseException] = None
        self.t0 = None

    def expected(self) -> int:
        return self.n - len([i for i in self.drop if i < self.n]) + len([i for i in self.duplicate if i < self.n])

    def run(self) -> None:
        try:
            self._run()
        except BaseException as e:        # surfaced by the caller through ``error``
            self.error = e

    def _wait_until(self, t: float) -> None:
        while True:
            now = time.perf_counter()
            if now >= t:
                return
            time.sleep(min(t - now, 0.001))

    def _run(self) -> None:
        import heapq
        self.t0 = time.perf_counter()
        rid = 0
        # stack starts (first frame due) in time order, taken strictly one
        # after the other; frame updates and completions of the stacks being
        # acquired, in time order
        starts, updates = [], []
        seq = 0
        for i in range(self.n):
            if i in self.drop:
                continue
            t_done = self.t0 + self.offsets[i] + self.delay_s.get(i, 0.0)
            nscan = self.shapes[int(self.order[i])][0]
            heapq.heappush(starts, (t_done - nscan / self.fps if self.fps else t_done, seq, i))
            seq += 1
        live = {}   # index -> [requests, time of the first frame, completion time, nscan, frames written]
        t_refused = None  # when the ring first refused the next stack
        while starts or updates:
            now = time.perf_counter()
            if starts and starts[0][0] <= now and (not updates or starts[0][0] <= updates[0][0]):
                t, _, i = starts[0]
                nscan, nrows, ncols, C = self.shapes[int(self.order[i])]
                copies = 2 if i in self.duplicate else 1
                off = self.ring.try_acquire(2 * nscan * nrows * ncols * C, refs=copies)
                if off is None:
                    # ring full: this stack (and every later one) waits and its
                    # lag grows, while the stacks being acquired keep writing
                    if t_refused is None:
                        t_refused = now
                        self.ring.stalls += 1
                    elif now - t_refused > self.ring_timeout:
                        raise TimeoutError("pinned ring full")
                    if not (updates and updates[0][0] <= now):
                        nxt = updates[0][0] - now if updates else 0.05
                        self.ring.wait_release(min(max(nxt, 0.0), 0.05))
                        continue
                    off = -1                   # due frame updates first
            else:
                off = -1
            if off >= 0:
                heapq.heappop(starts)
                if t_refused is not None:      # acquisition starts late: frames are due from now
                    t, t_refused = max(t, now), None
                host = self.ring.view(off, (nscan, nrows, ncols * C))
                t_done = self.t0 + self.offsets[i] + self.delay_s.get(i, 0.0)
                reqs = []
                for _ in range(copies):
                    reqs.append(Request(rid, nscan, nrows, ncols, C, host, t_arrival=t_done, ring=self.ring,
                                        ring_off=off, frames_ready=0 if self.fps else nscan))
                    rid += 1
                live[i] = [reqs, t, t_done, nscan, 0]
                if self.stream_frames:
                    for r in reqs:
                        self.server.submit(r)
                        self.delivered += 1
                heapq.heappush(updates, ((t if self.fps else t_done), seq, 1 if self.fps else 2, i))
                seq += 1
                continue
            if updates and updates[0][0] <= now:
                _, _, kind, i = heapq.heappop(updates)
                if kind == 1:                  # frames written so far, in whole chunks
                    reqs, t_first, t_done, nscan, written = live[i]
                    due = min(nscan, int((now - t_first) * self.fps))
                    if due < nscan:
                        due = due // self.chunk_frames * self.chunk_frames
                    if due > written:
                        live[i][4] = due
                        for r in reqs:
                            r.frames_ready = due
                    if due < nscan:
                        t_next = t_first + min(nscan, due + self.chunk_frames) / self.fps
                        heapq.heappush(updates, (t_next, seq, 1, i))
                    else:
                        heapq.heappush(updates, (t_done, seq, 2, i))
                    seq += 1
                else:                          # stack complete
                    reqs = live.pop(i)[0]
                    for r in reqs:
                        r.frames_ready = r.nscan
                    if not self.stream_frames:
                        for r in reqs:
                            self.server.submit(r)
                            self.delivered += 1
                continue
            nxt = min([q[0][0] for q in (starts, updates) if q])
            self._wait_until(nxt)


def serve_stats(server, t_first: float) -> dict:
    """Throughput and latency (arrival -> views in host memory) of the
    served requests, with the latency split into queueing (arrival -> copy
    issued), copy-in (-> projection launched) and the rest (-> views back)."""
    done = server.done
    lat = [r.latency_ms for r in done]
    t_last = max((r.t_done for r in done), default=t_first)
    span = max(t_last - t_first, 1e-9)
    ch = sum(r.channels for r in done)
    # a request streamed frame by frame is admitted before its stack is
    # complete: its queueing is then zero and its copy-in runs from arrival
    parts = {"queue": [max(0.0, r.t_admit - r.t_arrival) * 1e3 for r in done],
             "copy_in": [(r.t_launch - max(r.t_admit, r.t_arrival)) * 1e3 for r in done],
             "finish": [(r.t_done - r.t_launch) * 1e3 for r in done]}
    out = {"served": len(done), "rejected": len(server.rejected),
           "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "max_ms": max(lat) if lat else None,
           "stacks_per_s": len(done) / span, "volumes_per_s": ch / span, "span_s": span}
    timed = [r for r in done if r.t_h2d_end > 0.0]
    if timed:   # device clock of the copies: queued behind earlier copies, then copying
        parts["h2d_wait"] = [(r.t_h2d_start - max(r.t_admit, r.t_arrival)) * 1e3 for r in timed]
        parts["h2d_copy"] = [(r.t_h2d_end - r.t_h2d_start) * 1e3 for r in timed]
        parts["h2d_landed_to_launch"] = [(r.t_launch - r.t_h2d_end) * 1e3 for r in timed]
    for k, v in parts.items():
        out[f"{k}_p50_ms"] = percentile(v, 50)
        out[f"{k}_p99_ms"] = percentile(v, 99)
    if getattr(server, "ticks", 0):
        out["ticks"] = server.ticks
        out["host_set_ms_per_tick"] = server.host_set_s * 1e3 / server.ticks
    return out

