"""Live view of a stack that arrives frame by frame (Fig. 4).

The paper offers two refresh modes: global, where the projection is shown
once per complete stack, and rolling, where it is refreshed after every
camera exposure so that slow acquisitions (long exposures) still give a
responsive view.  ``RollingView`` serves both from two device frame buffers:
each new frame n is copied in and the voxels whose lower plane is n - 1 are
folded into the projections (``opm_stream_pair``); the frame after the last
closes the stack.  In rolling mode every push returns the projections so
far; in global mode only the push that completes a stack does.

A third mode, sliding, keeps the latest frame of every scan position in a
device stack buffer (frame n of the current stack replaces frame n of the
previous one), so the view always spans a full stack: the newest frames
where they exist, the previous stack's elsewhere (zeros before the first
stack completes).  After new frame m the view is the projection of pairs
-1 .. m - 1 (new frames only), pair m (new frame m, old frame m + 1) and
pairs m + 1 .. nscan - 1 (old frames only).  The maximum is associative
and exact, so the view is kept as three parts:
  * R, the running maximum of the new stack's complete pairs;
  * slot p, the previous stack's suffix maximum over its pairs p ..
    nscan - 1 (built in one pass when that stack completed), until the new
    stack's pair p overwrites it with its own partial projection;
  * the mixed pair m, folded into the view directly.
One opm_sliding_push call per frame does it in the library: two pair
passes, one zeroing and two elementwise maxima instead of a whole
re-projection, and the view equals opm_project of the mixed stack bit for
bit.  The completing frame also builds the next suffixes (nscan - 2
maxima).  With a z-sum the mode re-projects the buffer after every frame
instead (sums would change their rounding order).
"""
from __future__ import annotations

from typing import Optional

from . import Plan, opm_sliding_push, opm_stream_begin, opm_stream_pair


class RollingView:
    """Accumulates the z-MIP / y-MIP (and optionally z-sum) of successive
    stacks of ``plan``'s shape, one uint16 frame [nrows][ncols] per push."""

    def __init__(self, plan: Plan, mode: str = "rolling", zsum: bool = False, stream=None):
        import torch
        if mode not in ("rolling", "global", "sliding"):
            raise ValueError("mode must be 'rolling', 'global' or 'sliding'")
        self.torch = torch
        self.plan, self.mode = plan, mode
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        dev = torch.device("cuda", torch.cuda.current_device())
        if mode == "sliding":
            self.stack = torch.zeros(plan.raw_shape, dtype=torch.int16, device=dev).view(torch.uint16)
            self.frames = []
        else:
            self.frames = [torch.empty((plan.nrows, plan.ncols), dtype=torch.uint16, device=dev) for _ in range(2)]
        zn, P = plan.ny * plan.nx, plan.ny * plan.nx + plan.nz * plan.nx
        self.fast_sliding = mode == "sliding" and not zsum
        if self.fast_sliding:
            # opm_sliding_push's buffers, each a z-MIP followed by a y-MIP, all
            # zero at first (the projection of the all-zero stack)
            self.run = torch.zeros(P, dtype=torch.float32, device=dev)
            self.slots = torch.zeros((plan.nscan, P), dtype=torch.float32, device=dev)
            self.view = torch.zeros(P, dtype=torch.float32, device=dev)
            self.zmip = self.view[:zn].view(plan.ny, plan.nx)
            self.ymip = self.view[zn:].view(plan.nz, plan.nx)
        else:
            self.zmip = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=dev)
            self.ymip = torch.empty((plan.nz, plan.nx), dtype=torch.float32, device=dev)
        self.zsum = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=dev) if zsum else None
        self.n = 0            # frames of the current stack received so far
        self.stacks = 0       # completed stacks

    def _outs(self):
        return self.zmip, self.zsum, self.ymip

    def push(self, frame) -> Optional[dict]:
        """Adds the next frame (uint16 [nrows][ncols], host or device).
        Returns {"zmip", "ymip"[, "zsum"], "frames", "complete"} (device
        tensors, valid until the next push) when the mode publishes a view."""
        torch = self.torch
        p = self.plan
        if tuple(frame.shape) != (p.nrows, p.ncols) or frame.dtype != torch.uint16:
            raise ValueError(f"frame must be uint16 {(p.nrows, p.ncols)}")
        if self.mode == "sliding":
            return self._push_sliding(frame)
        cur = self.frames[self.n % 2]
        with torch.cuda.stream(self.stream):
            cur.view(torch.int16).copy_(frame.view(torch.int16), non_blocking=True)
        zmip, zsum, ymip = self._outs()
        if self.n == 0:
            opm_stream_begin(p, zmip, zsum, ymip, self.stream)
            opm_stream_pair(p, None, cur, -1, zmip, zsum, ymip, self.stream)
        else:
            opm_stream_pair(p, self.frames[(self.n - 1) % 2], cur, self.n - 1, zmip, zsum, ymip, self.stream)
        self.n += 1
        complete = self.n == p.nscan
        if complete:
            opm_stream_pair(p, cur, None, p.nscan - 1, zmip, zsum, ymip, self.stream)
            self.n = 0
            self.stacks += 1
        if self.mode == "rolling" or complete:
            out = {"zmip": zmip, "ymip": ymip, "frames": p.nscan if complete else self.n, "complete": complete}
            if zsum is not None:
                out["zsum"] = zsum
            return out
        return None

    def _push_sliding(self, frame) -> dict:
        torch = self.torch
        p = self.plan
        m = self.n
        with torch.cuda.stream(self.stream):
            self.stack[m].view(torch.int16).copy_(frame.view(torch.int16), non_blocking=True)
        if self.fast_sliding:
            opm_sliding_push(p, self.stack, m, self.run, self.slots, self.view, self.stream)
        else:
            from . import opm_project
            opm_project(p, self.stack, self.zmip, self.zsum, self.ymip, None, self.stream)
        self.n += 1
        complete = self.n == p.nscan
        if complete:
            self.n = 0
            self.stacks += 1
        out = {"zmip": self.zmip, "ymip": self.ymip, "frames": p.nscan if complete else self.n,
               "complete": complete, "stacks": self.stacks}
        if self.zsum is not None:
            out["zsum"] = self.zsum
        return out
