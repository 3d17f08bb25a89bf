"""Runs one kernel of the library a few times on a named stack, for a
profiler to capture (``ncu -k regex:<kernel> -c <n> python -m
paper_2211_00645_gb300.profile_case ...``).

  --kernel project   fused z-MIP + y-MIP live view (uint16 in)
  --kernel deskew    full deskewed FP32 volume
  --kernel batch     batched live view over a mix of serving-sized stacks
  --kernel fused     volume + z-MIP + y-MIP in one pass (opm_deskew_mip)
  --kernel sheet     the sheet-frame view with the shear of Eq. 1 (opm_sheet_project)
  --kernel pair      one plane-pair update of the plane-by-plane view (opm_stream_pair)
  --kernel batch1    the named stack alone through the persistent batch kernel
  --kernel adjoint   skew adjoint of an FP32 volume (opm_skew_adjoint)
  --kernel mipbwd    z-MIP backward scatter onto the raw grid (opm_mip_backward)
                     (--kchunk, --ctas: its launch shape)
  --nscan N          override the stack's scan-plane count (smaller captures)

Content: the named configuration's Poisson+blob stack for project/deskew
(``opm_synth.raw_stack``); repeated stack tiles for batch.  Prints one JSON
line with the shapes and the mean event-timed duration of the launches.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=["project", "deskew", "fused", "sheet", "pair", "batch", "batch1", "adjoint", "mipbwd"], required=True)
    ap.add_argument("--kchunk", type=int, default=0)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--config", default="liveview_200x512x2048")
    ap.add_argument("--nscan", type=int, default=0)
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    import opm_synth
    import paper_2211_00645_gb300 as opm
    opm.load()
    s = torch.cuda.current_stream()
    if args.kernel == "batch":
        shapes = opm_synth.serve_shapes(6, seed=11)      # 2.6 GB of raw stacks
        items, keep = [], []
        for (n, r, c, C) in shapes:
            plan = opm.Plan(n, r, c, 35.0, 0.3, 0.1)
            host = opm_synth.tiled_stack((n, r, c * C), seed=11)
            raw = torch.from_numpy(host.view(np.int16)).cuda().view(torch.uint16)
            for ch in range(C):
                items.append({"plan": plan, "raw": raw[:, :, ch * c:], "row_pitch": C * c, "plane_pitch": r * C * c,
                              "zmip": torch.empty((plan.ny, plan.nx), device="cuda"),
                              "ymip": torch.empty((plan.nz, plan.nx), device="cuda")})
            keep.append(raw)
        b = opm.Batch(max_items=len(items), max_units=1 << 22)
        b.set(items, args.kchunk)
        b.upload()
        desc = {"items": len(items), "shapes": shapes, "kchunk": args.kchunk, "ctas": args.ctas, **b.info()}

        def launch():
            b.launch(args.ctas, s)
    else:
        cfg = opm_synth.CONFIGS[args.config]
        if args.nscan:
            cfg = dataclasses.replace(cfg, nscan=args.nscan)
        R = opm_synth.raw_stack(cfg)
        plan = opm.Plan(cfg.nscan, cfg.nrows, cfg.ncols, cfg.theta_deg, cfg.step, cfg.pixel)
        raw = torch.from_numpy(R.view(np.int16)).cuda().view(torch.uint16)
        desc = {"config": cfg.name, "raw": list(cfg.shape), "grid": [plan.nz, plan.ny, plan.nx]}
        if args.kernel == "batch1":
            item = {"plan": plan, "raw": raw, "zmip": torch.empty((plan.ny, plan.nx), device="cuda"),
                    "ymip": torch.empty((plan.nz, plan.nx), device="cuda")}
            b = opm.Batch(max_items=1, max_units=1 << 22)
            b.set([item], args.kchunk)
            b.upload()
            desc.update({"kchunk": args.kchunk, "ctas": args.ctas, **b.info()})

            def launch():
                b.launch(args.ctas, s)
        elif args.kernel in ("adjoint", "mipbwd"):
            g = torch.Generator(device="cuda").manual_seed(1)
            r = torch.empty(plan.raw_shape, device="cuda")
            if args.kernel == "adjoint":
                v = torch.randn(plan.vol_shape, generator=g, device="cuda")

                def launch():
                    opm.opm_skew_adjoint(plan, v, r, s)
            else:
                gz = torch.randn((plan.ny, plan.nx), generator=g, device="cuda")
                argz = torch.randint(0, plan.nz, (plan.ny, plan.nx), generator=g, device="cuda", dtype=torch.int32)

                def launch():
                    opm.opm_mip_backward(plan, gz, argz, r, s)
        elif args.kernel == "pair":
            zmip = torch.zeros((plan.ny, plan.nx), device="cuda")
            ymip = torch.zeros((plan.nz, plan.nx), device="cuda")
            mid = cfg.nscan // 2

            def launch():
                opm.opm_stream_pair(plan, raw[mid], raw[mid + 1], mid, zmip, None, ymip, s)
        elif args.kernel == "sheet":
            import math
            shear = cfg.step * math.cos(math.radians(cfg.theta_deg)) / cfg.pixel
            out = opm.opm_sheet_project(raw, shear)

            def launch():
                opm.opm_sheet_project(raw, shear, out=out, stream=s)
        elif args.kernel == "fused":
            vol = torch.empty(plan.vol_shape, device="cuda")
            zmip = torch.empty((plan.ny, plan.nx), device="cuda")
            ymip = torch.empty((plan.nz, plan.nx), device="cuda")

            def launch():
                opm.opm_deskew_mip(plan, raw, vol, None, zmip, ymip, s)
        elif args.kernel == "project":
            zmip = torch.empty((plan.ny, plan.nx), device="cuda")
            ymip = torch.empty((plan.nz, plan.nx), device="cuda")

            def launch():
                opm.opm_project(plan, raw, zmip, None, ymip, None, s)
        else:
            vol = torch.empty(plan.vol_shape, device="cuda")

            def launch():
                opm.opm_deskew(plan, raw, vol, s)
    for _ in range(args.warmup):
        launch()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.launches + 1)]
    ev[0].record(s)
    for i in range(args.launches):
        launch()
        ev[i + 1].record(s)
    torch.cuda.synchronize()
    us = [ev[i].elapsed_time(ev[i + 1]) * 1e3 for i in range(args.launches)]
    print(json.dumps({"kernel": args.kernel, **desc, "mean_us": round(float(np.mean(us)), 2)}), flush=True)


if __name__ == "__main__":
    main()
