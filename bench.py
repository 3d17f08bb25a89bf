"""Benchmark of the OPM deskew library on the live-view stack.

Workload (one step): the fused live view of the 200 scan planes x 512 rows x
2048 columns uint16 stack (theta 35 deg, step 0.3 um, pixel 0.1 um,
Poisson(100) + 2000 blobs): deskew + z-MIP + y-MIP in one opm_project call,
with no volume in memory.  Metric: deskew GB/s of algorithmic bytes (raw read
once + both projections written once), its fraction of the measured HBM copy
bandwidth, and volumes/s.  The separate full FP32 volume run of the same
stack (alone, beside the live view, and as one fused kernel) is reported
under "volume"; the other workloads under their own keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload.  Under torchrun every rank processes its own
stack (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import opm_synth  # noqa: E402

WORKLOAD = "liveview_200x512x2048"
METRIC = "deskew GB/s (fused deskew + z-MIP + y-MIP live view, algorithmic bytes)"
UNIT = "GB/s"

# Sources each timed kernel is compiled from: a change to any of them voids
# the stored ncu traffic figure.
KERNEL_SOURCES = {
    "periodic": ["csrc/opm_project.cu", "csrc/opm_periodic.cuh", "csrc/opm_gen.cuh", "csrc/opm_tma.cuh",
                 "csrc/opm_common.cuh", "csrc/opm_internal.h", "csrc/opm_sched.h", "csrc/opm_plan.cu",
                 "../include/opm.h"],
    "liveview": ["csrc/opm_project.cu", "csrc/opm_tma.cuh", "csrc/opm_common.cuh", "csrc/opm_internal.h",
                 "csrc/opm_sched.h", "csrc/opm_plan.cu", "../include/opm.h"],
    "volume_f32": ["csrc/opm_deskew.cu", "csrc/opm_common.cuh", "csrc/opm_internal.h", "csrc/opm_sched.h",
                   "../include/opm.h"],
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per full-size
# launch from ncu captures, keyed by the hash of the kernel's sources at
# capture time (reported as null once a source has changed).  periodic:
# captured at full size (448.58 MB read, 9.17 MB written, 76.8 M warp
# instructions).  volume_f32:
# captured with 100 scan planes (213.11 MB read, 2963.51 MB written) and
# scaled to 200 planes, reads by the raw bytes (x2.0) and writes by the
# volume bytes (x1.4161).
NCU_TRAFFIC = {
    "periodic": {"src_sha": "0916abe0e7ee", "bytes_per_launch": 457752064, "warp_insts_per_launch": 76816242},
    "volume_f32": {"src_sha": "4eff36766d3d", "bytes_per_launch": 4622836946},
}

L2_BYTES = 129 * 10**6  # L2 of the GB300 (bytes)


def _tree_sha():
    """Hash of every library source and header (identifies the build measured)."""
    h = hashlib.sha1()
    for d in (os.path.join(ROOT, "paper_2211_00645_gb300", "csrc"), os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:12]


def _src_sha(kernel):
    h = hashlib.sha1()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.normpath(os.path.join(ROOT, "paper_2211_00645_gb300", rel)), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


# Derived issue peak: one warp instruction per scheduler per cycle at the
# maximum SM clock (152 SMs x 4 schedulers x 2.07 GHz).
ISSUE_PEAK = 152 * 4 * 2.07e9


def issue_bound(tr, ms_step):
    """The step against the instruction-issue roofline (the fused path may be
    issue-bound): ncu's warp instructions per launch over the derived issue
    peak, as a time floor and a fraction of the measured time."""
    if not tr or "warp_insts_per_launch" not in tr:
        return None
    floor_us = tr["warp_insts_per_launch"] / ISSUE_PEAK * 1e6
    return {"warp_insts_per_launch": tr["warp_insts_per_launch"], "peak_warp_insts_per_s": ISSUE_PEAK,
            "floor_us": round(floor_us, 2), "frac": round(floor_us / (ms_step * 1e3), 4)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(cfg, ny):
    raw = 2 * cfg.nscan * cfg.nrows * cfg.ncols
    live = raw + 4 * ny * cfg.ncols + 4 * cfg.nrows * cfg.ncols       # zmip + ymip
    vol = raw + 4 * cfg.nrows * ny * cfg.ncols                        # FP32 volume
    return live, vol


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            self.f.close()
            os.unlink(self.f.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for nm, val in zip(names, r[5:9]):
                if "Active" in val and "Not" not in val:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def run_reference(args):
    """The FP64 oracle timed on the host cores, per step on a bounded sample."""
    import oracle as O

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    cfg = opm_synth.CONFIGS[WORKLOAD]
    Rfull = opm_synth.raw_stack(cfg)
    # size the per-step sample so that warm-up + timed steps fit the budget
    cal = 16
    gc = O.geometry(cfg.nscan, cfg.nrows, cal, cfg.theta_deg, cfg.step, cfg.pixel)
    Rc = Rfull[:, :, :cal].astype(np.float64)
    t0 = time.perf_counter()
    O.project(Rc, gc)
    t_col = (time.perf_counter() - t0) / cal
    ncol = int(args.ref_budget_s / ((args.steps + args.warmup) * t_col))
    ncol = max(8, min(args.ref_cols, ncol))
    R = Rfull[:, :, :ncol].astype(np.float64)
    g = O.geometry(cfg.nscan, cfg.nrows, ncol, cfg.theta_deg, cfg.step, cfg.pixel)
    sub = opm_synth.StackConfig("r", cfg.nscan, cfg.nrows, ncol, cfg.theta_deg, cfg.step, cfg.pixel,
                                0, (1, 1), (1, 1))
    live, _ = algorithmic_bytes(sub, g.ny)
    for _ in range(args.warmup):
        O.project(R, g)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.project(R, g)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    value = live / t / 1e9
    sample = f"first {ncol} of {cfg.ncols} x-columns of the {WORKLOAD} stack (x-columns are independent)"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(R, cfg, cols, budget_s=20.0):
    import oracle as O
    Rs = R[:, :, :cols].astype(np.float64)
    g = O.geometry(cfg.nscan, cfg.nrows, cols, cfg.theta_deg, cfg.step, cfg.pixel)
    sub = opm_synth.StackConfig("s", cfg.nscan, cfg.nrows, cols, cfg.theta_deg, cfg.step, cfg.pixel,
                                0, (1, 1), (1, 1))
    live, _ = algorithmic_bytes(sub, g.ny)
    t0 = time.perf_counter()
    O.project(Rs, g)
    t = time.perf_counter() - t0
    return {"value": round(live / t / 1e9, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {cols} of {cfg.ncols} x-columns (z-MIP + y-MIP of the oracle's volume, {t:.1f} s)"}


def _oracle_chunk(job):
    """Worker of cpu_baseline_all_cores: the oracle on one block of x-columns."""
    import oracle as O
    R, geo = job
    g = O.geometry(*geo)
    t0 = time.perf_counter()
    O.project(R, g)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(R, cfg, cols=None):
    """The same oracle run on every host core at once: the stack's x-columns
    are independent, so each process takes one block of columns (processes
    started with spawn, after the GPU work)."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    cols = cols or cfg.ncols
    blocks = np.array_split(np.arange(cols), ncores)
    jobs = [(R[:, :, b[0]:b[-1] + 1].astype(np.float64),
             (cfg.nscan, cfg.nrows, len(b), cfg.theta_deg, cfg.step, cfg.pixel)) for b in blocks if len(b)]
    sub = opm_synth.StackConfig("a", cfg.nscan, cfg.nrows, cols, cfg.theta_deg, cfg.step, cfg.pixel,
                                0, (1, 1), (1, 1))
    import oracle as O
    live, _ = algorithmic_bytes(sub, O.geometry(cfg.nscan, cfg.nrows, cols, cfg.theta_deg, cfg.step,
                                                cfg.pixel).ny)
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        pool.map(_oracle_chunk, [(j[0][:, :, :1], j[1][:2] + (1,) + j[1][3:]) for j in jobs])  # start-up
        t0 = time.perf_counter()
        pool.map(_oracle_chunk, jobs)
        t = time.perf_counter() - t0
    return {"value": round(live / t / 1e9, 4), "unit": UNIT, "cores": len(jobs), "kind": "oracle",
            "sample": f"first {cols} of {cfg.ncols} x-columns in {len(jobs)} processes ({t:.1f} s)"}


def tune_serving(torch, plans, ring):
    """Launch shape of the batched server, tuned on six stacks of the serving
    mix (one tick's worth) copied to the device."""
    from paper_2211_00645_gb300.tune import Tuner
    items, keep = [], []
    for (n, r, c, C) in opm_synth.serve_shapes(6, seed=11):
        plan = plans.get(n, r, c)
        off = ring.acquire(2 * n * r * c * C)
        raw = ring.view(off, (n, r, c * C)).view(torch.int16).cuda().view(torch.uint16)
        ring.release(off)
        keep.append(raw)
        for ch in range(C):
            items.append({"plan": plan, "raw": raw[:, :, ch * c:], "row_pitch": C * c, "plane_pitch": r * C * c,
                          "zmip": torch.empty((plan.ny, plan.nx), device="cuda"),
                          "ymip": torch.empty((plan.nz, plan.nx), device="cuda")})
    e = Tuner().tune(items, reps=3)
    del items, keep
    torch.cuda.empty_cache()
    return e


def batch_bench(torch, opm, fixed=None):
    """One tick of the batched server on device-resident inputs: the six
    stacks of the serving mix (seeded shapes; uniform random uint16 made on
    the device), each channel an item of one batch, z-MIP + y-MIP.  The
    autotuner times every kernel shape x kchunk x CTAs-per-SM candidate and
    keeps the fastest; ``fixed`` = (shape name, kchunk, ctas) times that
    configuration alone instead (profiler captures)."""
    from paper_2211_00645_gb300.tune import SHAPE_IDS, Tuner
    plans = {}
    items, keep = [], []
    g = torch.Generator(device="cuda").manual_seed(11)
    for (n, r, c, C) in opm_synth.serve_shapes(6, seed=11):
        plan = plans.setdefault((n, r, c), opm.Plan(n, r, c, 35.0, 0.3, 0.1))
        raw = torch.randint(0, 4096, (n, r, c * C), generator=g, device="cuda", dtype=torch.int32)
        raw = raw.to(torch.int16).view(torch.uint16)
        keep.append(raw)
        for ch in range(C):
            items.append({"plan": plan, "raw": raw[:, :, ch * c:], "row_pitch": C * c, "plane_pitch": r * C * c,
                          "zmip": torch.empty((plan.ny, plan.nx), device="cuda"),
                          "ymip": torch.empty((plan.nz, plan.nx), device="cuda")})
    raw_b = sum(2 * k.numel() for k in keep)
    out = {"workload": "serving mix: 6 stacks, 2 channels each (theta 35, step 0.3, pixel 0.1), "
                       "z-MIP + y-MIP per channel, one batch", "items": len(items), "raw_bytes": raw_b}
    def time_config(shape_id, kchunk, ctas):
        b = opm.Batch(max_items=len(items), max_units=1 << 24)
        b.set(items, kchunk, shape_id)
        b.upload()
        s = torch.cuda.current_stream()
        for _ in range(3):
            b.launch(ctas, s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(10):
            b.launch(ctas, s)
        e1.record(s)
        e1.synchronize()
        b.check()
        info = b.info()
        return round(e0.elapsed_time(e1) * 100, 2), info

    if fixed:
        shape, kchunk, ctas = fixed
        us, _ = time_config(SHAPE_IDS[shape], kchunk, ctas)
        out["fixed"] = {"shape": shape, "kchunk": kchunk, "ctas_per_sm": ctas, "us": us}
    else:
        # what a caller gets without the tuner: shape, kchunk and CTAs left at 0
        us, info = time_config(opm.OPM_SHAPE_AUTO, 0, 0)
        out["default"] = {"shape": opm.SHAPE_NAMES[info["shape"]], "units": info["units"], "us": us}
        e = Tuner().tune(items, reps=5, warmup=2)
        out["tuned"] = {k: e[k] for k in ("shape", "kchunk", "ctas_per_sm", "us")}
        out["candidates_us"] = e["candidates"]
        out["tuned"]["GBps_raw"] = round(raw_b / (e["us"] * 1e-6) / 1e9, 1)
    del items, keep
    torch.cuda.empty_cache()
    return out


def xshard_bench(torch, opm, cfg, raw, stream, t_whole):
    """The x-column partition of one stack (dist.xshard), measured on one GPU:
    the live view of one rank's columns for 2, 4 and 8 ranks, against the
    whole stack's step.  Each rank would run its part on its own GPU with no
    exchange, so whole / (N x part) is the partition's efficiency before the
    gather for display."""
    from paper_2211_00645_gb300 import dist as pdist
    out = {"what": "live view of rank 0's columns (contiguous copy), timed alone; no collective",
           "whole_us": round(t_whole * 1e6, 2)}
    for n in (2, 4, 8):
        x0, x1 = pdist.xshard(cfg.ncols, 0, n)
        part = raw[:, :, x0:x1].contiguous()
        # copies enough that the rotation exceeds twice L2: every launch reads from HBM
        ncopy = max(2, -(-2 * int(L2_BYTES) // (part.numel() * 2)))
        parts = [part] + [part.clone() for _ in range(ncopy - 1)]
        plan = opm.Plan(cfg.nscan, cfg.nrows, x1 - x0, cfg.theta_deg, cfg.step, cfg.pixel)
        z = torch.empty((plan.ny, plan.nx), device="cuda")
        y = torch.empty((plan.nz, plan.nx), device="cuda")
        for i in range(3):
            opm.opm_project(plan, parts[i % ncopy], z, None, y, None, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10 * ncopy
        e0.record(stream)
        for i in range(reps):
            opm.opm_project(plan, parts[i % ncopy], z, None, y, None, stream)
        e1.record(stream)
        e1.synchronize()
        opm.opm_plan_check(plan)
        t = e0.elapsed_time(e1) / reps * 1e-3
        out[f"ranks_{n}"] = {"columns": x1 - x0, "unit_rows": opm.opm_plan_schedule(plan)[2],
                             "part_us": round(t * 1e6, 2), "copies": ncopy,
                             "efficiency": round(t_whole / (n * t), 3)}
        del part, parts, z, y
    torch.cuda.empty_cache()
    return out


def adjoint_bench(torch, opm, peak, shape=None):
    """Forward deskew, skew adjoint and z-MIP backward (FP32) on the
    differentiable workload 128 x 256 x 256 (theta 30, step 0.4, pixel
    0.115; ``shape`` = (nscan, nrows, ncols) replaces its size), each launch
    timed alone with CUDA events after a write of twice the L2 size, against
    its algorithmic bytes."""
    c = opm_synth.CONFIGS["diff_128x256x256"]
    n, rows, cols = shape or (c.nscan, c.nrows, c.ncols)
    p = opm.Plan(n, rows, cols, c.theta_deg, c.step, c.pixel)
    s = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(p.raw_shape, generator=g, device="cuda")
    v = torch.empty(p.vol_shape, device="cuda")
    r = torch.empty(p.raw_shape, device="cuda")
    gz = torch.randn((p.ny, p.nx), generator=g, device="cuda")
    argz = torch.randint(0, p.nz, (p.ny, p.nx), generator=g, device="cuda", dtype=torch.int32)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    raw_b, vol_b = 4 * x.numel(), 4 * v.numel()
    calls = {
        "forward_f32": (lambda: opm.opm_deskew(p, x, v, s), raw_b + vol_b),
        "skew_adjoint_f32": (lambda: opm.opm_skew_adjoint(p, v, r, s), vol_b + raw_b),
        "mip_backward": (lambda: opm.opm_mip_backward(p, gz, argz, r, s), 8 * gz.numel() + raw_b),
    }
    out = {"workload": f"diff_{n}x{rows}x{cols}", "grid": [p.nz, p.ny, p.nx],
           "timing": "each launch alone, after writing 2 x L2 bytes"}
    reps = 20
    for name, (fn, nbytes) in calls.items():
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in ev:
            flush.fill_(1)
            e0.record(s)
            fn()
            e1.record(s)
        torch.cuda.synchronize()
        t = sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps * 1e-3
        out[name] = {"bytes": nbytes, "us": round(t * 1e6, 2), "GBps": round(nbytes / t / 1e9, 1),
                     "frac": round(nbytes / t / 1e9 / peak, 4)}
    return out


def large_bench(torch, opm, peak):
    """The large-volume workload 1000 x 1024 x 2048 uint16 (theta 45, step
    0.2, pixel 0.115): the FP32 volume, the round-to-nearest uint16 volume and
    the z-MIP written in one pass (opm_deskew_mip), timed with CUDA events
    against raw + both volumes + z-MIP bytes."""
    c = opm_synth.CONFIGS["large_1000x1024x2048"]
    p = opm.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    s = torch.cuda.current_stream()
    host = opm_synth.tiled_stack((c.nscan, c.nrows, c.ncols), seed=c.seed)
    raw = torch.from_numpy(host.view(np.int16)).cuda().view(torch.uint16)
    del host
    vol = torch.empty(p.vol_shape, device="cuda")
    vol16 = torch.empty(p.vol_shape, dtype=torch.int16, device="cuda").view(torch.uint16)
    zmip = torch.empty((p.ny, p.nx), device="cuda")
    nbytes = 2 * raw.numel() + 6 * vol.numel() + 4 * zmip.numel()
    os.environ["OPM_ONE_PASS_FUSED"] = "1"
    try:
        p_fused = opm.Plan(c.nscan, c.nrows, c.ncols, c.theta_deg, c.step, c.pixel)
    finally:
        os.environ.pop("OPM_ONE_PASS_FUSED", None)

    def timed(plan, n=10):
        for _ in range(3):
            opm.opm_deskew_mip(plan, raw, vol, vol16, zmip, None, s)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(n):
            opm.opm_deskew_mip(plan, raw, vol, vol16, zmip, None, s)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n * 1e-3

    t = timed(p)
    t_fused = timed(p_fused)
    del p_fused
    out = {"workload": "large_1000x1024x2048", "grid": [p.nz, p.ny, p.nx],
           "call": "opm_deskew_mip (FP32 volume + uint16 volume + z-MIP in one call)", "bytes": nbytes,
           "us": round(t * 1e6, 1), "GBps": round(nbytes / t / 1e9, 1), "frac": round(nbytes / t / 1e9 / peak, 4),
           "volumes_per_s": round(1.0 / t, 2),
           "fused_kernel_us": round(t_fused * 1e6, 1), "fused_kernel_frac": round(nbytes / t_fused / 1e9 / peak, 4)}
    del raw, vol, vol16, zmip
    torch.cuda.empty_cache()
    return out


def rolling_bench(torch, opm, plan, host_raw, raw):
    """Frame-by-frame live view of the live-view stack (Fig. 4 rolling and
    global modes): every frame is copied in from pinned host memory and its
    plane pair folded into the projections.  Reported: the device time per
    frame, the latency from the last frame's copy to a complete view, and
    the same latency for the whole-stack path (copy the stack, then one fused
    projection)."""
    s = torch.cuda.current_stream()
    frames = [torch.empty((plan.nrows, plan.ncols), dtype=torch.uint16, device="cuda") for _ in range(2)]
    z = torch.empty((plan.ny, plan.nx), device="cuda")
    y = torch.empty((plan.nz, plan.nx), device="cuda")

    def one_stack(ev=None):
        opm.opm_stream_begin(plan, z, None, y, s)
        for n in range(plan.nscan):
            cur = frames[n % 2]
            if ev is not None and n == plan.nscan - 1:
                ev[0].record(s)
            cur.view(torch.int16).copy_(host_raw[n], non_blocking=True)
            opm.opm_stream_pair(plan, frames[(n - 1) % 2] if n else None, cur, n - 1, z, None, y, s)
        opm.opm_stream_pair(plan, frames[(plan.nscan - 1) % 2], None, plan.nscan - 1, z, None, y, s)
        if ev is not None:
            ev[1].record(s)

    for _ in range(2):
        one_stack()
    torch.cuda.synchronize()
    reps = 5
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for r in range(reps):
        one_stack(ev[r])
    t1.record(s)
    torch.cuda.synchronize()
    stack_ms = t0.elapsed_time(t1) / reps
    last_us = statistics.median(e[0].elapsed_time(e[1]) for e in ev) * 1e3
    # kernels alone, frames resident
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(s)
    for n in range(-1, plan.nscan):
        opm.opm_stream_pair(plan, raw[n] if n >= 0 else None, raw[n + 1] if n + 1 < plan.nscan else None, n, z,
                            None, y, s)
    k1.record(s)
    torch.cuda.synchronize()
    pair_us = k0.elapsed_time(k1) * 1e3 / (plan.nscan + 1)
    # whole-stack path: copy the stack in, then the fused projection
    w0 = torch.cuda.Event(enable_timing=True)
    w1 = torch.cuda.Event(enable_timing=True)
    wz = torch.empty_like(z)
    wy = torch.empty_like(y)
    w0.record(s)
    for _ in range(reps):
        raw.view(torch.int16).copy_(host_raw, non_blocking=True)
        opm.opm_project(plan, raw, wz, None, wy, None, s)
    w1.record(s)
    torch.cuda.synchronize()
    assert torch.equal(z, wz) and torch.equal(y, wy)
    whole_ms = w0.elapsed_time(w1) / reps
    # sliding view (a full stack of the newest frames after every frame): one
    # stack of pushes through RollingView, copy in included, after a first
    # stack; against copying the frame and re-projecting the stack buffer
    from paper_2211_00645_gb300.rolling import RollingView
    sv = RollingView(plan, mode="sliding", stream=s)
    hframes = host_raw.view(torch.uint16)  # pinned, the uint16 bits
    for n in range(plan.nscan):
        sv.push(hframes[n])
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(s)
    for n in range(plan.nscan):
        sv.push(hframes[n])
    q1.record(s)
    torch.cuda.synchronize()
    slide_us = q0.elapsed_time(q1) * 1e3 / plan.nscan
    assert torch.equal(sv.zmip, wz) and torch.equal(sv.ymip, wy)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(s)
    for n in range(plan.nscan):
        raw[n].view(torch.int16).copy_(host_raw[n], non_blocking=True)
        opm.opm_project(plan, raw, wz, None, wy, None, s)
    r1.record(s)
    torch.cuda.synchronize()
    reproj_us = r0.elapsed_time(r1) * 1e3 / plan.nscan
    del sv
    return {"frames": plan.nscan, "frame_bytes": plan.nrows * plan.ncols * 2,
            "per_frame_us": round(stack_ms * 1e3 / plan.nscan, 2), "pair_kernel_us": round(pair_us, 2),
            "max_camera_fps": round(plan.nscan / (stack_ms * 1e-3)),
            "last_frame_to_view_us": round(last_us, 1), "whole_stack_copy_then_project_ms": round(whole_ms, 3),
            "identical_to_whole_stack": True,
            "sliding": {"per_frame_us": round(slide_us, 2), "max_camera_fps": round(1e6 / slide_us),
                        "reproject_per_frame_us": round(reproj_us, 2),
                        "what": "full-stack view after every frame: running max + previous stack's suffix "
                                "maxima + the mixed pair, against copy + opm_project of the stack buffer"}}


def serve_bench(args, torch):
    """Serving comparison on the batched-serving workload: the live-view
    server against the plain per-stack path, first at Poisson arrivals of
    ``serve_rate`` stacks/s, then with every stack arriving at once."""
    from paper_2211_00645_gb300.serve import Camera, LiveViewServer, PinnedRing, PlainServer, PlanCache, \
        serve_stats
    from paper_2211_00645_gb300.tune import SHAPE_IDS
    shapes = opm_synth.serve_shapes(256, seed=11)
    plans = PlanCache(35.0, 0.3, 0.1)
    for (n, r, c, _) in set(shapes):
        plans.get(n, r, c)
    ring = PinnedRing(args.serve_ring_gb << 30, seed=11)
    budget = args.serve_budget_gb << 30
    tuned = tune_serving(torch, plans, ring)

    def link_gbs():
        """Pinned host -> device copy rate (the serving bound): the best of
        three timings (CUDA events) of three 2 GB copies each."""
        n = min(ring.nbytes, 2 << 30)
        dst = torch.empty(n, dtype=torch.uint8, device="cuda")
        s = torch.cuda.current_stream()
        dst.copy_(ring.buf[:n])
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(3):
                dst.copy_(ring.buf[:n], non_blocking=True)
            e1.record(s)
            e1.synchronize()
            best = max(best, 3 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        del dst
        return round(best, 1)

    link0 = link_gbs()
    out = {"workload": "serving: ROIs rows {256,512,1024} x cols {512,1024,2048}, planes 50..400, 2 channels, "
                       "theta 35, step 0.3, pixel 0.1; z-MIP + y-MIP per channel",
           "budget_bytes": budget, "ring_bytes": ring.nbytes,
           "camera": f"paced: each stack acquired frame by frame at {args.serve_fps:g} frames/s, complete at its "
                     "Poisson time; the batched server copies frames as they are written, the plain server "
                     "copies the complete stack; saturated: every stack complete at once",
           "latency": "stack complete (last frame written) -> both views of every channel in host memory"}
    phases = [("paced", args.serve_rate, args.serve_paced), ("saturated", None, args.serve_saturated)]

    def one(make, rate, n, seed, fps=None, stream=False):
        srv = make()
        cam = Camera(srv, ring, shapes, n, rate, seed=seed, fps=fps, stream_frames=stream)
        cam.start()
        srv.run(cam.expected(), timeout_s=600)
        cam.join(timeout=60)
        if cam.error is not None:
            raise cam.error
        torch.cuda.synchronize()
        st = serve_stats(srv, cam.t0)
        if isinstance(srv, LiveViewServer):
            st["mean_batch"] = round(float(np.mean(srv.batch_sizes)), 2)
            st["peak_device_bytes"] = srv.peak_in_use
        st["ring_stalls"] = ring.stalls
        return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}

    out["tuned"] = tuned
    mean_raw = sum(2 * n * r * c * C for (n, r, c, C) in shapes) / len(shapes)
    makers = {"batched": lambda: LiveViewServer(plans, budget, keep_results=False, kchunk=tuned["kchunk"],
                                                ctas_per_sm=tuned["ctas_per_sm"],
                                                shape=SHAPE_IDS[tuned["shape"]]),
              "plain": lambda: PlainServer(plans, keep_results=False)}
    for name, make in makers.items():
        one(make, None, 16, seed=1)                                   # warm-up: allocators, plans
        for phase, rate, n in phases:
            if n > 0:
                ring.stalls = 0
                fps = args.serve_fps if rate else None
                out.setdefault(phase, {"rate_per_s": rate, "stacks": n})[name] = one(
                    make, rate, n, seed=2, fps=fps, stream=(name == "batched" and fps is not None))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    link1 = link_gbs()
    out["h2d_link_gbs"] = {"before": link0, "after": link1}
    out["mean_raw_bytes"] = round(mean_raw)
    # the link's capacity: the better of the two measurements on an idle device
    out["link_bound_stacks_per_s"] = round(max(link0, link1) * 1e9 / mean_raw, 1)
    return out


def one_pass(torch, opm, cfg, raw, vol, zmip, ymip, stream, vol_b, live_b, peak):
    """The FP32 volume and the live view from the single fused kernel (raw
    read once): a plan made with OPM_ONE_PASS_FUSED=1."""
    os.environ["OPM_ONE_PASS_FUSED"] = "1"
    try:
        plan_f = opm.Plan(cfg.nscan, cfg.nrows, cfg.ncols, cfg.theta_deg, cfg.step, cfg.pixel)
    finally:
        os.environ.pop("OPM_ONE_PASS_FUSED", None)
    for _ in range(3):
        opm.opm_deskew_mip(plan_f, raw, vol, None, zmip, ymip, stream)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(20):
        opm.opm_deskew_mip(plan_f, raw, vol, None, zmip, ymip, stream)
    f1.record(stream)
    torch.cuda.synchronize()
    t_one = f0.elapsed_time(f1) / 20 * 1e-3
    del plan_f
    one_b = vol_b + live_b - 2 * cfg.nscan * cfg.nrows * cfg.ncols
    return {"call": "opm_deskew_mip, single fused kernel (plan made with OPM_ONE_PASS_FUSED=1)",
            "bytes": one_b, "us": round(t_one * 1e6, 2), "GBps": round(one_b / t_one / 1e9, 1),
            "frac": round(one_b / t_one / 1e9 / peak, 4)}


def sheet_bench(torch, opm, cfg, raw, stream, peak):
    """The paper's own sheet-frame view (the shear of Eq. 1) of the stack."""
    import math as _m
    shear = cfg.step * _m.cos(_m.radians(cfg.theta_deg)) / cfg.pixel
    sheet = opm.opm_sheet_project(raw, shear, stream=stream)
    for _ in range(3):
        opm.opm_sheet_project(raw, shear, out=sheet, stream=stream)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(20):
        opm.opm_sheet_project(raw, shear, out=sheet, stream=stream)
    s1.record(stream)
    torch.cuda.synchronize()
    opm.opm_sheet_check()
    t_sheet = s0.elapsed_time(s1) / 20 * 1e-3
    sheet_b = 2 * cfg.nscan * cfg.nrows * cfg.ncols + 4 * sheet.numel()
    out = {"call": "opm_sheet_project", "shear_rows_per_frame": round(shear, 6),
           "out": list(sheet.shape), "bytes": sheet_b, "us": round(t_sheet * 1e6, 2),
           "GBps": round(sheet_b / t_sheet / 1e9, 1), "frac": round(sheet_b / t_sheet / 1e9 / peak, 4)}
    del sheet
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="opm", choices=["opm", "reference"])
    ap.add_argument("--ref-cols", type=int, default=256)
    ap.add_argument("--ref-budget-s", type=float, default=150.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 1000 x 1024 x 2048 one-pass volume")
    ap.add_argument("--serve-paced", type=int, default=200, help="stacks at Poisson arrivals (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-saturated", type=int, default=1800, help="stacks arriving at once (0: skip)")
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--serve-ring-gb", type=int, default=16,
                    help="pinned host ring of the camera (8 GB stalls acquisitions at 20 stacks/s)")
    ap.add_argument("--serve-fps", type=float, default=2000.0, help="camera frame rate of the paced phase")
    ap.add_argument("--nscan", type=int, default=0,
                    help="scan planes of the live-view stack (0: the workload's 200; smaller for profiler captures)")
    ap.add_argument("--diff-shape", default="",
                    help="nscan,nrows,ncols of the differentiable section (default 128,256,256)")
    ap.add_argument("--only", default="all",
                    help="comma list of the sections run after the live-view step: volume, sheet, "
                         "differentiable, rolling, xshard, large, batch, serving, cpu (or all, none)")
    ap.add_argument("--batch-config", default="",
                    help="shape,kchunk,ctas (e.g. per_j32x2,256,4): time that batch configuration instead of tuning")
    args = ap.parse_args()
    sections = {"volume", "sheet", "differentiable", "rolling", "xshard", "large", "batch", "serving", "cpu"}
    only = sections if args.only == "all" else set() if args.only == "none" else set(args.only.split(","))
    if only - sections:
        ap.error(f"unknown sections {sorted(only - sections)}")
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2211_00645_gb300 as opm
    from paper_2211_00645_gb300 import build as opm_build
    from paper_2211_00645_gb300 import dist as pdist

    ws, rank, local = pdist.env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    opm_build.build()
    opm.load()

    cfg = opm_synth.CONFIGS[WORKLOAD]
    if args.nscan:
        import dataclasses
        cfg = dataclasses.replace(cfg, nscan=args.nscan)
    R = opm_synth.raw_stack(cfg)
    plan = opm.Plan(cfg.nscan, cfg.nrows, cfg.ncols, cfg.theta_deg, cfg.step, cfg.pixel)
    live_b, vol_b = algorithmic_bytes(cfg, plan.ny)

    host_raw = torch.from_numpy(R.view(np.int16)).pin_memory()            # uint16 bits
    raw = torch.empty(plan.raw_shape, dtype=torch.uint16, device=dev)
    raw.view(torch.int16).copy_(host_raw)
    zmip = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=dev)
    ymip = torch.empty((plan.nz, plan.nx), dtype=torch.float32, device=dev)
    vol = None  # the FP32 volume: allocated for the volume section, after serving (the step never writes one)
    host_z = torch.empty((plan.ny, plan.nx), dtype=torch.float32).pin_memory()
    host_y = torch.empty((plan.nz, plan.nx), dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream()

    def step():
        # the live view: deskew + z-MIP + y-MIP in one call, no volume in memory
        opm.opm_project(plan, raw, zmip, None, ymip, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    opm.opm_plan_check(plan)

    # ---- device-resident timing of the step (CUDA events on the launching stream)
    K = args.steps
    sampler = ClockSampler(torch.cuda.current_device())
    if rank == 0:
        sampler.start()
    pdist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(K):
        step()
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if rank == 0 else None
    total_ms = t_start.elapsed_time(t_end)
    ms_step = pdist.max_over_ranks(total_ms / K, device=dev)
    opm.opm_plan_check(plan)

    opm.opm_plan_check(plan)

    # ---- end to end through the C ABI: every step copies its stack in from
    # pinned host memory and both projections back out (the bytes of the
    # metric are the live view's: raw in, z-MIP and y-MIP out).  Two device stack
    # buffers: the copy of step i + 1 (copy stream) overlaps the compute of
    # step i (compute stream).
    E = max(10, K // 10)
    raws = [raw, torch.empty_like(raw)]
    copy_s = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def step_on(r):
        opm.opm_project(plan, r, zmip, None, ymip, None, stream)

    # two untimed pipelined steps first: the copy stream's first use
    for b in range(2):
        with torch.cuda.stream(copy_s):
            raws[b].view(torch.int16).copy_(host_raw, non_blocking=True)
        copied[b].record(copy_s)
        stream.wait_event(copied[b])
        step_on(raws[b])
        host_z.copy_(zmip, non_blocking=True)
        host_y.copy_(ymip, non_blocking=True)
    torch.cuda.synchronize()
    pdist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_s.wait_event(e0)
    for i in range(E):
        b = i % 2
        if i >= 2:
            copy_s.wait_event(freed[b])           # step i - 2 is done with this buffer
        with torch.cuda.stream(copy_s):
            raws[b].view(torch.int16).copy_(host_raw, non_blocking=True)
        copied[b].record(copy_s)
        stream.wait_event(copied[b])
        step_on(raws[b])
        freed[b].record(stream)
        host_z.copy_(zmip, non_blocking=True)
        host_y.copy_(ymip, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = pdist.max_over_ranks(e0.elapsed_time(e1) / E, device=dev)
    del raws

    if rank != 0:
        dist.destroy_process_group()
        return

    peak, peak_src = peaks()
    value = ws * live_b / (ms_step * 1e-3) / 1e9
    path = opm.opm_plan_path(plan)
    kname = {opm.OPM_PATH_PERIODIC: "periodic", opm.OPM_PATH_FAST: "liveview"}.get(path[0], "liveview_general")
    tr = NCU_TRAFFIC.get(kname)
    full_size = args.nscan in (0, 200)  # the captured traffic is that of the full 200-plane launch
    traffic = tr["bytes_per_launch"] if tr and tr["src_sha"] == _src_sha(kname) and full_size else None
    ach = live_b / (ms_step * 1e-3) / 1e9
    pair_b = live_b + vol_b
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16->f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.nscan else f"{WORKLOAD} with {cfg.nscan} scan planes",
                   "raw": [cfg.nscan, cfg.nrows, cfg.ncols], "theta_deg": cfg.theta_deg,
                   "step_um": cfg.step, "pixel_um": cfg.pixel, "grid": [plan.nz, plan.ny, plan.nx],
                   "step": "fused deskew + z-MIP + y-MIP live view, one opm_project call, no volume in memory",
                   "kernel_path": {"path": kname, "pixel_over_step": f"{path[1]}/{path[2]}" if path[1] else None,
                                   "unit_rows": opm.opm_plan_schedule(plan)[2]},
                   "l2": "input larger than L2 (raw 419 MB)",
                   "parallelism": f"{ws} independent stacks" if ws > 1 else "1 GPU"},
        "volumes_per_s": round(ws / (ms_step * 1e-3), 2),
        "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4), "traffic": traffic,
                     "kernel": f"k_project_{'per' if kname == 'periodic' else 'fast'} + k_init_outputs "
                               "(one opm_project call, timed together)",
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "issue": issue_bound(tr if traffic is not None else None, ms_step)},
        "e2e": {"value": round(ws * live_b / (e2e_ms * 1e-3) / 1e9, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(host_raw.numel() * 2),
                "d2h_bytes_per_step": int((host_z.numel() + host_y.numel()) * 4),
                "ms_per_step": round(e2e_ms, 4)},
        "gpu_launches": 2 * K,
        "host": {"cores": os.cpu_count(), "library_sources_sha": _tree_sha()},
        "clocks": clocks,
    }
    # Serving runs first among the sections, right after the step: its host
    # threads and copies were slowed by what ran before it in the process
    # (sections that allocate and free GB of device buffers), while serving
    # alone after the step measured cleanly.  The stack stays where the step
    # allocated it for the sections after serving.
    if "serving" in only:
        torch.cuda.empty_cache()
        line["serving"] = serve_bench(args, torch)
    # ---- the separate full FP32 volume run of the same stack: the volume alone,
    # and volume + live view from one opm_deskew_mip call (side by side)
    if "volume" in only:
        vol = torch.empty(plan.vol_shape, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            opm.opm_deskew(plan, raw, vol, stream)
            opm.opm_deskew_mip(plan, raw, vol, None, zmip, ymip, stream)
        KV = max(20, K // 8)
        v0, v1, v2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        v0.record(stream)
        for _ in range(KV):
            opm.opm_deskew(plan, raw, vol, stream)
        v1.record(stream)
        for _ in range(KV):
            opm.opm_deskew_mip(plan, raw, vol, None, zmip, ymip, stream)
        v2.record(stream)
        torch.cuda.synchronize()
        t_vol = v0.elapsed_time(v1) / KV * 1e-3
        t_pair = v1.elapsed_time(v2) / KV * 1e-3
        opm.opm_plan_check(plan)
    vtr = NCU_TRAFFIC.get("volume_f32")
    if vol is not None:
        line["volume"] = {
            "what": "the separate full FP32 volume run of the same stack (512 x 1021 x 2048)",
            "deskew_f32": {"bytes": vol_b, "us": round(t_vol * 1e6, 2), "GBps": round(vol_b / t_vol / 1e9, 1),
                           "frac": round(vol_b / t_vol / 1e9 / peak, 4), "volumes_per_s": round(1.0 / t_vol, 1),
                           "traffic": (vtr["bytes_per_launch"] if vtr and vtr["src_sha"] == _src_sha("volume_f32")
                                       and full_size else None)},
            "deskew_mip_side_by_side": {"call": "opm_deskew_mip (volume + live view, the two kernels side by side)",
                                        "bytes": pair_b, "us": round(t_pair * 1e6, 2),
                                        "GBps": round(pair_b / t_pair / 1e9, 1),
                                        "frac": round(pair_b / t_pair / 1e9 / peak, 4)},
            "one_pass_fused": one_pass(torch, opm, cfg, raw, vol, zmip, ymip, stream, vol_b, live_b, peak),
        }
        vol = None
        torch.cuda.empty_cache()
    if "sheet" in only:
        line["sheet_view"] = sheet_bench(torch, opm, cfg, raw, stream, peak)
    if "differentiable" in only:
        dshape = tuple(int(v) for v in args.diff_shape.split(",")) if args.diff_shape else None
        line["differentiable"] = adjoint_bench(torch, opm, peak, dshape)
    if "rolling" in only:
        line["rolling"] = rolling_bench(torch, opm, plan, host_raw, raw)
    if "large" in only and not args.no_large:
        line["large_volume"] = large_bench(torch, opm, peak)
    if "batch" in only:
        bc = args.batch_config.split(",") if args.batch_config else None
        line["batch"] = batch_bench(torch, opm, (bc[0], int(bc[1]), int(bc[2])) if bc else None)
    if "xshard" in only:
        line["xshard"] = xshard_bench(torch, opm, cfg, raw, stream, ms_step * 1e-3)
    if "cpu" in only and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(R, cfg, args.ref_cols)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(R, cfg)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
