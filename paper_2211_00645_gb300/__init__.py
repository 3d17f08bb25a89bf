"""Python binding of libopm.so, the sm_103a OPM deskew library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/opm.h``.  PyTorch provides
device memory and streams.  The functions ``opm_*`` mirror the C entry points
one to one (tensors in place of pointers, the current torch stream by
default); ``deskew``/``project``/``skew_adjoint``/``mip_backward`` allocate
their outputs with torch and call them.

There is no CPU fallback: if the library has not been built, or no CUDA device
is present, these functions raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libopm.so")

OPM_OK, OPM_ERR_INVALID_ARG, OPM_ERR_UNSUPPORTED, OPM_ERR_CUDA, OPM_ERR_OUT_OF_MEMORY, OPM_ERR_INTERNAL = range(6)
OPM_INTERP_LINEAR, OPM_INTERP_NEAREST = 0, 1
OPM_U16, OPM_F32, OPM_F64 = 0, 1, 2

_STATUS = {
    OPM_ERR_INVALID_ARG: "OPM_ERR_INVALID_ARG",
    OPM_ERR_UNSUPPORTED: "OPM_ERR_UNSUPPORTED",
    OPM_ERR_CUDA: "OPM_ERR_CUDA",
    OPM_ERR_OUT_OF_MEMORY: "OPM_ERR_OUT_OF_MEMORY",
    OPM_ERR_INTERNAL: "OPM_ERR_INTERNAL",
}

class opm_batch_item(ctypes.Structure):
    """Mirror of the C struct opm_batch_item."""
    _fields_ = [("plan", ctypes.c_void_p), ("raw", ctypes.c_void_p), ("row_pitch", ctypes.c_int64),
                ("plane_pitch", ctypes.c_int64), ("zmip", ctypes.c_void_p), ("ymip", ctypes.c_void_p),
                ("zsum", ctypes.c_void_p), ("argz", ctypes.c_void_p)]


# Every symbol the header declares, with its ctypes signature.
_SIGS = {
    "opm_plan_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "opm_plan_shape": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 4),
    "opm_plan_path": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 3),
    "opm_plan_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "opm_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "opm_deskew": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_void_p]),
    "opm_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5),
    "opm_sheet_rows": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int64)]),
    "opm_sheet_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "opm_sheet_check": (ctypes.c_int, []),
    "opm_max_combine": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_void_p]),
    "opm_sliding_push": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 4),
    "opm_warp_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "opm_deskew_mip": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5),
    "opm_stream_begin": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "opm_stream_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "opm_deskew_dual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "opm_skew_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p]),
    "opm_mip_backward": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "opm_plan_check": (ctypes.c_int, [ctypes.c_void_p]),
    "opm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)]),
    "opm_batch_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "opm_batch_upload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "opm_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "opm_batch_launch_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "opm_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "opm_batch_check": (ctypes.c_int, [ctypes.c_void_p]),
    "opm_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "opm_batch_project_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_void_p]),
    "opm_last_error": (ctypes.c_char_p, []),
    "opm_version": (ctypes.c_int, []),
}

_lib: Optional[ctypes.CDLL] = None


class OpmError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libopm.so (built by ``paper_2211_00645_gb300.build``) once."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, func: str):
    if status != OPM_OK:
        raise OpmError(status, func, load().opm_last_error().decode(errors="replace"))


class Plan:
    """Owns an ``opm_plan*``; destroyed with the object."""

    def __init__(self, nscan, nrows, ncols, theta_deg, step, pixel, interp=OPM_INTERP_LINEAR):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.opm_plan_create(int(nscan), int(nrows), int(ncols), float(theta_deg), float(step),
                                   float(pixel), int(interp), ctypes.byref(h)), "opm_plan_create")
        self._h = h
        self.nscan, self.nrows, self.ncols = int(nscan), int(nrows), int(ncols)
        self.theta_deg, self.step, self.pixel, self.interp = float(theta_deg), float(step), float(pixel), int(interp)
        self.nz, self.ny, self.nx, self.J0 = opm_plan_shape(self)

    @property
    def handle(self):
        return self._h

    @property
    def raw_shape(self):
        return (self.nscan, self.nrows, self.ncols)

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().opm_plan_destroy(self._h), "opm_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def opm_plan_create(nscan, nrows, ncols, theta_deg, step, pixel, interp=OPM_INTERP_LINEAR) -> Plan:
    return Plan(nscan, nrows, ncols, theta_deg, step, pixel, interp)


def opm_plan_shape(plan: Plan):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load().opm_plan_shape(plan.handle, *[ctypes.byref(x) for x in v]), "opm_plan_shape")
    return tuple(int(x.value) for x in v)


OPM_PATH_GENERAL, OPM_PATH_FAST, OPM_PATH_PERIODIC = 0, 1, 2

# opm_shape: kernel shapes of the batched launch (same results, different speed)
OPM_SHAPE_AUTO, OPM_SHAPE_FAST_J8X4, OPM_SHAPE_PER_J32X2, OPM_SHAPE_PER_J16X2, OPM_SHAPE_GEN_J8X4 = 0, 1, 2, 3, 4
SHAPE_NAMES = {OPM_SHAPE_AUTO: "auto", OPM_SHAPE_FAST_J8X4: "fast_j8x4", OPM_SHAPE_PER_J32X2: "per_j32x2",
               OPM_SHAPE_PER_J16X2: "per_j16x2", OPM_SHAPE_GEN_J8X4: "gen_j8x4"}


def opm_plan_path(plan: Plan):
    """``opm_plan_path``: (path, p, q) of the live-view kernel the plan takes
    (OPM_PATH_GENERAL / _FAST / _PERIODIC; p/q = pixel/step of the periodic
    kernel, else 0, 0)."""
    v = [ctypes.c_int() for _ in range(3)]
    _check(load().opm_plan_path(plan.handle, *[ctypes.byref(x) for x in v]), "opm_plan_path")
    return tuple(x.value for x in v)


def opm_plan_schedule(plan: Plan):
    """``opm_plan_schedule``: (units, lists, rows per unit) of the plan's
    live-view schedule; all 0 without one."""
    n = ctypes.c_int64()
    l, r = ctypes.c_int(), ctypes.c_int()
    _check(load().opm_plan_schedule(plan.handle, ctypes.byref(n), ctypes.byref(l), ctypes.byref(r)),
           "opm_plan_schedule")
    return n.value, l.value, r.value


def opm_plan_destroy(plan: Plan):
    plan.close()


def opm_plan_check(plan: Plan):
    _check(load().opm_plan_check(plan.handle), "opm_plan_check")


# ------------------------------------------------------------------ tensors
def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    m = {torch.uint16: OPM_U16, torch.float32: OPM_F32, torch.float64: OPM_F64}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype} (uint16, float32 or float64)")
    return m[t.dtype]


def _ptr(t, shape=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    dev = _torch().cuda.current_device()
    if t.device.index != dev:
        # the plan lives on the current device; a kernel there must not be
        # handed another GPU's memory
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def opm_deskew(plan: Plan, raw, vol, stream=None):
    _check(load().opm_deskew(plan.handle, _ptr(raw, plan.raw_shape, "raw"), _dtype_code(raw),
                             _ptr(vol, plan.vol_shape, "vol"), _dtype_code(vol), _stream(stream)), "opm_deskew")


def opm_sheet_rows(nscan: int, nrows: int, shear: float) -> int:
    rows = ctypes.c_int64()
    _check(load().opm_sheet_rows(int(nscan), int(nrows), float(shear), ctypes.byref(rows)), "opm_sheet_rows")
    return rows.value


def opm_sheet_project(raw, shear: float, out=None, stream=None):
    """Sheet-frame view of raw [nscan][nrows][ncols] (uint16 or float32 CUDA
    tensor); returns out [opm_sheet_rows(...)][ncols] float32."""
    torch = _torch()
    nscan, nrows, ncols = raw.shape
    H = opm_sheet_rows(nscan, nrows, shear)
    if out is None:
        out = torch.empty((H, ncols), dtype=torch.float32, device=raw.device)
    _check(load().opm_sheet_project(_ptr(raw, None, "raw"), _dtype_code(raw), nscan, nrows, ncols, float(shear),
                                    _ptr(out, (H, ncols), "out"), H, _stream(stream)), "opm_sheet_project")
    return out


def opm_max_combine(out, a, b, stream=None):
    """``opm_max_combine``: out = max(a, b) elementwise (float32 CUDA tensors of
    one shape; out may be a or b)."""
    torch = _torch()
    for t, name in ((out, "out"), (a, "a"), (b, "b")):
        if t.dtype != torch.float32:
            raise TypeError(f"{name} must be float32")
    n = out.numel()
    if a.numel() != n or b.numel() != n:
        raise ValueError("out, a and b must hold the same number of values")
    _check(load().opm_max_combine(_ptr(out, None, "out"), _ptr(a, None, "a"), _ptr(b, None, "b"), n,
                                  _stream(stream)), "opm_max_combine")
    return out


def opm_sliding_push(plan: Plan, stack, m: int, run, slots, view, stream=None):
    """``opm_sliding_push`` on CUDA tensors: stack uint16 [nscan][nrows][ncols],
    run and view float32 [P], slots float32 [nscan][P], P = ny nx + nz nx."""
    P = plan.ny * plan.nx + plan.nz * plan.nx
    _check(load().opm_sliding_push(plan.handle, _ptr(stack, plan.raw_shape, "stack"), int(m),
                                   _ptr(run, (P,), "run"), _ptr(slots, (plan.nscan, P), "slots"),
                                   _ptr(view, (P,), "view"), _stream(stream)), "opm_sliding_push")


def opm_sheet_check():
    """``opm_sheet_check``: raises OpmError (OPM_ERR_INTERNAL) when a sheet-view
    ring wait on the current device gave up since the last check."""
    _check(load().opm_sheet_check(), "opm_sheet_check")


def opm_warp_rows(inp, out_rows: int, a: float, b: float, out=None, stream=None):
    torch = _torch()
    H, ncols = inp.shape
    if inp.dtype != torch.float32:
        raise TypeError("in must be float32")
    if out is None:
        out = torch.empty((out_rows, ncols), dtype=torch.float32, device=inp.device)
    _check(load().opm_warp_rows(_ptr(inp, None, "in"), H, ncols, _ptr(out, (out_rows, ncols), "out"), int(out_rows),
                                float(a), float(b), _stream(stream)), "opm_warp_rows")
    return out


def opm_deskew_mip(plan: Plan, raw, vol_f32=None, vol_u16=None, zmip=None, ymip=None, stream=None):
    torch = _torch()
    if vol_f32 is not None and vol_f32.dtype != torch.float32:
        raise TypeError("vol_f32 must be float32")
    if vol_u16 is not None and vol_u16.dtype != torch.uint16:
        raise TypeError("vol_u16 must be uint16")
    pj = (plan.ny, plan.nx)
    _check(load().opm_deskew_mip(plan.handle, _ptr(raw, plan.raw_shape, "raw"), _dtype_code(raw),
                                 _ptr(vol_f32, plan.vol_shape, "vol_f32"), _ptr(vol_u16, plan.vol_shape, "vol_u16"),
                                 _ptr(zmip, pj, "zmip"), _ptr(ymip, (plan.nz, plan.nx), "ymip"), _stream(stream)),
           "opm_deskew_mip")


def opm_stream_begin(plan: Plan, zmip=None, zsum=None, ymip=None, stream=None):
    pj = (plan.ny, plan.nx)
    _check(load().opm_stream_begin(plan.handle, _ptr(zmip, pj, "zmip"), _ptr(zsum, pj, "zsum"),
                                   _ptr(ymip, (plan.nz, plan.nx), "ymip"), _stream(stream)), "opm_stream_begin")


def opm_stream_pair(plan: Plan, plane_lo, plane_hi, n: int, zmip=None, zsum=None, ymip=None, stream=None):
    """Frames are uint16 CUDA tensors [nrows][ncols] (None outside the stack)."""
    fr = (plan.nrows, plan.ncols)
    pj = (plan.ny, plan.nx)
    _check(load().opm_stream_pair(plan.handle, _ptr(plane_lo, fr, "plane_lo"), _ptr(plane_hi, fr, "plane_hi"), int(n),
                                  _ptr(zmip, pj, "zmip"), _ptr(zsum, pj, "zsum"), _ptr(ymip, (plan.nz, plan.nx), "ymip"),
                                  _stream(stream)), "opm_stream_pair")


def opm_deskew_dual(plan: Plan, raw, vol_f32, vol_u16, stream=None):
    torch = _torch()
    if vol_f32.dtype != torch.float32 or vol_u16.dtype != torch.uint16:
        raise TypeError("vol_f32 must be float32 and vol_u16 uint16")
    _check(load().opm_deskew_dual(plan.handle, _ptr(raw, plan.raw_shape, "raw"), _dtype_code(raw),
                                  _ptr(vol_f32, plan.vol_shape, "vol_f32"), _ptr(vol_u16, plan.vol_shape, "vol_u16"),
                                  _stream(stream)), "opm_deskew_dual")


def opm_project(plan: Plan, raw, zmip=None, zsum=None, ymip=None, argz=None, stream=None):
    torch = _torch()
    for t, nm in ((zmip, "zmip"), (zsum, "zsum"), (ymip, "ymip")):
        if t is not None and t.dtype != torch.float32:
            raise TypeError(f"{nm} must be float32")
    if argz is not None and argz.dtype != torch.int32:
        raise TypeError("argz must be int32")
    pj = (plan.ny, plan.nx)
    _check(load().opm_project(plan.handle, _ptr(raw, plan.raw_shape, "raw"), _dtype_code(raw),
                              _ptr(zmip, pj, "zmip"), _ptr(zsum, pj, "zsum"),
                              _ptr(ymip, (plan.nz, plan.nx), "ymip"), _ptr(argz, pj, "argz"),
                              _stream(stream)), "opm_project")


def opm_skew_adjoint(plan: Plan, vol, raw_out, stream=None):
    if vol.dtype != raw_out.dtype:
        raise TypeError("vol and raw_out must share a dtype")
    _check(load().opm_skew_adjoint(plan.handle, _ptr(vol, plan.vol_shape, "vol"),
                                   _ptr(raw_out, plan.raw_shape, "raw_out"), _dtype_code(vol),
                                   _stream(stream)), "opm_skew_adjoint")


def opm_mip_backward(plan: Plan, g_zmip, argz, g_raw, stream=None):
    torch = _torch()
    if g_zmip.dtype != torch.float32 or g_raw.dtype != torch.float32 or argz.dtype != torch.int32:
        raise TypeError("g_zmip/g_raw must be float32 and argz int32")
    pj = (plan.ny, plan.nx)
    _check(load().opm_mip_backward(plan.handle, _ptr(g_zmip, pj, "g_zmip"), _ptr(argz, pj, "argz"),
                                   _ptr(g_raw, plan.raw_shape, "g_raw"), _stream(stream)), "opm_mip_backward")


# ------------------------------------------------------- allocating helpers
def deskew(plan: Plan, raw, out_dtype=None, stream=None):
    torch = _torch()
    if out_dtype is None:
        out_dtype = torch.float64 if raw.dtype == torch.float64 else torch.float32
    vol = torch.empty(plan.vol_shape, dtype=out_dtype, device=raw.device)
    opm_deskew(plan, raw, vol, stream)
    return vol


def project(plan: Plan, raw, zmip=True, zsum=False, ymip=False, argz=False, stream=None):
    """Returns a dict with the requested projections."""
    torch = _torch()
    dev = raw.device
    out = {}
    if zmip:
        out["zmip"] = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=dev)
    if zsum:
        out["zsum"] = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=dev)
    if ymip:
        out["ymip"] = torch.empty((plan.nz, plan.nx), dtype=torch.float32, device=dev)
    if argz:
        out["argz"] = torch.empty((plan.ny, plan.nx), dtype=torch.int32, device=dev)
    opm_project(plan, raw, out.get("zmip"), out.get("zsum"), out.get("ymip"), out.get("argz"), stream)
    return out


def skew_adjoint(plan: Plan, vol, stream=None):
    torch = _torch()
    raw = torch.empty(plan.raw_shape, dtype=vol.dtype, device=vol.device)
    opm_skew_adjoint(plan, vol, raw, stream)
    return raw


def mip_backward(plan: Plan, g_zmip, argz, stream=None):
    torch = _torch()
    g = torch.empty(plan.raw_shape, dtype=torch.float32, device=g_zmip.device)
    opm_mip_backward(plan, g_zmip, argz, g, stream)
    return g


# ----------------------------------------------------------------- batches
def _batch_items(items):
    """C array of opm_batch_item for dicts {plan, raw, zmip?, ymip?, zsum?,
    argz?, row_pitch?, plane_pitch?}, and the objects it points into."""
    arr = (opm_batch_item * max(1, len(items)))()
    keep = []
    for i, it in enumerate(items):
        raw = it["raw"]
        if not raw.is_cuda:
            raise ValueError("raw must be a CUDA tensor")
        outs = [it.get(k) for k in ("zmip", "ymip", "zsum", "argz")]
        ptrs = [o.data_ptr() if o is not None else None for o in outs]
        arr[i] = opm_batch_item(it["plan"].handle.value, raw.data_ptr(), int(it.get("row_pitch", 0)),
                                int(it.get("plane_pitch", 0)), *ptrs)
        keep.append((it["plan"], raw, *outs))
    return arr, keep


def batch_project_static(items, kchunk: int = 0, ctas_per_sm: int = 0, check: bool = False, stream=None):
    """``opm_batch_project_static``: the batched live view of ``items`` (dicts
    as for ``Batch.set``) in one call that allocates no device memory, for
    callers that must not allocate (a fixed memory plan, a per-frame
    deadline).  At most 64 items and 65536 work units; calls that overlap on
    one device race."""
    arr, _ = _batch_items(items)
    _check(load().opm_batch_project_static(ctypes.cast(arr, ctypes.c_void_p), len(items), int(kchunk),
                                           int(ctas_per_sm), int(bool(check)), _stream(stream)),
           "opm_batch_project_static")


class Batch:
    """Owns an ``opm_batch*``: persistent launches of the fused projections
    (z-MIP, y-MIP, z-sum, arg-max) over many uint16 stacks, channels
    (strided ROIs) and ROIs."""

    def __init__(self, max_items: int, max_units: int = 1 << 20):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.opm_batch_create(int(max_items), int(max_units), ctypes.byref(h)), "opm_batch_create")
        self._h = h
        self.max_items = int(max_items)
        self._keep = []

    @property
    def handle(self):
        return self._h

    def set(self, items, kchunk: int = 0, shape: int = OPM_SHAPE_AUTO):
        """items: sequence of dicts {plan, raw, zmip?, ymip?, zsum?, argz?,
        row_pitch?, plane_pitch?}; raw is a uint16 CUDA tensor (a view is
        fine: its data pointer is the ROI origin and the pitches are
        elements).  shape: an OPM_SHAPE_* kernel shape."""
        arr, keep = _batch_items(items)
        _check(load().opm_batch_set(self._h, ctypes.cast(arr, ctypes.c_void_p), len(items), int(kchunk),
                                    int(shape)), "opm_batch_set")
        self._keep = keep

    def upload(self, stream=None):
        _check(load().opm_batch_upload(self._h, _stream(stream)), "opm_batch_upload")

    def launch(self, ctas_per_sm: int = 0, stream=None):
        _check(load().opm_batch_launch(self._h, int(ctas_per_sm), _stream(stream)), "opm_batch_launch")

    def launch_graph(self, ctas_per_sm: int = 0, stream=None):
        """``opm_batch_launch_graph``: the launch through the batch's CUDA graph."""
        _check(load().opm_batch_launch_graph(self._h, int(ctas_per_sm), _stream(stream)), "opm_batch_launch_graph")

    def run(self, ctas_per_sm: int = 0, stream=None, graph: bool = False):
        self.upload(stream)
        if graph:
            self.launch_graph(ctas_per_sm, stream)
        else:
            self.launch(ctas_per_sm, stream)

    def info(self):
        n = ctypes.c_int()
        u = ctypes.c_int64()
        sm = ctypes.c_int()
        gc = ctypes.c_int()
        sh = ctypes.c_int()
        _check(load().opm_batch_info(self._h, ctypes.byref(n), ctypes.byref(u), ctypes.byref(sm), ctypes.byref(gc),
                                     ctypes.byref(sh)), "opm_batch_info")
        return {"items": n.value, "units": u.value, "smem_bytes": sm.value, "graph_captures": gc.value,
                "shape": sh.value}

    def check(self):
        _check(load().opm_batch_check(self._h), "opm_batch_check")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().opm_batch_destroy(self._h), "opm_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
