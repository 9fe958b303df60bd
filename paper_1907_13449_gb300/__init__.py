"""GB300 light-field depth with semi-global matching -- Python binding of liblfsgm.so.

Thin ctypes marshalling over the C ABI in ``include/lfsgm.h``: every function named
``lfsgm_*`` here calls the C entry point of the same name with the device pointers of
the torch tensors it is given.  All arithmetic runs in the library's CUDA kernels; there
is no CPU fallback, and ``load()`` raises if the library is missing.

Method: Anisimov, Wasenmueller, Stricker, "Rapid Light Field Depth Estimation with
Semi-Global Matching", ICCP 2019 (initial map Sec. III-D, final map Sec. III-E,
post-processing Sec. III-F).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblfsgm.so")
_lock = threading.Lock()
_lib = None

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NO_MEMORY", 3: "WORKSPACE", 4: "CUDA", 5: "UNSUPPORTED",
          6: "TIMEOUT", 7: "DEVICE_CHECK"}


class LfsgmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lfsgm error {STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    """Mirror of ``lfsgm_config``."""
    _fields_ = [("U", C.c_int32), ("V", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
                ("uc", C.c_int32), ("vc", C.c_int32), ("census_w", C.c_int32),
                ("dmin", C.c_double), ("dmax", C.c_double), ("coarse_labels", C.c_int32),
                ("init_views", C.c_int32), ("phi", C.c_double), ("fill_passes", C.c_int32),
                ("fine_labels", C.c_int32), ("fine_radius", C.c_int32), ("w_l2", C.c_float),
                ("w_census", C.c_float), ("p1_frac", C.c_double), ("p2_frac", C.c_double),
                ("subpixel", C.c_int32), ("softmin_tau", C.c_float), ("paths", C.c_int32),
                ("edge_threshold", C.c_float), ("channels", C.c_int32), ("boundless", C.c_int32),
                ("fine_radius_far", C.c_int32)]


def make_config(p) -> Config:
    """``Config`` from any object carrying the method's parameter names (views are
    [V][U][H][W] for one channel, [V][U][C][H][W] for ``channels`` = 3)."""
    return Config(U=p.U, V=p.V, H=p.H, W=p.W, uc=getattr(p, "uc", -1), vc=getattr(p, "vc", -1),
                  census_w=p.census_w, dmin=p.dmin, dmax=p.dmax, coarse_labels=p.coarse_labels,
                  init_views=p.init_views, phi=p.phi, fill_passes=p.fill_passes,
                  fine_labels=p.fine_labels, fine_radius=p.fine_radius, w_l2=p.w_l2,
                  w_census=p.w_census, p1_frac=p.p1_frac, p2_frac=p.p2_frac, subpixel=p.subpixel,
                  softmin_tau=p.softmin_tau, paths=getattr(p, "paths", 8),
                  edge_threshold=getattr(p, "edge_threshold", 0.0), channels=getattr(p, "channels", 1),
                  boundless=getattr(p, "boundless", 0), fine_radius_far=getattr(p, "fine_radius_far", 0))


EXPORTS = ["lfsgm_create", "lfsgm_destroy", "lfsgm_workspace_size", "lfsgm_set_workspace",
           "lfsgm_max_nnz", "lfsgm_initial_disparity", "lfsgm_cost_volume", "lfsgm_sgm_aggregate",
           "lfsgm_wta_subpixel", "lfsgm_backward", "lfsgm_sync", "lfsgm_last_error",
           "lfsgm_launch_count", "lfsgm_set_profiling", "lfsgm_kernel_times", "lfsgm_depth_host",
           "lfsgm_depth", "lfsgm_cost_volume_noalloc", "lfsgm_batch_create", "lfsgm_batch_run",
           "lfsgm_batch_times", "lfsgm_batch_kernel_nodes", "lfsgm_batch_last_error",
           "lfsgm_batch_destroy", "lfsgm_median_filter", "lfsgm_batch_workspace_size", "lfsgm_batch_create_ws",
           "lfsgm_set_tuning", "lfsgm_batch_knobs", "lfsgm_autotune", "lfsgm_sgm_aggregate_record",
           "lfsgm_backward_recorded", "lfsgm_set_sgm_warps", "lfsgm_get_tuning", "lfsgm_batch_sgm_warps",
           "lfsgm_set_sgm_split", "lfsgm_get_sgm_split", "lfsgm_batch_sgm_split"]


def load(build_if_missing: bool = False):
    """Load liblfsgm.so (raises if it is missing and not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if build_if_missing:
                from . import _build
                _build.build()
            else:
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        P, vp, i32, i64, f32 = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_float
        L.lfsgm_create.argtypes = [P(Config), vp, P(vp)]
        L.lfsgm_destroy.argtypes = [vp]
        L.lfsgm_workspace_size.argtypes = [vp, P(C.c_size_t)]
        L.lfsgm_set_workspace.argtypes = [vp, vp, C.c_size_t]
        L.lfsgm_max_nnz.argtypes = [vp, P(i64)]
        L.lfsgm_initial_disparity.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, P(i64)]
        L.lfsgm_cost_volume.argtypes = [vp, vp, vp, vp, vp, vp]
        L.lfsgm_sgm_aggregate.argtypes = [vp, vp, vp, vp, vp, f32, f32, vp]
        L.lfsgm_wta_subpixel.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.lfsgm_backward.argtypes = [vp, vp, vp, vp, vp, vp, f32, f32, vp, vp, vp, vp, vp]
        L.lfsgm_sgm_aggregate_record.argtypes = [vp, vp, vp, vp, vp, f32, f32, vp]
        L.lfsgm_backward_recorded.argtypes = [vp, vp, vp, vp, vp, vp, vp, f32, f32, vp, vp, vp, vp, vp]
        L.lfsgm_set_sgm_warps.argtypes = [vp, i32]
        L.lfsgm_set_sgm_split.argtypes = [vp, i32]
        L.lfsgm_get_sgm_split.argtypes = [vp, C.POINTER(i32)]
        L.lfsgm_get_tuning.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.lfsgm_batch_sgm_warps.argtypes = [vp, vp]
        L.lfsgm_batch_sgm_split.argtypes = [vp, vp]
        L.lfsgm_sync.argtypes = [vp]
        L.lfsgm_last_error.argtypes = [vp]
        L.lfsgm_last_error.restype = C.c_char_p
        L.lfsgm_launch_count.argtypes = [vp]
        L.lfsgm_launch_count.restype = i64
        L.lfsgm_set_profiling.argtypes = [vp, i32]
        L.lfsgm_kernel_times.argtypes = [vp, P(C.c_char_p), P(f32), i32, P(i32)]
        L.lfsgm_depth_host.argtypes = [vp, vp, vp, vp]
        L.lfsgm_depth.argtypes = [vp, vp, vp, vp]
        L.lfsgm_cost_volume_noalloc.argtypes = [P(Config), vp, vp, vp, vp, vp, vp]
        L.lfsgm_batch_create.argtypes = [i32, P(Config), P(vp), P(vp), vp, i32, P(vp)]
        L.lfsgm_batch_workspace_size.argtypes = [i32, P(Config), i32, P(C.c_size_t)]
        L.lfsgm_set_tuning.argtypes = [vp, i32, i32]
        L.lfsgm_autotune.argtypes = [vp, vp, P(i32), P(i32)]
        L.lfsgm_batch_knobs.argtypes = [vp, P(i32), P(i32)]
        L.lfsgm_batch_create_ws.argtypes = [i32, P(Config), P(vp), P(vp), vp, i32, vp, C.c_size_t, P(vp)]
        L.lfsgm_batch_run.argtypes = [vp]
        L.lfsgm_batch_times.argtypes = [vp, P(C.c_double), P(C.c_double), P(i32)]
        L.lfsgm_batch_kernel_nodes.argtypes = [vp]
        L.lfsgm_batch_kernel_nodes.restype = i64
        L.lfsgm_batch_last_error.argtypes = [vp]
        L.lfsgm_batch_last_error.restype = C.c_char_p
        L.lfsgm_batch_destroy.argtypes = [vp]
        L.lfsgm_median_filter.argtypes = [vp, vp, vp]
        for name in EXPORTS:
            if name not in ("lfsgm_last_error", "lfsgm_launch_count", "lfsgm_batch_kernel_nodes",
                            "lfsgm_batch_last_error"):
                getattr(L, name).restype = i32
        _lib = L
        return L


def _check(st: int, h=None):
    if st != OK:
        raise LfsgmError(st, (load().lfsgm_last_error(h) or b"").decode())


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _hptr(a, name="array"):
    """Host pointer of a contiguous CPU tensor or numpy array."""
    import numpy as np
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"{name} must be a tensor or ndarray")


# ------------------------------------------------------------------ C ABI, same names
def lfsgm_create(cfg, stream=None):
    """Handle for one light-field shape.  ``cfg``: Config or an object with the parameter
    names.  ``stream``: a torch.cuda.Stream (None -> torch's current stream)."""
    import torch
    L = load()
    if not isinstance(cfg, Config):
        cfg = make_config(cfg)
    if stream is None:
        stream = torch.cuda.current_stream()
    h = C.c_void_p()
    st = L.lfsgm_create(C.byref(cfg), C.c_void_p(stream.cuda_stream), C.byref(h))
    _check(st, None)
    return h


def lfsgm_destroy(h):
    _check(load().lfsgm_destroy(h), None)


def lfsgm_workspace_size(h) -> int:
    n = C.c_size_t()
    _check(load().lfsgm_workspace_size(h, C.byref(n)), h)
    return n.value


def lfsgm_set_workspace(h, ws):
    _check(load().lfsgm_set_workspace(h, _ptr(ws, name="workspace"), ws.numel() * ws.element_size()), h)


def lfsgm_max_nnz(h) -> int:
    n = C.c_int64()
    _check(load().lfsgm_max_nnz(h, C.byref(n)), h)
    return n.value


def lfsgm_initial_disparity(h, views, Pc1, Pc2, lo, cnt, off, dinit=None, maps=None, want_nnz=False):
    import torch
    nnz = C.c_int64(-1)
    st = load().lfsgm_initial_disparity(
        h, _ptr(views, torch.float32, "views"), int(Pc1), int(Pc2), _ptr(lo, torch.int32, "lo"),
        _ptr(cnt, torch.int32, "cnt"), _ptr(off, torch.int64, "off"), _ptr(dinit, torch.float32, "dinit"),
        _ptr(maps, torch.int32, "maps"), C.byref(nnz) if want_nnz else None)
    _check(st, h)
    return nnz.value if want_nnz else None


def lfsgm_cost_volume(h, views, lo, cnt, off, cost):
    import torch
    _check(load().lfsgm_cost_volume(h, _ptr(views, torch.float32, "views"), _ptr(lo, torch.int32, "lo"),
                                    _ptr(cnt, torch.int32, "cnt"), _ptr(off, torch.int64, "off"),
                                    _ptr(cost, torch.float32, "cost")), h)


def lfsgm_sgm_aggregate(h, cost, lo, cnt, off, P1, P2, agg):
    import torch
    _check(load().lfsgm_sgm_aggregate(h, _ptr(cost, torch.float32, "cost"), _ptr(lo, torch.int32, "lo"),
                                      _ptr(cnt, torch.int32, "cnt"), _ptr(off, torch.int64, "off"),
                                      float(P1), float(P2), _ptr(agg, torch.float32, "agg")), h)


def lfsgm_wta_subpixel(h, agg, lo, cnt, off, label, disp):
    import torch
    _check(load().lfsgm_wta_subpixel(h, _ptr(agg, torch.float32, "agg"), _ptr(lo, torch.int32, "lo"),
                                     _ptr(cnt, torch.int32, "cnt"), _ptr(off, torch.int64, "off"),
                                     _ptr(label, torch.int32, "label"), _ptr(disp, torch.float32, "disp")), h)


def lfsgm_backward(h, views, cost, lo, cnt, off, P1, P2, grad_disp, grad_cost, grad_P1, grad_P2,
                   grad_views=None):
    import torch
    f = torch.float32
    _check(load().lfsgm_backward(h, _ptr(views, f, "views"), _ptr(cost, f, "cost"),
                                 _ptr(lo, torch.int32, "lo"), _ptr(cnt, torch.int32, "cnt"),
                                 _ptr(off, torch.int64, "off"), float(P1), float(P2),
                                 _ptr(grad_disp, f, "grad_disp"), _ptr(grad_cost, f, "grad_cost"),
                                 _ptr(grad_P1, f, "grad_P1"), _ptr(grad_P2, f, "grad_P2"),
                                 _ptr(grad_views, f, "grad_views")), h)


def lfsgm_sgm_aggregate_record(h, cost, lo, cnt, off, P1, P2, agg):
    """lfsgm_sgm_aggregate on explicit penalties that also records the branches for
    lfsgm_backward_recorded."""
    import torch
    _check(load().lfsgm_sgm_aggregate_record(h, _ptr(cost, torch.float32, "cost"), _ptr(lo, torch.int32, "lo"),
                                             _ptr(cnt, torch.int32, "cnt"), _ptr(off, torch.int64, "off"),
                                             float(P1), float(P2), _ptr(agg, torch.float32, "agg")), h)


def lfsgm_backward_recorded(h, views, cost, agg, lo, cnt, off, P1, P2, grad_disp, grad_cost, grad_P1, grad_P2,
                            grad_views=None):
    import torch
    f = torch.float32
    _check(load().lfsgm_backward_recorded(h, _ptr(views, f, "views"), _ptr(cost, f, "cost"), _ptr(agg, f, "agg"),
                                          _ptr(lo, torch.int32, "lo"), _ptr(cnt, torch.int32, "cnt"),
                                          _ptr(off, torch.int64, "off"), float(P1), float(P2),
                                          _ptr(grad_disp, f, "grad_disp"), _ptr(grad_cost, f, "grad_cost"),
                                          _ptr(grad_P1, f, "grad_P1"), _ptr(grad_P2, f, "grad_P2"),
                                          _ptr(grad_views, f, "grad_views")), h)


def lfsgm_median_filter(h, disp, out):
    """3 x 3 median of the disparity map (Sec. III-F), border values repeated."""
    import torch
    _check(load().lfsgm_median_filter(h, _ptr(disp, torch.float32, "disp"), _ptr(out, torch.float32, "out")), h)


def lfsgm_sync(h):
    _check(load().lfsgm_sync(h), h)


def lfsgm_last_error(h) -> str:
    return (load().lfsgm_last_error(h) or b"").decode()


def lfsgm_launch_count(h) -> int:
    return int(load().lfsgm_launch_count(h))


def lfsgm_set_profiling(h, enable: bool):
    _check(load().lfsgm_set_profiling(h, 1 if enable else 0), h)


def lfsgm_kernel_times(h, cap: int = 4096):
    names = (C.c_char_p * cap)()
    ms = (C.c_float * cap)()
    n = C.c_int32()
    _check(load().lfsgm_kernel_times(h, names, ms, cap, C.byref(n)), h)
    return [(names[i].decode(), float(ms[i])) for i in range(n.value)]


def lfsgm_depth_host(h, views_host, disp_host, label_host=None):
    _check(load().lfsgm_depth_host(h, _hptr(views_host, "views_host"), _hptr(disp_host, "disp_host"),
                                   None if label_host is None else _hptr(label_host, "label_host")), h)


def lfsgm_depth(h, views, disp=None, label=None):
    import torch
    _check(load().lfsgm_depth(h, _ptr(views, torch.float32, "views"), _ptr(disp, torch.float32, "disp"),
                              _ptr(label, torch.int32, "label")), h)


def lfsgm_cost_volume_noalloc(cfg, views, lo, cnt, off, cost, stream=None):
    """lfsgm_cost_volume without a handle and without any device allocation, for callers
    that run under a fixed device-memory budget (scratch lives in a static 32 MiB device
    array inside the library; calls that overlap on the GPU race on it)."""
    import torch
    if not isinstance(cfg, Config):
        cfg = make_config(cfg)
    if stream is None:
        stream = torch.cuda.current_stream()
    st = load().lfsgm_cost_volume_noalloc(
        C.byref(cfg), C.c_void_p(stream.cuda_stream), _ptr(views, torch.float32, "views"),
        _ptr(lo, torch.int32, "lo"), _ptr(cnt, torch.int32, "cnt"), _ptr(off, torch.int64, "off"),
        _ptr(cost, torch.float32, "cost"))
    if st != OK:
        raise LfsgmError(st, "lfsgm_cost_volume_noalloc: " + {1: "invalid config or null buffer",
                                                              5: "light field too large for the static scratch"
                                                                 " (or in colour)",
                                                              4: "CUDA error"}.get(st, ""))


# ------------------------------------------------------------------ batches (not in the paper)
def _bcheck(st: int, b=None):
    if st != OK:
        raise LfsgmError(st, (load().lfsgm_batch_last_error(b) or b"").decode())


def _configs(cfgs):
    n = len(cfgs)
    return n, (Config * n)(*[c if isinstance(c, Config) else make_config(c) for c in cfgs])


def lfsgm_batch_create(cfgs, views, disp, stream=None, branches=0, ws=None):
    """One CUDA graph running the whole depth pipeline of every light field.  ``cfgs``: list of
    Config (or parameter objects); ``views``/``disp``: lists of device float32 tensors
    ([V,U,H,W] and [H*W]) whose addresses are baked into the graph.  ``branches`` <= 0 lets the
    library time 1, 2, 4, 8, 16 concurrent branches and keep the fastest.  ``ws``: an optional
    caller-owned device buffer (uint8 tensor, lfsgm_batch_workspace_size bytes) for the scratch
    (lfsgm_batch_create_ws)."""
    import torch
    n, arr = _configs(cfgs)
    if n < 1 or len(views) != n or len(disp) != n:
        raise ValueError("need equally long, non-empty cfgs, views and disp")
    vptr = (C.c_void_p * n)(*[_ptr(v, torch.float32, "views") for v in views])
    dptr = (C.c_void_p * n)(*[_ptr(d, torch.float32, "disp") for d in disp])
    if stream is None:
        stream = torch.cuda.current_stream()
    b = C.c_void_p()
    if ws is None:
        _bcheck(load().lfsgm_batch_create(n, arr, vptr, dptr, C.c_void_p(stream.cuda_stream), int(branches),
                                          C.byref(b)), None)
    else:
        _bcheck(load().lfsgm_batch_create_ws(n, arr, vptr, dptr, C.c_void_p(stream.cuda_stream), int(branches),
                                             _ptr(ws, torch.uint8, "ws"), ws.numel(), C.byref(b)), None)
    return b


def lfsgm_batch_create_ws(cfgs, views, disp, ws, stream=None, branches=0):
    """lfsgm_batch_create with the scratch in the caller's buffer ``ws`` (uint8 device tensor)."""
    return lfsgm_batch_create(cfgs, views, disp, stream, branches, ws=ws)


def lfsgm_batch_workspace_size(cfgs, branches=0) -> int:
    """Bytes of caller-owned scratch a batch of these configurations needs (no device work)."""
    n, arr = _configs(cfgs)
    out = C.c_size_t()
    _bcheck(load().lfsgm_batch_workspace_size(n, arr, int(branches), C.byref(out)), None)
    return int(out.value)


def lfsgm_set_tuning(h, row_kw=0, list_ctas_per_sm=0):
    """Speed knobs of a handle: the row cost kernel's label span (36 or 44; 0 = 36) and the list
    kernel's CTAs per SM (0 = default)."""
    _check(load().lfsgm_set_tuning(h, int(row_kw), int(list_ctas_per_sm)), h)


def lfsgm_autotune(h, views):
    """Tune the handle's speed knobs on ``views`` (device tensor); returns (row_kw, list_ctas_per_sm)."""
    import torch
    kw = C.c_int32()
    lc = C.c_int32()
    _check(load().lfsgm_autotune(h, _ptr(views, torch.float32, "views"), C.byref(kw), C.byref(lc)), h)
    return int(kw.value), int(lc.value)


def lfsgm_set_sgm_warps(h, warps_per_cta=0):
    """Speed knob of the fine SGM: scanlines (warps) per CTA, 2, 4 or 8 (0 = 4)."""
    _check(load().lfsgm_set_sgm_warps(h, int(warps_per_cta)), h)


def lfsgm_set_sgm_split(h, min_wide=0):
    """Speed knob of the fine SGM: scanlines crossing at least min_wide windows wider than 32
    labels run on all warps of a CTA (0: none)."""
    _check(load().lfsgm_set_sgm_split(h, int(min_wide)), h)


def lfsgm_get_sgm_split(h):
    """The handle's SGM split threshold (0: off)."""
    v = C.c_int32()
    _check(load().lfsgm_get_sgm_split(h, C.byref(v)), h)
    return int(v.value)


def lfsgm_get_tuning(h):
    """The handle's speed knobs: (row_kw, list_ctas_per_sm, sgm_warps)."""
    kw, lc, sw = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().lfsgm_get_tuning(h, C.byref(kw), C.byref(lc), C.byref(sw)), h)
    return int(kw.value), int(lc.value), int(sw.value)


def lfsgm_batch_sgm_warps(b, n):
    """The fine SGM's warps per CTA of each light field of a batch (numpy int32 array)."""
    import numpy as np
    w = np.zeros(n, np.int32)
    _bcheck(load().lfsgm_batch_sgm_warps(b, w.ctypes.data_as(C.c_void_p)), b)
    return w


def lfsgm_batch_sgm_split(b, n):
    """The fine SGM's split threshold of each light field of a batch (numpy int32 array; 0: off)."""
    import numpy as np
    w = np.zeros(n, np.int32)
    _bcheck(load().lfsgm_batch_sgm_split(b, w.ctypes.data_as(C.c_void_p)), b)
    return w


def lfsgm_batch_knobs(b, n):
    """(row_kw, list_ctas_per_sm) per light field of a batch, as numpy int32 arrays."""
    import numpy as np
    kw = np.zeros(n, np.int32)
    lc = np.zeros(n, np.int32)
    _bcheck(load().lfsgm_batch_knobs(b, kw.ctypes.data_as(C.POINTER(C.c_int32)),
                                     lc.ctypes.data_as(C.POINTER(C.c_int32))), b)
    return kw, lc


def lfsgm_batch_run(b):
    _bcheck(load().lfsgm_batch_run(b), b)


def lfsgm_batch_times(b, n):
    """(start_ms, end_ms, branches): per light field, when its pipeline started and ended
    relative to the start of the last batch run (synchronises)."""
    import numpy as np
    s = np.zeros(n, np.float64)
    e = np.zeros(n, np.float64)
    k = C.c_int32()
    _bcheck(load().lfsgm_batch_times(b, s.ctypes.data_as(C.POINTER(C.c_double)),
                                     e.ctypes.data_as(C.POINTER(C.c_double)), C.byref(k)), b)
    return s, e, k.value


def lfsgm_batch_kernel_nodes(b) -> int:
    return int(load().lfsgm_batch_kernel_nodes(b))


def lfsgm_batch_last_error(b) -> str:
    return (load().lfsgm_batch_last_error(b) or b"").decode()


def lfsgm_batch_destroy(b):
    _bcheck(load().lfsgm_batch_destroy(b), None)


class LightFieldBatch:
    """Owns the batch graph, the output disparity maps and references to the input views."""

    def __init__(self, params, views, branches=0, stream=None, ws=None):
        import torch
        self.params = list(params)
        self.views = [v.contiguous() for v in views]
        self.disp = [torch.empty(p.H * p.W, dtype=torch.float32, device=v.device)
                     for p, v in zip(self.params, self.views)]
        self.ws = ws                  # caller-owned scratch (kept alive with the batch)
        self.b = lfsgm_batch_create(self.params, self.views, self.disp, stream, branches, ws=ws)
        self.n = len(self.params)

    def run(self):
        lfsgm_batch_run(self.b)
        return self.disp

    def times(self):
        return lfsgm_batch_times(self.b, self.n)

    def knobs(self):
        """(row_kw, list_ctas_per_sm, sgm_warps, sgm_split) per light field, numpy int32 arrays."""
        kw, lc = lfsgm_batch_knobs(self.b, self.n)
        return kw, lc, lfsgm_batch_sgm_warps(self.b, self.n), lfsgm_batch_sgm_split(self.b, self.n)

    @property
    def kernel_nodes(self):
        return lfsgm_batch_kernel_nodes(self.b)

    def close(self):
        if self.b is not None:
            lfsgm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ differentiation (not in the paper)
def _autograd():
    import torch

    class SGMSoftArgmin(torch.autograd.Function):
        """disp = soft-argmin(SGM(cost; P1, P2)) on the windows held by ``L`` (a LightFieldDepth
        created with subpixel=2); backward = lfsgm_backward (grad wrt cost, P1, P2)."""

        @staticmethod
        def forward(ctx, cost, P1, P2, L):
            p1, p2 = float(P1), float(P2)
            cost = cost.contiguous()
            agg = torch.empty_like(cost)
            lfsgm_sgm_aggregate_record(L.h, cost, L.lo, L.cnt, L.off, p1, p2, agg)
            L.recorded = (cost.data_ptr(), agg.data_ptr(), (p1, p2))
            disp = torch.empty(L.N, dtype=torch.float32, device=cost.device)
            lfsgm_wta_subpixel(L.h, agg, L.lo, L.cnt, L.off, None, disp)
            ctx.save_for_backward(cost, agg)
            ctx.pen, ctx.L = (p1, p2), L
            return disp

        @staticmethod
        def backward(ctx, gdisp):
            cost, agg = ctx.saved_tensors
            L = ctx.L
            gcost = torch.empty_like(cost)
            gp = torch.zeros(2, dtype=torch.float32, device=cost.device)
            _backward_saved(L, None, cost, agg, ctx.pen, gdisp.contiguous(), gcost, gp, None)
            return _needed(ctx, gcost, gp[0], gp[1])

    class DepthFromViews(torch.autograd.Function):
        """disp = soft-argmin(SGM(cost_volume(views); P1, P2)) on the windows held by ``L``;
        backward = lfsgm_backward (grad wrt views through the l2 term, P1, P2)."""

        @staticmethod
        def forward(ctx, views, P1, P2, L):
            p1, p2 = float(P1), float(P2)
            L.cost_volume(views)
            cost = L.cost.clone()            # L.cost is overwritten by the next forward
            agg = torch.empty_like(cost)
            lfsgm_sgm_aggregate_record(L.h, cost, L.lo, L.cnt, L.off, p1, p2, agg)
            L.recorded = (cost.data_ptr(), agg.data_ptr(), (p1, p2))
            disp = torch.empty(L.N, dtype=torch.float32, device=views.device)
            lfsgm_wta_subpixel(L.h, agg, L.lo, L.cnt, L.off, None, disp)
            ctx.save_for_backward(views, cost, agg)
            ctx.pen, ctx.L = (p1, p2), L
            return disp

        @staticmethod
        def backward(ctx, gdisp):
            views, cost, agg = ctx.saved_tensors
            L = ctx.L
            gcost = torch.empty_like(cost)
            gviews = torch.empty_like(views)
            gp = torch.zeros(2, dtype=torch.float32, device=views.device)
            _backward_saved(L, views, cost, agg, ctx.pen, gdisp.contiguous(), gcost, gp, gviews)
            return _needed(ctx, gviews, gp[0], gp[1])

    return SGMSoftArgmin, DepthFromViews


def _needed(ctx, *grads):
    """The gradients of the inputs that want one (plain-number penalties get None)."""
    return tuple(g if need else None for g, need in zip(grads, ctx.needs_input_grad)) + (None,)


def _backward_saved(L, views, cost, agg, pen, gdisp, gcost, gp, gviews):
    """The backward on the forward's record when it is still the handle's last one (one handle
    records one forward at a time), else with the SGM recomputed."""
    if L.recorded == (cost.data_ptr(), agg.data_ptr(), pen):
        lfsgm_backward_recorded(L.h, views, cost, agg, L.lo, L.cnt, L.off, pen[0], pen[1], gdisp, gcost, gp[0:1],
                                gp[1:2], gviews)
    else:
        lfsgm_backward(L.h, views, cost, L.lo, L.cnt, L.off, pen[0], pen[1], gdisp, gcost, gp[0:1], gp[1:2], gviews)
        L.recorded = None             # lfsgm_backward records over the handle's scratch


def sgm_softargmin(cost, P1, P2, L):
    """Differentiable soft-argmin disparity of the SGM-aggregated cost (see SGMSoftArgmin)."""
    return _autograd()[0].apply(cost, P1, P2, L)


def depth_from_views(views, P1, P2, L):
    """Differentiable soft-argmin disparity from the views on fixed windows (see DepthFromViews)."""
    return _autograd()[1].apply(views, P1, P2, L)


# ------------------------------------------------------------------ convenience wrapper
class LightFieldDepth:
    """Owns a handle and the windowed buffers of one light-field shape and runs the
    stages in the paper's order.  Buffers are torch CUDA tensors."""

    def __init__(self, params, stream=None, device="cuda"):
        import torch
        self.params = params
        self.device = torch.device(device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.h = lfsgm_create(params, self.stream)
        self.recorded = None          # (cost, agg, penalties) of the handle's SGM record, if still valid
        N = params.H * params.W
        self.N = N
        self.max_nnz = lfsgm_max_nnz(self.h)
        i32, i64, f32 = torch.int32, torch.int64, torch.float32
        self.lo = torch.empty(N, dtype=i32, device=self.device)
        self.cnt = torch.empty(N, dtype=i32, device=self.device)
        self.off = torch.empty(N + 1, dtype=i64, device=self.device)
        self.dinit = torch.empty(N, dtype=f32, device=self.device)
        self.maps = torch.empty(4, N, dtype=i32, device=self.device)
        self.cost = torch.empty(self.max_nnz, dtype=f32, device=self.device)
        self.agg = torch.empty(self.max_nnz, dtype=f32, device=self.device)
        self.label = torch.empty(N, dtype=i32, device=self.device)
        self.disp = torch.empty(N, dtype=f32, device=self.device)

    def initial(self, views, Pc1=0, Pc2=0, want_nnz=False):
        return lfsgm_initial_disparity(self.h, views, Pc1, Pc2, self.lo, self.cnt, self.off, self.dinit,
                                       self.maps, want_nnz)

    def cost_volume(self, views):
        lfsgm_cost_volume(self.h, views, self.lo, self.cnt, self.off, self.cost)

    def aggregate(self, P1=-1.0, P2=-1.0):
        lfsgm_sgm_aggregate(self.h, self.cost, self.lo, self.cnt, self.off, P1, P2, self.agg)

    def wta(self):
        lfsgm_wta_subpixel(self.h, self.agg, self.lo, self.cnt, self.off, self.label, self.disp)

    def forward(self, views, Pc=(0, 0), P=(-1.0, -1.0)):
        self.initial(views, *Pc)
        self.cost_volume(views)
        self.aggregate(*P)
        self.wta()
        return self.disp

    def close(self):
        if self.h is not None:
            lfsgm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
