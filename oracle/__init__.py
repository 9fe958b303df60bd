"""FP64 CPU oracle of the light-field SGM depth method (Anisimov, Wasenmueller,
Stricker, ICCP 2019) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_1907_13449_gb300``): the arithmetic lives in ``lfsgm_oracle.c`` (plain
loops, double precision, built with ``-ffp-contract=off``), and this module only
marshals numpy arrays and composes the stages in the paper's order
(Sec. III-D initial map -> Sec. III-E final map -> Sec. III-F post-processing).

Every function here either calls one C stage or chains stages exactly as the
paper orders them; see ``lfsgm_oracle.c`` for the per-equation citations.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfsgm_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

DIRECTIONS = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1),
              (2, 1), (-2, -1), (2, -1), (-2, 1), (1, 2), (-1, -2), (1, -2), (-1, 2))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math, OpenMP over rows)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(C.Structure):
    _fields_ = [("U", C.c_int32), ("V", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
                ("uc", C.c_int32), ("vc", C.c_int32), ("census_w", C.c_int32),
                ("dmin", C.c_double), ("dmax", C.c_double), ("Lc", C.c_int32),
                ("init_views", C.c_int32), ("phi", C.c_double), ("fill_passes", C.c_int32),
                ("G", C.c_int32), ("R", C.c_int32), ("w_l2", C.c_double), ("w_census", C.c_double),
                ("paths", C.c_int32), ("edge_threshold", C.c_float), ("channels", C.c_int32),
                ("boundless", C.c_int32), ("R_far", C.c_int32)]


def make_cfg(p) -> Cfg:
    """Oracle config from any object with the method's parameter names
    (``lfsynth.LFParams`` or the library's config dataclass).  Views are
    [V][U][H][W] for one channel and [V][U][C][H][W] for C = 3 (RGB)."""
    channels = int(getattr(p, "channels", 1) or 1)
    if channels not in (1, 3):
        raise ValueError(f"channels must be 1 or 3, got {channels}")
    return Cfg(U=p.U, V=p.V, H=p.H, W=p.W, uc=p.uc, vc=p.vc, census_w=p.census_w,
               dmin=p.dmin, dmax=p.dmax, Lc=p.coarse_labels, init_views=p.init_views,
               phi=p.phi, fill_passes=p.fill_passes, G=p.fine_labels, R=p.fine_radius,
               w_l2=p.w_l2, w_census=p.w_census, paths=getattr(p, "paths", 8),
               edge_threshold=getattr(p, "edge_threshold", 0.0), channels=channels,
               boundless=int(getattr(p, "boundless", 0)), R_far=int(getattr(p, "fine_radius_far", 0)))


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            P = C.POINTER
            L.or_label_disp.restype = C.c_double
            L.or_set_threads.argtypes = [C.c_int]
            L.or_median3.argtypes = [C.c_int, C.c_int, P(C.c_double), P(C.c_double)]
            L.or_set_threads.restype = C.c_int
            L.or_label_disp.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int]
            L.or_shift.argtypes = [C.c_int, C.c_double, P(C.c_int), P(C.c_double), P(C.c_int)]
            L.or_census.argtypes = [P(C.c_double), C.c_int, C.c_int, C.c_int, P(C.c_uint64)]
            L.or_hamming.restype = C.c_int
            L.or_hamming.argtypes = [C.c_uint64, C.c_uint64]
            L.or_census_all.argtypes = [P(Cfg), P(C.c_double), P(C.c_uint64)]
            L.or_arm_views.restype = C.c_int
            L.or_arm_views.argtypes = [P(Cfg), C.c_int, P(C.c_int)]
            L.or_coarse_cost.restype = C.c_int
            L.or_coarse_cost.argtypes = [P(Cfg), P(C.c_uint64), C.c_int, P(C.c_int64)]
            L.or_int_penalties.argtypes = [C.c_int64, C.c_int64, C.c_double, C.c_double,
                                           P(C.c_int64), P(C.c_int64)]
            L.or_sgm_int_path.argtypes = [C.c_int, C.c_int, C.c_int, P(C.c_int64), C.c_int64,
                                          C.c_int64, C.c_int, P(C.c_int64)]
            L.or_sgm_int.argtypes = [C.c_int, C.c_int, C.c_int, P(C.c_int64), C.c_int64, C.c_int64,
                                     C.c_int, P(C.c_int64)]
            L.or_wta_int.argtypes = [C.c_size_t, C.c_int, P(C.c_int64), P(C.c_int32)]
            L.or_fuse.argtypes = [C.c_size_t, C.c_int, P(C.c_int32), C.c_double, P(C.c_double)]
            L.or_hole_fill.argtypes = [C.c_int, C.c_int, C.c_int, P(C.c_double)]
            L.or_windows.argtypes = [P(Cfg), C.c_size_t, P(C.c_double), P(C.c_uint8), P(C.c_int32), P(C.c_int32)]
            L.or_radius.restype = C.c_int
            L.or_radius.argtypes = [P(Cfg), C.c_int64]
            L.or_sobel_edges.argtypes = [C.c_int, C.c_int, P(C.c_float), C.c_float, P(C.c_uint8)]
            L.or_cost_volume.argtypes = [P(Cfg), P(C.c_double), P(C.c_uint64), P(C.c_int32),
                                         P(C.c_int32), P(C.c_int64), P(C.c_double)]
            L.or_softargmin_backward.argtypes = [P(Cfg), C.c_size_t, P(C.c_int32), P(C.c_int32), P(C.c_int64),
                                                 P(C.c_double), P(C.c_double), C.c_double, P(C.c_double)]
            L.or_sgm_bounded_path_backward.argtypes = [C.c_int, C.c_int, P(C.c_int32), P(C.c_int32),
                                                       P(C.c_int64), P(C.c_double), C.c_double, C.c_double,
                                                       C.c_int, P(C.c_double), P(C.c_double), P(C.c_double),
                                                       P(C.c_double)]
            L.or_cost_backward_views.argtypes = [P(Cfg), P(C.c_double), P(C.c_int32), P(C.c_int32),
                                                 P(C.c_int64), P(C.c_double), P(C.c_double)]
            L.or_sgm_bounded_path.argtypes = [C.c_int, C.c_int, P(C.c_int32), P(C.c_int32),
                                              P(C.c_int64), P(C.c_double), C.c_double, C.c_double,
                                              C.c_int, C.c_int, P(C.c_double)]
            L.or_sgm_bounded.argtypes = [C.c_int, C.c_int, P(C.c_int32), P(C.c_int32), P(C.c_int64),
                                         P(C.c_double), C.c_double, C.c_double, C.c_int, P(C.c_double)]
            L.or_wta_subpixel.argtypes = [P(Cfg), C.c_size_t, P(C.c_int32), P(C.c_int32),
                                          P(C.c_int64), P(C.c_double), C.c_int, C.c_double,
                                          P(C.c_int32), P(C.c_double), P(C.c_double)]
    return _lib


# ----------------------------------------------------------------- small helpers
def label_disp(dmin: float, dmax: float, L: int, k: int) -> float:
    return lib().or_label_disp(dmin, dmax, L, k)


def shift(a: int, d: float):
    """(ox, fx, nx) of the shift a*d under the oracle's shift rule."""
    o, n, f = C.c_int(), C.c_int(), C.c_double()
    lib().or_shift(a, d, C.byref(o), C.byref(f), C.byref(n))
    return o.value, f.value, n.value


def census(img: np.ndarray, w: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    out = np.zeros((H, W), np.uint64)
    lib().or_census(_ptr(img, C.c_double), H, W, w, _ptr(out, C.c_uint64))
    return out


def hamming(a: int, b: int) -> int:
    return lib().or_hamming(int(a), int(b))


def census_all(cfg: Cfg, views: np.ndarray) -> np.ndarray:
    views = np.ascontiguousarray(views, dtype=np.float64)
    out = np.zeros(views.shape, np.uint64)
    lib().or_census_all(C.byref(cfg), _ptr(views, C.c_double), _ptr(out, C.c_uint64))
    return out


def arm_views(cfg: Cfg, arm: int):
    buf = (C.c_int * 1024)()
    n = lib().or_arm_views(C.byref(cfg), arm, buf)
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]


def coarse_cost(cfg: Cfg, cen: np.ndarray, arm: int):
    """int64 [H*W, Lc] arm cost (Eq. 7) or None for an empty arm."""
    out = np.zeros((cfg.H * cfg.W, cfg.Lc), np.int64)
    n = lib().or_coarse_cost(C.byref(cfg), _ptr(cen, C.c_uint64), arm, _ptr(out, C.c_int64))
    return out if n > 0 else None


def int_penalties(total: int, count: int, p1f: float, p2f: float):
    a, b = C.c_int64(), C.c_int64()
    lib().or_int_penalties(int(total), int(count), p1f, p2f, C.byref(a), C.byref(b))
    return a.value, b.value


def sgm_int_path(H, W, Cv: np.ndarray, P1: int, P2: int, direction: int) -> np.ndarray:
    Cv = np.ascontiguousarray(Cv, dtype=np.int64)
    out = np.zeros_like(Cv)
    lib().or_sgm_int_path(H, W, Cv.shape[-1], _ptr(Cv, C.c_int64), P1, P2, direction,
                          _ptr(out, C.c_int64))
    return out


def sgm_int(H, W, Cv: np.ndarray, P1: int, P2: int, paths: int = 8) -> np.ndarray:
    Cv = np.ascontiguousarray(Cv, dtype=np.int64)
    out = np.zeros_like(Cv)
    lib().or_sgm_int(H, W, Cv.shape[-1], _ptr(Cv, C.c_int64), P1, P2, int(paths), _ptr(out, C.c_int64))
    return out


def wta_int(Cs: np.ndarray) -> np.ndarray:
    Cs = np.ascontiguousarray(Cs, dtype=np.int64)
    out = np.zeros(Cs.shape[0], np.int32)
    lib().or_wta_int(Cs.shape[0], Cs.shape[1], _ptr(Cs, C.c_int64), _ptr(out, C.c_int32))
    return out


def fuse(maps: np.ndarray, phi: float) -> np.ndarray:
    maps = np.ascontiguousarray(maps, dtype=np.int32)
    n, N = maps.shape
    out = np.zeros(N, np.float64)
    lib().or_fuse(N, n, _ptr(maps, C.c_int32), phi, _ptr(out, C.c_double))
    return out


def hole_fill(dinit: np.ndarray, H: int, W: int, passes: int) -> np.ndarray:
    d = np.array(dinit, dtype=np.float64, copy=True).reshape(-1)
    lib().or_hole_fill(H, W, passes, _ptr(d, C.c_double))
    return d


def sobel_edges(I: np.ndarray, threshold: float) -> np.ndarray:
    """Edge mask of the reference view for the border exclusion (Sec. III-D), FP32 Sobel.
    ``I`` is [H][W], or [C][H][W]: a pixel is an edge iff it is one in any channel."""
    I = np.ascontiguousarray(I, dtype=np.float32)
    if I.ndim == 3:
        return np.logical_or.reduce([sobel_edges(I[ch], threshold) for ch in range(I.shape[0])])
    H, W = I.shape
    out = np.zeros((H, W), np.uint8)
    lib().or_sobel_edges(H, W, _ptr(I, C.c_float), float(threshold), _ptr(out, C.c_uint8))
    return out.astype(bool)


def radius(cfg: Cfg, gc: int) -> int:
    """Border threshold lambda of a window centred on fine label gc (constant unless R_far > 0)."""
    return int(lib().or_radius(C.byref(cfg), int(gc)))


def windows(cfg: Cfg, dinit: np.ndarray, edge=None):
    d = np.ascontiguousarray(dinit, dtype=np.float64).reshape(-1)
    lo = np.zeros(d.size, np.int32)
    cnt = np.zeros(d.size, np.int32)
    e = None if edge is None else np.ascontiguousarray(edge, dtype=np.uint8).reshape(-1)
    lib().or_windows(C.byref(cfg), d.size, _ptr(d, C.c_double), None if e is None else _ptr(e, C.c_uint8),
                     _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32))
    return lo, cnt


def offsets(cnt: np.ndarray) -> np.ndarray:
    off = np.zeros(cnt.size + 1, np.int64)
    np.cumsum(cnt.reshape(-1), out=off[1:])
    return off


def cost_volume(cfg: Cfg, views: np.ndarray, lo: np.ndarray, cnt: np.ndarray, cen=None):
    """(off, cost) with cost[off[p] + j] = C(p, lo[p] + j) (Eq. 12 + Eq. 15).  Views are
    taken in double precision (float32 inputs convert exactly)."""
    views = np.ascontiguousarray(views, dtype=np.float64)
    if cen is None:
        cen = census_all(cfg, views)
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = offsets(cnt)
    cost = np.zeros(int(off[-1]), np.float64)
    lib().or_cost_volume(C.byref(cfg), _ptr(views, C.c_double), _ptr(cen, C.c_uint64),
                         _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32), _ptr(off, C.c_int64),
                         _ptr(cost, C.c_double))
    return off, cost


def sgm_bounded_path(H, W, lo, cnt, off, cost, P1, P2, direction, normalised=True):
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(off, dtype=np.int64)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    out = np.zeros_like(cost)
    lib().or_sgm_bounded_path(H, W, _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32), _ptr(off, C.c_int64),
                              _ptr(cost, C.c_double), float(P1), float(P2), direction,
                              1 if normalised else 0, _ptr(out, C.c_double))
    return out


def threads() -> int:
    """Threads the oracle's parallel loops use (OpenMP default: all cores)."""
    return int(lib().or_set_threads(0))


def set_threads(n: int) -> int:
    """Set the threads of the oracle's parallel loops (results do not depend on it)."""
    return int(lib().or_set_threads(int(n)))


def sgm_bounded(H, W, lo, cnt, off, cost, P1, P2, paths: int = 8):
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(off, dtype=np.int64)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    out = np.zeros_like(cost)
    lib().or_sgm_bounded(H, W, _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32), _ptr(off, C.c_int64),
                         _ptr(cost, C.c_double), float(P1), float(P2), int(paths), _ptr(out, C.c_double))
    return out


def wta_subpixel(cfg: Cfg, lo, cnt, off, Cs, mode=1, tau=0.1):
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(off, dtype=np.int64)
    Cs = np.ascontiguousarray(Cs, dtype=np.float64)
    N = lo.size
    label = np.zeros(N, np.int32)
    disp = np.zeros(N, np.float64)
    gap = np.zeros(N, np.float64)
    lib().or_wta_subpixel(C.byref(cfg), N, _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32),
                          _ptr(off, C.c_int64), _ptr(Cs, C.c_double), mode, tau,
                          _ptr(label, C.c_int32), _ptr(disp, C.c_double), _ptr(gap, C.c_double))
    return label, disp, gap


# --------------------------------------------------------- composed stages
def initial_disparity(cfg: Cfg, views: np.ndarray, penalties=None, p1f=0.05, p2f=0.5, cen=None):
    """Sec. III-D in order: census of the cross views, per-arm cost (Eq. 7), SGM per
    arm (Eq. 8-9), WTA (Eq. 10), fusion with threshold phi, median hole filling,
    borders (Eq. 11).  ``penalties``: None -> per-arm (P1, P2) derived from the arm's
    mean cost with fractions (p1f, p2f); or a list of one (P1, P2) per arm."""
    views = np.ascontiguousarray(views, dtype=np.float32)
    if cen is None:
        cen = census_all(cfg, views)
    H, W, N = cfg.H, cfg.W, cfg.H * cfg.W
    if cfg.boundless:
        # boundary-less search (Sec. IV-E): no initial map, every window is the whole range
        nan = np.full(N, np.nan)
        lo, cnt = windows(cfg, nan)
        return {"maps": np.zeros((0, N), np.int32), "arms": [], "penalties": [], "fused": nan,
                "dinit": nan, "lo": lo, "cnt": cnt, "census": cen}
    maps, pens, arms = [], [], []
    for arm in range(4):
        ca = coarse_cost(cfg, cen, arm)
        if ca is None:
            continue
        if penalties is None:
            P1, P2 = int_penalties(int(ca.sum()), ca.size, p1f, p2f)
        else:
            P1, P2 = penalties[arm]
        Cs = sgm_int(H, W, ca, P1, P2, cfg.paths)
        maps.append(wta_int(Cs))
        pens.append((P1, P2))
        arms.append(arm)
    maps = np.stack(maps)
    fused = fuse(maps, cfg.phi)
    filled = hole_fill(fused, H, W, cfg.fill_passes)
    edge = None
    if cfg.edge_threshold > 0:
        edge = sobel_edges(views[cfg.vc, cfg.uc], cfg.edge_threshold)
    lo, cnt = windows(cfg, filled, edge)
    return {"maps": maps, "arms": arms, "penalties": pens, "fused": fused,
            "dinit": filled, "lo": lo, "cnt": cnt, "census": cen}


def depth(cfg: Cfg, views: np.ndarray, fine_penalties=None, p1f=0.05, p2f=0.5, mode=1, tau=0.1,
          coarse_penalties=None):
    """The whole method: initial map, bounded cost (Eq. 12 + 15), bounded SGM, WTA and
    sub-pixel refinement.  ``fine_penalties``: None -> (p1f, p2f) x mean active cost."""
    init = initial_disparity(cfg, views, coarse_penalties, p1f, p2f)
    off, cost = cost_volume(cfg, views, init["lo"], init["cnt"], init["census"])
    if fine_penalties is None:
        mean = float(cost.mean())
        P1, P2 = p1f * mean, p2f * mean
    else:
        P1, P2 = fine_penalties
    Cs = sgm_bounded(cfg.H, cfg.W, init["lo"], init["cnt"], off, cost, P1, P2, cfg.paths)
    label, disp, gap = wta_subpixel(cfg, init["lo"], init["cnt"], off, Cs, mode, tau)
    out = dict(init)
    out.update(off=off, cost=cost, P1=P1, P2=P2, Cs=Cs, label=label, disp=disp, gap=gap)
    return out


# ------------------------------------------------------- adjoint (not in the paper)
def softargmin(cfg: Cfg, lo, cnt, off, Cs, tau):
    _, disp, _ = wta_subpixel(cfg, lo, cnt, off, Cs, mode=2, tau=tau)
    return disp


def softargmin_backward(cfg: Cfg, lo, cnt, off, Cs, gd, tau):
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(off, dtype=np.int64)
    Cs = np.ascontiguousarray(Cs, dtype=np.float64)
    gd = np.ascontiguousarray(gd, dtype=np.float64).reshape(-1)
    out = np.zeros_like(Cs)
    lib().or_softargmin_backward(C.byref(cfg), lo.size, _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32),
                                 _ptr(off, C.c_int64), _ptr(Cs, C.c_double), _ptr(gd, C.c_double), tau,
                                 _ptr(out, C.c_double))
    return out


def sgm_backward(H, W, lo, cnt, off, cost, P1, P2, gCs, paths: int = 8):
    """(dLoss/dcost, dLoss/dP1, dLoss/dP2) from dLoss/dC_s, one direction at a time."""
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(off, dtype=np.int64)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    gCs = np.ascontiguousarray(gCs, dtype=np.float64)
    gC = np.zeros_like(cost)
    g1, g2 = C.c_double(0.0), C.c_double(0.0)
    for r in range(paths):
        lib().or_sgm_bounded_path_backward(H, W, _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32), _ptr(off, C.c_int64),
                                           _ptr(cost, C.c_double), float(P1), float(P2), r, _ptr(gCs, C.c_double),
                                           _ptr(gC, C.c_double), C.byref(g1), C.byref(g2))
    return gC, g1.value, g2.value


def cost_backward_views(cfg: Cfg, views, lo, cnt, off, gcost):
    views = np.ascontiguousarray(views, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(off, dtype=np.int64)
    gcost = np.ascontiguousarray(gcost, dtype=np.float64)
    out = np.zeros(views.shape, np.float64)
    lib().or_cost_backward_views(C.byref(cfg), _ptr(views, C.c_double), _ptr(lo, C.c_int32), _ptr(cnt, C.c_int32),
                                 _ptr(off, C.c_int64), _ptr(gcost, C.c_double), _ptr(out, C.c_double))
    return out


def loss_from_cost(cfg: Cfg, lo, cnt, cost, P1, P2, gd, tau):
    """Loss = sum_p gd(p) dhat(p) with dhat the soft-argmin of the SGM-aggregated cost."""
    off = offsets(cnt)
    Cs = sgm_bounded(cfg.H, cfg.W, lo, cnt, off, cost, P1, P2, cfg.paths)
    return float(np.dot(np.asarray(gd, np.float64).reshape(-1), softargmin(cfg, lo, cnt, off, Cs, tau)))


def backward(cfg: Cfg, views, lo, cnt, cost, P1, P2, gd, tau):
    """All gradients of Loss = sum_p gd(p) dhat(p): (dcost, dP1, dP2, dviews)."""
    off = offsets(cnt)
    Cs = sgm_bounded(cfg.H, cfg.W, lo, cnt, off, cost, P1, P2, cfg.paths)
    gCs = softargmin_backward(cfg, lo, cnt, off, Cs, gd, tau)
    gC, g1, g2 = sgm_backward(cfg.H, cfg.W, lo, cnt, off, cost, P1, P2, gCs, cfg.paths)
    gV = cost_backward_views(cfg, views, lo, cnt, off, gC)
    return gC, g1, g2, gV


def median3(disp: np.ndarray) -> np.ndarray:
    """3 x 3 median of a disparity map [H][W] (Sec. III-F), border pixels repeated; FP64."""
    d = np.ascontiguousarray(disp, dtype=np.float64)
    H, W = d.shape
    out = np.empty_like(d)
    lib().or_median3(H, W, _ptr(d, C.c_double), _ptr(out, C.c_double))
    return out
