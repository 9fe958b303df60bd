"""Seeded synthetic light fields shaped like the method's workloads.

This module only makes inputs: it renders piecewise-planar scenes into a
``views[v][u][y][x]`` float32 array and returns the method's parameters for the
workload.  It holds none of the depth method's arithmetic and is shared by the
oracle side (tests, CPU baseline) and the CUDA side (tests, bench, smoke).

Geometry convention: a scene point seen at reference pixel (x, y) with
disparity d appears in view (u, v) at (x + (u-uc) d, y + (v-vc) d).  A view
pixel (X, Y) is rendered by solving, for every plane, for the reference point
that lands on it, keeping the nearest plane (largest d) whose back-projected
point lies inside its own region (the farthest plane fills holes), and sampling
that plane's texture there bilinearly.  Then Gaussian noise, an optional
vignetting gain and a clip to [0, 1] are applied.

Voronoi regions are rasterised at 1/4 px (the scene's region map is that raster).
Seeds: ``np.random.SeedSequence(seed).spawn(3)`` gives the texture, geometry and
noise streams; the workloads use ``seed = 1000 * workload_index + lf_index``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class LFParams:
    """Sizes and method parameters of one workload (names follow the paper)."""
    U: int
    V: int
    H: int
    W: int
    census_w: int
    dmin: float
    dmax: float
    coarse_labels: int          # Lc, inclusive grid over [dmin, dmax]
    fine_labels: int            # G, inclusive grid over [dmin, dmax]
    fine_radius: int            # lambda in fine labels (window = 2R+1 labels)
    init_views: int = 1         # 1: whole cross arms, 0: the 4 extreme views
    phi: float = 3.0            # fusion threshold (coarse labels)
    fill_passes: int = 2
    w_l2: float = 1.0
    w_census: float = -1.0      # -1 -> 1 / census bits
    p1_frac: float = 0.05
    p2_frac: float = 0.5
    subpixel: int = 1
    softmin_tau: float = 0.1
    paths: int = 8              # SGM directions: 8, or the paper's 16 (Sec. IV-C)
    edge_threshold: float = 0.0 # Sobel edge exclusion from the borders (Sec. III-D); 0 = off
    channels: int = 1           # 1 (grey) or 3 (RGB: views[v][u][c][y][x])
    boundless: int = 0          # 1: no initial map, every window is the whole range (Sec. IV-E)
    fine_radius_far: int = 0    # > 0: lambda at d = dmin, moving linearly to fine_radius at dmax
    uc: int = -1
    vc: int = -1
    name: str = ""

    def __post_init__(self):
        if self.uc < 0:
            self.uc = (self.U - 1) // 2
        if self.vc < 0:
            self.vc = (self.V - 1) // 2
        if self.w_census < 0:
            self.w_census = 1.0 / (self.census_w * self.census_w - 1)

    @property
    def N(self) -> int:
        return self.H * self.W

    @property
    def fine_step(self) -> float:
        return (self.dmax - self.dmin) / (self.fine_labels - 1)


@dataclasses.dataclass
class Plane:
    a: float          # disparity at the centre (cx, cy)
    b: float = 0.0    # slope over the image width
    c: float = 0.0    # slope over the image height

    def disp(self, x, y, W, H):
        return self.a + self.b * (x - 0.5 * (W - 1)) / W + self.c * (y - 0.5 * (H - 1)) / H


def _blur121(t: np.ndarray) -> np.ndarray:
    p = np.pad(t, 1, mode="edge")
    t = 0.25 * p[:-2, 1:-1] + 0.5 * p[1:-1, 1:-1] + 0.25 * p[2:, 1:-1]
    p = np.pad(t, ((0, 0), (1, 1)), mode="edge")
    return 0.25 * p[:, :-2] + 0.5 * p[:, 1:-1] + 0.25 * p[:, 2:]


def _sample(tex: np.ndarray, margin: int, idx: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bilinear lookup in texture ``idx`` at reference coordinates (clamped to the texture)."""
    _, th, tw = tex.shape
    gx = np.clip(x + margin, 0.0, tw - 1.000001)
    gy = np.clip(y + margin, 0.0, th - 1.000001)
    x0 = np.floor(gx).astype(np.int64)
    y0 = np.floor(gy).astype(np.int64)
    fx = gx - x0
    fy = gy - y0
    t00 = tex[idx, y0, x0]
    t10 = tex[idx, y0, x0 + 1]
    t01 = tex[idx, y0 + 1, x0]
    t11 = tex[idx, y0 + 1, x0 + 1]
    return (1 - fy) * ((1 - fx) * t00 + fx * t10) + fy * ((1 - fx) * t01 + fx * t11)


def render(p: LFParams, planes, region, textures, margin, noise_rng, sigma, vignette=False):
    """Render views[v][u][y][x] (float32; views[v][u][c][y][x] for colour textures) and the
    reference-view disparity (float64).

    ``region(i, x, y)`` -> bool array: is reference point (x, y) on plane i.
    ``textures[i]``: texture of plane i on the reference grid plus ``margin`` ([th][tw], or
    [C][th][tw] for C colour channels, each sampled at the same points)."""
    U, V, H, W = p.U, p.V, p.H, p.W
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    tex = np.stack(textures)
    colour = tex.ndim == 4
    C = tex.shape[1] if colour else 1
    views = np.zeros((V, U, C, H, W) if colour else (V, U, H, W), np.float32)
    gt = None
    for v in range(V):
        for u in range(U):
            a, b = u - p.uc, v - p.vc
            best_d = np.full((H, W), -np.inf)
            far_d = np.full((H, W), np.inf)
            best = [np.zeros((H, W), np.int64), np.zeros((H, W)), np.zeros((H, W))]
            far = [np.zeros((H, W), np.int64), np.zeros((H, W)), np.zeros((H, W))]
            for i, pl in enumerate(planes):
                # X = x + a*d(x,y), Y = y + b*d(x,y), with d affine in (x, y): 2x2 solve
                kx, ky = pl.b / W, pl.c / H
                k0 = pl.a - kx * 0.5 * (W - 1) - ky * 0.5 * (H - 1)
                m00, m01 = 1.0 + a * kx, a * ky
                m10, m11 = b * kx, 1.0 + b * ky
                r0, r1 = X - a * k0, Y - b * k0
                det = m00 * m11 - m01 * m10
                x = (m11 * r0 - m01 * r1) / det
                y = (m00 * r1 - m10 * r0) / det
                d = pl.disp(x, y, W, H)
                take = region(i, x, y) & (d > best_d)
                best_d = np.where(take, d, best_d)
                for arr, val in zip(best, (i, x, y)):
                    arr[take] = val if np.isscalar(val) else val[take]
                fall = d < far_d
                far_d = np.where(fall, d, far_d)
                for arr, val in zip(far, (i, x, y)):
                    arr[fall] = val if np.isscalar(val) else val[fall]
            hole = ~np.isfinite(best_d)
            idx, xs, ys = (np.where(hole, f, bb) for f, bb in zip(far, best))
            if colour:
                img = np.stack([_sample(tex[:, ch], margin, idx, xs, ys) for ch in range(C)])
            else:
                img = _sample(tex, margin, idx, xs, ys)
            if a == 0 and b == 0:
                gt = np.where(hole, far_d, best_d)
            if sigma > 0:
                img = img + noise_rng.normal(0.0, sigma, size=img.shape)
            if vignette:
                rho2 = (a * a + b * b) / float(max(p.uc, 1) ** 2 + max(p.vc, 1) ** 2)
                r2 = ((X - 0.5 * (W - 1)) ** 2 + (Y - 0.5 * (H - 1)) ** 2) / (
                    (0.5 * (W - 1)) ** 2 + (0.5 * (H - 1)) ** 2)
                img = img * (1.0 - 0.3 * rho2 * (0.5 + 0.5 * r2))
            views[v, u] = np.clip(img, 0.0, 1.0).astype(np.float32)
    return views, gt


def _streams(seed: int):
    ss = np.random.SeedSequence(seed).spawn(3)
    return [np.random.default_rng(s) for s in ss]


# ------------------------------------------------------------------ workloads
def tiny_params(**kw) -> LFParams:
    """5x5 x 64x64, census 5x5, coarse 32 labels on [-2,2], fine +-0.25 by 0.05."""
    d = dict(U=5, V=5, H=64, W=64, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=32,
             fine_labels=81, fine_radius=5, name="tiny 5x5x64x64")
    d.update(kw)
    return LFParams(**d)


def bench_params(**kw) -> LFParams:
    """9x9 x 512x512, census 7x7, coarse 100 labels on [-4,4] over 17 cross views,
    fine +-0.3 px by 0.02 px (31 labels, 401 on the whole range)."""
    d = dict(U=9, V=9, H=512, W=512, census_w=7, dmin=-4.0, dmax=4.0, coarse_labels=100,
             fine_labels=401, fine_radius=15, name="bench 9x9x512x512")
    d.update(kw)
    return LFParams(**d)


def plenoptic_params(**kw) -> LFParams:
    """15x15 x 434x625, census 7x7, coarse 64 labels on [-1.5,1.5] over 29 cross views,
    fine +-0.15 px by 0.01 px (31 labels, 301 on the whole range)."""
    d = dict(U=15, V=15, H=434, W=625, census_w=7, dmin=-1.5, dmax=1.5, coarse_labels=64,
             fine_labels=301, fine_radius=15, name="plenoptic 15x15x434x625")
    d.update(kw)
    return LFParams(**d)


def epfl_params(**kw) -> LFParams:
    """EPFL-shaped (Sec. IV-E): 3x3 x 541x376, narrow baseline (disparity in [-1, 1] px), 32 coarse
    labels over 5 cross views, fine +-0.3 px by 0.02 (101 labels).  The fine cost is l2 + census:
    with |u - uc| <= 1 the census term, sampled at the nearest integer shift, is the same for
    every label within half a pixel, so census alone cannot place these disparities."""
    d = dict(U=3, V=3, H=376, W=541, census_w=7, dmin=-1.0, dmax=1.0, coarse_labels=32,
             fine_labels=101, fine_radius=15, name="epfl 3x3x376x541")
    d.update(kw)
    return LFParams(**d)


def middlebury_params(**kw) -> LFParams:
    """Middlebury-shaped (Sec. IV-E): 7 views in a row (U=7, V=1) of a half-size 555x650 image,
    wide baseline (disparity in [0, 12] px per view step), census cost, boundary-less search
    (no initial map: every window is the whole range), 121 fine labels by 0.1 px (64 coarse
    labels, unused)."""
    d = dict(U=7, V=1, H=555, W=650, census_w=7, dmin=0.0, dmax=12.0, coarse_labels=64,
             fine_labels=121, fine_radius=5, boundless=1, w_l2=0.0, w_census=1.0,
             name="middlebury 7x1x555x650")
    d.update(kw)
    return LFParams(**d)


def tiny(lf_index: int = 0, params: LFParams | None = None):
    """Uniform-noise texture on 3 fronto-parallel planes (-1.5 background, 0.25 centre
    rectangle, 1.75 inner rectangle), noise sigma 0.01."""
    p = params or tiny_params()
    tex_rng, geo_rng, noise_rng = _streams(1000 * 0 + lf_index)
    margin = int(math.ceil(max(abs(p.dmin), abs(p.dmax)) * max(p.U, p.V))) + 2
    th, tw = p.H + 2 * margin, p.W + 2 * margin
    textures = [tex_rng.uniform(0.05, 0.95, size=(th, tw)) for _ in range(3)]
    if p.channels > 1:       # further channels drawn after the grey ones (grey scenes unchanged)
        extra = [[tex_rng.uniform(0.05, 0.95, size=(th, tw)) for _ in range(p.channels - 1)] for _ in range(3)]
        textures = [np.stack([t] + e) for t, e in zip(textures, extra)]
    planes = [Plane(-1.5), Plane(0.25), Plane(1.75)]
    H, W = p.H, p.W
    rects = [None, (W * 0.25, H * 0.25, W * 0.75, H * 0.75), (W * 0.40, H * 0.375, W * 0.60, H * 0.625)]

    def region(i, x, y):
        if rects[i] is None:
            return np.ones(x.shape, bool)
        x0, y0, x1, y1 = rects[i]
        return (x >= x0) & (x < x1) & (y >= y0) & (y < y1)

    views, gt = render(p, planes, region, textures, margin, noise_rng, 0.01)
    return views, gt, p


def voronoi_scene(p: LFParams, seed: int, n_planes: int, a_range, slope, clamp, sigma,
                  vignette=False):
    tex_rng, geo_rng, noise_rng = _streams(seed)
    margin = int(math.ceil(max(abs(p.dmin), abs(p.dmax)) * max(p.U, p.V))) + 2
    th, tw = p.H + 2 * margin, p.W + 2 * margin
    textures = [_blur121(tex_rng.uniform(0.0, 1.0, size=(th, tw))) for _ in range(n_planes)]
    if p.channels > 1:       # further channels drawn after the grey ones (grey scenes unchanged)
        extra = [[_blur121(tex_rng.uniform(0.0, 1.0, size=(th, tw))) for _ in range(p.channels - 1)]
                 for _ in range(n_planes)]
        textures = [np.stack([t] + e) for t, e in zip(textures, extra)]
    sites = np.stack([geo_rng.uniform(0, p.W, n_planes), geo_rng.uniform(0, p.H, n_planes)], 1)
    planes = []
    for _ in range(n_planes):
        a = geo_rng.uniform(*a_range)
        b = geo_rng.uniform(-slope, slope)
        c = geo_rng.uniform(-slope, slope)
        # keep the plane inside [-clamp, clamp] over the image
        ext = 0.5 * (abs(b) + abs(c))
        a = float(np.clip(a, -clamp + ext, clamp - ext))
        planes.append(Plane(a, b, c))

    # Voronoi cells of the sites, rasterised at 1/4 px over the texture domain
    q = 4
    gy, gx = np.mgrid[0:th * q, 0:tw * q].astype(np.float32) / q - margin
    d2 = np.stack([(gx - sites[j, 0]) ** 2 + (gy - sites[j, 1]) ** 2 for j in range(n_planes)])
    cell = np.argmin(d2, axis=0).astype(np.int8)
    del d2, gx, gy

    def region(i, x, y):
        qx = np.clip(np.rint((x + margin) * q).astype(np.int64), 0, tw * q - 1)
        qy = np.clip(np.rint((y + margin) * q).astype(np.int64), 0, th * q - 1)
        return cell[qy, qx] == i

    views, gt = render(p, planes, region, textures, margin, noise_rng, sigma, vignette)
    return views, gt


def bench(lf_index: int = 0, params: LFParams | None = None):
    """8 slanted textured planes on the Voronoi cells of 8 seeded sites, disparity in
    [-4, 4] px, texture = uniform noise blurred by [1,2,1]/4, noise sigma 0.01."""
    p = params or bench_params()
    views, gt = voronoi_scene(p, 1000 * 1 + lf_index, 8, (-3.4, 3.4), 0.5, 4.0, 0.01)
    return views, gt, p


def plenoptic(lf_index: int = 0, params: LFParams | None = None):
    """8 planes, disparity in [-1.5, 1.5] px, noise sigma 0.02, vignetting on outer views."""
    p = params or plenoptic_params()
    views, gt = voronoi_scene(p, 1000 * 2 + lf_index, 8, (-1.2, 1.2), 0.3, 1.5, 0.02, vignette=True)
    return views, gt, p


def epfl(lf_index: int = 0, params: LFParams | None = None):
    """8 slanted planes with disparity in [-0.9, 0.9] px, noise sigma 0.01."""
    p = params or epfl_params()
    views, gt = voronoi_scene(p, 1000 * 5 + lf_index, 8, (-0.8, 0.8), 0.2, 0.9, 0.01)
    return views, gt, p


def middlebury(lf_index: int = 0, params: LFParams | None = None):
    """8 slanted planes with disparity in [0.5, 11.5] px per view step, noise sigma 0.01."""
    p = params or middlebury_params()
    views, gt = voronoi_scene(p, 1000 * 6 + lf_index, 8, (1.5, 10.5), 1.0, 11.5, 0.01)
    return views, gt, p


def integer_planes(U=5, V=5, H=48, W=48, disps=(-1.0, 0.0, 1.0), seed=7, **kw):
    """Noise-free fronto-parallel planes with integer disparity: every view is an exact
    integer shift of a seeded uniform texture (nested rectangles, one per plane)."""
    d = dict(U=U, V=V, H=H, W=W, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=33,
             fine_labels=81, fine_radius=5, name=f"integer planes {U}x{V}x{H}x{W}")
    d.update(kw)
    p = LFParams(**d)
    tex_rng, _, noise_rng = _streams(seed)
    margin = int(math.ceil(max(abs(p.dmin), abs(p.dmax)) * max(p.U, p.V))) + 2
    th, tw = p.H + 2 * margin, p.W + 2 * margin
    textures = [tex_rng.uniform(0.05, 0.95, size=(th, tw)) for _ in disps]
    if p.channels > 1:       # further channels drawn after the grey ones (grey scenes unchanged)
        extra = [[tex_rng.uniform(0.05, 0.95, size=(th, tw)) for _ in range(p.channels - 1)] for _ in disps]
        textures = [np.stack([t] + e) for t, e in zip(textures, extra)]
    order = np.argsort(disps)
    planes = [Plane(float(disps[i])) for i in order]
    n = len(planes)

    def region(i, x, y):
        if i == 0:
            return np.ones(x.shape, bool)
        f = 0.5 * i / n
        return (x >= W * f) & (x < W * (1 - f)) & (y >= H * f) & (y < H * (1 - f))

    views, gt = render(p, planes, region, textures, margin, noise_rng, 0.0)
    return views, gt, p


def random_views(U, V, H, W, seed=0, lo=0.0, hi=1.0, channels=1):
    """Plain i.i.d. uniform views (for stage-level tests that need no scene);
    [V][U][C][H][W] when ``channels`` > 1."""
    rng = np.random.default_rng(seed)
    shape = (V, U, H, W) if channels == 1 else (V, U, channels, H, W)
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


WORKLOADS = {"tiny": tiny, "bench": bench, "plenoptic": plenoptic, "epfl": epfl, "middlebury": middlebury}
PARAMS = {"tiny": tiny_params, "bench": bench_params, "plenoptic": plenoptic_params, "epfl": epfl_params,
          "middlebury": middlebury_params}


# ------------------------------------------------------------------ device-side rendering
def _scene(p: LFParams, seed: int, n_planes: int, a_range, slope, clamp):
    """Textures, Voronoi sites and planes of a Voronoi scene (the draws of ``voronoi_scene``)."""
    tex_rng, geo_rng, _ = _streams(seed)
    margin = int(math.ceil(max(abs(p.dmin), abs(p.dmax)) * max(p.U, p.V))) + 2
    th, tw = p.H + 2 * margin, p.W + 2 * margin
    textures = [_blur121(tex_rng.uniform(0.0, 1.0, size=(th, tw))) for _ in range(n_planes)]
    sites = np.stack([geo_rng.uniform(0, p.W, n_planes), geo_rng.uniform(0, p.H, n_planes)], 1)
    planes = []
    for _ in range(n_planes):
        a = geo_rng.uniform(*a_range)
        b = geo_rng.uniform(-slope, slope)
        c = geo_rng.uniform(-slope, slope)
        ext = 0.5 * (abs(b) + abs(c))
        planes.append(Plane(float(np.clip(a, -clamp + ext, clamp - ext)), b, c))
    return textures, sites, planes, margin


def voronoi_scene_torch(p: LFParams, seed: int, n_planes: int, a_range, slope, clamp, sigma,
                        vignette=False, device="cpu", noise_seed=None):
    """The scene of ``voronoi_scene`` rendered with torch on ``device`` (float64 geometry).

    Same textures, sites and planes; the Voronoi cell of a point is that of its nearest 1/4-px
    raster position, computed directly instead of through the raster.  The noise comes from a
    ``torch.Generator`` seeded with ``noise_seed`` (default: ``seed``), so it differs from the
    NumPy stream of ``voronoi_scene``; with ``sigma = 0`` both renderers agree up to rounding.
    Returns views [V][U][H][W] float32 on ``device``."""
    import torch
    dev = torch.device(device)
    f64 = torch.float64
    textures, sites, planes, margin = _scene(p, seed, n_planes, a_range, slope, clamp)
    U, V, H, W = p.U, p.V, p.H, p.W
    tex = torch.from_numpy(np.stack(textures)).to(dev)
    ntex, th, tw = tex.shape
    flat = tex.reshape(-1)
    sx = torch.tensor(sites[:, 0], dtype=f64, device=dev).view(-1, 1, 1, 1)
    sy = torch.tensor(sites[:, 1], dtype=f64, device=dev).view(-1, 1, 1, 1)
    Y, X = torch.meshgrid(torch.arange(H, dtype=f64, device=dev), torch.arange(W, dtype=f64, device=dev),
                          indexing="ij")
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed if noise_seed is None else noise_seed)
    q = 4

    def cell(x, y):
        qx = torch.clamp(torch.round((x + margin) * q), 0, tw * q - 1) / q - margin
        qy = torch.clamp(torch.round((y + margin) * q), 0, th * q - 1) / q - margin
        d2 = (qx.unsqueeze(0) - sx) ** 2 + (qy.unsqueeze(0) - sy) ** 2
        return torch.argmin(d2, dim=0)

    def sample(idx, x, y):
        gx = torch.clamp(x + margin, 0.0, tw - 1.000001)
        gy = torch.clamp(y + margin, 0.0, th - 1.000001)
        x0 = torch.floor(gx)
        y0 = torch.floor(gy)
        fx, fy = gx - x0, gy - y0
        base = idx * (th * tw) + y0.long() * tw + x0.long()
        t00, t10 = flat[base], flat[base + 1]
        t01, t11 = flat[base + tw], flat[base + tw + 1]
        return (1 - fy) * ((1 - fx) * t00 + fx * t10) + fy * ((1 - fx) * t01 + fx * t11)

    views = torch.empty((V, U, H, W), dtype=torch.float32, device=dev)
    a = (torch.arange(U, dtype=f64, device=dev) - p.uc).view(U, 1, 1)     # one row of views at a time
    if vignette:
        r2 = ((X - 0.5 * (W - 1)) ** 2 + (Y - 0.5 * (H - 1)) ** 2) / ((0.5 * (W - 1)) ** 2 + (0.5 * (H - 1)) ** 2)
    for v in range(V):
        b = float(v - p.vc)
        best_d = torch.full((U, H, W), -float("inf"), dtype=f64, device=dev)
        far_d = torch.full((U, H, W), float("inf"), dtype=f64, device=dev)
        bi = torch.zeros((U, H, W), dtype=torch.long, device=dev)
        fi = torch.zeros_like(bi)
        bx, by, fxv, fyv = (torch.zeros((U, H, W), dtype=f64, device=dev) for _ in range(4))
        for i, pl in enumerate(planes):
            # X = x + a*d(x,y), Y = y + b*d(x,y), with d affine in (x, y): 2x2 solve per view
            kx, ky = pl.b / W, pl.c / H
            k0 = pl.a - kx * 0.5 * (W - 1) - ky * 0.5 * (H - 1)
            m00, m01 = 1.0 + a * kx, a * ky
            m10, m11 = b * kx, 1.0 + b * ky
            r0, r1 = X - a * k0, Y - b * k0
            det = m00 * m11 - m01 * m10
            x = (m11 * r0 - m01 * r1) / det
            y = (m00 * r1 - m10 * r0) / det
            d = pl.disp(x, y, W, H)
            take = (cell(x, y) == i) & (d > best_d)
            best_d = torch.where(take, d, best_d)
            bi = torch.where(take, torch.full_like(bi, i), bi)
            bx = torch.where(take, x, bx)
            by = torch.where(take, y, by)
            fall = d < far_d
            far_d = torch.where(fall, d, far_d)
            fi = torch.where(fall, torch.full_like(fi, i), fi)
            fxv = torch.where(fall, x, fxv)
            fyv = torch.where(fall, y, fyv)
        hole = ~torch.isfinite(best_d)
        img = sample(torch.where(hole, fi, bi), torch.where(hole, fxv, bx), torch.where(hole, fyv, by))
        if sigma > 0:
            img = img + sigma * torch.randn((U, H, W), generator=gen, dtype=f64, device=dev)
        if vignette:
            rho2 = (a * a + b * b) / float(max(p.uc, 1) ** 2 + max(p.vc, 1) ** 2)
            img = img * (1.0 - 0.3 * rho2 * (0.5 + 0.5 * r2))
        views[v] = torch.clamp(img, 0.0, 1.0).to(torch.float32)
    return views


# Shape classes of the mixed batch: 5x5 x 256^2, 9x9 x 512^2, 4x4 camera-array frames of
# 1280x720 and 15x15 x 434x625 plenoptic images, each with its own disparity range, fine grid
# and scene statistics.
BATCH_CLASSES = (
    dict(U=5, V=5, H=256, W=256, dmin=-2.0, dmax=2.0, fine_labels=201, fine_radius=10,
         scene=((-1.7, 1.7), 0.4, 2.0, 0.01, False), name="5x5x256x256"),
    dict(U=9, V=9, H=512, W=512, dmin=-4.0, dmax=4.0, fine_labels=401, fine_radius=15,
         scene=((-3.4, 3.4), 0.5, 4.0, 0.01, False), name="9x9x512x512"),
    dict(U=4, V=4, H=720, W=1280, dmin=-6.0, dmax=6.0, fine_labels=241, fine_radius=8,
         scene=((-5.0, 5.0), 0.8, 6.0, 0.01, False), name="4x4x720x1280"),
    dict(U=15, V=15, H=434, W=625, dmin=-1.5, dmax=1.5, fine_labels=301, fine_radius=15,
         scene=((-1.2, 1.2), 0.3, 1.5, 0.02, True), name="15x15x434x625"),
)


def batch_params(i: int) -> LFParams:
    """Light field i of the mixed batch: shape class i mod 4, census 5x5 / 7x7 alternating
    every 4 light fields, coarse labels cycling 16, 32, 64, 128 every 8."""
    c = BATCH_CLASSES[i % 4]
    census = (5, 7)[(i // 4) % 2]
    lc = (16, 32, 64, 128)[(i // 8) % 4]
    return LFParams(U=c["U"], V=c["V"], H=c["H"], W=c["W"], census_w=census, dmin=c["dmin"], dmax=c["dmax"],
                    coarse_labels=lc, fine_labels=c["fine_labels"], fine_radius=c["fine_radius"],
                    name=f'{c["name"]} census {census} Lc {lc}')


def batch_lf(i: int, device="cpu", scale: float = 1.0):
    """Views of light field i of the mixed batch (seed 1000 * 4 + i), rendered on ``device``.
    ``scale`` < 1 shrinks H and W (for tests)."""
    p = batch_params(i)
    if scale != 1.0:
        p = dataclasses.replace(p, H=max(16, int(round(p.H * scale))), W=max(16, int(round(p.W * scale))))
    a_range, slope, clamp, sigma, vig = BATCH_CLASSES[i % 4]["scene"]
    views = voronoi_scene_torch(p, 1000 * 4 + i, 8, a_range, slope, clamp, sigma, vig, device=device)
    return views, p
