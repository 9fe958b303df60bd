"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: census/Hamming, coarse maps, windows and labels bit-exact (labels: except where the
oracle's own decision is a near-tie, gap <= 1e-5 * scale); l2 and aggregated costs within
1e-5 relative to the per-pixel scale; sub-pixel disparity within 1e-3 px."""
import dataclasses

import numpy as np
import pytest

import lfsynth
import oracle
from lf_helpers import (DISP_TOL, RTOL, TIE_REL, best_of, csr_rel_err, gather, label_mismatch,
                        pad4_offsets)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def tiny_case():
    views, gt, p = lfsynth.tiny()
    cfg = oracle.make_cfg(p)
    ref = oracle.depth(cfg, views, p1f=p.p1_frac, p2f=p.p2_frac)
    return views, gt, p, cfg, ref


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _np(t):
    return t.detach().cpu().numpy()


def _run_initial(lf, p, views, Pc=(0, 0)):
    import torch
    h = lf.lfsgm_create(p)
    N = p.H * p.W
    lo = torch.empty(N, dtype=torch.int32, device="cuda")
    cnt = torch.empty_like(lo)
    off = torch.empty(N + 1, dtype=torch.int64, device="cuda")
    dinit = torch.empty(N, dtype=torch.float32, device="cuda")
    maps = torch.full((4, N), -7, dtype=torch.int32, device="cuda")
    nnz = lf.lfsgm_initial_disparity(h, _dev(views), Pc[0], Pc[1], lo, cnt, off, dinit, maps, want_nnz=True)
    lf.lfsgm_sync(h)
    out = dict(lo=_np(lo), cnt=_np(cnt), off=_np(off), dinit=_np(dinit), maps=_np(maps), nnz=nnz)
    lf.lfsgm_destroy(h)
    return out


def _check_initial(g, ref, p):
    n = len(ref["arms"])
    assert np.array_equal(g["maps"][:n], ref["maps"]), "coarse WTA maps differ"
    assert np.array_equal(g["lo"], ref["lo"])
    assert np.array_equal(g["cnt"], ref["cnt"])
    rd = ref["dinit"].astype(np.float32)
    assert np.array_equal(np.isnan(g["dinit"]), np.isnan(rd))
    ok = ~np.isnan(rd)
    assert np.array_equal(g["dinit"][ok], rd[ok])
    assert np.array_equal(g["off"], pad4_offsets(ref["cnt"]))
    assert g["nnz"] == g["off"][-1]
    assert np.all(g["off"][:-1] % 4 == 0)


# --------------------------------------------------------------------- initial pass
def test_initial_disparity_tiny_bitexact(gpu_lib, tiny_case):
    views, gt, p, cfg, ref = tiny_case
    g = _run_initial(gpu_lib, p, views)
    _check_initial(g, ref, p)


@pytest.mark.parametrize("variant", ["explicit_pen", "paper_4_views", "census7_odd_shape", "one_pass",
                                     "row_lf", "max_coarse_labels", "two_coarse_labels", "paths16",
                                     "sobel_edges"])
def test_initial_disparity_variants(gpu_lib, variant):
    Pc = (0, 0)
    if variant == "explicit_pen":
        views, _, p = lfsynth.tiny()
        Pc = (2, 9)
    elif variant == "paper_4_views":
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(init_views=0))
    elif variant == "census7_odd_shape":
        p = lfsynth.tiny_params(H=37, W=45, census_w=7, coarse_labels=97, fine_labels=101, fine_radius=7)
        views, _, p = lfsynth.tiny(params=p)
    elif variant == "one_pass":
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(fill_passes=1, phi=1.0))
    elif variant == "max_coarse_labels":   # Lc = 256: eight labels per lane, 16-byte rows
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(coarse_labels=256))
    elif variant == "two_coarse_labels":   # the smallest grid: the label step is the whole range
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(coarse_labels=2))
    elif variant == "paths16":             # the paper's 16 SGM directions (Sec. IV-C)
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(paths=16, H=41, W=53))
    elif variant == "sobel_edges":         # edge exclusion from the borders (Sec. III-D)
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(edge_threshold=1.5))
        assert 0.05 < oracle.sobel_edges(views[p.vc, p.uc], 1.5).mean() < 0.95
    else:  # a 3-D light field: one row of 7 views (Middlebury-like)
        p = lfsynth.tiny_params(U=7, V=1, H=30, W=70, coarse_labels=130)
        views, _, p = lfsynth.tiny(params=p)
    cfg = oracle.make_cfg(p)
    pens = None if Pc[0] <= 0 else [Pc] * 4
    ref = oracle.initial_disparity(cfg, views, pens, p.p1_frac, p.p2_frac)
    g = _run_initial(gpu_lib, p, views, Pc)
    _check_initial(g, ref, p)


# ----------------------------------------------------------------------- cost volume
def _gpu_cost(lf, p, views, lo, cnt, row_kw=0):
    import torch
    h = lf.lfsgm_create(p)
    if row_kw:
        lf.lfsgm_set_tuning(h, row_kw, 16)
    off = pad4_offsets(cnt)
    cost = torch.full((int(off[-1]),), float("nan"), dtype=torch.float32, device="cuda")
    lf.lfsgm_cost_volume(h, _dev(views), _dev(lo, torch.int32), _dev(cnt, torch.int32), _dev(off), cost)
    lf.lfsgm_sync(h)
    lf.lfsgm_destroy(h)
    c = _np(cost)
    # padding slots are written with 0
    pad = np.ones(c.size, bool)
    pad[np.repeat(off[:-1], cnt) + (np.arange(int(np.sum(cnt))) - np.repeat(np.cumsum(cnt) - cnt, cnt))] = False
    assert np.all(c[pad] == 0.0)
    return off, c


def test_cost_volume_tiny(gpu_lib, tiny_case):
    views, gt, p, cfg, ref = tiny_case
    off, c = _gpu_cost(gpu_lib, p, views, ref["lo"], ref["cnt"])
    err = csr_rel_err(gather(c, off, ref["cnt"]), ref["cost"], ref["cnt"])
    assert err < RTOL, err


@pytest.mark.parametrize("row_kw", [36, 44])
def test_cost_volume_with_each_row_span(gpu_lib, tiny_case, row_kw):
    """The speed knobs (row kernel label span 36 / 44, list kernel CTAs per SM) change which kernel
    computes a window, not the cost: both match the oracle (Eq. 12 + Eq. 15)."""
    views, gt, p, cfg, ref = tiny_case
    off, c = _gpu_cost(gpu_lib, p, views, ref["lo"], ref["cnt"], row_kw=row_kw)
    err = csr_rel_err(gather(c, off, ref["cnt"]), ref["cost"], ref["cnt"])
    assert err < RTOL, err
    h = gpu_lib.lfsgm_create(p)
    with pytest.raises(gpu_lib.LfsgmError, match="row_kw"):
        gpu_lib.lfsgm_set_tuning(h, 40, 0)
    gpu_lib.lfsgm_destroy(h)


def test_cost_census_only_is_exact(gpu_lib):
    views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(w_l2=0.0, w_census=1.0, census_w=7))
    cfg = oracle.make_cfg(p)
    rng = np.random.default_rng(1)
    lo = rng.integers(0, 60, p.N).astype(np.int32)
    cnt = rng.integers(1, 22, p.N).astype(np.int32)
    o_off, o_cost = oracle.cost_volume(cfg, views, lo, cnt)
    off, c = _gpu_cost(gpu_lib, p, views, lo, cnt)
    assert np.array_equal(gather(c, off, cnt).astype(np.float64), o_cost)


@pytest.mark.parametrize("census_w", [5, 7])
def test_census_with_ties_and_signed_zeros_is_exact(gpu_lib, census_w):
    """Views quantised to 4 levels (many equal neighbours) with a quarter of the zeros stored as
    -0.0: xi = [centre > neighbour] is false for equal values, +0 and -0 included (Eq. 3)."""
    p = lfsynth.tiny_params(U=5, V=5, H=40, W=56, w_l2=0.0, w_census=1.0, census_w=census_w)
    rng = np.random.default_rng(3)
    views = (rng.integers(0, 4, (p.V, p.U, p.H, p.W)) / 3.0).astype(np.float32)
    neg = (views == 0.0) & (rng.random(views.shape) < 0.25)
    views[neg] = -0.0
    assert np.signbit(views).any()
    cfg = oracle.make_cfg(p)
    lo = rng.integers(0, 60, p.N).astype(np.int32)
    cnt = rng.integers(1, 22, p.N).astype(np.int32)
    o_off, o_cost = oracle.cost_volume(cfg, views, lo, cnt)
    off, c = _gpu_cost(gpu_lib, p, views, lo, cnt)
    assert np.array_equal(gather(c, off, cnt).astype(np.float64), o_cost)
    g = _run_initial(gpu_lib, p, views)
    ref = oracle.initial_disparity(cfg, views, None, p.p1_frac, p.p2_frac)
    assert np.array_equal(g["maps"][:len(ref["arms"])], ref["maps"])


@pytest.mark.parametrize("shape", [(5, 5, 33, 47), (3, 3, 1, 40), (9, 9, 20, 1), (4, 4, 17, 29)])
def test_cost_volume_ragged_windows(gpu_lib, shape):
    U, V, H, W = shape
    p = lfsynth.LFParams(U=U, V=V, H=H, W=W, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=32,
                         fine_labels=81, fine_radius=5)
    views = lfsynth.random_views(U, V, H, W, seed=H * W)
    rng = np.random.default_rng(H + W)
    lo = rng.integers(0, 81, p.N).astype(np.int32)
    cnt = np.minimum(rng.integers(1, 40, p.N), 81 - lo).astype(np.int32)
    cnt[::7] = 81
    lo[::7] = 0                      # whole-range pixels
    lo[1::11] = 80
    cnt[1::11] = 1                   # one-label windows at the top of the range
    cfg = oracle.make_cfg(p)
    _, o_cost = oracle.cost_volume(cfg, views, lo, cnt)
    off, c = _gpu_cost(gpu_lib, p, views, lo, cnt)
    err = csr_rel_err(gather(c, off, cnt), o_cost, cnt)
    assert err < RTOL, err


def test_cost_volume_max_fine_labels(gpu_lib):
    """G = 4096 fine labels (the largest grid): ragged windows anywhere in the range, including
    whole-range pixels (4096 labels, 128 list chunks each) and windows at both ends."""
    p = lfsynth.LFParams(U=5, V=5, H=24, W=40, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=32,
                         fine_labels=4096, fine_radius=15)
    views = lfsynth.random_views(5, 5, 24, 40, seed=11)
    rng = np.random.default_rng(12)
    lo = rng.integers(0, 4096, p.N).astype(np.int32)
    cnt = np.minimum(rng.integers(1, 40, p.N), 4096 - lo).astype(np.int32)
    cnt[::53] = 4096
    lo[::53] = 0
    lo[5::17] = 0
    lo[9::19] = 4096 - cnt[9::19]
    cfg = oracle.make_cfg(p)
    _, o_cost = oracle.cost_volume(cfg, views, lo, cnt)
    off, c = _gpu_cost(gpu_lib, p, views, lo, cnt)
    err = csr_rel_err(gather(c, off, cnt), o_cost, cnt)
    assert err < RTOL, err


# ------------------------------------------------------------------------------ SGM
def _gpu_sgm(lf, p, cost32, lo, cnt, P1, P2, split=0):
    import torch
    h = lf.lfsgm_create(p)
    lf.lfsgm_set_sgm_split(h, split)
    off = pad4_offsets(cnt)
    full = np.zeros(int(off[-1]), np.float32)
    full[np.repeat(off[:-1], cnt) + (np.arange(int(np.sum(cnt))) - np.repeat(np.cumsum(cnt) - cnt, cnt))] = cost32
    agg = torch.full_like(_dev(full), float("nan"))
    lf.lfsgm_sgm_aggregate(h, _dev(full), _dev(lo, torch.int32), _dev(cnt, torch.int32), _dev(off), P1, P2, agg)
    lf.lfsgm_sync(h)
    lf.lfsgm_destroy(h)
    return off, _np(agg)


@pytest.mark.parametrize("paths", [8, 16])
def test_sgm_tiny(gpu_lib, tiny_case, paths):
    views, gt, p, cfg, ref = tiny_case
    p = dataclasses.replace(p, paths=paths)
    c32 = ref["cost"].astype(np.float32)
    P1, P2 = np.float32(ref["P1"]), np.float32(ref["P2"])
    o_Cs = oracle.sgm_bounded(p.H, p.W, ref["lo"], ref["cnt"], ref["off"], c32.astype(np.float64),
                              float(P1), float(P2), paths)
    off, agg = _gpu_sgm(gpu_lib, p, c32, ref["lo"], ref["cnt"], P1, P2)
    err = csr_rel_err(gather(agg, off, ref["cnt"]), o_Cs, ref["cnt"])
    assert err < RTOL, err


@pytest.mark.parametrize("paths", [8, 16])
def test_sgm_zero_penalties_is_paths_times_cost(gpu_lib, tiny_case, paths):
    views, gt, p, cfg, ref = tiny_case
    p = dataclasses.replace(p, paths=paths)
    c32 = ref["cost"].astype(np.float32)
    off, agg = _gpu_sgm(gpu_lib, p, c32, ref["lo"], ref["cnt"], 0.0, 0.0)
    g = gather(agg, off, ref["cnt"]).astype(np.float64)
    assert np.max(np.abs(g - paths * c32) / np.maximum(paths * c32, 1e-30)) < 1e-6


@pytest.mark.parametrize("paths", [8, 16])
@pytest.mark.parametrize("shape", [(1, 50), (50, 1), (2, 31), (3, 70), (23, 37), (64, 9)])
def test_sgm_ragged_and_wide_windows(gpu_lib, shape, paths):
    H, W = shape
    G = 150
    p = lfsynth.LFParams(U=3, V=3, H=H, W=W, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=32,
                         fine_labels=G, fine_radius=5, paths=paths)
    rng = np.random.default_rng(H * 100 + W)
    lo = rng.integers(0, G, H * W).astype(np.int32)
    cnt = np.minimum(rng.integers(1, 40, H * W), G - lo).astype(np.int32)
    wide = rng.random(H * W) < 0.15
    lo[wide] = rng.integers(0, 20, wide.sum())
    cnt[wide] = np.minimum(rng.integers(33, G, wide.sum()), G - lo[wide])   # multi-chunk rows
    off_o = oracle.offsets(cnt)
    cost = rng.uniform(0, 30, int(off_o[-1])).astype(np.float32)
    P1, P2 = np.float32(1.7), np.float32(9.5)
    o_Cs = oracle.sgm_bounded(H, W, lo, cnt, off_o, cost.astype(np.float64), float(P1), float(P2), paths)
    off, agg = _gpu_sgm(gpu_lib, p, cost, lo, cnt, P1, P2)
    err = csr_rel_err(gather(agg, off, cnt), o_Cs, cnt)
    assert err < RTOL, err
    # scanlines crossing two or more wide windows split across a CTA's warps: the same bits
    _, agg2 = _gpu_sgm(gpu_lib, p, cost, lo, cnt, P1, P2, split=2)
    assert np.array_equal(agg, agg2, equal_nan=True)


_DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1),
         (2, 1), (-2, -1), (2, -1), (-2, 1), (1, 2), (-1, -2), (1, -2), (-1, 2)]


def _wide_per_scanline(wide, paths):
    """Windows wider than 32 labels on each scanline (keyed by direction and start pixel: walk back
    from a pixel until its predecessor leaves the image)."""
    H, W = wide.shape
    counts = {}
    for y, x in zip(*np.nonzero(wide)):
        for r, (dx, dy) in enumerate(_DIRS[:paths]):
            tx = x // dx if dx > 0 else ((W - 1 - x) // -dx if dx < 0 else 1 << 30)
            ty = y // dy if dy > 0 else ((H - 1 - y) // -dy if dy < 0 else 1 << 30)
            t = min(tx, ty)
            key = (r, x - t * dx, y - t * dy)
            counts[key] = counts.get(key, 0) + 1
    return np.array(list(counts.values()))


@pytest.mark.parametrize("paths", [8, 16])
def test_sgm_split_scanlines_give_the_same_bits(gpu_lib, paths):
    """lfsgm_set_sgm_split: a scanline that crosses many windows wider than 32 labels runs on all the
    warps of a CTA, which share each wide step's chunks.  Whole wide rows (one of whole-range
    windows, one the image's last) and columns, a narrow run inside a wide row, and scattered wide
    windows: the aggregate is the same bit for bit with the split off (the default), at the
    autotuner's threshold, at one that splits more scanlines, and at ones that qualify too many
    (none split), also in the recording form; and it matches the oracle."""
    import torch
    H, W, G = 40, 56, 150
    p = lfsynth.LFParams(U=3, V=3, H=H, W=W, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=32,
                         fine_labels=G, fine_radius=5, paths=paths)
    rng = np.random.default_rng(4056 + paths)
    lo = rng.integers(0, G, H * W).astype(np.int32)
    cnt = np.minimum(rng.integers(1, 33, H * W), G - lo).astype(np.int32)
    wide = (rng.random(H * W) < 0.04).reshape(H, W)
    wide[[3, 17, H - 1], :] = True
    wide[:, [0, 41]] = True
    wide[3, 10:30] = False
    wide = wide.ravel()
    lo[wide] = rng.integers(0, 20, wide.sum())
    cnt[wide] = np.minimum(rng.integers(33, G + 1, wide.sum()), G - lo[wide])
    lo.reshape(H, W)[17, :] = 0                      # a run of identical whole-range windows
    cnt.reshape(H, W)[17, :] = G
    per = _wide_per_scanline((cnt > 32).reshape(H, W), paths)
    assert 1 <= np.sum(per >= 24) <= 256 and np.sum(per >= 1) > 256    # split at 24, too many at 1
    off_o = oracle.offsets(cnt)
    cost = rng.uniform(0, 30, int(off_o[-1])).astype(np.float32)
    P1, P2 = np.float32(1.7), np.float32(9.5)
    o_Cs = oracle.sgm_bounded(H, W, lo, cnt, off_o, cost.astype(np.float64), float(P1), float(P2), paths)
    off = pad4_offsets(cnt)
    full = np.zeros(int(off[-1]), np.float32)
    full[np.repeat(off[:-1], cnt) + (np.arange(int(np.sum(cnt))) - np.repeat(np.cumsum(cnt) - cnt, cnt))] = cost
    cd, lod, cntd, offd = _dev(full), _dev(lo, torch.int32), _dev(cnt, torch.int32), _dev(off)
    h = gpu_lib.lfsgm_create(p)
    runs = []
    for min_wide, warps, rec in ((0, 4, False), (24, 4, False), (24, 8, False), (24, 2, False), (6, 4, False),
                                 (3, 8, False), (1, 4, False), (0, 4, True), (24, 8, True), (6, 2, True)):
        gpu_lib.lfsgm_set_sgm_split(h, min_wide)
        gpu_lib.lfsgm_set_sgm_warps(h, warps)
        agg = torch.full_like(cd, float("nan"))
        (gpu_lib.lfsgm_sgm_aggregate_record if rec else gpu_lib.lfsgm_sgm_aggregate)(h, cd, lod, cntd, offd, P1, P2, agg)
        runs.append(((min_wide, warps, rec), agg))
    with pytest.raises(gpu_lib.LfsgmError):
        gpu_lib.lfsgm_set_sgm_split(h, -1)
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)
    base = runs[0][1]
    for knobs, agg in runs[1:]:
        diff = torch.nonzero(base != agg).flatten()
        assert diff.numel() == 0, (knobs, int(diff.numel()), diff[:8].tolist())
    err = csr_rel_err(gather(_np(base), off, cnt), o_Cs, cnt)
    assert err < RTOL, err


def test_sgm_derived_penalties(gpu_lib, tiny_case):
    views, gt, p, cfg, ref = tiny_case
    c32 = ref["cost"].astype(np.float32)
    mean = float(c32.astype(np.float64).mean())
    o_Cs = oracle.sgm_bounded(p.H, p.W, ref["lo"], ref["cnt"], ref["off"], c32.astype(np.float64),
                              p.p1_frac * mean, p.p2_frac * mean)
    off, agg = _gpu_sgm(gpu_lib, p, c32, ref["lo"], ref["cnt"], -1.0, -1.0)
    err = csr_rel_err(gather(agg, off, ref["cnt"]), o_Cs, ref["cnt"])
    assert err < RTOL, err


# -------------------------------------------------------------------------------- WTA
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_wta_subpixel_on_identical_input(gpu_lib, tiny_case, mode):
    import torch
    views, gt, p, cfg, ref = tiny_case
    Cs32 = ref["Cs"].astype(np.float32)
    o_label, o_disp, _ = oracle.wta_subpixel(cfg, ref["lo"], ref["cnt"], ref["off"], Cs32.astype(np.float64),
                                             mode=mode, tau=p.softmin_tau)
    pp = lfsynth.tiny_params(subpixel=mode)
    h = gpu_lib.lfsgm_create(pp)
    off = pad4_offsets(ref["cnt"])
    full = np.zeros(int(off[-1]), np.float32)
    cnt = ref["cnt"]
    full[np.repeat(off[:-1], cnt) + (np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt))] = Cs32
    label = torch.empty(p.N, dtype=torch.int32, device="cuda")
    disp = torch.empty(p.N, dtype=torch.float32, device="cuda")
    gpu_lib.lfsgm_wta_subpixel(h, _dev(full), _dev(ref["lo"], torch.int32), _dev(cnt, torch.int32), _dev(off),
                               label, disp)
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)
    assert np.array_equal(_np(label), o_label)
    assert np.max(np.abs(_np(disp) - o_disp)) < DISP_TOL


# ---------------------------------------------------------------------- end to end
def _gpu_depth(lf, p, views):
    import torch
    h = lf.lfsgm_create(p)
    label = torch.empty(p.N, dtype=torch.int32, device="cuda")
    disp = torch.empty(p.N, dtype=torch.float32, device="cuda")
    lf.lfsgm_depth(h, _dev(views), disp, label)
    lf.lfsgm_sync(h)
    n = lf.lfsgm_launch_count(h)
    lf.lfsgm_destroy(h)
    return _np(label), _np(disp), n


def _check_end_to_end(g_label, g_disp, ref, p):
    best = best_of(ref["Cs"], ref["off"], ref["cnt"], ref["label"], ref["lo"])
    bad, ties = label_mismatch(g_label, ref["label"], ref["gap"], best)
    assert bad == 0, f"{bad} decided labels differ ({ties} near-ties differ)"
    same = g_label == ref["label"]
    assert np.max(np.abs(g_disp[same] - ref["disp"][same])) < DISP_TOL
    return ties


def test_depth_end_to_end_tiny(gpu_lib, tiny_case):
    views, gt, p, cfg, ref = tiny_case
    g_label, g_disp, n = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)
    assert n > 10


@pytest.mark.parametrize("kind", ["epfl", "middlebury"])
def test_depth_end_to_end_real_world_shapes(gpu_lib, kind):
    """EPFL-shaped (3x3 views) and Middlebury-shaped (a row of 7 views, boundary-less search)
    light fields, census cost only (Eq. 15), at reduced image size."""
    if kind == "epfl":
        views, gt, p = lfsynth.epfl(params=lfsynth.epfl_params(H=94, W=135))
    else:
        views, gt, p = lfsynth.middlebury(params=lfsynth.middlebury_params(H=70, W=81))
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


def test_depth_end_to_end_16_paths(gpu_lib):
    views, gt, p = lfsynth.tiny(params=lfsynth.tiny_params(paths=16))
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


def test_depth_end_to_end_paper_4_views(gpu_lib):
    """The paper's initial views (the four extreme views only): the whole-method chain transforms
    the inner cross views in its cost stage (the initial pass never touched them)."""
    views, gt, p = lfsynth.tiny(params=lfsynth.tiny_params(init_views=0))
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


def test_depth_end_to_end_integer_planes_exact(gpu_lib):
    views, gt, p = lfsynth.integer_planes(H=96, W=96)
    cfg = oracle.make_cfg(p)
    ref = oracle.depth(cfg, views)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


@pytest.mark.parametrize("shape", [(1, 1), (1, 70), (45, 1), (37, 129), (512, 512)])
def test_median_filter_bit_exact(gpu_lib, shape):
    """3 x 3 median (Sec. III-F) of an FP32 map with many ties: the selection is exact."""
    import torch
    H, W = shape
    p = lfsynth.tiny_params(H=H, W=W)
    rng = np.random.default_rng(H * 1000 + W)
    d = rng.normal(size=(H, W)).astype(np.float32)
    d[rng.random((H, W)) < 0.3] = 0.25
    h = gpu_lib.lfsgm_create(p)
    out = torch.full((H * W,), float("nan"), dtype=torch.float32, device="cuda")
    gpu_lib.lfsgm_median_filter(h, _dev(d.reshape(-1)), out)
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)
    ref = oracle.median3(d.astype(np.float64)).astype(np.float32)
    assert np.array_equal(_np(out).reshape(H, W), ref)


def test_median_filter_after_depth_matches_oracle(gpu_lib, tiny_case):
    """The paper's chain ends with the median: compare where the oracle's WTA decisions of the
    whole 3 x 3 neighbourhood are not near-ties."""
    import torch
    views, gt, p, cfg, ref = tiny_case
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    h = gpu_lib.lfsgm_create(p)
    out = torch.empty(p.N, dtype=torch.float32, device="cuda")
    gpu_lib.lfsgm_median_filter(h, _dev(g_disp), out)
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)
    o = oracle.median3(ref["disp"].reshape(p.H, p.W))
    best = best_of(ref["Cs"], ref["off"], ref["cnt"], ref["label"], ref["lo"])
    bad = (ref["gap"] <= TIE_REL * np.maximum(1.0, np.abs(best))).reshape(p.H, p.W)
    bad = np.pad(bad, 1, mode="edge")
    near = np.zeros((p.H, p.W), bool)
    for dy in range(3):
        for dx in range(3):
            near |= bad[dy:dy + p.H, dx:dx + p.W]
    assert (~near).mean() > 0.9
    assert np.max(np.abs(_np(out).reshape(p.H, p.W) - o)[~near]) < DISP_TOL


def test_depth_host_matches_device(gpu_lib, tiny_case):
    import torch
    views, gt, p, cfg, ref = tiny_case
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    h = gpu_lib.lfsgm_create(p)
    vh = torch.from_numpy(np.ascontiguousarray(views)).pin_memory()
    dh = torch.empty(p.N, dtype=torch.float32).pin_memory()
    lh = torch.empty(p.N, dtype=torch.int32).pin_memory()
    gpu_lib.lfsgm_depth_host(h, vh, dh, lh)
    gpu_lib.lfsgm_destroy(h)
    # the same kernels on the same input: bit-identical (the SGM's direction sum does not depend
    # on the order of its atomics)
    assert np.array_equal(lh.numpy(), g_label)
    assert np.array_equal(dh.numpy(), g_disp, equal_nan=True)


@pytest.mark.parametrize("paths", [8, 16])
def test_sgm_aggregate_is_reproducible_at_bench_shape(gpu_lib, paths):
    """9x9 x 512x512, 31-label windows: aggregations of the same cost volume are bit-identical (the
    8 or 16 directions add into C_s with atomics in whatever order they arrive), also across the
    SGM's warps-per-CTA speed knob."""
    import dataclasses

    import torch
    views, _, p = lfsynth.bench()
    p = dataclasses.replace(p, paths=paths)
    L = gpu_lib.LightFieldDepth(p)
    vd = torch.from_numpy(views).cuda()
    L.initial(vd)
    L.cost_volume(vd)
    nnz = int(L.off[-1].item())
    runs = []
    # three runs with the default CTA size, then one with each other size of the SGM's speed knob:
    # a scanline's arithmetic does not depend on which CTA runs it
    for w in (0, 0, 0, 2, 8):
        gpu_lib.lfsgm_set_sgm_warps(L.h, w)
        L.aggregate(-1.0, -1.0)
        torch.cuda.synchronize()
        runs.append(L.agg[:nnz].clone())
    assert gpu_lib.lfsgm_get_tuning(L.h)[2] == 8
    # and with the border scanlines that cross many whole-range windows split across a CTA's warps
    assert gpu_lib.lfsgm_get_sgm_split(L.h) == 0
    gpu_lib.lfsgm_set_sgm_split(L.h, 24)
    L.aggregate(-1.0, -1.0)
    torch.cuda.synchronize()
    runs.append(L.agg[:nnz].clone())
    gpu_lib.lfsgm_sync(L.h)
    with pytest.raises(gpu_lib.LfsgmError):
        gpu_lib.lfsgm_set_sgm_warps(L.h, 3)
    L.close()
    for r in runs[1:]:
        diff = torch.nonzero(runs[0] != r).flatten()
        assert diff.numel() == 0, (int(diff.numel()), diff[:8].tolist(), runs[0][diff[:8]].tolist(), r[diff[:8]].tolist())


def test_argument_errors_are_reported(gpu_lib, tiny_case):
    import torch
    views, gt, p, cfg, ref = tiny_case
    h = gpu_lib.lfsgm_create(p)
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    i = torch.zeros(16, dtype=torch.int32, device="cuda")
    o = torch.zeros(17, dtype=torch.int64, device="cuda")
    with pytest.raises(gpu_lib.LfsgmError, match="P2 >= P1|P1 <= P2"):
        gpu_lib.lfsgm_sgm_aggregate(h, x, i, i, o, 5.0, 1.0, x)
    with pytest.raises(gpu_lib.LfsgmError, match="P2 >= P1"):
        gpu_lib.lfsgm_initial_disparity(h, x, 5, 1, i, i, o)
    with pytest.raises(TypeError):
        gpu_lib.lfsgm_cost_volume(h, x, x, i, o, x)
    # windowed rows are read and written as 16-byte vectors: a shifted base is refused on the host
    with pytest.raises(gpu_lib.LfsgmError, match="16-byte aligned"):
        gpu_lib.lfsgm_wta_subpixel(h, x[1:], i, i, o, i, x)
    with pytest.raises(gpu_lib.LfsgmError, match="16-byte aligned"):
        gpu_lib.lfsgm_sgm_aggregate(h, x, i, i, o, -1.0, -1.0, x[2:])
    with pytest.raises(gpu_lib.LfsgmError, match="16-byte aligned"):
        gpu_lib.lfsgm_cost_volume(h, x, i, i, o, x[3:])
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)


# ------------------------------------------------------------- full size (bench shape)
@pytest.fixture(scope="session")
def bench_case():
    views, gt, p = lfsynth.bench()
    cfg = oracle.make_cfg(p)
    ref = oracle.depth(cfg, views, p1f=p.p1_frac, p2f=p.p2_frac)
    return views, gt, p, cfg, ref


def _full_parity(gpu_lib, views, p, ref):
    lf = gpu_lib.LightFieldDepth(p)
    vd = _dev(views)
    nnz = lf.initial(vd, want_nnz=True)
    g = dict(lo=_np(lf.lo), cnt=_np(lf.cnt), off=_np(lf.off), dinit=_np(lf.dinit), maps=_np(lf.maps), nnz=nnz)
    _check_initial(g, ref, p)
    lf.cost_volume(vd)
    cost = _np(lf.cost)
    err = csr_rel_err(gather(cost, g["off"], g["cnt"]), ref["cost"], g["cnt"])
    assert err < RTOL, err
    lf.aggregate(-1.0, -1.0)
    agg = _np(lf.agg)
    err = csr_rel_err(gather(agg, g["off"], g["cnt"]), ref["Cs"], g["cnt"])
    assert err < RTOL, err
    lf.wta()
    _check_end_to_end(_np(lf.label), _np(lf.disp), ref, p)
    lf.close()


def test_bench_shape_full_parity(gpu_lib, bench_case):
    """9x9 x 512x512, census 7x7, 100 coarse labels, 31-label windows: the same stage chain
    as the benchmark, compared with the oracle on every pixel."""
    views, gt, p, cfg, ref = bench_case
    _full_parity(gpu_lib, views, p, ref)


def test_plenoptic_shape_full_parity(gpu_lib):
    """15x15 x 434x625 (225 views, vignetting, noise 0.02), census 7x7, 64 coarse labels over 29
    views, 31-label windows on a 301-label grid: every pixel against the oracle."""
    views, gt, p = lfsynth.plenoptic()
    cfg = oracle.make_cfg(p)
    ref = oracle.depth(cfg, views, p1f=p.p1_frac, p2f=p.p2_frac)
    _full_parity(gpu_lib, views, p, ref)


def test_autotune_picks_valid_knobs_and_keeps_the_depth(gpu_lib, tiny_case):
    """lfsgm_autotune sets the handle's three speed knobs to values from their candidate sets
    (lfsgm_get_tuning reads them back), and the depth afterwards is the default knobs' depth: bit
    for bit with the default label span (the list kernel's CTA count and the SGM's CTA size do
    not change the arithmetic), else to rounding (a window may move between the row and the list
    kernel, which add the views in different FP32 orders)."""
    import torch
    views, gt, p, cfg, ref = tiny_case
    h = gpu_lib.lfsgm_create(p)
    vd = _dev(views)
    label0 = torch.empty(p.N, dtype=torch.int32, device="cuda")
    disp0 = torch.empty(p.N, dtype=torch.float32, device="cuda")
    gpu_lib.lfsgm_depth(h, vd, disp0, label0)
    kw, lc = gpu_lib.lfsgm_autotune(h, vd)
    assert kw in (36, 44) and lc in (0, 8, 12, 24)
    tuned = gpu_lib.lfsgm_get_tuning(h)
    assert tuned[:2] == (kw, lc) and tuned[2] in (2, 4, 8)
    assert gpu_lib.lfsgm_get_sgm_split(h) in (0, 24)
    label1 = torch.empty_like(label0)
    disp1 = torch.empty_like(disp0)
    gpu_lib.lfsgm_depth(h, vd, disp1, label1)
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)
    d0, d1, l0, l1 = _np(disp0), _np(disp1), _np(label0), _np(label1)
    if kw == 36:
        assert np.array_equal(l0, l1) and np.array_equal(d0, d1, equal_nan=True)
    else:
        same = l0 == l1
        assert np.mean(same) >= 0.99
        ok = same & np.isfinite(d0) & np.isfinite(d1)
        assert np.abs(d0[ok] - d1[ok]).max() <= 1e-3
