"""Parity of the colour (C = 3) CUDA path with the FP64 oracle, through the C ABI.

Colour follows Sec. III-B/C: census of every channel with the Hamming distances summed, and the
l2 term as the Euclidean norm of the colour difference.  Bars as for one channel: census costs,
coarse maps, windows and labels bit-exact (labels: except where the oracle's own decision is a
near-tie); l2 and aggregated costs within 1e-5 relative to the per-pixel scale; sub-pixel
disparity within 1e-3 px; gradients per element within the bar of tests/test_gpu_backward.py."""
import dataclasses

import numpy as np
import pytest

import lfsynth
import oracle
from lf_helpers import (DISP_TOL, GRAD_ABS, GRAD_MASS, GRAD_TOL_P, RTOL, TIE_REL, best_of, csr_rel_err, err_stats,
                        gather, grad_tol, needed_rel, pad4_offsets)
from test_gpu_parity import (_check_end_to_end, _check_initial, _dev, _full_parity, _gpu_cost, _gpu_depth,
                             _np, _run_initial)

pytestmark = pytest.mark.gpu
TAU = 0.1


def _rgb_tiny(lf_index=0, **kw):
    return lfsynth.tiny(lf_index, params=lfsynth.tiny_params(channels=3, **kw))


@pytest.fixture(scope="module")
def rgb_case():
    views, gt, p = _rgb_tiny()
    assert views.shape == (5, 5, 3, 64, 64)
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    return views, gt, p, ref


@pytest.mark.parametrize("variant", ["default", "paper_4_views", "census7_odd_shape", "paths16", "sobel_edges"])
def test_rgb_initial_disparity_bitexact(gpu_lib, variant):
    kw = {"paper_4_views": dict(init_views=0),
          "census7_odd_shape": dict(H=37, W=45, census_w=7, coarse_labels=97, fine_labels=101, fine_radius=7),
          "paths16": dict(paths=16, H=41, W=53),
          "sobel_edges": dict(edge_threshold=1.5)}.get(variant, {})
    views, _, p = _rgb_tiny(**kw)
    cfg = oracle.make_cfg(p)
    if variant == "sobel_edges":
        e_rgb = oracle.sobel_edges(views[p.vc, p.uc], 1.5)
        e_0 = oracle.sobel_edges(views[p.vc, p.uc, 0], 1.5)
        assert 0.05 < e_rgb.mean() < 0.95 and (e_rgb & ~e_0).any()   # the other channels add edges
    ref = oracle.initial_disparity(cfg, views, None, p.p1_frac, p.p2_frac)
    _check_initial(_run_initial(gpu_lib, p, views), ref, p)


def test_rgb_cost_volume_tiny(gpu_lib, rgb_case):
    views, gt, p, ref = rgb_case
    off, c = _gpu_cost(gpu_lib, p, views, ref["lo"], ref["cnt"])
    err = csr_rel_err(gather(c, off, ref["cnt"]), ref["cost"], ref["cnt"])
    assert err < RTOL, err


@pytest.mark.parametrize("census_w", [5, 7])
def test_rgb_census_cost_is_exact_with_ties_and_signed_zeros(gpu_lib, census_w):
    """Census term alone, views quantised to 4 levels per channel with some zeros stored as -0.0:
    the summed Hamming distances are integers and must match exactly."""
    p = lfsynth.tiny_params(H=40, W=56, w_l2=0.0, w_census=1.0, census_w=census_w, channels=3)
    rng = np.random.default_rng(5)
    views = (rng.integers(0, 4, (p.V, p.U, 3, p.H, p.W)) / 3.0).astype(np.float32)
    views[(views == 0.0) & (rng.random(views.shape) < 0.25)] = -0.0
    cfg = oracle.make_cfg(p)
    lo = rng.integers(0, 60, p.N).astype(np.int32)
    cnt = rng.integers(1, 22, p.N).astype(np.int32)
    _, o_cost = oracle.cost_volume(cfg, views, lo, cnt)
    off, c = _gpu_cost(gpu_lib, p, views, lo, cnt)
    assert np.array_equal(gather(c, off, cnt).astype(np.float64), o_cost)
    g = _run_initial(gpu_lib, p, views)
    ref = oracle.initial_disparity(cfg, views, None, p.p1_frac, p.p2_frac)
    assert np.array_equal(g["maps"][:len(ref["arms"])], ref["maps"])


@pytest.mark.parametrize("shape", [(5, 5, 33, 47), (3, 3, 1, 40), (9, 9, 20, 1), (4, 4, 17, 29)])
def test_rgb_cost_volume_ragged_windows(gpu_lib, shape):
    U, V, H, W = shape
    p = lfsynth.LFParams(U=U, V=V, H=H, W=W, census_w=5, dmin=-2.0, dmax=2.0, coarse_labels=32,
                         fine_labels=81, fine_radius=5, channels=3)
    views = lfsynth.random_views(U, V, H, W, seed=H * W, channels=3)
    rng = np.random.default_rng(H + W)
    lo = rng.integers(0, 81, p.N).astype(np.int32)
    cnt = np.minimum(rng.integers(1, 40, p.N), 81 - lo).astype(np.int32)
    cnt[::7] = 81
    lo[::7] = 0
    lo[1::11] = 80
    cnt[1::11] = 1
    _, o_cost = oracle.cost_volume(oracle.make_cfg(p), views, lo, cnt)
    off, c = _gpu_cost(gpu_lib, p, views, lo, cnt)
    err = csr_rel_err(gather(c, off, cnt), o_cost, cnt)
    assert err < RTOL, err


def test_rgb_depth_end_to_end_tiny(gpu_lib, rgb_case):
    views, gt, p, ref = rgb_case
    g_label, g_disp, n = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


def test_rgb_depth_end_to_end_16_paths_and_edges(gpu_lib):
    views, gt, p = _rgb_tiny(1, paths=16, edge_threshold=1.5)
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


def test_rgb_bench_like_shape_full_parity(gpu_lib):
    """9x9 x 128x160 colour light field with the benchmark's method parameters (census 7x7, 100
    coarse labels, 31-label windows on a 401-label grid): every stage, every pixel."""
    views, gt, p = lfsynth.bench(params=lfsynth.bench_params(H=128, W=160, channels=3))
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    _full_parity(gpu_lib, views, p, ref)


def test_rgb_depth_host_matches_device(gpu_lib, rgb_case):
    import torch
    views, gt, p, ref = rgb_case
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    h = gpu_lib.lfsgm_create(p)
    vh = torch.from_numpy(np.ascontiguousarray(views)).pin_memory()
    dh = torch.empty(p.N, dtype=torch.float32).pin_memory()
    lh = torch.empty(p.N, dtype=torch.int32).pin_memory()
    gpu_lib.lfsgm_depth_host(h, vh, dh, lh)
    gpu_lib.lfsgm_destroy(h)
    assert np.array_equal(lh.numpy(), g_label)
    assert np.array_equal(dh.numpy(), g_disp, equal_nan=True)


@pytest.mark.parametrize("windows", ["narrow", "ragged"])
def test_rgb_backward_matches_oracle_adjoint(gpu_lib, windows):
    import torch
    p = lfsynth.LFParams(U=7, V=7, H=32, W=40, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=9,
                         fine_labels=41, fine_radius=8, w_l2=1.0, w_census=1.0 / 24, subpixel=2,
                         softmin_tau=TAU, channels=3)
    rng = np.random.default_rng(31)
    views = rng.uniform(0.0, 1.0, (7, 7, 3, 32, 40)).astype(np.float32)
    if windows == "narrow":
        lo = np.full(p.N, 12, np.int32)
        cnt = np.full(p.N, 16, np.int32)
    else:
        cnt = rng.choice(np.array([5, 16, 31, 33, 40], np.int32), size=p.N).astype(np.int32)
        lo = (rng.random(p.N) * (p.fine_labels - cnt + 1)).astype(np.int32)
    gd = rng.normal(size=p.N).astype(np.float32)
    cfg = oracle.make_cfg(p)
    off_o, cost_o = oracle.cost_volume(cfg, views, lo, cnt)
    P1, P2 = np.float32(0.05 * cost_o.mean()), np.float32(0.5 * cost_o.mean())
    gC_o, g1_o, g2_o, gV_o = oracle.backward(cfg, views, lo, cnt, cost_o, float(P1), float(P2), gd, TAU)
    L = gpu_lib.LightFieldDepth(p)
    L.lo.copy_(torch.from_numpy(lo))
    L.cnt.copy_(torch.from_numpy(cnt))
    L.off.copy_(torch.from_numpy(pad4_offsets(cnt)))
    vd = torch.from_numpy(views).cuda()
    L.cost_volume(vd)
    gcost = torch.empty_like(L.cost)
    gviews = torch.full_like(vd, float("nan"))
    g1 = torch.zeros(1, device="cuda")
    g2 = torch.zeros(1, device="cuda")
    gpu_lib.lfsgm_backward(L.h, vd, L.cost, L.lo, L.cnt, L.off, float(P1), float(P2), torch.from_numpy(gd).cuda(),
                           gcost, g1, g2, gviews)
    gpu_lib.lfsgm_sync(L.h)
    gC = gather(gcost.cpu().numpy(), pad4_offsets(cnt), cnt)
    gV = gviews.cpu().numpy()
    vs = np.abs(gV_o).max()
    # per element, the bar of tests/test_gpu_backward.py (view gradients grouped by channel plane)
    eC = needed_rel(gC, gC_o, cnt, GRAD_ABS)
    eV = needed_rel(gV, gV_o, np.full(p.U * p.V * 3, p.H * p.W), GRAD_ABS)
    tol = grad_tol(oracle.sgm_bounded(p.H, p.W, lo, cnt, off_o, cost_o, float(P1), float(P2)).max(), TAU)
    print(f"rgb backward {windows}, bar {tol:.2e}, needed relative tolerance: dcost", err_stats(eC),
          "dviews", err_stats(eV))
    assert eC.max() <= tol, err_stats(eC)
    assert eV.max() <= tol, err_stats(eV)
    mass = GRAD_MASS / GRAD_TOL_P * np.abs(gC_o).sum()
    assert abs(g1.item() - g1_o) <= GRAD_TOL_P * (abs(g1_o) + mass), (g1.item(), g1_o)
    assert abs(g2.item() - g2_o) <= GRAD_TOL_P * (abs(g2_o) + mass), (g2.item(), g2_o)
    # every channel of the reference view receives gradient
    assert all(np.abs(gV[p.vc, p.uc, ch]).max() > 0.1 * vs for ch in range(3))
    L.close()


def test_rgb_and_grey_light_fields_in_one_batch(gpu_lib):
    import torch
    members = [_rgb_tiny(0), lfsynth.tiny(1), _rgb_tiny(2, H=40, W=72)]
    views = [torch.from_numpy(v).cuda() for v, _, _ in members]
    b = gpu_lib.LightFieldBatch([m[2] for m in members], views, branches=2)
    disp = [d.cpu().numpy() for d in b.run()]
    torch.cuda.synchronize()
    b.close()
    for d, (v, _, p) in zip(disp, members):
        ref = oracle.depth(oracle.make_cfg(p), v, p1f=p.p1_frac, p2f=p.p2_frac)
        best = best_of(ref["Cs"], ref["off"], ref["cnt"], ref["label"], ref["lo"])
        decided = ref["gap"] > TIE_REL * np.maximum(1.0, np.abs(best))
        assert decided.sum() > 0.9 * p.N
        assert np.max(np.abs(d - ref["disp"])[decided]) < DISP_TOL, p.name


def test_rgb_is_unsupported_without_a_handle(gpu_lib):
    import torch
    p = lfsynth.tiny_params(channels=3)
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    o = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(gpu_lib.LfsgmError, match="colour"):
        gpu_lib.lfsgm_cost_volume_noalloc(p, x, i, i, o, x)
    with pytest.raises(gpu_lib.LfsgmError):
        gpu_lib.lfsgm_create(dataclasses.replace(p, channels=2))


def test_rgb_boundless_with_depth_dependent_radius_variants(gpu_lib):
    """Colour with the window variants: the boundary-less search (every window the whole range,
    list kernel only) and, separately, the depth-dependent border threshold."""
    views, gt, p = _rgb_tiny(3, H=40, W=44, boundless=1)
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)
    views, gt, p = _rgb_tiny(4, fine_radius=2, fine_radius_far=7)
    ref = oracle.initial_disparity(oracle.make_cfg(p), views, None, p.p1_frac, p.p2_frac)
    _check_initial(_run_initial(gpu_lib, p, views), ref, p)
