"""Window variants on the GPU against the oracle, through the C ABI: the depth-dependent border
threshold (Sec. IV-F; windows bit-exact) and the boundary-less search (Sec. IV-E; no initial map,
every window the whole range)."""
import dataclasses

import numpy as np
import pytest

import lfsynth
import oracle
from test_gpu_parity import _check_end_to_end, _check_initial, _gpu_depth, _run_initial

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("radii", [(2, 8), (8, 2), (5, 5), (0, 12)])
def test_depth_dependent_radius_windows_bitexact(gpu_lib, radii):
    R, R_far = radii
    views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(fine_radius=R, fine_radius_far=R_far))
    cfg = oracle.make_cfg(p)
    ref = oracle.initial_disparity(cfg, views, None, p.p1_frac, p.p2_frac)
    g = _run_initial(gpu_lib, p, views)
    _check_initial(g, ref, p)
    if R != R_far:
        assert len(np.unique(ref["cnt"][ref["cnt"] < p.fine_labels])) > 2     # the radius varies


def test_depth_dependent_radius_end_to_end(gpu_lib):
    views, _, p = lfsynth.tiny(1, params=lfsynth.tiny_params(fine_radius=3, fine_radius_far=9))
    ref = oracle.depth(oracle.make_cfg(p), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, _ = _gpu_depth(gpu_lib, p, views)
    _check_end_to_end(g_label, g_disp, ref, p)


def test_boundless_initial_pass_writes_whole_range_windows_only(gpu_lib):
    views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(boundless=1, edge_threshold=1.5))
    g = _run_initial(gpu_lib, p, views)
    assert np.all(g["lo"] == 0) and np.all(g["cnt"] == p.fine_labels)
    assert np.all(np.isnan(g["dinit"]))
    assert np.all(g["maps"] == -7)                     # untouched
    ref = oracle.initial_disparity(oracle.make_cfg(p), views, None, p.p1_frac, p.p2_frac)
    _check_initial(g, ref, p)


def test_boundless_depth_matches_oracle_with_fewer_launches(gpu_lib):
    views, _, p = lfsynth.tiny(2, params=lfsynth.tiny_params(H=48, W=56))
    pb = dataclasses.replace(p, boundless=1)
    ref = oracle.depth(oracle.make_cfg(pb), views, p1f=p.p1_frac, p2f=p.p2_frac)
    g_label, g_disp, n_free = _gpu_depth(gpu_lib, pb, views)
    _check_end_to_end(g_label, g_disp, ref, pb)
    _, _, n_bounded = _gpu_depth(gpu_lib, p, views)
    assert n_free < n_bounded - 5                      # no census / coarse cost / SGM / WTA / fill


@pytest.mark.parametrize("kind", ["corner_reference", "boundless"])
def test_depth_host_matches_device(gpu_lib, kind):
    """lfsgm_depth_host uploads the cross views first and the other views on a second stream
    (four rectangles of the view grid, some empty when the reference view sits in a corner);
    the result equals the device-buffer entry point."""
    import torch
    from test_gpu_parity import _dev, _np
    if kind == "corner_reference":
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(uc=0, vc=4, H=40, W=48))
    else:
        views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(boundless=1, H=40, W=48))
    h = gpu_lib.lfsgm_create(p)
    label = torch.empty(p.N, dtype=torch.int32, device="cuda")
    disp = torch.empty(p.N, dtype=torch.float32, device="cuda")
    gpu_lib.lfsgm_depth(h, _dev(views), disp, label)
    vh = torch.from_numpy(np.ascontiguousarray(views)).pin_memory()
    dh = torch.empty(p.N, dtype=torch.float32).pin_memory()
    lh = torch.empty(p.N, dtype=torch.int32).pin_memory()
    for _ in range(2):                                  # twice: the buffer is reused
        gpu_lib.lfsgm_depth_host(h, vh, dh, lh)
        assert np.array_equal(lh.numpy(), _np(label))
        assert np.max(np.abs(dh.numpy() - _np(disp))) < 1e-5
    gpu_lib.lfsgm_sync(h)
    gpu_lib.lfsgm_destroy(h)


def test_boundless_and_bounded_light_fields_in_one_batch(gpu_lib):
    """A batch branch shares its workspace between a boundary-less light field (no initial pass)
    and bounded ones (their cost stage reuses the initial pass's census planes)."""
    import torch
    from lf_helpers import DISP_TOL, TIE_REL, best_of
    members = [lfsynth.tiny(5, params=lfsynth.tiny_params(boundless=1, H=40, W=48)),
               lfsynth.tiny(6, params=lfsynth.tiny_params(H=48, W=40, init_views=0)),
               lfsynth.tiny(7, params=lfsynth.tiny_params(H=36, W=52, fine_radius=3, fine_radius_far=8))]
    views = [torch.from_numpy(v).cuda() for v, _, _ in members]
    b = gpu_lib.LightFieldBatch([m[2] for m in members], views, branches=1)
    disp = [d.cpu().numpy() for d in b.run()]
    torch.cuda.synchronize()
    b.close()
    for d, (v, _, p) in zip(disp, members):
        ref = oracle.depth(oracle.make_cfg(p), v, p1f=p.p1_frac, p2f=p.p2_frac)
        best = best_of(ref["Cs"], ref["off"], ref["cnt"], ref["label"], ref["lo"])
        decided = ref["gap"] > TIE_REL * np.maximum(1.0, np.abs(best))
        assert decided.sum() > 0.9 * p.N
        assert np.max(np.abs(d - ref["disp"])[decided]) < DISP_TOL, p.name
