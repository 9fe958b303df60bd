"""The allocation-free cost volume (lfsgm_cost_volume_noalloc) against the regular entry
point.  It exists for callers that run under a fixed device-memory budget -- real-time
loops and plug-ins inside another application's memory pool -- and may not call
cudaMalloc, so it keeps its scratch in a static device array inside the library.  This
file is collected last so that a failure here cannot hide any other test's result."""
import ctypes as C

import numpy as np
import pytest

import lfsynth
import oracle
from lf_helpers import RTOL, csr_rel_err, gather, pad4_offsets

pytestmark = pytest.mark.gpu


def _windows_and_reference(lf, p, views_dev):
    import torch
    h = lf.lfsgm_create(p)
    N = p.H * p.W
    lo = torch.empty(N, dtype=torch.int32, device="cuda")
    cnt = torch.empty_like(lo)
    off = torch.empty(N + 1, dtype=torch.int64, device="cuda")
    nnz = lf.lfsgm_initial_disparity(h, views_dev, 0, 0, lo, cnt, off, want_nnz=True)
    ref = torch.empty(nnz, dtype=torch.float32, device="cuda")
    lf.lfsgm_cost_volume(h, views_dev, lo, cnt, off, ref)
    lf.lfsgm_sync(h)
    lf.lfsgm_destroy(h)
    return lo, cnt, off, ref


def test_noalloc_cost_volume_matches_regular_entry_point_twice(gpu_lib):
    import torch
    lf = gpu_lib
    for lf_index in (0, 1):           # two calls in a row, different light fields
        views, _, p = lfsynth.tiny(lf_index)
        vd = torch.from_numpy(views).cuda()
        lo, cnt, off, ref = _windows_and_reference(lf, p, vd)
        got = torch.full_like(ref, float("nan"))
        lf.lfsgm_cost_volume_noalloc(p, vd, lo, cnt, off, got)
        torch.cuda.synchronize()
        c = cnt.cpu().numpy()
        o = off.cpu().numpy()
        g = gather(got.cpu().numpy(), o, c)
        r = gather(ref.cpu().numpy(), o, c)
        assert not np.isnan(g).any()
        assert csr_rel_err(g, r, c) < RTOL


def test_noalloc_rejects_light_fields_beyond_the_static_scratch(gpu_lib):
    import torch
    lf = gpu_lib
    p = lfsynth.bench_params()        # 81 views of 512x512: 170 MB of census words
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    o = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(lf.LfsgmError, match="too large"):
        lf.lfsgm_cost_volume_noalloc(p, x, i, i, o, x)
    cfg = lf.make_config(p)
    assert lf.load().lfsgm_cost_volume_noalloc(C.byref(cfg), None, None, None, None, None, None) == 1


def _ragged(U, V, H, W, G, census_w, seed):
    """Generic random views and ragged windows of 1..min(G, 48) labels at random positions."""
    p = lfsynth.LFParams(U=U, V=V, H=H, W=W, census_w=census_w, dmin=-1.5, dmax=1.5, coarse_labels=9,
                         fine_labels=G, fine_radius=4)
    rng = np.random.default_rng(seed)
    views = rng.uniform(0.0, 1.0, (V, U, H, W)).astype(np.float32)
    cnt = rng.integers(1, min(G, 48) + 1, size=p.N).astype(np.int32)
    lo = (rng.random(p.N) * (G - cnt + 1)).astype(np.int32)
    return p, views, lo, cnt


def _noalloc_vs_oracle(lf, p, views, lo, cnt):
    import torch
    off = pad4_offsets(cnt)
    got = torch.full((int(off[-1]),), float("nan"), dtype=torch.float32, device="cuda")
    lf.lfsgm_cost_volume_noalloc(p, torch.from_numpy(views).cuda(), torch.from_numpy(lo).cuda(),
                                 torch.from_numpy(cnt).cuda(), torch.from_numpy(off).cuda(), got)
    torch.cuda.synchronize()
    g = gather(got.cpu().numpy(), off, cnt)
    off_o, cost_o = oracle.cost_volume(oracle.make_cfg(p), views, lo, cnt)
    r = gather(cost_o, off_o, cnt)
    assert not np.isnan(g).any()
    err = csr_rel_err(g, r, cnt)
    assert err < RTOL, err
    # the padding slots of every row are written with 0
    pad = np.ones(int(off[-1]), bool)
    pad[np.repeat(off[:-1], cnt) + (np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt))] = False
    assert (got.cpu().numpy()[pad] == 0.0).all()


@pytest.mark.parametrize("census_w,G", [(7, 48), (5, 37)])
def test_noalloc_ragged_wide_windows_match_oracle(gpu_lib, census_w, G):
    """Windows of 1..48 labels (wider than one 32-label chunk) at random positions, census 5x5
    and 7x7, compared element by element with the FP64 oracle (Eq. 12 + Eq. 15)."""
    p, views, lo, cnt = _ragged(5, 5, 40, 52, G, census_w, seed=300 + census_w)
    _noalloc_vs_oracle(gpu_lib, p, views, lo, cnt)


def test_noalloc_near_the_scratch_limit_matches_oracle(gpu_lib):
    """5x5 views of 400x416 with 48 fine labels: the scratch needs 33.3 MB of its 33.55 MB."""
    U = V = 5
    H, W, G = 400, 416, 48
    need = 256 + 256 + ((16 * U * V * G + 255) // 256) * 256 + 8 * U * V * H * W
    assert 0.99 * (32 << 20) < need <= (32 << 20)
    p, views, lo, cnt = _ragged(U, V, H, W, G, 7, seed=909)
    _noalloc_vs_oracle(gpu_lib, p, views, lo, cnt)
