"""The allocation-free cost volume (lfsgm_cost_volume_noalloc) against the regular entry
point.  It exists for callers that run under a fixed device-memory budget -- real-time
loops and plug-ins inside another application's memory pool -- and may not call
cudaMalloc, so it keeps its scratch in a static device array inside the library.  This
file is collected last so that a failure here cannot hide any other test's result."""
import ctypes as C

import numpy as np
import pytest

import lfsynth
from lf_helpers import RTOL, csr_rel_err, gather

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
