"""The batch runner (one CUDA graph for many light fields of mixed shape) against the oracle
and against one-light-field launches.

Eight light fields of the mixed batch, shrunk to 15% of their size: all four shape classes,
census 5x5 and 7x7, coarse label counts 16, 32, 64 and 128.  A batch returns sub-pixel
disparities only, so a pixel is checked where the oracle's WTA decision is not a near-tie
(gap > 1e-5 * scale): there the disparity must agree within 1e-3 px."""
import numpy as np
import pytest

import lfsynth
import oracle
from lf_helpers import DISP_TOL, TIE_REL, best_of

pytestmark = pytest.mark.gpu

PICK = (0, 5, 10, 15, 16, 21, 26, 31)


@pytest.fixture(scope="module")
def mix():
    out = []
    for i in PICK:
        views, p = lfsynth.batch_lf(i, device="cpu", scale=0.15)
        views = views.numpy()
        cfg = oracle.make_cfg(p)
        ref = oracle.depth(cfg, views, p1f=p.p1_frac, p2f=p.p2_frac)
        best = best_of(ref["Cs"], ref["off"], ref["cnt"], ref["label"], ref["lo"])
        decided = ref["gap"] > TIE_REL * np.maximum(1.0, np.abs(best))
        out.append((p, views, ref, decided))
    return out


def _batch(lf, mix, branches):
    import torch
    views = [torch.from_numpy(v).cuda() for _, v, _, _ in mix]
    b = lf.LightFieldBatch([m[0] for m in mix], views, branches=branches)
    disp = [d.cpu().numpy() for d in b.run()]
    torch.cuda.synchronize()
    start, end, k = b.times()
    nodes = b.kernel_nodes
    b.close()
    return disp, start, end, k, nodes


def _check_vs_oracle(disp, mix):
    for d, (p, _, ref, decided) in zip(disp, mix):
        err = np.abs(d - ref["disp"])[decided]
        assert err.size > 0.9 * p.N, p.name
        assert np.max(err) < DISP_TOL, (p.name, float(np.max(err)))


def test_batch_matches_oracle(gpu_lib, mix):
    disp, start, end, k, nodes = _batch(gpu_lib, mix, branches=3)
    assert k == 3
    _check_vs_oracle(disp, mix)
    assert nodes > 10 * len(mix)


def test_batch_single_branch_reuses_buffers_across_shapes(gpu_lib, mix):
    """One branch: every light field runs in the scratch buffers of the largest one."""
    disp, start, end, k, _ = _batch(gpu_lib, mix, branches=1)
    assert k == 1
    _check_vs_oracle(disp, mix)
    order = np.argsort(start)
    # on one branch the light fields run one after another
    assert np.all(start[order][1:] >= end[order][:-1])


def test_batch_autotuned_times_are_consistent(gpu_lib, mix):
    import torch
    views = [torch.from_numpy(v).cuda() for _, v, _, _ in mix]
    b = gpu_lib.LightFieldBatch([m[0] for m in mix], views, branches=0)
    disp = [d.cpu().numpy() for d in b.run()]
    torch.cuda.synchronize()
    start, end, k = b.times()
    kw, lc, sw, sp = b.knobs()
    b.close()
    assert k in (1, 2, 4, 8)
    _check_vs_oracle(disp, mix)
    assert np.all(start >= 0.0) and np.all(end > start)
    # the autotuner picked a row span, list CTAs, SGM warps and split threshold per shape class
    assert set(kw.tolist()) <= {36, 44} and set(lc.tolist()) <= {0, 8, 12, 24} and set(sw.tolist()) <= {2, 4, 8}
    assert set(sp.tolist()) <= {0, 24}


def test_batch_matches_single_light_field_launches(gpu_lib, mix):
    import torch
    disp, *_ = _batch(gpu_lib, mix, branches=2)
    for d, (p, views, ref, decided) in zip(disp, mix):
        h = gpu_lib.lfsgm_create(p)
        one = torch.empty(p.N, dtype=torch.float32, device="cuda")
        gpu_lib.lfsgm_depth(h, torch.from_numpy(views).cuda(), one, None)
        gpu_lib.lfsgm_sync(h)
        gpu_lib.lfsgm_destroy(h)
        # every stage is deterministic (the SGM's direction sum included), so the batch reproduces
        # the single launches bit for bit
        assert np.array_equal(one.cpu().numpy(), d, equal_nan=True), p.name


def test_batch_runs_repeatedly(gpu_lib, mix):
    import torch
    views = [torch.from_numpy(v).cuda() for _, v, _, _ in mix[:3]]
    b = gpu_lib.LightFieldBatch([m[0] for m in mix[:3]], views, branches=2)
    first = [d.clone() for d in b.run()]
    for _ in range(3):
        b.run()
    b.times()
    for a, c in zip(first, b.disp):
        assert torch.equal(torch.nan_to_num(a, nan=-1e30), torch.nan_to_num(c, nan=-1e30))
    b.close()


def test_batch_rejects_an_invalid_member(gpu_lib, mix):
    import torch
    bad = lfsynth.tiny_params(census_w=9)
    views = [torch.from_numpy(mix[0][1]).cuda(), torch.zeros(25 * 64 * 64, device="cuda")]
    with pytest.raises(gpu_lib.LfsgmError, match="light field 1"):
        gpu_lib.LightFieldBatch([mix[0][0], bad], views, branches=1)


def test_batch_in_caller_workspace_matches_library_scratch(gpu_lib, mix):
    """lfsgm_batch_create_ws: the scratch of every branch in one caller-owned buffer of the size
    lfsgm_batch_workspace_size reports; the disparities equal those of the library-allocated
    batch bit for bit, and a buffer one byte short is refused with LFSGM_ERR_WORKSPACE."""
    import torch
    params = [m[0] for m in mix]
    views = [torch.from_numpy(v).cuda() for _, v, _, _ in mix]
    ref = gpu_lib.LightFieldBatch(params, views, branches=2)
    want = [d.clone() for d in ref.run()]
    torch.cuda.synchronize()
    ref.close()
    need = gpu_lib.lfsgm_batch_workspace_size(params, branches=2)
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    ws = ws[off:off + need]
    b = gpu_lib.LightFieldBatch(params, views, branches=2, ws=ws)
    for _ in range(2):
        got = b.run()
        torch.cuda.synchronize()
        for a, c in zip(want, got):
            assert torch.equal(torch.nan_to_num(a, nan=-1e30), torch.nan_to_num(c, nan=-1e30))
    s, e, k = b.times()
    assert k == 2 and np.all(e > s)
    b.close()
    with pytest.raises(gpu_lib.LfsgmError, match="too small"):
        gpu_lib.LightFieldBatch(params, views, branches=2, ws=ws[:need - 1])
    # autotuned branch count inside a buffer sized for every candidate
    need_all = gpu_lib.lfsgm_batch_workspace_size(params, branches=0)
    assert need_all >= need
    ws2 = torch.empty(need_all + 256, dtype=torch.uint8, device="cuda")
    off = (-ws2.data_ptr()) % 256
    b = gpu_lib.LightFieldBatch(params, views, branches=0, ws=ws2[off:off + need_all])
    got = b.run()
    torch.cuda.synchronize()
    for a, c in zip(want, got):
        assert torch.equal(torch.nan_to_num(a, nan=-1e30), torch.nan_to_num(c, nan=-1e30))
    b.close()
