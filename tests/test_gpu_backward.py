"""GPU adjoint (lfsgm_backward, through the C ABI) against the oracle's FP64 adjoint, which is
itself pinned by finite differences (tests/test_oracle_adjoint.py).

Every gradient element is compared with the oracle's: |gpu - oracle| <= rel * scale + abs * G, with
scale = max(|x|, mean |x| over the element's group) -- the group being the pixel's window for
dLoss/dcost and the view plane for dLoss/dviews -- and G the largest oracle gradient of that kind.

Tolerances.  The GPU aggregates in FP32 and feeds exp(-C_s / tau) into the soft-argmin.  An
absolute error e of C_s becomes a relative error e / tau of the weights, and e is a few FP32
unit roundoffs u of C_s, so the weights carry ~u C_s / tau: with tau = 0.1 and C_s up to 550
(grey) or 1350 (colour) here, 3e-4 .. 8e-4.  The SGM adjoint then adds contributions of either
sign; where they cancel, an element keeps the FP32 rounding of the terms it summed, which is a
fraction of the largest gradient rather than of its own size.  Hence the relative part
grad_tol = 16 u max(C_s) / tau (lf_helpers) plus GRAD_ABS of the largest gradient.  Measured, the
needed relative part is 0 (the absolute part covers it) for 99 % of the elements; its maximum is
1.5e-3 in dcost and 2.1e-3 in dviews (grey, against a bar of 5.2e-3 .. 5.8e-3) and 6.1e-3
(colour, against 1.1e-2).  dLoss/dP1 and dLoss/dP2 sum signed adjoints over every cell and
direction; each summand carries the weights' relative error, which does not cancel with the
sum, so their bar adds GRAD_MASS of sum |dLoss/dcost| (measured: 1.4e-5 of it at worst).  Where
C_s / tau is of order one (views of small contrast, tau = 1) the same kernels are held to
GRAD_TOL_EXACT per element."""
import numpy as np
import pytest

import lfsynth
import oracle
from lf_helpers import (GRAD_ABS, GRAD_MASS, GRAD_TOL_P, err_stats, gather, grad_tol, group_rel_err, needed_rel,
                        pad4_offsets)

pytestmark = pytest.mark.gpu
TAU = 0.1
GRAD_TOL_EXACT = 1e-5    # per element, C_s / tau ~ 1


def _setup(seed=2024, contrast=1.0, w_census=1.0 / 24, tau=TAU):
    p = lfsynth.LFParams(U=7, V=7, H=32, W=32, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=9,
                         fine_labels=41, fine_radius=8, w_l2=1.0, w_census=w_census, subpixel=2, softmin_tau=tau)
    rng = np.random.default_rng(seed)
    views = (contrast * rng.uniform(0.0, 1.0, (7, 7, 32, 32))).astype(np.float32)
    lo = np.full(p.N, 12, np.int32)
    cnt = np.full(p.N, 16, np.int32)
    gd = rng.normal(size=p.N).astype(np.float32)
    return p, views, lo, cnt, gd


def _gpu_holder(lf, p, lo, cnt):
    import torch
    L = lf.LightFieldDepth(p)
    L.lo.copy_(torch.from_numpy(lo))
    L.cnt.copy_(torch.from_numpy(cnt))
    L.off.copy_(torch.from_numpy(pad4_offsets(cnt)))
    return L


def _run_gpu_backward(lf, p, views, lo, cnt, P1, P2, gd, tau, recorded=False):
    """dLoss/dcost (active slots), dP1, dP2, dLoss/dviews from the library: lfsgm_backward, or with
    recorded=True the training form (lfsgm_sgm_aggregate_record, then lfsgm_backward_recorded)."""
    import torch
    L = _gpu_holder(lf, p, lo, cnt)
    vd = torch.from_numpy(views).cuda()
    L.cost_volume(vd)
    gcost = torch.empty_like(L.cost)
    gviews = torch.empty_like(vd)
    g1 = torch.zeros(1, device="cuda")
    g2 = torch.zeros(1, device="cuda")
    if recorded:
        lf.lfsgm_sgm_aggregate_record(L.h, L.cost, L.lo, L.cnt, L.off, float(P1), float(P2), L.agg)
        lf.lfsgm_backward_recorded(L.h, vd, L.cost, L.agg, L.lo, L.cnt, L.off, float(P1), float(P2),
                                   torch.from_numpy(gd).cuda(), gcost, g1, g2, gviews)
    else:
        lf.lfsgm_backward(L.h, vd, L.cost, L.lo, L.cnt, L.off, float(P1), float(P2), torch.from_numpy(gd).cuda(),
                          gcost, g1, g2, gviews)
    lf.lfsgm_sync(L.h)
    gC = gather(gcost.cpu().numpy(), pad4_offsets(cnt), cnt)
    out = gC, g1.item(), g2.item(), gviews.cpu().numpy()
    L.close()
    return out


def _cs_max(p, lo, cnt, off_o, cost_o, P1, P2):
    return oracle.sgm_bounded(p.H, p.W, lo, cnt, off_o, cost_o, float(P1), float(P2), p.paths).max()


def _elem_errors(p, cnt, gC, gC_o, gV, gV_o, abs_frac=GRAD_ABS):
    """The relative tolerance each element needs beside the absolute part (dcost, dviews)."""
    planes = np.full(p.U * p.V * p.channels, p.H * p.W)
    return needed_rel(gC, gC_o, cnt, abs_frac), needed_rel(gV, gV_o, planes, abs_frac)


def _penalties(cost_o):
    return np.float32(0.05 * cost_o.mean()), np.float32(0.5 * cost_o.mean())


@pytest.mark.parametrize("recorded", [False, True], ids=["recompute", "recorded"])
def test_backward_matches_oracle_adjoint(gpu_lib, recorded):
    p, views, lo, cnt, gd = _setup()
    cfg = oracle.make_cfg(p)
    off_o, cost_o = oracle.cost_volume(cfg, views, lo, cnt)
    P1, P2 = _penalties(cost_o)
    gC_o, g1_o, g2_o, gV_o = oracle.backward(cfg, views, lo, cnt, cost_o, float(P1), float(P2), gd, TAU)
    gC, g1, g2, gV = _run_gpu_backward(gpu_lib, p, views, lo, cnt, P1, P2, gd, TAU, recorded)
    eC, eV = _elem_errors(p, cnt, gC, gC_o, gV, gV_o)
    tol = grad_tol(_cs_max(p, lo, cnt, off_o, cost_o, P1, P2), TAU)
    print(f"backward 7x7x32x32 tau 0.1, bar {tol:.2e}, needed relative tolerance: dcost", err_stats(eC),
          "dviews", err_stats(eV), "plain relative error: dcost", err_stats(group_rel_err(gC, gC_o, cnt)))
    assert eC.max() <= tol, err_stats(eC)
    assert eV.max() <= tol, err_stats(eV)
    assert abs(g1 - g1_o) <= GRAD_TOL_P * max(abs(g1_o), 1e-3), (g1, g1_o)
    assert abs(g2 - g2_o) <= GRAD_TOL_P * max(abs(g2_o), 1e-3), (g2, g2_o)
    # exact invariant: per-pixel sums of dLoss/dcost vanish (normalised SGM + shift-invariant softmax)
    scale = np.abs(gC_o).max()
    assert np.abs(gC.reshape(p.N, 16).sum(1)).max() <= 1e-5 * scale * 16


@pytest.mark.parametrize("seed", [2024, 7])
def test_backward_low_amplification_matches_oracle_per_element(gpu_lib, seed):
    """Views of contrast 0.01, a small census weight and tau = 1 keep C_s / tau near one, so FP32
    rounding of the aggregate is not amplified by the softmax: every element of dLoss/dcost and
    dLoss/dviews agrees with the FP64 adjoint to GRAD_TOL_EXACT of its scale."""
    tau = 1.0
    p, views, lo, cnt, gd = _setup(seed=seed, contrast=0.01, w_census=1e-4, tau=tau)
    cfg = oracle.make_cfg(p)
    off_o, cost_o = oracle.cost_volume(cfg, views, lo, cnt)
    P1, P2 = _penalties(cost_o)
    gC_o, g1_o, g2_o, gV_o = oracle.backward(cfg, views, lo, cnt, cost_o, float(P1), float(P2), gd, tau)
    gC, g1, g2, gV = _run_gpu_backward(gpu_lib, p, views, lo, cnt, P1, P2, gd, tau)
    # dcost: purely relative; dviews: plus 1e-6 of the largest view gradient (each view pixel sums
    # ~10^2 signed FP32 terms, measured 1.8e-5 of its scale at worst without that part)
    eC, _ = _elem_errors(p, cnt, gC, gC_o, gV, gV_o, abs_frac=0.0)
    _, eV = _elem_errors(p, cnt, gC, gC_o, gV, gV_o, abs_frac=1e-6)
    print(f"backward low amplification seed {seed}: dcost", err_stats(eC), "dviews", err_stats(eV),
          "dP1", g1, g1_o, "dP2", g2, g2_o)
    assert eC.max() <= GRAD_TOL_EXACT, err_stats(eC)
    assert eV.max() <= GRAD_TOL_EXACT, err_stats(eV)
    mass = np.abs(gC_o).sum()
    assert abs(g1 - g1_o) <= GRAD_TOL_EXACT * (abs(g1_o) + 1e-3 * mass), (g1, g1_o)
    assert abs(g2 - g2_o) <= GRAD_TOL_EXACT * (abs(g2_o) + 1e-3 * mass), (g2, g2_o)


def _ragged_case(kind, seed=77):
    """Windows of 5-40 labels at random positions (narrow windows go through the tile kernel,
    wider ones through the per-chunk kernel); 'wide_range' spreads them over a +-12 px range so
    that a tile's tap footprint no longer fits its shared-memory box."""
    if kind == "mixed":
        p = lfsynth.LFParams(U=7, V=7, H=32, W=40, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=9,
                             fine_labels=41, fine_radius=8, w_l2=1.0, w_census=1.0 / 24, subpixel=2,
                             softmin_tau=TAU)
    else:
        p = lfsynth.LFParams(U=7, V=7, H=32, W=40, census_w=5, dmin=-12.0, dmax=12.0, coarse_labels=9,
                             fine_labels=97, fine_radius=8, w_l2=1.0, w_census=1.0 / 24, subpixel=2,
                             softmin_tau=TAU)
    rng = np.random.default_rng(seed)
    views = rng.uniform(0.0, 1.0, (p.V, p.U, p.H, p.W)).astype(np.float32)
    cnt = rng.choice(np.array([5, 16, 31, 33, 40], np.int32), size=p.N).astype(np.int32)
    lo = (rng.random(p.N) * (p.fine_labels - cnt + 1)).astype(np.int32)
    gd = rng.normal(size=p.N).astype(np.float32)
    return p, views, lo, cnt, gd


@pytest.mark.parametrize("kind", ["mixed", "wide_range", "mixed_16_paths", "mixed_recorded",
                                  "mixed_16_paths_recorded"])
def test_backward_ragged_windows_match_oracle(gpu_lib, kind):
    import dataclasses
    recorded = kind.endswith("_recorded")
    kind = kind.replace("_recorded", "")
    p, views, lo, cnt, gd = _ragged_case(kind.replace("_16_paths", ""))
    if kind.endswith("16_paths"):
        p = dataclasses.replace(p, paths=16)
    cfg = oracle.make_cfg(p)
    off_o, cost_o = oracle.cost_volume(cfg, views, lo, cnt)
    P1, P2 = _penalties(cost_o)
    gC_o, g1_o, g2_o, gV_o = oracle.backward(cfg, views, lo, cnt, cost_o, float(P1), float(P2), gd, TAU)
    gC, g1, g2, gV = _run_gpu_backward(gpu_lib, p, views, lo, cnt, P1, P2, gd, TAU, recorded)
    eC, eV = _elem_errors(p, cnt, gC, gC_o, gV, gV_o)
    tol = grad_tol(_cs_max(p, lo, cnt, off_o, cost_o, P1, P2), TAU)
    print(f"backward ragged {kind}, bar {tol:.2e}, needed relative tolerance: dcost", err_stats(eC),
          "dviews", err_stats(eV))
    assert eC.max() <= tol, err_stats(eC)
    assert eV.max() <= tol, err_stats(eV)
    # dLoss/dP1, dLoss/dP2 are signed sums over every cell and direction (see the module docstring)
    mass = GRAD_MASS / GRAD_TOL_P * np.abs(gC_o).sum()
    assert abs(g1 - g1_o) <= GRAD_TOL_P * (abs(g1_o) + mass), (g1, g1_o, mass)
    assert abs(g2 - g2_o) <= GRAD_TOL_P * (abs(g2_o) + mass), (g2, g2_o, mass)


def test_backward_bench_band_matches_oracle(gpu_lib):
    """Rows 192..255 of the 9x9 x 512x512 bench light field (census 7x7, 401 fine labels), with the
    31-label windows of the oracle's own initial pass on that band: the GPU adjoint against the FP64
    adjoint at the bench configuration (tau = 0.1).

    On a real scene a few decisions of the adjoint sit on a kink: the SGM minimum has near-ties
    (two branches within FP32 rounding of each other), and |I_ref - sample| has samples within
    FP32 rounding of I_ref.  There the FP32 and FP64 adjoints pick different subgradients, both
    correct.  So the per-element bar of the other tests must hold for all but 1e-4 of the elements
    (measured: 6 of 1.1 M cost gradients, 19 of 2.7 M view gradients), and the total absolute
    difference must stay below 1e-3 of the total gradient mass (measured 1.5e-4, 1.7e-4)."""
    views_full, _, pb = lfsynth.bench()
    y0, rows = 192, 64
    band = np.ascontiguousarray(views_full[:, :, y0:y0 + rows, :])
    p = lfsynth.LFParams(**{**pb.__dict__, "H": rows, "subpixel": 2, "softmin_tau": TAU})
    cfg = oracle.make_cfg(p)
    init = oracle.initial_disparity(cfg, band, None, p.p1_frac, p.p2_frac)
    lo, cnt = init["lo"].astype(np.int32), init["cnt"].astype(np.int32)
    off_o, cost_o = oracle.cost_volume(cfg, band, lo, cnt, init["census"])
    P1, P2 = _penalties(cost_o)
    gd = np.random.default_rng(11).normal(size=p.N).astype(np.float32)
    gC_o, g1_o, g2_o, gV_o = oracle.backward(cfg, band, lo, cnt, cost_o, float(P1), float(P2), gd, TAU)
    tol = grad_tol(_cs_max(p, lo, cnt, off_o, cost_o, P1, P2), TAU)
    for recorded in (False, True):
        gC, g1, g2, gV = _run_gpu_backward(gpu_lib, p, band, lo, cnt, P1, P2, gd, TAU, recorded)
        eC, eV = _elem_errors(p, cnt, gC, gC_o, gV, gV_o)
        print(f"backward bench band (recorded {recorded}), bar {tol:.2e}, needed relative tolerance: dcost",
              err_stats(eC), "dviews", err_stats(eV), "beyond the bar:", int((eC > tol).sum()),
              int((eV > tol).sum()), "dP1", g1, g1_o, "dP2", g2, g2_o)
        for e, g, o in ((eC, gC, gC_o), (eV, gV, gV_o)):
            assert np.mean(e > tol) <= 1e-4, err_stats(e)
            assert np.abs(g.astype(np.float64).reshape(-1) - o.reshape(-1)).sum() <= 1e-3 * np.abs(o).sum()
        mass = GRAD_MASS / GRAD_TOL_P * np.abs(gC_o).sum()
        assert abs(g1 - g1_o) <= GRAD_TOL_P * (abs(g1_o) + mass), (g1, g1_o, mass)
        assert abs(g2 - g2_o) <= GRAD_TOL_P * (abs(g2_o) + mass), (g2, g2_o, mass)


def test_autograd_functions_match_direct_call(gpu_lib):
    import torch
    p, views, lo, cnt, gd = _setup(seed=5)
    L = _gpu_holder(gpu_lib, p, lo, cnt)
    vd = torch.from_numpy(views).cuda().requires_grad_(True)
    P1 = torch.tensor(0.3, device="cuda", requires_grad=True)
    P2 = torch.tensor(2.5, device="cuda", requires_grad=True)
    disp = gpu_lib.depth_from_views(vd, P1, P2, L)
    g = torch.from_numpy(gd).cuda()
    (disp * g).sum().backward()
    # the same through the cost-level function
    cost = L.cost.clone().requires_grad_(True)
    P1b = torch.tensor(0.3, device="cuda", requires_grad=True)
    P2b = torch.tensor(2.5, device="cuda", requires_grad=True)
    disp2 = gpu_lib.sgm_softargmin(cost, P1b, P2b, L)
    (disp2 * g).sum().backward()
    # the aggregate is deterministic, so both routes give the same disparities
    assert torch.equal(disp, disp2)
    assert abs(P1.grad.item() - P1b.grad.item()) <= GRAD_TOL_P * max(1.0, abs(P1b.grad.item()))
    assert abs(P2.grad.item() - P2b.grad.item()) <= GRAD_TOL_P * max(1.0, abs(P2b.grad.item()))
    assert torch.isfinite(vd.grad).all() and vd.grad.abs().sum() > 0
    # soft-argmin forward agrees with the oracle
    cfg = oracle.make_cfg(p)
    off_o, cost_o = oracle.cost_volume(cfg, views, lo, cnt)
    Cs = oracle.sgm_bounded(p.H, p.W, lo, cnt, off_o, cost_o, 0.3, 2.5)
    d_o = oracle.softargmin(cfg, lo, cnt, off_o, Cs, TAU)
    assert np.abs(disp.detach().cpu().numpy() - d_o).max() < 1e-3
    L.close()


def test_backward_bench_shape_invariants(gpu_lib):
    """9x9 x 512x512 with 31-label windows from the initial pass: gradients are finite and the
    per-pixel sums of dLoss/dcost vanish (up to FP32 rounding)."""
    import torch
    views, gt, p = lfsynth.bench()
    p.subpixel = 2
    L = gpu_lib.LightFieldDepth(p)
    vd = torch.from_numpy(views).cuda()
    L.initial(vd)
    L.cost_volume(vd)
    mean = float(L.cost[:int(L.off[-1].item())].double().sum().item()) / float(L.cnt.sum().item())
    P1, P2 = 0.05 * mean, 0.5 * mean
    gd = torch.randn(p.N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    gcost = torch.empty_like(L.cost)
    gviews = torch.empty_like(vd)
    g1 = torch.zeros(1, device="cuda")
    g2 = torch.zeros(1, device="cuda")
    gpu_lib.lfsgm_backward(L.h, vd, L.cost, L.lo, L.cnt, L.off, P1, P2, gd, gcost, g1, g2, gviews)
    gpu_lib.lfsgm_sync(L.h)
    cnt = L.cnt.cpu().numpy()
    off = L.off.cpu().numpy()
    gC = gather(gcost.cpu().numpy(), off, cnt)
    assert np.isfinite(gC).all() and np.isfinite(gviews.cpu().numpy()).all()
    starts = np.cumsum(cnt) - cnt
    sums = np.add.reduceat(gC.astype(np.float64), starts)
    scale = np.add.reduceat(np.abs(gC).astype(np.float64), starts)
    # the sums vanish in exact arithmetic; in FP32 the adjoint is carried along 512-step paths
    # (8 of them per pixel) and the softmax weights carry FP32 rounding of the aggregate
    # amplified by C_s / tau, so residuals of order n * eps_32 ~ 3e-5 of the global scale occur
    # (observed 0.9e-5 .. 1.7e-5)
    assert np.abs(sums).max() <= 1e-4 * scale.max(), (np.abs(sums).max(), scale.max())
    L.close()


def test_recorded_aggregate_and_backward_agree_with_the_plain_calls(gpu_lib):
    """lfsgm_sgm_aggregate_record writes the same aggregate as lfsgm_sgm_aggregate, bit for bit, and
    lfsgm_backward_recorded gives lfsgm_backward's gradients: the same kernels on the same branch
    record, up to the order of the atomic additions into dLoss/dcost and dLoss/dviews."""
    import torch
    p, views, lo, cnt, gd = _ragged_case("mixed", seed=5)
    L = _gpu_holder(gpu_lib, p, lo, cnt)
    vd = torch.from_numpy(views).cuda()
    L.cost_volume(vd)
    P1, P2 = 0.2, 1.7
    agg_plain = torch.empty_like(L.cost)
    gpu_lib.lfsgm_sgm_aggregate(L.h, L.cost, L.lo, L.cnt, L.off, P1, P2, agg_plain)
    gpu_lib.lfsgm_sgm_aggregate_record(L.h, L.cost, L.lo, L.cnt, L.off, P1, P2, L.agg)
    nnz = int(L.off[-1].item())
    assert torch.equal(agg_plain[:nnz], L.agg[:nnz])
    g = torch.from_numpy(gd).cuda()
    out = []
    for recorded in (True, False):
        gcost = torch.zeros_like(L.cost)
        gviews = torch.empty_like(vd)
        gp = torch.zeros(2, device="cuda")
        if recorded:
            gpu_lib.lfsgm_backward_recorded(L.h, vd, L.cost, L.agg, L.lo, L.cnt, L.off, P1, P2, g, gcost, gp[0:1],
                                            gp[1:2], gviews)
        else:
            gpu_lib.lfsgm_backward(L.h, vd, L.cost, L.lo, L.cnt, L.off, P1, P2, g, gcost, gp[0:1], gp[1:2], gviews)
        gpu_lib.lfsgm_sync(L.h)
        out.append((gcost[:nnz].double(), gviews.double(), gp.double()))
    for a, b in zip(out[0], out[1]):
        assert (a - b).abs().max().item() <= 1e-5 * max(b.abs().max().item(), 1e-30), (a - b).abs().max()
    L.close()


def test_recorded_backward_refuses_a_stale_record(gpu_lib):
    """lfsgm_backward_recorded returns an error, and launches nothing, unless the handle's last
    record was taken on the same buffers and penalties (another recording or an lfsgm_backward
    in between replaces it)."""
    import torch
    p, views, lo, cnt, gd = _setup(seed=3)
    L = _gpu_holder(gpu_lib, p, lo, cnt)
    vd = torch.from_numpy(views).cuda()
    L.cost_volume(vd)
    g = torch.from_numpy(gd).cuda()
    gcost = torch.empty_like(L.cost)
    gp = torch.zeros(2, device="cuda")
    other = L.cost.clone()

    def recorded(cost=None, agg=None, P1=0.3, P2=2.5):
        gpu_lib.lfsgm_backward_recorded(L.h, None, L.cost if cost is None else cost, L.agg if agg is None else agg,
                                        L.lo, L.cnt, L.off, P1, P2, g, gcost, gp[0:1], gp[1:2], None)

    with pytest.raises(RuntimeError):
        recorded()                                    # nothing recorded yet
    gpu_lib.lfsgm_sgm_aggregate_record(L.h, L.cost, L.lo, L.cnt, L.off, 0.3, 2.5, L.agg)
    n0 = gpu_lib.lfsgm_launch_count(L.h)
    for kw in ({"P1": 0.31}, {"P2": 2.4}, {"cost": other}, {"agg": torch.empty_like(L.agg)}):
        with pytest.raises(RuntimeError):
            recorded(**kw)
    assert gpu_lib.lfsgm_launch_count(L.h) == n0
    recorded()
    recorded()                                        # the record survives its backward
    gpu_lib.lfsgm_backward(L.h, None, L.cost, L.lo, L.cnt, L.off, 0.3, 2.5, g, gcost, gp[0:1], gp[1:2], None)
    with pytest.raises(RuntimeError):
        recorded()                                    # lfsgm_backward recorded over it
    gpu_lib.lfsgm_sync(L.h)
    L.close()


def test_autograd_interleaved_forwards_fall_back_to_recompute(gpu_lib):
    """Two forwards on one handle before their backwards: the second forward's record replaces the
    first's, so the first backward recomputes the SGM; both match a single forward + backward."""
    import torch
    p, views, lo, cnt, gd = _setup(seed=9)
    L = _gpu_holder(gpu_lib, p, lo, cnt)
    vd = torch.from_numpy(views).cuda()
    L.cost_volume(vd)
    g = torch.from_numpy(gd).cuda()
    grads = []
    for pen in ((0.3, 2.5), (0.2, 1.5)):
        c = L.cost.clone().requires_grad_(True)
        (gpu_lib.sgm_softargmin(c, *pen, L) * g).sum().backward()
        grads.append(c.grad)
    c1 = L.cost.clone().requires_grad_(True)
    c2 = L.cost.clone().requires_grad_(True)
    d1 = gpu_lib.sgm_softargmin(c1, 0.3, 2.5, L)
    d2 = gpu_lib.sgm_softargmin(c2, 0.2, 1.5, L)
    (d1 * g).sum().backward()                         # record of d2 on the handle: recomputes
    (d2 * g).sum().backward()                         # its own record was replaced: recomputes
    nnz = int(L.off[-1].item())
    for a, b in ((c1.grad, grads[0]), (c2.grad, grads[1])):
        assert (a[:nnz] - b[:nnz]).abs().max().item() <= 1e-5 * b[:nnz].abs().max().item()
    L.close()
