"""Pins of the oracle's FP64 adjoint (soft-argmin -> bounded SGM over 8 or 16 paths -> l2/census cost
-> views) against central finite differences in FP64 and exact invariants.

Workload: 7x7 views of 32x32, every pixel searching one dense 16-label window (the initial
pass is bypassed), Loss = sum_p gd(p) dhat(p) with gd ~ N(0,1) and dhat the soft-argmin
(tau = 0.1) of the aggregated cost.  Inputs are generic (continuous random textures), so
per-path minima are distinct and no |difference| or census comparison sits at a switch."""
import numpy as np
import pytest

import lfsynth
import oracle

TAU = 0.1


@pytest.fixture(scope="module", params=[8, 16], ids=["8paths", "16paths"])
def case(request):
    p = lfsynth.LFParams(U=7, V=7, H=32, W=32, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=9,
                         fine_labels=41, fine_radius=8, w_l2=1.0, w_census=1.0 / 24, paths=request.param)
    cfg = oracle.make_cfg(p)
    rng = np.random.default_rng(2024)
    views = rng.uniform(0.0, 1.0, (7, 7, 32, 32))
    # a fronto-parallel shift structure plus noise keeps the costs informative
    lo = np.full(p.N, 12, np.int32)
    cnt = np.full(p.N, 16, np.int32)
    off, cost = oracle.cost_volume(cfg, views, lo, cnt)
    mean = cost.mean()
    P1, P2 = 0.05 * mean, 0.5 * mean
    gd = rng.normal(size=p.N)
    grads = oracle.backward(cfg, views, lo, cnt, cost, P1, P2, gd, TAU)
    return p, cfg, views, lo, cnt, off, cost, P1, P2, gd, grads


def _loss_cost(case, cost=None, P1=None, P2=None):
    p, cfg, views, lo, cnt, off, c0, p1, p2, gd, _ = case
    return oracle.loss_from_cost(cfg, lo, cnt, c0 if cost is None else cost, p1 if P1 is None else P1,
                                 p2 if P2 is None else P2, gd, TAU)


def _loss_views(case, views):
    p, cfg, _, lo, cnt, off, _, P1, P2, gd, _ = case
    _, cost = oracle.cost_volume(cfg, views, lo, cnt)
    return oracle.loss_from_cost(cfg, lo, cnt, cost, P1, P2, gd, TAU)


def _close(a, b, rel=2e-4, abs_=2e-7):
    return abs(a - b) <= abs_ + rel * max(abs(a), abs(b))


def test_grad_cost_matches_finite_differences(case):
    p, cfg, views, lo, cnt, off, cost, P1, P2, gd, (gC, g1, g2, gV) = case
    rng = np.random.default_rng(7)
    idx = list(rng.choice(cost.size, 24, replace=False))
    idx += list(np.argsort(-np.abs(gC))[:8])          # the largest gradients too
    h = 1e-5
    for k in idx:
        cp, cm = cost.copy(), cost.copy()
        cp[k] += h
        cm[k] -= h
        fd = (_loss_cost(case, cost=cp) - _loss_cost(case, cost=cm)) / (2 * h)
        assert _close(fd, gC[k]), (k, fd, gC[k])


def test_grad_penalties_match_finite_differences(case):
    p, cfg, views, lo, cnt, off, cost, P1, P2, gd, (gC, g1, g2, gV) = case
    h = 1e-6
    fd1 = (_loss_cost(case, P1=P1 + h) - _loss_cost(case, P1=P1 - h)) / (2 * h)
    fd2 = (_loss_cost(case, P2=P2 + h) - _loss_cost(case, P2=P2 - h)) / (2 * h)
    assert _close(fd1, g1), (fd1, g1)
    assert _close(fd2, g2), (fd2, g2)
    assert g1 != 0.0 and g2 != 0.0


def test_grad_views_match_finite_differences(case):
    p, cfg, views, lo, cnt, off, cost, P1, P2, gd, (gC, g1, g2, gV) = case
    rng = np.random.default_rng(11)
    picks = [(3, 3, 16, 16), (3, 3, 5, 27)]                      # reference view pixels
    picks += [tuple(int(v) for v in (rng.integers(7), rng.integers(7), rng.integers(2, 30), rng.integers(2, 30)))
              for _ in range(8)]
    flat = np.abs(gV).reshape(-1)
    big = np.unravel_index(np.argsort(-flat)[:4], gV.shape)
    picks += list(zip(*[b.tolist() for b in big]))
    h = 1e-6
    for (v, u, y, x) in picks:
        vp, vm = views.copy(), views.copy()
        vp[v, u, y, x] += h
        vm[v, u, y, x] -= h
        fd = (_loss_views(case, vp) - _loss_views(case, vm)) / (2 * h)
        assert _close(fd, gV[v, u, y, x], rel=5e-4, abs_=1e-6), ((v, u, y, x), fd, gV[v, u, y, x])


def test_softargmin_gradient_sums_to_zero_per_pixel(case):
    """Adding a constant to a pixel's aggregated costs leaves its softmax unchanged."""
    p, cfg, views, lo, cnt, off, cost, P1, P2, gd, _ = case
    Cs = oracle.sgm_bounded(p.H, p.W, lo, cnt, off, cost, P1, P2, p.paths)
    gCs = oracle.softargmin_backward(cfg, lo, cnt, off, Cs, gd, TAU)
    assert np.allclose(gCs.reshape(p.N, 16).sum(1), 0.0, atol=1e-12)


def test_sgm_cost_gradient_sums_to_zero_per_pixel(case):
    """A constant added to all of a pixel's costs shifts L_r at that pixel only (the
    normalised recurrence removes it downstream), so C_s(p) shifts by (paths) times the constant
    and every soft-argmin is unchanged: the per-pixel sums of dLoss/dcost vanish."""
    p, cfg, views, lo, cnt, off, cost, P1, P2, gd, (gC, g1, g2, gV) = case
    assert np.allclose(gC.reshape(p.N, 16).sum(1), 0.0, atol=1e-10)
