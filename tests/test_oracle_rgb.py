"""Pins of the oracle's colour (C = 3) path: census per channel with the Hamming distances
summed, and the l2 term as the Euclidean norm of the colour difference (Sec. III-B/C, Eq. 6,
Eq. 12), against closed forms, brute force and exact reductions to the one-channel path."""
import numpy as np
import pytest

import lfsynth
import oracle


def _params(U=5, V=5, H=16, W=16, **kw):
    d = dict(U=U, V=V, H=H, W=W, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=9,
             fine_labels=21, fine_radius=3, w_l2=1.0, w_census=1.0 / 24)
    d.update(kw)
    return lfsynth.LFParams(**d)


def _full(p):
    return np.zeros(p.N, np.int32), np.full(p.N, p.fine_labels, np.int32)


def test_colour_l2_closed_form_on_linear_ramps():
    """Channel c of view (u,v) is alpha_c (x - a d0) + beta_c (y - b d0) + gamma_c: a plane at d0
    seen through a linear colour texture.  Bilinear sampling is exact, so away from the border
    the colour difference is (alpha_c a + beta_c b)(d - d0) per channel and
    C_l2(p, d) = |d - d0| sum_views sqrt(sum_c (alpha_c a + beta_c b)^2); a per-channel sum of
    absolute values would give a different number."""
    U = V = 5
    H = W = 24
    alpha = (0.013, -0.021, 0.004)
    beta = (-0.029, 0.017, 0.011)
    gamma = (0.5, 0.4, 0.6)
    d0 = 0.37
    uc, vc = 2, 2
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    views = np.zeros((V, U, 3, H, W), np.float32)
    for v in range(V):
        for u in range(U):
            a, b = u - uc, v - vc
            for c in range(3):
                views[v, u, c] = alpha[c] * (x - a * d0) + beta[c] * (y - b * d0) + gamma[c]
    p = _params(U, V, H, W, fine_labels=41, w_census=0.0, channels=3)
    cfg = oracle.make_cfg(p)
    lo, cnt = _full(p)
    off, cost = oracle.cost_volume(cfg, views, lo, cnt)
    ws = sum(np.sqrt(sum((alpha[c] * (u - uc) + beta[c] * (v - vc)) ** 2 for c in range(3)))
             for u in range(U) for v in range(V))
    m = 5
    for yy in range(m, H - m):
        for xx in range(m, W - m):
            pix = yy * W + xx
            for g in range(41):
                d = -1.0 + g * 0.05
                assert abs(cost[off[pix] + g] - ws * abs(d - d0)) < 2e-5


def test_colour_constant_views_give_the_3_4_5_norm():
    """Constant views: the census words are all zero and every non-reference view differs from
    the reference by (0.3, 0.4, 0): each contributes exactly the norm 0.5 at every label."""
    p = _params(U=3, V=3, H=6, W=7, channels=3, w_census=1.0)
    views = np.empty((3, 3, 3, 6, 7), np.float64)
    views[:, :] = np.array([0.25, 0.5, 0.75])[:, None, None]
    views[p.vc, p.uc] = np.array([0.55, 0.9, 0.75])[:, None, None]
    cfg = oracle.make_cfg(p)
    lo, cnt = _full(p)
    _, cost = oracle.cost_volume(cfg, views, lo, cnt)
    assert np.allclose(cost, 8 * 0.5, rtol=1e-15, atol=0)


def test_colour_census_cost_brute_force_bits():
    """Coarse (Eq. 7) and fine census (Eq. 15) costs by direct pixel comparisons per channel:
    a bit of channel c differs when xi(Iref_c(p), Iref_c(p+o)) != xi(Iv_c(q), Iv_c(q+o))."""
    p = _params(U=3, V=3, H=6, W=7, coarse_labels=5, fine_labels=9, fine_radius=1, init_views=1,
                channels=3, w_l2=0.0, w_census=1.0)
    views = lfsynth.random_views(3, 3, 6, 7, seed=17, channels=3)
    cfg = oracle.make_cfg(p)
    cen = oracle.census_all(cfg, views)
    h = p.census_w // 2
    offs = [(dx, dy) for dy in range(-h, h + 1) for dx in range(-h, h + 1) if (dx, dy) != (0, 0)]

    def px(img, x, y):
        return float(img[min(max(y, 0), p.H - 1), min(max(x, 0), p.W - 1)])

    def bits(ref, img, x, y, qx, qy):
        return sum(int((px(ref, x, y) > px(ref, x + dx, y + dy)) != (px(img, qx, qy) > px(img, qx + dx, qy + dy)))
                   for dx, dy in offs)

    def near(a, d):
        return int(np.floor(a * d + 0.5))

    for arm in range(4):
        got = oracle.coarse_cost(cfg, cen, arm)
        (u, v), = oracle.arm_views(cfg, arm)
        for yy in range(p.H):
            for xx in range(p.W):
                for k in range(p.coarse_labels):
                    d = -1.0 + k * 0.5
                    qx = min(max(xx + near(u - p.uc, d), 0), p.W - 1)
                    qy = min(max(yy + near(v - p.vc, d), 0), p.H - 1)
                    want = sum(bits(views[p.vc, p.uc, c], views[v, u, c], xx, yy, qx, qy) for c in range(3))
                    assert got[yy * p.W + xx, k] == want
    lo, cnt = _full(p)
    off, cost = oracle.cost_volume(cfg, views, lo, cnt)
    for pix in (0, 9, 23, 41):
        yy, xx = divmod(pix, p.W)
        for g in range(p.fine_labels):
            d = -1.0 + g * 0.25
            want = 0
            for v in range(3):
                for u in range(3):
                    if (u, v) == (p.uc, p.vc):
                        continue
                    qx = min(max(xx + near(u - p.uc, d), 0), p.W - 1)
                    qy = min(max(yy + near(v - p.vc, d), 0), p.H - 1)
                    want += sum(bits(views[p.vc, p.uc, c], views[v, u, c], xx, yy, qx, qy) for c in range(3))
            assert cost[off[pix] + g] == want


def test_colour_with_constant_extra_channels_equals_grey():
    """Channels (I, k1, k2) with k1, k2 constant: the constant channels add nothing to census or
    to the norm, so every cost equals the one-channel cost of I."""
    p1 = _params(U=5, V=5, H=12, W=13)
    p3 = _params(U=5, V=5, H=12, W=13, channels=3)
    grey = lfsynth.random_views(5, 5, 12, 13, seed=3)
    rgb = np.empty((5, 5, 3, 12, 13), np.float32)
    rgb[:, :, 0] = grey
    rgb[:, :, 1] = 0.25
    rgb[:, :, 2] = 0.75
    lo, cnt = _full(p1)
    c1, c3 = oracle.make_cfg(p1), oracle.make_cfg(p3)
    _, cost1 = oracle.cost_volume(c1, grey, lo, cnt)
    _, cost3 = oracle.cost_volume(c3, rgb, lo, cnt)
    assert np.array_equal(cost1, cost3)
    for arm in range(4):
        assert np.array_equal(oracle.coarse_cost(c1, oracle.census_all(c1, grey), arm),
                              oracle.coarse_cost(c3, oracle.census_all(c3, rgb), arm))


def test_colour_channel_permutation_invariance():
    """Census sum and Euclidean norm are symmetric in the channels: permuting them in every view
    changes no cost (up to the order of the three-term sum of squares).  A reference channel
    paired with another view's different channel would break this."""
    p = _params(U=5, V=5, H=12, W=13, channels=3)
    rgb = lfsynth.random_views(5, 5, 12, 13, seed=8, channels=3)
    cfg = oracle.make_cfg(p)
    lo, cnt = _full(p)
    _, a = oracle.cost_volume(cfg, rgb, lo, cnt)
    _, b = oracle.cost_volume(cfg, np.ascontiguousarray(rgb[:, :, [2, 0, 1]]), lo, cnt)
    assert np.allclose(a, b, rtol=1e-14, atol=0)
    assert not np.allclose(a, oracle.cost_volume(oracle.make_cfg(_params(U=5, V=5, H=12, W=13)),
                                                 rgb[:, :, 0], lo, cnt)[1])


def test_colour_identical_channels_scale_the_costs():
    """Three identical channels: census costs triple and the norm is sqrt(3) |delta|; with the
    census term alone and every penalty tripled, SGM and the sub-pixel step are homogeneous, so
    the whole method returns the one-channel labels and disparities exactly."""
    views, gt, pg = lfsynth.integer_planes(H=40, W=40, w_l2=0.0, w_census=1.0)
    p3 = lfsynth.LFParams(**{**pg.__dict__, "channels": 3})
    rgb = np.repeat(views[:, :, None], 3, axis=2)
    c1, c3 = oracle.make_cfg(pg), oracle.make_cfg(p3)
    for arm in range(4):
        a = oracle.coarse_cost(c1, oracle.census_all(c1, views), arm)
        b = oracle.coarse_cost(c3, oracle.census_all(c3, rgb), arm)
        assert np.array_equal(3 * a, b)
    g = oracle.depth(c1, views, coarse_penalties=[(2, 20)] * 4, fine_penalties=(1.0, 10.0))
    r = oracle.depth(c3, rgb, coarse_penalties=[(6, 60)] * 4, fine_penalties=(3.0, 30.0))
    assert np.array_equal(3 * g["cost"], r["cost"])
    assert np.array_equal(g["label"], r["label"]) and np.array_equal(g["disp"], r["disp"])
    pl = lfsynth.LFParams(**{**pg.__dict__, "w_l2": 1.0, "w_census": 0.0})
    pl3 = lfsynth.LFParams(**{**pl.__dict__, "channels": 3})
    lo, cnt = g["lo"], g["cnt"]
    _, l1 = oracle.cost_volume(oracle.make_cfg(pl), views, lo, cnt)
    _, l3 = oracle.cost_volume(oracle.make_cfg(pl3), rgb, lo, cnt)
    assert np.allclose(l3, np.sqrt(3.0) * l1, rtol=1e-14, atol=0)


def test_colour_edges_are_the_union_of_channel_edges():
    """A pixel is excluded from the borders when any channel's Sobel magnitude passes the
    threshold; constant channels contribute none."""
    H, W = 9, 12
    img = np.full((3, H, W), 0.4)
    img[2, :, 6:] = 1.0                     # a step of 0.6 in the third channel only: gx = 2.4
    e = oracle.sobel_edges(img, 2.3)
    assert e[:, 5].all() and e[:, 6].all() and e.sum() == 2 * H
    img[0, 4:, :] = 0.0                     # a horizontal step of 0.4 in the first channel: gy = 1.6
    e2 = oracle.sobel_edges(img, 1.0)
    assert np.array_equal(e2, oracle.sobel_edges(img[0], 1.0) | oracle.sobel_edges(img[2], 1.0))
    assert e2[3].all() and e2[4].all()


def test_colour_rejects_other_channel_counts():
    with pytest.raises(ValueError):
        oracle.make_cfg(_params(channels=2))


def test_colour_view_gradient_matches_finite_differences():
    """Adjoint of the Euclidean norm (Eq. 12 over three channels): d||delta||/d delta_c =
    delta_c / ||delta||, checked through the whole loss against central differences."""
    tau = 0.1
    p = _params(U=5, V=5, H=14, W=14, channels=3)
    cfg = oracle.make_cfg(p)
    rng = np.random.default_rng(99)
    views = rng.uniform(0.0, 1.0, (5, 5, 3, 14, 14))
    lo = np.full(p.N, 4, np.int32)
    cnt = np.full(p.N, 12, np.int32)
    off, cost = oracle.cost_volume(cfg, views, lo, cnt)
    P1, P2 = 0.05 * cost.mean(), 0.5 * cost.mean()
    gd = rng.normal(size=p.N)
    _, _, _, gV = oracle.backward(cfg, views, lo, cnt, cost, P1, P2, gd, tau)
    assert gV.shape == views.shape

    def loss(vw):
        _, c = oracle.cost_volume(cfg, vw, lo, cnt)
        return oracle.loss_from_cost(cfg, lo, cnt, c, P1, P2, gd, tau)

    picks = [(2, 2, c, 7, 7) for c in range(3)] + [(0, 4, 1, 3, 9), (4, 1, 2, 10, 2), (3, 2, 0, 6, 6)]
    flat = np.abs(gV).reshape(-1)
    picks += [tuple(int(i) for i in t) for t in zip(*np.unravel_index(np.argsort(-flat)[:3], gV.shape))]
    h = 1e-6
    for t in picks:
        vp, vm = views.copy(), views.copy()
        vp[t] += h
        vm[t] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        assert abs(fd - gV[t]) <= 1e-6 + 5e-4 * max(abs(fd), abs(gV[t])), (t, fd, gV[t])
