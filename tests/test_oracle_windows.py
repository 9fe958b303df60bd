"""Pins of the oracle's window variants: the boundary-less search of Sec. IV-E (no initial map,
every window is the whole range) and the depth-dependent border threshold proposed in Sec. IV-F
(a larger lambda for small disparities), here linear in the window centre and rounded half up."""
import dataclasses

import numpy as np

import lfsynth
import oracle


def _cfg(G=41, R=2, R_far=6, **kw):
    p = lfsynth.LFParams(U=3, V=3, H=4, W=4, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=5,
                         fine_labels=G, fine_radius=R, fine_radius_far=R_far, **kw)
    return oracle.make_cfg(p)


def test_radius_hand_cases():
    """lambda(gc) = R + round_half_up((R_far - R)(G-1-gc)/(G-1)) worked by hand for G = 41."""
    up = _cfg(R=2, R_far=6)
    # gc: 40 -> 2 (near end), 0 -> 6 (far end), 20 -> 2 + 2, 30 -> 2 + 1, 35 -> 2 + round(0.5) = 3,
    # 25 -> 2 + round(1.5) = 4, 39 -> 2 + round(0.1) = 2
    for gc, want in [(40, 2), (0, 6), (20, 4), (30, 3), (35, 3), (25, 4), (39, 2)]:
        assert oracle.radius(up, gc) == want, gc
    down = _cfg(R=6, R_far=2)
    # decreasing towards the far end: 35 -> 6 + round(-0.5) = 6, 25 -> 6 + round(-1.5) = 5, 0 -> 2
    for gc, want in [(40, 6), (35, 6), (25, 5), (0, 2), (20, 4)]:
        assert oracle.radius(down, gc) == want, gc
    flat = _cfg(R=3, R_far=0)           # off: the constant threshold of Eq. 11
    assert all(oracle.radius(flat, g) == 3 for g in range(41))
    same = _cfg(R=4, R_far=4)
    assert all(oracle.radius(same, g) == 4 for g in range(41))


def test_windows_with_depth_dependent_radius():
    """Coarse grid of 5 labels on [-1, 1] (D_init k/8 coarse units), fine grid G = 41: the
    centre gc = round(D_init * 40 / 4) and the window [gc - lambda(gc), gc + lambda(gc)] clamped."""
    cfg = _cfg(R=2, R_far=6)
    dinit = np.array([0.0, 4.0, 2.0, 3.0, 1.0, np.nan])
    lo, cnt = oracle.windows(cfg, dinit)
    assert (lo[0], cnt[0]) == (0, 7)            # gc 0, lambda 6: [0, 6]
    assert (lo[1], cnt[1]) == (38, 3)           # gc 40, lambda 2: [38, 40]
    assert (lo[2], cnt[2]) == (16, 9)           # gc 20, lambda 4: [16, 24]
    assert (lo[3], cnt[3]) == (27, 7)           # gc 30, lambda 3: [27, 33]
    assert (lo[4], cnt[4]) == (5, 11)           # gc 10, lambda 2 + round(3.0) = 5: [5, 15]
    assert (lo[5], cnt[5]) == (0, 41)           # discarded: whole range


def test_boundless_windows_cover_the_range():
    cfg = _cfg(R=2, R_far=6, boundless=1)
    lo, cnt = oracle.windows(cfg, np.array([0.0, 2.0, np.nan, 4.0]))
    assert np.all(lo == 0) and np.all(cnt == 41)


def test_boundless_depth_equals_whole_range_windows():
    """The boundary-less search skips the initial map; its result equals the bounded method's
    when the radius covers the grid (every window is then the whole range as well)."""
    views, _, p = lfsynth.tiny(params=lfsynth.tiny_params(H=24, W=28, fine_labels=41, fine_radius=41))
    wide = oracle.depth(oracle.make_cfg(p), views)
    assert np.all(wide["cnt"] == 41)
    free = oracle.depth(oracle.make_cfg(dataclasses.replace(p, boundless=1, fine_radius=2)), views)
    assert len(free["arms"]) == 0 and np.all(np.isnan(free["dinit"]))
    assert np.array_equal(free["lo"], wide["lo"]) and np.array_equal(free["cnt"], wide["cnt"])
    assert np.array_equal(free["cost"], wide["cost"])
    assert np.array_equal(free["label"], wide["label"]) and np.array_equal(free["disp"], wide["disp"])
