"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, identities, brute force on tiny inputs, hand-worked fixtures).
None of these compares the oracle with itself or with the CUDA library."""
import itertools
import os

import numpy as np
import pytest

import lfsynth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def popcount(x: int) -> int:
    return bin(int(x)).count("1")


# ------------------------------------------------------------------ shift rule
def test_label_grid_endpoints_and_spacing():
    for dmin, dmax, L in [(-4.0, 4.0, 401), (-2.0, 2.0, 32), (-1.5, 1.5, 301)]:
        ds = [oracle.label_disp(dmin, dmax, L, k) for k in range(L)]
        assert ds[0] == dmin
        assert abs(ds[-1] - dmax) < 1e-12
        assert np.allclose(np.diff(ds), (dmax - dmin) / (L - 1), atol=1e-13)


def test_shift_integer_and_half_integer_exact():
    # bench fine grid: d_g = -4 + g/50; a*d_g is a multiple of 1/2 iff a*(g-200) % 25 == 0
    for a in range(-4, 5):
        for g in range(401):
            d = oracle.label_disp(-4.0, 4.0, 401, g)
            o, f, n = oracle.shift(a, d)
            assert 0.0 <= f < 1.0
            exact = a * (g - 200)  # s = exact / 50
            assert abs(o + f - exact / 50.0) < 1e-12
            if exact % 25 == 0:            # integer or half-integer shift
                assert f in (0.0, 0.5)
                assert o == (exact // 25) // 2 if f == 0.0 else True
            # nearest integer, halves upward
            assert n == int(np.floor(exact / 50.0 + 0.5 + (1e-12 if exact % 25 == 0 else 0)))


def test_shift_nearest_rounds_half_up():
    assert oracle.shift(1, 0.5) == (0, 0.5, 1)
    assert oracle.shift(1, -0.5) == (-1, 0.5, 0)
    assert oracle.shift(3, 0.5) == (1, 0.5, 2)
    assert oracle.shift(-2, 0.75) == (-2, 0.5, -1)


# ---------------------------------------------------------------------- census
def _ramp7(centre):
    img = np.array([[10 * y + x for x in range(7)] for y in range(7)], np.float32)
    img[3, 3] = centre
    return img


def test_census_hand_worked_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "census_hand.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for name, w, centre, hexv in rows:
        img = _ramp7(float(centre))
        got = oracle.census(img, int(w))[3, 3]
        assert int(got) == int(hexv, 16), name


def test_census_constant_image_is_zero():
    img = np.full((9, 11), 0.37, np.float32)
    for w in (5, 7):
        assert not oracle.census(img, w).any()


def test_census_invariant_under_increasing_map():
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 1, (20, 23)).astype(np.float32)
    f = (img.astype(np.float64) ** 3 + 2 * img).astype(np.float32)
    # f is strictly increasing on [0,1] and float32-representable differences stay ordered
    assert np.all(np.argsort(img, axis=None) == np.argsort(f, axis=None))
    for w in (5, 7):
        assert np.array_equal(oracle.census(img, w), oracle.census(f, w))


def test_census_negation_complements_interior():
    rng = np.random.default_rng(2)
    img = rng.permutation(20 * 20).reshape(20, 20).astype(np.float32)  # distinct values
    for w in (5, 7):
        h, nb = w // 2, w * w - 1
        a = oracle.census(img, w)[h:-h, h:-h]
        b = oracle.census(-img, w)[h:-h, h:-h]
        mask = np.uint64((1 << nb) - 1)
        assert np.array_equal(b, (~a) & mask)


def test_hamming_identities():
    rng = np.random.default_rng(3)
    words = [int(x) for x in rng.integers(0, 1 << 48, 40)]
    nb = 48
    mask = (1 << nb) - 1
    for a, b in itertools.product(words[:12], repeat=2):
        assert oracle.hamming(a, a) == 0
        assert oracle.hamming(a, b) == oracle.hamming(b, a) == popcount(a ^ b)
        assert oracle.hamming(a, (~b) & mask) == nb - oracle.hamming(a, b)
    for a, b, c in itertools.combinations(words[:10], 3):
        assert oracle.hamming(a, c) <= oracle.hamming(a, b) + oracle.hamming(b, c)


# ----------------------------------------------------------------- coarse cost
def test_coarse_cost_brute_force_bits():
    """Eq. 7 by direct pixel comparisons (no packed words): for each census offset o,
    a bit differs when xi(Iref(p), Iref(p+o)) != xi(Iv(q), Iv(q+o)), q = p + nearest shift."""
    p = lfsynth.LFParams(U=3, V=3, H=7, W=8, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=9,
                         fine_labels=9, fine_radius=1, init_views=1)
    views = lfsynth.random_views(3, 3, 7, 8, seed=5)
    cfg = oracle.make_cfg(p)
    cen = oracle.census_all(cfg, views)
    h = p.census_w // 2
    offs = [(dx, dy) for dy in range(-h, h + 1) for dx in range(-h, h + 1) if (dx, dy) != (0, 0)]

    def px(img, x, y):
        return float(img[min(max(y, 0), p.H - 1), min(max(x, 0), p.W - 1)])

    ref = views[p.vc, p.uc]
    for arm in range(4):
        got = oracle.coarse_cost(cfg, cen, arm)
        uv = oracle.arm_views(cfg, arm)
        assert len(uv) == 1
        u, v = uv[0]
        img = views[v, u]
        for y in range(p.H):
            for x in range(p.W):
                for k in range(p.coarse_labels):
                    d = -1.0 + k * 0.25
                    nx = int(np.floor((u - p.uc) * d + 0.5))
                    ny = int(np.floor((v - p.vc) * d + 0.5))
                    qx = min(max(x + nx, 0), p.W - 1)
                    qy = min(max(y + ny, 0), p.H - 1)
                    bits = 0
                    for dx, dy in offs:
                        r = px(ref, x, y) > px(ref, x + dx, y + dy)
                        s = px(img, qx, qy) > px(img, qx + dx, qy + dy)
                        bits += int(r != s)
                    assert got[y * p.W + x, k] == bits


def test_arm_views_order_and_extremes():
    p = lfsynth.bench_params()
    cfg = oracle.make_cfg(p)
    arms = [oracle.arm_views(cfg, a) for a in range(4)]
    assert [len(a) for a in arms] == [4, 4, 4, 4]
    assert arms[0][-1] == (4, 0) and arms[1][-1] == (4, 8)     # up, down
    assert arms[2][-1] == (0, 4) and arms[3][-1] == (8, 4)     # left, right
    cfg.init_views = 0
    assert [oracle.arm_views(cfg, a) for a in range(4)] == [[(4, 0)], [(4, 8)], [(0, 4)], [(8, 4)]]


def test_int_penalties():
    assert oracle.int_penalties(1000, 10, 0.05, 0.5) == (5, 50)
    assert oracle.int_penalties(10, 10, 0.05, 0.5) == (1, 1)        # P1 >= 1, P2 >= P1
    assert oracle.int_penalties(300, 10, 0.05, 0.5) == (2, 15)      # 1.5 -> 2 (half up)


# ------------------------------------------------------------------------- SGM
def _pairwise_V(P1, P2):
    def V(a, b):
        return 0 if a == b else (P1 if abs(a - b) == 1 else P2)
    return V


def _path_pixels(H, W, x, y, dx, dy):
    seq = []
    while 0 <= x < W and 0 <= y < H:
        seq.append((x, y))
        x, y = x - dx, y - dy
    return seq[::-1]


@pytest.mark.parametrize("direction", range(16))
def test_sgm_bounded_brute_force_path_energy(direction):
    """min over labels of the printed (unnormalised) Eq. 8 at the end of a path equals
    the minimum over all label sequences along the path of sum C + sum V, V = 0/P1/P2
    for |dg| = 0/1/>=2, with every label inside its pixel's window (Sec. III-E)."""
    rng = np.random.default_rng(10 + direction)
    H, W = 4, 4
    lo = rng.integers(0, 4, H * W).astype(np.int32)
    cnt = rng.integers(1, 4, H * W).astype(np.int32)
    off = oracle.offsets(cnt)
    cost = rng.uniform(0, 3, int(off[-1]))
    P1, P2 = 0.4, 1.3
    V = _pairwise_V(P1, P2)
    L = oracle.sgm_bounded_path(H, W, lo, cnt, off, cost, P1, P2, direction, normalised=False)
    dx, dy = oracle.DIRECTIONS[direction]
    for y in range(H):
        for x in range(W):
            path = _path_pixels(H, W, x, y, dx, dy)
            idx = [yy * W + xx for xx, yy in path]
            choices = [range(lo[i], lo[i] + cnt[i]) for i in idx]
            best = {}
            for seq in itertools.product(*choices):
                e = sum(cost[off[i] + g - lo[i]] for i, g in zip(idx, seq))
                e += sum(V(seq[k - 1], seq[k]) for k in range(1, len(seq)))
                best[seq[-1]] = min(best.get(seq[-1], np.inf), e)
            p = idx[-1]
            for g, e in best.items():
                assert abs(L[off[p] + g - lo[p]] - e) < 1e-12


@pytest.mark.parametrize("direction", [0, 3, 4, 7, 8, 11, 12, 15])
def test_sgm_int_brute_force_path_energy(direction):
    rng = np.random.default_rng(30 + direction)
    H, W, Lb = 3, 4, 3
    Cv = rng.integers(0, 9, (H * W, Lb)).astype(np.int64)
    P1, P2 = 2, 5
    V = _pairwise_V(P1, P2)
    Lr = oracle.sgm_int_path(H, W, Cv, P1, P2, direction)
    dx, dy = oracle.DIRECTIONS[direction]
    for y in range(H):
        for x in range(W):
            idx = [yy * W + xx for xx, yy in _path_pixels(H, W, x, y, dx, dy)]
            best = np.inf
            for seq in itertools.product(range(Lb), repeat=len(idx)):
                e = sum(int(Cv[i, g]) for i, g in zip(idx, seq))
                e += sum(V(seq[k - 1], seq[k]) for k in range(1, len(seq)))
                best = min(best, e)
            # normalised form: L_norm(p_k) = L_printed(p_k) - sum_{i<k} min_g L_norm(p_i)
            shift = sum(int(Lr[i].min()) for i in idx[:-1])
            assert int(Lr[idx[-1]].min()) + shift == best
    # normalised values stay in [C, C + P2]
    assert np.all(Lr - Cv >= 0) and np.all(Lr - Cv <= P2)


def test_sgm_normalised_is_shifted_unnormalised():
    rng = np.random.default_rng(4)
    H, W = 5, 6
    lo = rng.integers(0, 5, H * W).astype(np.int32)
    cnt = rng.integers(1, 6, H * W).astype(np.int32)
    off = oracle.offsets(cnt)
    cost = rng.uniform(0, 5, int(off[-1]))
    for r in range(16):
        a = oracle.sgm_bounded_path(H, W, lo, cnt, off, cost, 0.5, 2.0, r, True)
        b = oracle.sgm_bounded_path(H, W, lo, cnt, off, cost, 0.5, 2.0, r, False)
        for p in range(H * W):
            sa, sb = a[off[p]:off[p + 1]], b[off[p]:off[p + 1]]
            d = sb - sa
            assert np.ptp(d) < 1e-9                        # per-pixel constant shift
            assert np.argmin(sa) == np.argmin(sb)
            assert np.all(sa - cost[off[p]:off[p + 1]] >= -1e-12)
            assert np.all(sa - cost[off[p]:off[p + 1]] <= 2.0 + 1e-12)


def test_sgm_zero_penalties_gives_eight_times_cost_exactly():
    rng = np.random.default_rng(6)
    H, W = 6, 7
    lo = rng.integers(0, 30, H * W).astype(np.int32)
    cnt = rng.integers(1, 9, H * W).astype(np.int32)
    off = oracle.offsets(cnt)
    cost = rng.uniform(0, 40, int(off[-1]))
    Cs = oracle.sgm_bounded(H, W, lo, cnt, off, cost, 0.0, 0.0)
    assert np.array_equal(Cs, 8.0 * cost)
    assert np.array_equal(oracle.sgm_bounded(H, W, lo, cnt, off, cost, 0.0, 0.0, paths=16), 16.0 * cost)
    Ci = rng.integers(0, 200, (H * W, 11)).astype(np.int64)
    assert np.array_equal(oracle.sgm_int(H, W, Ci, 0, 0), 8 * Ci)
    assert np.array_equal(oracle.sgm_int(H, W, Ci, 0, 0, paths=16), 16 * Ci)


def test_sgm_full_window_matches_int_version():
    """With every window the whole range and integer costs, the bounded FP64 SGM and
    the integer SGM are the same recurrence."""
    rng = np.random.default_rng(8)
    H, W, Lb = 5, 5, 6
    Ci = rng.integers(0, 30, (H * W, Lb)).astype(np.int64)
    lo = np.zeros(H * W, np.int32)
    cnt = np.full(H * W, Lb, np.int32)
    off = oracle.offsets(cnt)
    for paths in (8, 16):
        a = oracle.sgm_int(H, W, Ci, 3, 11, paths)
        b = oracle.sgm_bounded(H, W, lo, cnt, off, Ci.reshape(-1).astype(np.float64), 3.0, 11.0, paths)
        assert np.array_equal(a.reshape(-1).astype(np.float64), b)


# ------------------------------------------------------------- WTA + subpixel
def _cfg1(G=41, dmin=-2.0, dmax=2.0):
    p = lfsynth.LFParams(U=3, V=3, H=1, W=1, census_w=5, dmin=dmin, dmax=dmax, coarse_labels=5,
                         fine_labels=G, fine_radius=5)
    return oracle.make_cfg(p)


def _wta_int_row(row):
    Cs = np.ascontiguousarray(np.asarray(row, np.int64).reshape(1, -1))
    return int(oracle.wta_int(Cs)[0])


def test_coarse_wta_hand_cases_lowest_label_on_ties():
    """Eq. 10 on the integer coarse sums: D(p) = argmin_k C_s(p,k).  The paper does not say which
    label wins a tie; the reading is the lowest one.  Hand cases put the tie at the first label,
    in the middle, at the last two labels, and across the whole row."""
    cases = [
        ([5, 5, 7, 9], 0),                       # tie at the first label
        ([9, 3, 8, 3, 4], 1),                    # tie in the middle, later copy ignored
        ([8, 6, 9, 2, 2], 3),                    # tie on the last two labels
        ([4, 4, 4, 4, 4, 4], 0),                 # every label ties
        ([7], 0),                                # one label
        ([9, 8, 7, 6, 5, 1], 5),                 # strict minimum on the last label
        ([1, 2, 3, 4], 0),                       # strict minimum on the first label
        ([3, 1, 2, 1, 1, 0, 0], 5),              # the lowest value wins before any tie rule
        ([2 ** 40 + 1, 2 ** 40, 2 ** 40 + 2], 1),  # int64 sums, beyond 32 bits
    ]
    for row, want in cases:
        assert _wta_int_row(row) == want, (row, want)


def test_coarse_wta_matches_first_minimum_brute_force():
    """Random integer rows with many ties (values from a small range) against numpy.argmin, whose
    documented rule returns the first occurrence of the minimum, and against a scan for the
    smallest index whose value equals the row minimum."""
    rng = np.random.default_rng(131)
    for L, hi in [(2, 2), (3, 3), (16, 4), (100, 6), (256, 3), (97, 1000)]:
        Cs = rng.integers(0, hi, size=(400, L)).astype(np.int64)
        got = oracle.wta_int(Cs)
        assert np.array_equal(got, np.argmin(Cs, axis=1))
        first = np.array([int(np.flatnonzero(r == r.min())[0]) for r in Cs])
        assert np.array_equal(got, first)


def test_subpixel_recovers_parabola_vertex():
    cfg = _cfg1()
    step = 4.0 / 40
    rng = np.random.default_rng(9)
    for _ in range(50):
        lo, cnt = 7, 9
        g0 = lo + 2 + rng.uniform(0.6, cnt - 3.6)      # vertex strictly inside
        gs = np.arange(lo, lo + cnt)
        Cs = 3.7 * (gs - g0) ** 2 + 1.25
        label, disp, gap = oracle.wta_subpixel(cfg, np.array([lo]), np.array([cnt]),
                                               np.array([0, cnt]), Cs, mode=1)
        assert label[0] == int(np.floor(g0 + 0.5))
        assert abs(disp[0] - (-2.0 + g0 * step)) < 1e-12


def test_subpixel_conditions_and_ties():
    cfg = _cfg1()
    off = np.array([0, 4])
    # cnt < 5 -> no interpolation
    label, disp, _ = oracle.wta_subpixel(cfg, np.array([3]), np.array([4]), off,
                                         np.array([4.0, 1.0, 2.0, 5.0]), mode=1)
    assert label[0] == 4 and disp[0] == -2.0 + 4 * 0.1
    # winner on the window edge -> no interpolation; ties -> lowest label
    off = np.array([0, 6])
    label, disp, gap = oracle.wta_subpixel(cfg, np.array([10]), np.array([6]), off,
                                           np.array([1.0, 1.0, 2.0, 3.0, 4.0, 5.0]), mode=1)
    assert label[0] == 10 and disp[0] == -2.0 + 10 * 0.1 and gap[0] == 0.0
    # mode 0 -> integer label disparity
    label, disp, _ = oracle.wta_subpixel(cfg, np.array([10]), np.array([6]), off,
                                         np.array([3.0, 2.0, 1.0, 1.5, 4.0, 5.0]), mode=0)
    assert label[0] == 12 and disp[0] == -2.0 + 12 * 0.1


def test_softargmin_limits():
    cfg = _cfg1()
    off = np.array([0, 5])
    # equal costs -> mean of the window's disparities
    _, disp, _ = oracle.wta_subpixel(cfg, np.array([10]), np.array([5]), off, np.zeros(5), mode=2)
    assert abs(disp[0] - (-2.0 + 12 * 0.1)) < 1e-12
    # one cost far below the rest -> its disparity
    _, disp, _ = oracle.wta_subpixel(cfg, np.array([10]), np.array([5]), off,
                                     np.array([9.0, 9.0, 9.0, 0.0, 9.0]), mode=2, tau=0.1)
    assert abs(disp[0] - (-2.0 + 13 * 0.1)) < 1e-30 + 1e-12


# ------------------------------------------------------- fusion / fill / borders
def test_fusion_hand_cases():
    maps = np.array([[10, 10, 10, 5], [11, 14, 20, 5], [12, 10, 10, 5], [10, 10, 10, 7]], np.int32)
    d = oracle.fuse(maps, 3.0)
    assert d[0] == ((10 + 11) / 2 + 12) / 2 / 2 + 10 / 2      # 10 -> 10.5 -> 11.25 -> 10.625
    assert d[0] == 10.625
    assert np.isnan(d[1])                                       # |10 - 14| >= 3
    assert np.isnan(d[2])                                       # sticky: later agreement ignored
    assert d[3] == 6.0                                          # 5 -> 5 -> 5 -> (5+7)/2
    maps = np.array([[10], [13]], np.int32)
    assert np.isnan(oracle.fuse(maps, 3.0)[0])                  # strict inequality


def test_hole_fill_hand_cases():
    nan = np.nan
    d = np.array([[1, 2, 3], [4, nan, 5], [6, 7, 8]], np.float64)
    out = oracle.hole_fill(d, 3, 3, 1).reshape(3, 3)
    assert out[1, 1] == 4.0                                     # lower middle of 1..8
    # Jacobi: a hole whose only neighbours are holes stays in pass 1, filled in pass 2
    d = np.full((5, 5), nan)
    d[0, 0] = 3.0
    out1 = oracle.hole_fill(d, 5, 5, 1).reshape(5, 5)
    assert out1[0, 1] == 3.0 and out1[1, 1] == 3.0 and np.isnan(out1[0, 2])
    out2 = oracle.hole_fill(d, 5, 5, 2).reshape(5, 5)
    assert out2[0, 2] == 3.0 and out2[2, 2] == 3.0 and np.isnan(out2[0, 3])
    full = np.arange(12, dtype=np.float64)
    assert np.array_equal(oracle.hole_fill(full, 3, 4, 2), full)
    assert np.isnan(oracle.hole_fill(np.full(4, nan), 2, 2, 2)).all()


def test_windows_hand_cases():
    p = lfsynth.bench_params()
    cfg = oracle.make_cfg(p)
    dinit = np.array([0.0, 99.0, 50.0, np.nan, 0.125 * 3, 49.5])
    lo, cnt = oracle.windows(cfg, dinit)
    assert (lo[0], cnt[0]) == (0, 16)                  # saturated at d_min
    assert (lo[1], cnt[1]) == (385, 16)                # saturated at d_max
    assert (lo[2], cnt[2]) == (202 - 15, 31)           # d = -4 + 50*8/99 -> label 202.02
    assert (lo[3], cnt[3]) == (0, 401)                 # discarded -> whole range
    assert (lo[4], cnt[4]) == (0, 18)                  # 0.375 * 400/99 = 1.515 -> 2: [0, 17]
    assert (lo[5], cnt[5]) == (200 - 15, 31)           # 49.5 * 400/99 = 200 exactly


# -------------------------------------------------------------- cost volume
def _ramp_views(U, V, H, W, alpha, beta, gamma, d0):
    uc, vc = (U - 1) // 2, (V - 1) // 2
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    views = np.zeros((V, U, H, W), np.float32)
    for v in range(V):
        for u in range(U):
            a, b = u - uc, v - vc
            views[v, u] = alpha * (x - a * d0) + beta * (y - b * d0) + gamma
    return views


def test_cost_l2_closed_form_on_linear_ramp():
    """For I_uv(x,y) = alpha (x - a d0) + beta (y - b d0) + gamma (a plane at disparity d0
    seen through a linear texture), bilinear sampling is exact, so away from the image
    border C_l2(p, d) = sum_views |alpha a + beta b| |d - d0| (Eq. 1, 6, 12)."""
    U = V = 5
    H = W = 24
    alpha, beta, gamma, d0 = 0.013, -0.029, 0.5, 0.37
    views = _ramp_views(U, V, H, W, alpha, beta, gamma, d0)
    p = lfsynth.LFParams(U=U, V=V, H=H, W=W, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=5,
                         fine_labels=41, fine_radius=3, w_l2=1.0, w_census=0.0)
    cfg = oracle.make_cfg(p)
    N = H * W
    lo = np.full(N, 0, np.int32)
    cnt = np.full(N, 41, np.int32)
    off, cost = oracle.cost_volume(cfg, views, lo, cnt)
    ws = sum(abs(alpha * (u - 2) + beta * (v - 2)) for u in range(U) for v in range(V))
    m = 5  # |shift| <= 2 * 1.0 plus one tap
    for y in range(m, H - m):
        for x in range(m, W - m):
            pix = y * W + x
            for g in range(41):
                d = -1.0 + g * 0.05
                assert abs(cost[off[pix] + g] - ws * abs(d - d0)) < 2e-5


def test_cost_exact_zero_at_true_integer_label():
    views, gt, p = lfsynth.integer_planes(U=5, V=5, H=32, W=32, disps=(1.0,))
    cfg = oracle.make_cfg(p)
    N = p.N
    lo = np.zeros(N, np.int32)
    cnt = np.full(N, p.fine_labels, np.int32)
    off, cost = oracle.cost_volume(cfg, views, lo, cnt)
    g_true = int(round((1.0 - p.dmin) / p.fine_step))
    m = 2 * 2 + 2 + 1
    for y in range(m, p.H - m):
        for x in range(m, p.W - m):
            pix = y * p.W + x
            c = cost[off[pix]:off[pix + 1]]
            assert c[g_true] == 0.0
            assert np.argmin(c) == g_true


def test_census_only_cost_is_integer():
    views = lfsynth.random_views(3, 3, 10, 10, seed=11)
    p = lfsynth.LFParams(U=3, V=3, H=10, W=10, census_w=5, dmin=-1.0, dmax=1.0, coarse_labels=5,
                         fine_labels=9, fine_radius=1, w_l2=0.0, w_census=1.0)
    cfg = oracle.make_cfg(p)
    lo = np.zeros(100, np.int32)
    cnt = np.full(100, 9, np.int32)
    _, cost = oracle.cost_volume(cfg, views, lo, cnt)
    assert np.array_equal(cost, np.round(cost))
    assert cost.max() <= 8 * 24


# ----------------------------------------------------------------- end to end
def test_end_to_end_exact_integer_planes():
    """Noise-free fronto-parallel planes with integer disparity: the fine label of
    the true disparity must win at every pixel away from borders and depth edges."""
    views, gt, p = lfsynth.integer_planes(H=96, W=96)
    cfg = oracle.make_cfg(p)
    out = oracle.depth(cfg, views)
    g_true = np.rint((gt.reshape(-1) - p.dmin) / p.fine_step).astype(np.int32)
    m = 2 * 2 + p.census_w // 2 + 1     # parallax across a depth edge + census half-window
    gt2 = gt.reshape(p.H, p.W)
    edge = np.zeros_like(gt2, bool)
    for dy in range(-m, m + 1):
        for dx in range(-m, m + 1):
            edge |= np.roll(np.roll(gt2, dy, 0), dx, 1) != gt2
    ys, xs = np.mgrid[0:p.H, 0:p.W]
    inner = (~edge) & (ys >= m) & (ys < p.H - m) & (xs >= m) & (xs < p.W - m)
    assert inner.sum() > 300
    lab = out["label"].reshape(p.H, p.W)
    assert np.array_equal(lab[inner], g_true.reshape(p.H, p.W)[inner])
    disp = out["disp"].reshape(p.H, p.W)
    assert np.all(np.abs(disp[inner] - gt2[inner]) <= 0.5 * p.fine_step + 1e-12)


# ------------------------------------------------------------ post-processing (Sec. III-F)
def _median3_numpy(d):
    """Independent restatement: NumPy's median over edge-padded 3 x 3 windows."""
    p = np.pad(d, 1, mode="edge")
    H, W = d.shape
    win = np.stack([p[dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3)])
    return np.median(win, axis=0)


def test_median3_matches_padded_numpy_median():
    rng = np.random.default_rng(21)
    for shape in [(1, 1), (1, 9), (7, 1), (6, 11), (33, 20)]:
        d = rng.normal(size=shape)
        d[rng.random(shape) < 0.3] = 0.5           # ties
        assert np.array_equal(oracle.median3(d), _median3_numpy(d)), shape


def test_median3_removes_impulses_and_keeps_ramps():
    H, W = 12, 15
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    ramp = 0.25 * x - 0.5 * y + 3.0
    m = oracle.median3(ramp)
    # interior: the window values are ramp(p) + {a i + b j}, symmetric about ramp(p)
    assert np.array_equal(m[1:-1, 1:-1], ramp[1:-1, 1:-1])
    # a map varying along x only keeps its left and right border columns (6 of 9 values repeat)
    xr = np.broadcast_to(0.1 * x[0], (H, W)).copy()
    assert np.array_equal(oracle.median3(xr), xr)
    # isolated impulses on a constant background disappear
    c = np.full((H, W), 1.5)
    c[3, 4] = 100.0
    c[8, 10] = -7.0
    c[0, 0] = 9.0
    assert np.array_equal(oracle.median3(c), np.full((H, W), 1.5))


# -------------------------------------------------- edge exclusion from the borders (Sec. III-D)
def test_sobel_edges_on_constant_ramp_and_step():
    H, W = 9, 12
    assert not oracle.sobel_edges(np.full((H, W), 0.3), 1e-6).any()
    # linear ramp a x: gx = 8 a in the interior (the weights 1, 2, 1 over a central difference of 2a)
    a = 0.125
    ramp = np.broadcast_to(a * np.arange(W, dtype=np.float64), (H, W))
    e_lo = oracle.sobel_edges(ramp, 8 * a - 0.01)
    e_hi = oracle.sobel_edges(ramp, 8 * a + 0.01)
    assert e_lo[:, 1:-1].all() and not e_hi.any()
    # border columns see a one-sided difference a: gx = 4 a
    assert not e_lo[:, 0].any() and not e_lo[:, -1].any()
    # a vertical step of height 1 between columns 5 and 6: gx = 4 on both columns next to it
    step = np.zeros((H, W))
    step[:, 6:] = 1.0
    e = oracle.sobel_edges(step, 3.9)
    assert e[:, 5].all() and e[:, 6].all() and e.sum() == 2 * H


def test_edges_search_the_whole_range():
    p = lfsynth.tiny_params(H=8, W=8, edge_threshold=0.5)
    cfg = oracle.make_cfg(p)
    dinit = np.full(p.N, 3.0)
    edge = np.zeros(p.N, bool)
    edge[[5, 17, 60]] = True
    lo0, cnt0 = oracle.windows(cfg, dinit)
    lo, cnt = oracle.windows(cfg, dinit, edge)
    assert np.array_equal(lo[~edge], lo0[~edge]) and np.array_equal(cnt[~edge], cnt0[~edge])
    assert np.all(lo[edge] == 0) and np.all(cnt[edge] == p.fine_labels)
