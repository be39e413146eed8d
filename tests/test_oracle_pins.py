"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these re-types the oracle's own formula: each checks a closed form,
an invariant, a special case that reduces to a textbook/library routine, or
brute force on tiny inputs, chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails one of them.
"""
import itertools
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------- pyramid
def test_pyramid_weights_quantise_sigma1_gaussian(orc):
    w = orc.pyr_weights()
    g = np.exp(-0.5 * np.array([1.0, 0.0, 1.0]))
    g = 256.0 * g / g.sum()
    assert w.sum() == 256
    assert np.all(np.abs(w - g) <= 0.5)
    assert list(w) == [70, 116, 70]


def test_pyramid_constant_and_impulse(orc):
    img = np.full((9, 11), 77, np.uint8)
    out = orc.pyramid_down(img)
    assert out.shape == (5, 6) and np.all(out == 77)
    # an impulse at even (4, 4) lands on output (2, 2) with weight 116*116
    imp = np.zeros((12, 12), np.uint8)
    imp[4, 4] = 255
    o = orc.pyramid_down(imp).astype(np.int64)
    assert o[2, 2] == (255 * 116 * 116 + 32768) >> 16 == 52
    assert o.sum() == o[2, 2]
    # at odd x = 5 it is shared by outputs x = 2 and x = 3 (weights 70*116)
    imp2 = np.zeros((12, 12), np.uint8)
    imp2[4, 5] = 255
    o2 = orc.pyramid_down(imp2).astype(np.int64)
    assert o2[2, 2] == o2[2, 3] == (255 * 70 * 116 + 32768) >> 16 == 32
    assert o2.sum() == 64


# ---------------------------------------------------------------- census
def test_census_ramps_hand_computed(orc):
    x = np.tile(np.arange(20, dtype=np.uint8) * 3, (15, 1))
    c = orc.census(x)
    # horizontal ramp: exactly the taps with dx < 0 are darker
    row = 0b1111
    expect = sum(row << (9 * r) for r in range(7))
    assert int(c[7, 10]) == expect
    y = x.T.copy()
    c2 = orc.census(y)
    # vertical ramp: the three rows above (27 taps) are darker
    assert int(c2[10, 7]) == (1 << 27) - 1


def test_census_centre_bit_zero_and_max_distance(orc):
    g = np.random.default_rng(1)
    img = g.integers(0, 256, (30, 40), dtype=np.uint8)
    c = orc.census(img)
    assert not np.any(c & np.uint64(1 << 31))
    peak = np.zeros((9, 11), np.uint8)
    peak[4, 5] = 200
    a = orc.census(np.zeros_like(peak))[4, 5]
    b = orc.census(peak)[4, 5]
    assert orc.hamming(a, b) == 62
    assert orc.hamming(b, b) == 0


def test_census_invariant_under_increasing_map(orc):
    g = np.random.default_rng(2)
    img = g.integers(0, 200, (25, 33), dtype=np.uint8)
    f = np.sort(g.choice(256, 200, replace=False)).astype(np.uint8)   # strictly increasing
    assert np.array_equal(orc.census(img), orc.census(f[img]))


def test_popcount_hamming_matches_bit_loop(orc):
    g = np.random.default_rng(3)
    for _ in range(50):
        a, b = (int(v) for v in g.integers(0, 2 ** 63, 2, dtype=np.uint64))
        assert orc.hamming(a, b) == bin(a ^ b).count("1")


# ---------------------------------------------------------------- homography
def _pose(g):
    ax = g.normal(size=3) * 0.05
    th = np.linalg.norm(ax)
    k = ax / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
    return R, g.normal(size=3)


def test_homography_point_transfer(orc):
    g = np.random.default_rng(4)
    K = np.array([[500.0, 0, 319.5], [0, 510.0, 239.5], [0, 0, 1]])
    for _ in range(20):
        R, t = _pose(g)
        n = g.normal(size=3)
        n /= np.linalg.norm(n)
        n = n if n[2] < 0 else -n
        delta = g.uniform(5, 50)
        Hm = orc.homography(K, R, t, n, delta)
        for _ in range(10):
            # a point on n^T X + delta = 0
            X = g.normal(size=3) * 3.0
            X = X - (n @ X + delta) * n
            if X[2] < 0.5:
                continue
            pr = K @ X
            pr /= pr[2]
            Xk = R @ X + t
            pk = K @ Xk
            pk /= pk[2]
            q = Hm @ pr
            q /= q[2]
            assert np.allclose(q[:2], pk[:2], atol=1e-8, rtol=0)


def test_homography_identity_and_stereo_normal_case(orc):
    K = np.array([[300.0, 0, 100.0], [0, 300.0, 80.0], [0, 0, 1]])
    n = np.array([0.0, 0.0, -1.0])
    Hm = orc.homography(K, np.eye(3), np.zeros(3), n, 7.0)
    assert np.allclose(Hm, np.eye(3), atol=1e-14)
    b, Z = 0.4, 12.0
    Hm = orc.homography(K, np.eye(3), np.array([-b, 0.0, 0.0]), n, Z)
    for u, v in [(3.0, 4.0), (150.0, 20.0)]:
        q = Hm @ np.array([u, v, 1.0])
        q /= q[2]
        assert abs((u - q[0]) - 300.0 * b / Z) < 1e-10 and abs(q[1] - v) < 1e-10


# ---------------------------------------------------------------- warp
def test_warp_identity_integer_and_half_shifts(orc):
    g = np.random.default_rng(5)
    img = g.integers(0, 256, (20, 30), dtype=np.uint8)
    w, val = orc.warp_image(img, np.eye(3))
    assert val.all() and np.array_equal(w, img.astype(np.float64))
    T = np.array([[1, 0, 2.0], [0, 1, -1.0], [0, 0, 1]])
    w, val = orc.warp_image(img, T)
    exp = img[:-1, 2:].astype(np.float64)                 # value at (x+2, y-1)
    assert np.array_equal(w[1:, :-2], exp)
    assert val[1:, :-2].all() and not val[0].any() and not val[:, -2:].any()
    Th = np.array([[1, 0, 0.5], [0, 1, 0.0], [0, 0, 1]])
    w, _ = orc.warp_image(img, Th)
    exp = (img[:, :-1].astype(np.float64) + img[:, 1:]) / 2
    assert np.array_equal(w[:, :-1], exp)
    # a quarter-pixel shift gives (3 a + b) / 4: the value is not rounded
    Tq = np.array([[1, 0, 0.25], [0, 1, 0.0], [0, 0, 1]])
    w, _ = orc.warp_image(img, Tq)
    a = img.astype(np.float64)
    assert np.array_equal(w[:, :-1], 0.75 * a[:, :-1] + 0.25 * a[:, 1:])


def test_warp_matches_weight_sum_bilinear_at_real_positions(orc):
    """The lerp form equals the textbook weight-sum bilinear interpolation
    (1-a)(1-b) I00 + a(1-b) I01 + (1-a) b I10 + a b I11 up to rounding, at
    unrounded positions, and clamps to the image outside it."""
    g = np.random.default_rng(51)
    H, W = 25, 33
    img = g.integers(0, 256, (H, W), dtype=np.uint8)
    A = np.array([[0.93, 0.071, 1.37], [-0.052, 1.04, 0.83], [1e-3, -2e-3, 1.0]])
    w, val = orc.warp_image(img, A)
    I = img.astype(np.float64)
    for y in range(H):
        for x in range(W):
            q = A @ [x, y, 1.0]
            u, v = q[0] / q[2], q[1] / q[2]
            cu, cv = min(max(u, 0.0), W - 1.0), min(max(v, 0.0), H - 1.0)
            iu, iv = min(int(cu), W - 2), min(int(cv), H - 2)
            a, b = cu - iu, cv - iv
            want = ((1 - a) * (1 - b) * I[iv, iu] + a * (1 - b) * I[iv, iu + 1]
                    + (1 - a) * b * I[iv + 1, iu] + a * b * I[iv + 1, iu + 1])
            assert abs(w[y, x] - want) < 1e-11
            assert val[y, x] == (0 <= u <= W - 1 and 0 <= v <= H - 1)
    # a point behind the camera is invalid and reads the corner pixel (0, 0)
    back = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, -1.0]])
    w, val = orc.warp_image(img, back)
    assert not val.any() and np.all(w == I[0, 0])


def test_warp_bilinear_exact_on_ramp(orc):
    # I = 5x + 3y is reproduced by bilinear interpolation at any position
    # inside the image (up to rounding)
    xs, ys = np.meshgrid(np.arange(40), np.arange(30))
    img = (5 * xs + 3 * ys).astype(np.uint8)
    A = np.array([[0.9, 0.05, 1.3], [-0.04, 0.95, 2.1], [0.0, 0.0, 1.0]])
    w, val = orc.warp_image(img, A)
    for y in range(0, 20, 3):
        for x in range(0, 25, 4):
            if not val[y, x]:
                continue
            u = A[0] @ [x, y, 1]
            v = A[1] @ [x, y, 1]
            assert abs(w[y, x] - (5 * u + 3 * v)) < 1e-12


# ---------------------------------------------------------------- left/right
def test_left_right_combination(orc):
    assert orc.lr_combine(17, 1, 9, 1) == 9
    assert orc.lr_combine(3, 1, 40, 1) == 3
    # 2 left / 3 right: the left sum is rescaled to 3 images, half up
    assert orc.lr_combine(7, 2, 100, 3) == (7 * 3 + 1) // 2 == 11
    assert orc.lr_combine(100, 2, 13, 3) == 13
    assert orc.lr_combine(0, 0, 13, 2) == 13


# ---------------------------------------------------------------- cost volume
def test_cost_volume_identity_views_are_zero(orc):
    g = np.random.default_rng(6)
    img = g.integers(0, 256, (14, 17), dtype=np.uint8)
    K = np.array([[20.0, 0, 8.0], [0, 20.0, 6.5], [0, 0, 1]])
    R = np.stack([np.eye(3)] * 2)
    t = np.zeros((2, 3))
    S = orc.cost_volume(img, [img, img], [-1, 1], K, R, t, [0, 0, -1.0], 0.1, 0.05, 5)
    assert S.shape == (14, 17, 5) and not S.any()


def test_cost_volume_exact_disparity_plane(orc):
    # stereo normal case: the right camera sits b to the right, so a point at
    # depth Z moves by f b / Z px to the left; the right view is the reference
    # moved by 3 px: right(x) = ref(x + 3).  f, b and the plane distances are
    # binary fractions, so the homography of plane 3 moves every pixel by
    # exactly 3 px in FP64.
    g = np.random.default_rng(7)
    W, H, f, b = 40, 20, 64.0, 0.5
    big = g.integers(0, 256, (H, W + 12), dtype=np.uint8)
    ref = big[:, 6:6 + W]
    right = big[:, 9:9 + W]
    K = np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1]])
    drho = 1.0 / 32.0                  # f b rho_g = g px of disparity
    rho0 = 0.0
    S = orc.cost_volume(ref, [right], [1], K, np.eye(3)[None], np.array([[-b, 0, 0]]),
                        [0, 0, -1.0], rho0, drho, 6)
    inner = S[3:-3, 8:-4]
    assert not inner[..., 3].any()
    assert np.all(inner[..., 3] <= inner.min(axis=-1))
    # out-of-image centre samples cost the maximum 62
    assert np.all(S[:, :4, 5] == 62)


def test_cost_volume_windows_select_planes(orc):
    g = np.random.default_rng(8)
    img = g.integers(0, 256, (12, 16), dtype=np.uint8)
    nb = g.integers(0, 256, (12, 16), dtype=np.uint8)
    K = np.array([[25.0, 0, 7.5], [0, 25.0, 5.5], [0, 0, 1]])
    R = np.eye(3)[None]
    t = np.array([[0.3, 0.02, 0.01]])
    full = orc.cost_volume(img, [nb], [1], K, R, t, [0, 0, -1.0], 0.05, 0.01, 12)
    lo = g.integers(0, 12 - 4 + 1, (12, 16)).astype(np.int32)
    win = orc.cost_volume(img, [nb], [1], K, R, t, [0, 0, -1.0], 0.05, 0.01, 12, lo=lo, D=4, Ds=8)
    for y in range(12):
        for x in range(16):
            assert np.array_equal(win[y, x, :4], full[y, x, lo[y, x]:lo[y, x] + 4])
            assert not win[y, x, 4:].any()


# ---------------------------------------------------------------- SGM
DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]


def test_path_order(orc):
    assert [orc.path_dir(r) for r in range(8)] == DIRS


def test_sgm_zero_penalties_is_path_count_times_cost(orc):
    g = np.random.default_rng(9)
    S = g.integers(0, 63, (12, 16, 8)).astype(np.uint16)
    for paths in (8, 4):
        Sb = orc.sgm_aggregate(S, 0, 0, paths=paths)
        assert np.array_equal(Sb.astype(np.int64), paths * S.astype(np.int64))


def test_sgm_bound_every_voxel(orc):
    g = np.random.default_rng(10)
    S = g.integers(0, 63, (10, 13, 9)).astype(np.uint16)
    img = g.integers(0, 256, (10, 13), dtype=np.uint8)
    lut = orc.p2_table(12)
    for r in range(8):
        L = orc.sgm_path(S, r, 12, lut=lut, img=img).astype(np.int64)
        assert np.all(L >= S) and np.all(L <= S.astype(np.int64) + lut.max())
        # the minimum over hypotheses is attained: min_s L - min_s S in [0, P2]
        assert np.all(L.min(-1) >= S.min(-1))


def _sgm_line_quadratic(Sline, lo_line, di_line, P1, P2s, D):
    """Plain definition, O(D^2): L(p, s) = S + min_{s'} (L(p-r, s') + V) - M,
    with V on global plane indices g = lo + s (zero-cost at g' = g + di)."""
    out = []
    prev = None
    for i, Sp in enumerate(Sline):
        if prev is None:
            cur = Sp.astype(np.int64)
        else:
            M = prev.min()
            cur = np.zeros(D, np.int64)
            for s in range(D):
                gz = lo_line[i] + s + di_line[i]
                best = None
                for s2 in range(D):
                    gp = lo_line[i - 1] + s2
                    d = abs(gz - gp)
                    v = 0 if d == 0 else (P1 if d == 1 else max(P2s[i], P1))
                    c = prev[s2] + v
                    best = c if best is None else min(best, c)
                cur[s] = int(Sp[s]) + best - M
        out.append(cur)
        prev = cur
    return out


def _line(W, H, r, x, y):
    dx, dy = DIRS[r]
    while 0 <= x - dx < W and 0 <= y - dy < H:
        x, y = x - dx, y - dy
    pts = []
    while 0 <= x < W and 0 <= y < H:
        pts.append((x, y))
        x, y = x + dx, y + dy
    return pts


@pytest.mark.parametrize("variant", [0, 1])
def test_sgm_linear_form_equals_quadratic_definition(orc, variant):
    g = np.random.default_rng(11 + variant)
    H, W, D, G = 9, 11, 6, 14
    S = g.integers(0, 63, (H, W, D)).astype(np.uint16)
    lo = g.integers(0, G - D + 1, (H, W)).astype(np.int32)
    img = g.integers(0, 256, (H, W), dtype=np.uint8)
    dI = g.integers(-3, 4, (8, H, W)).astype(np.int8) if variant == 1 else None
    P1 = 7
    lut = orc.p2_table(P1)
    for r in range(8):
        L = orc.sgm_path(S, r, P1, lut=lut, lo=lo, dI=dI, img=img, variant=variant, dmax=8)
        for (x, y) in [(0, 0), (W - 1, H - 1), (3, 4), (W - 1, 0), (0, H - 1)]:
            pts = _line(W, H, r, x, y)
            Sl = [S[py, px] for px, py in pts]
            lol = [lo[py, px] for px, py in pts]
            dil = [0] + [int(dI[r, py, px]) if dI is not None else 0 for px, py in pts[1:]]
            P2s = [0] + [int(lut[abs(int(img[py, px]) - int(img[qy, qx]))])
                         for (px, py), (qx, qy) in zip(pts[1:], pts[:-1])]
            ref = _sgm_line_quadratic(Sl, lol, dil, P1, P2s, D)
            for (px, py), Lr in zip(pts, ref):
                assert np.array_equal(L[py, px].astype(np.int64), Lr), (r, px, py)


def test_sgm_brute_force_16x12x8(orc):
    """Exhaustive label enumeration on path prefixes of length <= 5: the
    normalised path cost at the prefix end equals (up to a constant) the
    minimum over all label sequences ending in s of sum S + sum V."""
    g = np.random.default_rng(12)
    H, W, D = 12, 16, 8
    S = g.integers(0, 63, (H, W, D)).astype(np.uint16)
    P1, P2 = 9, 31
    for r in range(8):
        L = orc.sgm_path(S, r, P1, p2=P2).astype(np.int64)
        for start in [(0, 0), (W - 1, H - 1), (5, 0), (0, 7), (W - 1, 4)]:
            pts = _line(W, H, r, *start)[:5]
            n = len(pts)
            seqs = np.array(list(itertools.product(range(D), repeat=n)))
            cost = np.zeros(len(seqs), np.int64)
            for i, (px, py) in enumerate(pts):
                cost += S[py, px][seqs[:, i]]
                if i:
                    d = np.abs(seqs[:, i] - seqs[:, i - 1])
                    cost += np.where(d == 0, 0, np.where(d == 1, P1, P2))
            best = np.full(D, np.iinfo(np.int64).max)
            np.minimum.at(best, seqs[:, -1], cost)
            ex, ey = pts[-1]
            lr = L[ey, ex]
            assert np.array_equal(lr - lr.min(), best - best.min()), (r, start)


def test_sgm_mirror_symmetry(orc):
    g = np.random.default_rng(13)
    S = g.integers(0, 63, (9, 12, 7)).astype(np.uint16)
    img = g.integers(0, 256, (9, 12), dtype=np.uint8)
    lut = orc.p2_table(11)
    a = orc.sgm_aggregate(S, 11, lut=lut, img=img)
    b = orc.sgm_aggregate(S[:, ::-1].copy(), 11, lut=lut, img=img[:, ::-1].copy())
    c = orc.sgm_aggregate(S[::-1].copy(), 11, lut=lut, img=img[::-1].copy())
    assert np.array_equal(a[:, ::-1], b)
    assert np.array_equal(a[::-1], c)
    t = orc.sgm_aggregate(S.transpose(1, 0, 2).copy(), 11, lut=lut, img=img.T.copy())
    assert np.array_equal(a.transpose(1, 0, 2), t)


def test_sgm_zero_jumps_reduce_to_planewise(orc):
    g = np.random.default_rng(14)
    S = g.integers(0, 63, (8, 10, 6)).astype(np.uint16)
    z = np.zeros((8, 8, 10), np.int8)
    a = orc.sgm_aggregate(S, 5, p2=40)
    b = orc.sgm_aggregate(S, 5, p2=40, dI=z, variant=1)
    assert np.array_equal(a, b)


def test_sgm_path_gradient_follows_a_slanted_valley(orc):
    # one-hot valley s = 2 + x along each row: the path-gradient variant keeps
    # the zero-cost transition on it, plane-wise SGM pays P1 per step
    H, W, D = 3, 8, 16
    S = np.full((H, W, D), 20, np.uint16)
    for x in range(W):
        S[:, x, 2 + x] = 0
    Lpg = orc.sgm_path(S, 0, 5, p2=50, variant=2, dmax=8)
    Lpw = orc.sgm_path(S, 0, 5, p2=50, variant=0)
    for x in range(W):
        assert Lpg[1, x, 2 + x] == 0 if x != 1 else Lpg[1, x, 2 + x] == 5
        if x >= 1:
            assert Lpw[1, x, 2 + x] == 5


def test_p2_table_closed_form(orc):
    lut = orc.p2_table(24, 8.0, 10.0)
    assert lut[0] == 24 * 9
    assert lut[10] == round(24 * (1 + 8 * math.exp(-1.0)))
    assert lut[255] == 24
    assert np.all(np.diff(lut.astype(int)) <= 0)


# ---------------------------------------------------------------- WTA / refine
def test_parabola_vertex_exact(orc):
    a, v = 3.0, 10.37
    xs = [11.0, 10.2, 9.6]
    cs = [a * (x - v) ** 2 + 1.0 for x in xs]
    assert abs(orc.parabola_vertex(xs[0], cs[0], xs[1], cs[1], xs[2], cs[2]) - v) < 1e-12
    # flat: stays at the winner
    assert orc.parabola_vertex(11.0, 5, 10.0, 5, 9.0, 5) == 10.0


def test_wta_ties_edges_and_depth(orc):
    K = np.array([[10.0, 0, 1.0], [0, 10.0, 1.0], [0, 0, 1]])
    rho0, drho = 0.1, 0.02
    Sb = np.array([[[5, 3, 3, 9], [2, 7, 7, 7], [9, 9, 9, 1]]], np.uint16)
    d, g = orc.wta_refine(Sb, K, [0, 0, -1.0], rho0, drho)
    assert list(g[0]) == [1, 0, 3]
    assert abs(d[0, 1] - 1 / rho0) < 1e-4 and abs(d[0, 2] - 1 / (rho0 + 3 * drho)) < 1e-4
    # pixel 0: winner 1 with neighbours (5, 3): vertex between delta(0..2)
    assert 1 / (rho0 + 2 * drho) <= d[0, 0] <= 1 / rho0
    lo = np.array([[2, 0, 5]], np.int32)
    d2, g2 = orc.wta_refine(Sb, K, [0, 0, -1.0], rho0, drho, lo=lo)
    assert list(g2[0]) == [3, 0, 8]


# ---------------------------------------------------------------- median
def test_median5_matches_numpy(orc):
    g = np.random.default_rng(15)
    d = g.normal(10, 3, (13, 17)).astype(np.float32)
    m = orc.median5(d)
    pad = np.pad(d, 2, mode="edge")
    for y in range(13):
        for x in range(17):
            assert m[y, x] == np.median(pad[y:y + 5, x:x + 5])


# ---------------------------------------------------------------- normals / confidence
def _plane_depth(n, delta, K, W, H):
    xs, ys = np.meshgrid(np.arange(W), np.arange(H))
    ray = np.stack([(xs - K[0, 2]) / K[0, 0], (ys - K[1, 2]) / K[1, 1], np.ones_like(xs, float)], -1)
    return (-delta / (ray @ n)).astype(np.float32)


def test_normals_of_analytic_planes(orc):
    K = np.array([[80.0, 0, 19.5], [0, 80.0, 14.5], [0, 0, 1]])
    for n in ([0, 0, -1.0], [0.3, -0.2, -0.93], [-0.5, 0.1, -0.86]):
        n = np.array(n) / np.linalg.norm(n)
        d = _plane_depth(n, 10.0, K, 40, 30)
        img = np.random.default_rng(0).integers(0, 256, (30, 40), dtype=np.uint8)
        sm, raw = orc.normals(d, img, K)
        assert np.allclose(raw[2:-2, 2:-2], n, atol=5e-5)   # FP32 depth input
        assert np.allclose(sm[2:-2, 2:-2], n, atol=5e-5)


def test_confidence_closed_forms(orc):
    ns = np.array([[[0, 0, -1.0], [0, math.sin(math.pi / 4), -math.cos(math.pi / 4)],
                    [math.sin(math.pi / 3), 0, -math.cos(math.pi / 3)], [1, 0, 0.0], [0, 0, 0.0]]],
                  np.float32)
    c = orc.confidence(ns)[0]
    assert abs(c[0] - 1) < 1e-6
    assert abs(c[1] - (math.cos(math.pi / 4) - 0.5) / 0.5) < 1e-6
    assert abs(c[2]) < 1e-6 and c[3] == 0 and c[4] == 0


# ---------------------------------------------------------------- window / dsn
def test_window_centres_on_plane_of_prior_depth(orc):
    K = np.array([[50.0, 0, 9.5], [0, 50.0, 7.5], [0, 0, 1]])
    rho0, drho, G, D = 0.02, 0.004, 40, 8
    gs = np.array([[0, 3, 10], [20, 36, 39]])
    dc = (1.0 / (rho0 + gs * drho)).astype(np.float32)
    lo = orc.window(dc, 6, 4, K, [0, 0, -1.0], rho0, drho, G, D)
    assert lo.shape == (4, 6)
    for y in range(4):
        for x in range(6):
            gc = gs[min(y // 2, 1), min(x // 2, 2)]
            assert lo[y, x] == min(max(gc - D // 2, 0), G - D)


def test_dsn_matches_analytic_plane_index_step(orc):
    W, H = 24, 18
    K = np.array([[40.0, 0, 11.5], [0, 40.0, 8.5], [0, 0, 1]])
    drho = 0.001
    for nv in ([0, 0, -1.0], [0.0, -0.6, -0.8], [0.4, 0.2, -0.89]):
        n = np.array(nv) / np.linalg.norm(nv)
        Kc = K.copy()
        Kc[:2] /= 2.0
        Wc, Hc = W // 2, H // 2
        dc = _plane_depth(n, 10.0, Kc, Wc, Hc)
        nc = np.broadcast_to(n.astype(np.float32), (Hc, Wc, 3)).copy()
        di = orc.dsn(dc, nc, W, H, K, drho, dmax=100)
        for r in range(8):
            dx, dy = DIRS[r]
            for (x, y) in [(6, 5), (13, 9), (20, 14)]:
                d = dc[y // 2, x // 2]
                P = d * np.array([(x - K[0, 2]) / K[0, 0], (y - K[1, 2]) / K[1, 1], 1.0])
                q = np.array([(x - dx - K[0, 2]) / K[0, 0], (y - dy - K[1, 2]) / K[1, 1], 1.0])
                lam = (n @ P) / (n @ q)
                ex = (1.0 / lam - 1.0 / d) / drho
                if abs(abs(ex) - math.floor(abs(ex)) - 0.5) < 1e-3:
                    continue
                assert di[r, y, x] == int(math.copysign(math.floor(abs(ex) + 0.5), ex)), (nv, r, x, y)
        if nv[0] == 0 and nv[1] == 0:
            assert not di.any()


# ---------------------------------------------------------------- scene level
def test_fronto_plane_scene_recovers_plane_index(orc):
    from paper_2112_00821_b300 import synth
    W, H, f = 48, 36, 60.0
    rho0, drho, G = 1 / 30.0, (1 / 8.0 - 1 / 30.0) / 31, 32
    gstar = 13
    z = 1.0 / (rho0 + gstar * drho)
    q = synth._quad([0, 0, z], [1, 0, 0], [0, 1, 0], (-1e9, 1e9), (-1e9, 1e9), 4.0 * z / f, 5)
    K = synth._K(W, H, f)
    ref = synth.render_view([q], K, np.eye(3), np.zeros(3), W, H)
    ts = [np.array([0.4, 0.0, 0.0]), np.array([-0.45, 0.05, 0.0])]
    nbrs = [synth.render_view([q], K, np.eye(3), t, W, H) for t in ts]
    S = orc.cost_volume(ref, nbrs, [-1, 1], K, np.stack([np.eye(3)] * 2), np.stack(ts),
                        [0, 0, -1.0], rho0, drho, G)
    Sb = orc.sgm_aggregate(S, 10, p2=120)
    d, g = orc.wta_refine(Sb, K, [0, 0, -1.0], rho0, drho)
    # rendering resamples the texture, so the warped neighbours match the
    # reference only up to uint8 rounding: nearly every inner pixel picks g*,
    # none is more than one plane off
    inner = g[6:-6, 8:-8]
    assert np.mean(inner == gstar) > 0.95 and np.all(np.abs(inner - gstar) <= 1)
    spacing = 1.0 / (rho0 + (gstar - 1) * drho) - z
    assert np.median(np.abs(d[6:-6, 8:-8] - z)) < 0.25 * spacing


def test_tiny_estimate_close_to_ground_truth(orc):
    # 64 planes span only ~7 px of disparity here (0.12 px per plane), so the
    # error is measured in plane indices rather than in relative depth
    from paper_2112_00821_b300 import synth
    sc, cfg = synth.workload("tiny_160x120_g64", 0)
    c = orc.make_config(levels=1, D=[64], p1=10, p2=120)
    d, n, conf = orc.estimate(sc, c)
    gt_idx = (1.0 / sc.depth_gt - sc.rho_far) / sc.drho
    est_idx = (1.0 / d - sc.rho_far) / sc.drho
    err = np.abs(est_idx - gt_idx)
    assert np.median(err) < 1.0
    assert np.mean(err < 3.0) > 0.85
    assert conf.min() >= 0 and conf.max() <= 1


def test_fronto_plane_exact_shift_views_give_exact_plane_index(orc):
    """A fronto-parallel textured plane at the depth of plane g*, seen by two
    purely translated views whose images are exact integer shifts of the
    reference: every pixel whose windows stay inside both views picks g*
    exactly once the smoothness term is on; with zero penalties g* attains
    the minimum everywhere (census ties at local extrema are legitimate)."""
    g = np.random.default_rng(16)
    W, H, f = 44, 30, 64.0
    big = g.integers(0, 256, (H, W + 20), dtype=np.uint8)
    ref = big[:, 10:10 + W]
    gstar, G = 2, 6
    z = 16.0
    # view 1 (right, b = 3 z / f): disparity 3; view 2 (left, b = -2 z / f): -2;
    # f, the baselines and the plane distances are binary fractions, so the
    # homographies of plane g* shift by exactly 3 and -2 px in FP64
    k1, k2 = 3, -2
    nb1 = big[:, 13:13 + W]            # nb1(x) = ref(x + 3)
    nb2 = big[:, 8:8 + W]              # nb2(x) = ref(x - 2)
    ts = np.array([[-k1 * z / f, 0, 0], [-k2 * z / f, 0, 0]])
    drho = 1.0 / 64.0                   # one plane step = 0.75 px of view-1 disparity
    rho0 = 1.0 / z - gstar * drho
    K = np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1]])
    S = orc.cost_volume(ref, [nb1, nb2], [1, -1], K, np.stack([np.eye(3)] * 2), ts,
                        [0, 0, -1.0], rho0, drho, G)
    inner = (slice(4, -4), slice(9, -9))
    assert np.all(S[inner][..., gstar] == 0)
    for p1, p2 in ((10, 120), (24, 200)):
        Sb = orc.sgm_aggregate(S, p1, p2=p2)
        _, gw = orc.wta_refine(Sb, K, [0, 0, -1.0], rho0, drho)
        assert np.all(gw[inner] == gstar), (p1, p2)


def test_normal_smoothing_commutes_with_mirroring(orc):
    """Mirroring depth and image about the principal point mirrors the smoothed
    normals (n_x changes sign): the window and its weights are symmetric (an
    off-by-one window or a one-sided difference breaks this)."""
    g = np.random.default_rng(21)
    W, H = 31, 23
    K = np.array([[50.0, 0, (W - 1) / 2], [0, 50.0, (H - 1) / 2], [0, 0, 1]])
    xs, ys = np.meshgrid(np.arange(W), np.arange(H))
    d = (15.0 + np.sin(xs / 5.0) + 0.5 * np.cos(ys / 4.0) + 0.3 * xs / W).astype(np.float32)
    img = g.integers(0, 256, (H, W), dtype=np.uint8)
    sm, _ = orc.normals(d, img, K, radius=2, beta=10.0)
    smf, _ = orc.normals(d[:, ::-1].copy(), img[:, ::-1].copy(), K, radius=2, beta=10.0)
    mir = smf[:, ::-1].copy()
    mir[..., 0] *= -1
    assert np.allclose(sm, mir, atol=1e-6)


def test_normal_smoothing_stops_at_image_edges(orc):
    """The appearance term exp(-dI / beta) with dI = 255, beta = 10 weighs a
    neighbour across a strong image edge by e^-25.5, so a pixel next to the
    edge keeps its own surface's normal; with a uniform image the neighbour
    across mixes in."""
    K = np.array([[60.0, 0, 15.5], [0, 60.0, 12.5], [0, 0, 1]])
    xs, ys = np.meshgrid(np.arange(32), np.arange(26))
    n1 = np.array([0.4, 0.0, -1.0]); n1 /= np.linalg.norm(n1)
    n2 = np.array([-0.4, 0.0, -1.0]); n2 /= np.linalg.norm(n2)
    d1 = _plane_depth(n1, 10.0, K, 32, 26)
    d2 = _plane_depth(n2, 10.0, K, 32, 26)
    d = np.where(xs <= 15, d1, d2).astype(np.float32)   # surface changes between 15 | 16
    img = np.where(xs <= 16, 0, 255).astype(np.uint8)   # image edge between 16 | 17
    sm, raw = orc.normals(d, img, K, radius=2, beta=10.0)
    # column 18: its window (16..20) holds column 16, whose raw normal straddles
    # the surface change, but 16 lies across the image edge
    assert np.allclose(raw[5:-5, 17:21], n2, atol=5e-5)
    # (the raw normals themselves carry ~0.01 degree of FP32-depth noise)
    assert np.degrees(np.max(np.arccos(np.clip(sm[5:-5, 18] @ n2, -1, 1)))) < 0.05
    sm_u, _ = orc.normals(d, np.full_like(img, 128), K, radius=2, beta=10.0)
    assert np.degrees(np.arccos(np.clip(sm_u[10, 18] @ n2, -1, 1))) > 0.5


# ------------------------------------------------------------------ normal smoothing weights
# Hand-built raw normal fields whose smoothed normal has a closed form; the
# expected values are written as numbers (sigma = radius = 2, beta = 10).

def _field(H=9, W=9):
    return np.zeros((H, W, 3)), np.full((H, W), 100, np.uint8)


def test_normal_smoothing_sigma_is_the_window_radius(orc):
    """Only the pixels at distance 1 and 2 right of p carry a normal, (1,0,0)
    and (0,1,0): the smoothed normal at p is their weights' direction, whose
    ratio is exp(-(4 - 1) / (2 sigma^2)) = exp(-3/8) = 0.687289 for sigma = 2
    (sigma = 1 would give 0.223130)."""
    nr, img = _field()
    nr[4, 5] = (1.0, 0.0, 0.0)
    nr[4, 6] = (0.0, 1.0, 0.0)
    n = orc.normals_smooth(nr, img)[4, 4]
    r = 0.6872892787909722
    assert np.allclose(n, [1.0 / math.sqrt(1 + r * r), r / math.sqrt(1 + r * r), 0.0], atol=1e-6)


def test_normal_smoothing_own_term_and_gaussian_factor(orc):
    """p's raw normal is (1,0,0), every other pixel's (0,1,0), flat image.  The
    smoothed sum is (1 + c) e_x + c S e_y with c = (2 pi sigma^2)^-1/2 =
    0.199471 and S = sum over the 24 other window pixels of exp(-d^2 / 8) =
    14.824923; its y/x ratio is c S / (1 + c) = 2.465373.  Dropping the
    standalone n_p term gives 14.8249, dropping the factor c gives 7.41246,
    leaving p out of the window sum gives 2.95714."""
    nr, img = _field()
    nr[...] = (0.0, 1.0, 0.0)
    nr[4, 4] = (1.0, 0.0, 0.0)
    n = orc.normals_smooth(nr, img)[4, 4]
    assert abs(n[2]) < 1e-7
    assert abs(n[1] / n[0] - 2.4653734) < 2e-6


def test_normal_smoothing_intensity_weight_beta(orc):
    """Neighbours left and right of p at distance 1 carry (0,0,1) and (0,1,0);
    the left one differs from p by 20 grey levels (once brighter, once
    darker): the ratio of the two weights is exp(-20 / beta) = exp(-2) =
    0.135335 for beta = 10."""
    for dI in (20, -20):
        nr, img = _field()
        nr[4, 3] = (0.0, 0.0, 1.0)
        nr[4, 5] = (0.0, 1.0, 0.0)
        img[4, 3] = 100 + dI
        n = orc.normals_smooth(nr, img)[4, 4]
        assert abs(n[0]) < 1e-7
        assert abs(n[2] / n[1] - 0.1353352832366127) < 1e-6


# ------------------------------------------------------------------ NCC 5x5
def test_ncc_perfect_affine_anti_and_flat_windows(orc):
    g = np.random.default_rng(31)
    a = g.integers(20, 120, 25)
    assert orc.ncc_window(a, a) == 0                         # identical windows
    assert orc.ncc_window(a, 2 * a + 3.25) == 0              # positive affine map
    assert orc.ncc_window(a, 255 - a) == 255                 # anti-correlated: truncated
    assert orc.ncc_window(np.full(25, 77), a) == 255         # flat reference window
    assert orc.ncc_window(a, np.full(25, 100.0)) == 255      # flat warped window


def test_ncc_matches_the_correlation_coefficient(orc):
    """Against numpy's correlation coefficient (a library routine, FP64)."""
    g = np.random.default_rng(32)
    diffs = []
    for _ in range(2000):
        a = g.integers(0, 256, 25)
        b = np.clip(a + g.uniform(-56, 56, 25), 0, 255)
        r = np.corrcoef(a.astype(float), b.astype(float))[0, 1]
        want = int(np.floor(255.0 * (1.0 - max(r, 0.0)) + 0.5))
        diffs.append(orc.ncc_window(a, b) - want)
    assert not np.any(diffs)


def test_ncc_cost_volume_identity_and_exact_plane(orc):
    g = np.random.default_rng(33)
    W, H, f = 40, 30, 64.0
    K = np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1]])
    ref = g.integers(0, 256, (H, W), dtype=np.uint8)
    S = orc.cost_volume(ref, [ref], [1], K, np.eye(3)[None], np.zeros((1, 3)), [0, 0, -1.0], 0.1, 0.01, 4,
                        cost=1)
    assert np.all(S == 0)                                    # identity views: ncc = 1 everywhere
    # exact-shift fronto scene (as for the census): the true plane costs 0;
    # f, the baselines and the plane distances are binary fractions, so the
    # true plane's homographies shift by exactly 3 and -2 px in FP64
    big = g.integers(0, 256, (H, W + 20), dtype=np.uint8)
    ref = big[:, 10:10 + W]
    gstar, G, z = 2, 6, 16.0
    k1, k2 = 3, -2
    nb1, nb2 = big[:, 13:13 + W], big[:, 8:8 + W]
    ts = np.array([[-k1 * z / f, 0, 0], [-k2 * z / f, 0, 0]])
    drho = 1.0 / 64.0
    rho0 = 1.0 / z - gstar * drho
    S = orc.cost_volume(ref, [nb1, nb2], [1, -1], K, np.stack([np.eye(3)] * 2), ts, [0, 0, -1.0], rho0, drho, G,
                        cost=1)
    inner = (slice(3, -3), slice(8, -8))
    assert np.all(S[inner][..., gstar] == 0)
    assert np.mean(S[inner].argmin(axis=-1) == gstar) > 0.99
    # sampled voxels agree with the full volume
    ys, xs = np.nonzero(np.ones((H, W), bool))
    sel = g.choice(xs.size, 200, replace=False)
    gs = g.integers(0, G, 200)
    v = orc.cost_at(ref, [nb1, nb2], [1, -1], K, np.stack([np.eye(3)] * 2), ts, [0, 0, -1.0], rho0, drho,
                    xs[sel], ys[sel], gs, cost=1)
    assert np.array_equal(v, S[ys[sel], xs[sel], gs])


# ------------------------------------------------------------------ post-filters (Sec. 2.6)
def test_dog_weights_quantise_a_7_tap_gaussian(orc):
    w = orc.dog_weights()
    g = np.exp(-0.5 * (np.arange(-3, 4) / 1.4) ** 2)
    assert w.sum() == 256 and np.array_equal(w, w[::-1])
    assert np.all(np.abs(w - 256 * g / g.sum()) <= 1.0)


def test_speckle_removes_small_4_connected_components(orc):
    m = np.zeros((12, 20), np.uint8)
    m[1, 1:7] = 1                         # 6 pixels: removed
    m[4, 1:8] = 1                         # 7 pixels: kept
    m[8, 8] = m[9, 9] = m[10, 10] = 1     # diagonal neighbours are separate components
    m[6:9, 14:17] = 1                     # 9 pixels: kept
    out = orc.speckle(m, 1, 7)
    assert out[1, 1:7].sum() == 0 and out[4, 1:8].all() and out[6:9, 14:17].all()
    assert out[8, 8] == out[9, 9] == out[10, 10] == 0
    # holes (0-components) below 21 pixels are filled, from 21 on they stay
    h = np.ones((12, 30), np.uint8)
    h[2:6, 2:7] = 0                       # 20 pixels: filled
    h[2:5, 12:19] = 0                     # 21 pixels: kept
    out = orc.speckle(h, 0, 21)
    assert out[2:6, 2:7].all() and not out[2:5, 12:19].any()


def test_dog_mask_flat_textured_and_island(orc):
    g = np.random.default_rng(41)
    assert orc.dog_mask(np.full((40, 50), 90, np.uint8)).sum() == 0          # no texture anywhere
    noise = g.integers(0, 256, (40, 50), dtype=np.uint8)
    assert orc.dog_mask(noise).mean() > 0.99                                 # textured everywhere
    img = np.full((60, 80), 100, np.uint8)
    img[20:40, 30:50] = g.integers(0, 256, (20, 20), dtype=np.uint8)         # a textured island
    m = orc.dog_mask(img)
    assert m[20:40, 30:50].all()                                             # kept (and dilated)
    assert m[:10].sum() == 0 and m[:, :15].sum() == 0                        # far flat areas masked out
    d = np.ones((60, 80), np.float32)
    n = np.ones((60, 80, 3), np.float32)
    c = np.ones((60, 80), np.float32)
    d2, n2, c2 = orc.apply_mask(m, d, n, c)
    assert np.all(d2[m == 0] == 0) and np.all(n2[m == 0] == 0) and np.all(c2[m == 0] == 0)
    assert np.all(d2[m == 1] == 1)


def _plane_maps(W, H, f, z, ts):
    """Depth maps of a fronto plane at depth z seen from translated cameras
    (a translation parallel to the plane keeps the depth z)."""
    K = np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1]])
    return K, [np.full((H, W), z, np.float32) for _ in ts]


def test_geometric_consistency_on_a_plane_and_its_outliers(orc):
    W, H, f, z = 64, 48, 60.0, 10.0
    ts = np.array([[0.5, 0, 0], [-0.5, 0, 0], [0, 0.4, 0], [0, -0.4, 0]])
    K, dks = _plane_maps(W, H, f, z, ts)
    R = np.stack([np.eye(3)] * 4)
    dref = np.full((H, W), z, np.float32)
    hits = orc.geo_hits(dref, K, dks, R, ts, eta_r=1.0)
    # shifts of f b / z = 3 (x) and 2.4 (y) pixels: a pixel is seen by every
    # view whose projection stays inside the image
    yy, xx = np.mgrid[0:H, 0:W]
    inside = [(xx + 3 <= W - 1 + 0.5), (xx - 3 >= -0.5), (yy + 2.4 <= H - 0.5), (yy - 2.4 >= -0.5)]
    assert np.array_equal(hits, sum(m.astype(np.uint8) for m in inside))
    # a wrong depth reprojects off: at 0.7 z the shifts are 4.29 (x) and 3.43
    # (y) px instead of 3 and 2.4, errors of 1.29 and 1.03 px: with eta_r = 1
    # every view misses
    bad = dref.copy()
    bad[10:20, 10:20] = 0.7 * z
    h2 = orc.geo_hits(bad, K, dks, R, ts, eta_r=1.0)
    assert np.all(h2[10:20, 10:20] == 0)
    assert np.array_equal(h2[30:, 30:], hits[30:, 30:])
    zero = dref.copy()
    zero[0:5] = 0.0
    assert orc.geo_hits(zero, K, dks, R, ts)[0:5].sum() == 0                 # invalid depth: no hits


# ---------------------------------------------------------------- plane selection (Sec. 2.2.2, Alg. 2)
def _rot(axis, deg):
    a = math.radians(deg)
    ax = np.asarray(axis, float) / np.linalg.norm(axis)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(a) * Kx + (1 - math.cos(a)) * Kx @ Kx


def _Kc(W, H, f):
    return np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1.0]])


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def _images_on_planes(K, R, t, n, deltas, W, H):
    """Image in camera (R, t) of the point where every reference pixel's ray
    meets each plane n^T X + delta = 0, by direct intersection and projection:
    array [planes][H][W][2]."""
    xs, ys = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
    rays = np.stack([xs, ys, np.ones_like(xs)], -1) @ np.linalg.inv(K).T
    s = -np.asarray(deltas)[:, None, None] / (rays @ n)[None]
    X = rays[None] * s[..., None]
    x = (X @ R.T + t) @ K.T
    return x[..., :2] / x[..., 2:]


def test_plane_bounds_fronto_are_the_depth_range(orc):
    K = _Kc(80, 60, 70.0)
    assert orc.plane_bounds(K, 80, 60, [0, 0, -1.0], 3.5, 47.0) == (3.5, 47.0)


@pytest.mark.parametrize("nv", [[0, -0.5, -1.0], [0.3, 0.2, -1.0], [-0.6, 0.0, -1.0]])
def test_plane_bounds_enclose_the_frustum(orc, nv):
    """Brute force: |n^T X| over random points of the frustum stays inside
    [delta_min, delta_max] and both bounds are reached at corners."""
    W, H, f, dmin, dmax = 80, 60, 70.0, 3.0, 40.0
    K, n = _Kc(W, H, f), _unit(nv)
    lo, hi = orc.plane_bounds(K, W, H, n, dmin, dmax)
    g = np.random.default_rng(61)
    px = np.stack([g.uniform(0, W - 1, 20000), g.uniform(0, H - 1, 20000), np.ones(20000)], -1)
    X = (px @ np.linalg.inv(K).T) * g.uniform(dmin, dmax, 20000)[:, None]
    a = np.abs(X @ n)
    assert a.min() >= lo - 1e-12 and a.max() <= hi + 1e-12
    corners = np.array([[u, v, 1.0] for v in (0, H - 1) for u in (0, W - 1)]) @ np.linalg.inv(K).T
    assert abs(np.abs(corners * dmin @ n).min() - lo) < 1e-12
    assert abs(np.abs(corners * dmax @ n).max() - hi) < 1e-12
    assert hi > dmax * min(np.abs(corners @ n)) + 1e-3          # max, not min, over the far corners


def test_plane_bounds_reject_rays_that_miss_the_planes(orc):
    with pytest.raises(ValueError):
        orc.plane_bounds(_Kc(80, 60, 70.0), 80, 60, [1.0, 0, 0], 3.0, 40.0)


def test_cross_ratio_rectified_stereo_closed_form(orc):
    """Rectified pair with baseline b: disparity f b / delta, so one-pixel
    steps are uniform in inverse distance: 1/delta_i = 1/delta_max + i/(f b)."""
    W, H, f, b = 64, 48, 400.0, 0.5
    d, k = orc.cross_ratio_planes(_Kc(W, H, f), W, H, np.eye(3)[None], [[-b, 0, 0]], [0, 0, -1.0], 5.0, 50.0)
    L = f * b / 5.0 - f * b / 50.0                                # 36 px: an integral segment
    assert k == 0 and len(d) == int(math.ceil(L)) + 1
    i = np.arange(len(d))
    assert np.allclose(1.0 / d, 1.0 / 50.0 + i / (f * b), rtol=1e-12, atol=0)
    assert d[0] == pytest.approx(50.0, rel=1e-14) and d[-1] == 5.0


def test_cross_ratio_ragged_segment_ends_on_the_near_plane(orc):
    W, H, f, b = 64, 48, 60.0, 0.5                               # segment 5.4 px
    d, _ = orc.cross_ratio_planes(_Kc(W, H, f), W, H, np.eye(3)[None], [[-b, 0, 0]], [0, 0, -1.0], 5.0, 50.0)
    assert len(d) == 7 and d[-1] == 5.0
    assert np.allclose(1.0 / d[:6], 1.0 / 50.0 + np.arange(6) / (f * b), rtol=1e-12, atol=0)


_POSES = {
    "two_sided": (np.stack([_rot([0, 1, 0], -5), _rot([0, 1, 0], 8)]),
                  np.array([[-0.4, 0.05, 0.1], [0.9, -0.1, 0.2]]), 4.0, 40.0),
    "forward": (np.stack([_rot([1, 0, 0], 3)]), np.array([[0.3, 0.0, -2.0]]), 5.0, 60.0),
    "oblique": (np.stack([_rot([1, 0.2, 0], 4), _rot([0.3, 1, 0], -6)]),
                np.array([[-0.7, 0.3, -0.2], [0.5, 0.6, 0.4]]), 6.0, 80.0),
}


@pytest.mark.parametrize("pose", sorted(_POSES))
@pytest.mark.parametrize("nv", [[0, 0, -1.0], [0, -0.5, -1.0], [0.3, 0.2, -1.0]])
def test_cross_ratio_steps_move_every_pixel_at_most_one_pixel(orc, pose, nv):
    """Direct intersection and projection (no cross-ratio): in camera k one
    corner moves exactly 1 px per step (the last step at most 1 px).  Fronto
    sweeps move no pixel of any camera by more than 1 px; for slanted sweeps
    the bound is exact only at p_ref, elsewhere it stays within 1.1 px."""
    W, H, f = 64, 48, 60.0
    R, t, dmin, dmax = _POSES[pose]
    K, n = _Kc(W, H, f), _unit(nv)
    lo, hi = orc.plane_bounds(K, W, H, n, dmin, dmax)
    d, k = orc.cross_ratio_planes(K, W, H, R, t, n, lo, hi)
    assert np.all(np.diff(d) < 0) and d[0] == pytest.approx(hi, rel=1e-12) and d[-1] == lo
    worst, exact = 0.0, False
    for c in range(len(R)):
        x = _images_on_planes(K, R[c], t[c], n, d, W, H)
        step = np.hypot(*np.moveaxis(np.diff(x, axis=0), -1, 0))     # [planes-1][H][W]
        worst = max(worst, step.max())
        if c == k:
            for (u, v) in [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1)]:
                s = step[:, v, u]
                exact |= bool(np.allclose(s[:-1], 1.0, atol=1e-9) and s[-1] <= 1.0 + 1e-9)
    assert exact and worst <= (1.0 + 1e-9 if nv == [0, 0, -1.0] else 1.1)


def test_cross_ratio_picks_the_camera_with_the_widest_disparity_range(orc):
    W, H, f = 64, 48, 200.0
    R = np.stack([np.eye(3)] * 3)
    t = np.array([[-0.2, 0, 0], [0.6, 0, 0], [-0.35, 0, 0]])
    d, k = orc.cross_ratio_planes(_Kc(W, H, f), W, H, R, t, [0, 0, -1.0], 5.0, 50.0)
    assert k == 1 and len(d) == int(math.ceil(f * 0.6 * (1 / 5.0 - 1 / 50.0))) + 1


def test_cross_ratio_rejects_a_camera_behind_the_nearest_plane(orc):
    with pytest.raises(ValueError):                               # C_k at z = 6 > delta_min = 5
        orc.cross_ratio_planes(_Kc(64, 48, 60.0), 64, 48, np.eye(3)[None], [[0.3, 0, -6.0]], [0, 0, -1.0],
                               5.0, 60.0)


def test_dsn_with_a_slanted_sweep_normal_matches_the_plane_index_step(orc):
    """R11 with sweep normal m: the step of 1/delta = -1/(m^T X) between P and
    where the predecessor ray meets the tangent plane."""
    W, H = 24, 18
    K = np.array([[40.0, 0, 11.5], [0, 40.0, 8.5], [0, 0, 1]])
    drho = 0.001
    for mv in ([0.0, -0.5, -1.0], [0.3, 0.2, -1.0]):
        m = _unit(mv)
        for nv in ([0, 0, -1.0], [0.0, -0.6, -0.8], [0.4, 0.2, -0.89]):
            n = _unit(nv)
            Kc = K.copy()
            Kc[:2] /= 2.0
            Wc, Hc = W // 2, H // 2
            dc = _plane_depth(n, 10.0, Kc, Wc, Hc)
            nc = np.broadcast_to(n.astype(np.float32), (Hc, Wc, 3)).copy()
            di = orc.dsn(dc, nc, W, H, K, drho, dmax=100, n=m)
            nonzero = 0
            for r in range(8):
                dx, dy = DIRS[r]
                for (x, y) in [(6, 5), (13, 9), (20, 14)]:
                    d = dc[y // 2, x // 2]
                    P = d * np.array([(x - K[0, 2]) / K[0, 0], (y - K[1, 2]) / K[1, 1], 1.0])
                    q = np.array([(x - dx - K[0, 2]) / K[0, 0], (y - dy - K[1, 2]) / K[1, 1], 1.0])
                    Q = q * (n @ P) / (n @ q)
                    ex = (-1.0 / (m @ Q) + 1.0 / (m @ P)) / drho
                    if abs(abs(ex) - math.floor(abs(ex)) - 0.5) < 1e-3:
                        continue
                    assert di[r, y, x] == int(math.copysign(math.floor(abs(ex) + 0.5), ex)), (mv, nv, r, x, y)
                    nonzero += di[r, y, x] != 0
            assert nonzero > 0                                    # a slanted sweep sees steps even on fronto planes


def test_oracle_results_do_not_depend_on_its_thread_count():
    """The oracle's parallel loops run over independent pixels and lines: one
    thread and all threads give the same estimate, bit for bit."""
    import oracle
    from paper_2112_00821_b300 import synth
    sc, cfg = synth.workload("tiny_160x120_g64", 0, want_gt=False)
    oc = oracle.make_config(**cfg)
    many = oracle.estimate(sc, oc)
    n0 = oracle.threads()
    oracle.threads(1)
    try:
        assert oracle.threads() == 1
        one = oracle.estimate(sc, oc)
    finally:
        oracle.threads(n0)
    for x, y in zip(many, one):
        assert np.array_equal(x, y)
