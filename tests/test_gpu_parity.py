"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: bit-exact for integer work (pyramid, census, cost volume given exact
warps, SGM, WTA index, median, window, index jumps); the FP32 warp against
the FP64 oracle at most 1e-4 of cost voxels differing; depth L1-rel <= 1e-3;
normals <= 0.5 degree; confidence within 2e-3 (it is a cosine of the normal,
so 0.5 degree moves it by at most 2 sin(60 deg) * 0.0087 = 0.015; the FP32
kernels land far inside that).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.Context()
    yield c
    c.close()


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def host(t, dtype=None):
    a = t.cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def rand_img(g, H, W):
    return g.integers(0, 256, (H, W), dtype=np.uint8)


# ------------------------------------------------------------------ pyramid / census
@pytest.mark.parametrize("H,W", [(120, 160), (17, 33), (1080, 1920), (3, 2)])
def test_pyramid_bit_exact(ctx, orc, H, W):
    g = np.random.default_rng(H * 7 + W)
    img = rand_img(g, H, W)
    out = host(ctx.pyramid_down(dev(img)))
    assert np.array_equal(out, orc.pyramid_down(img))


@pytest.mark.parametrize("H,W", [(120, 160), (29, 45), (540, 960)])
def test_census_bit_exact(ctx, orc, H, W):
    g = np.random.default_rng(H + W)
    img = rand_img(g, H, W)
    img[5:20, 5:25] = 100        # plateaus exercise the strict comparison
    out = host(ctx.census(dev(img)), np.uint64)
    assert np.array_equal(out, orc.census(img))


# ------------------------------------------------------------------ cost volume
def _shift_scene(seed, W=44, H=30, f=64.0):
    """Fronto views whose images are the reference shifted by 3 and -2 px; f,
    the baselines and the plane distances are binary fractions, so plane 2's
    homographies shift by exactly 3 and -2 px in FP64 and in the kernel."""
    g = np.random.default_rng(seed)
    big = rand_img(g, H, W + 20)
    ref = np.ascontiguousarray(big[:, 10:10 + W])
    nb1 = np.ascontiguousarray(big[:, 13:13 + W])
    nb2 = np.ascontiguousarray(big[:, 8:8 + W])
    z = 16.0
    k1, k2 = 3, -2
    ts = np.array([[-k1 * z / f, 0, 0], [-k2 * z / f, 0, 0]])
    drho = 1.0 / 64.0
    rho0 = 1.0 / z - 2 * drho
    K = np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1]])
    return ref, [nb1, nb2], [1, -1], K, np.stack([np.eye(3)] * 2), ts, rho0, drho


def test_cost_volume_exact_shift_views(ctx, orc):
    ref, nbrs, side, K, R, t, rho0, drho = _shift_scene(3)
    n = [0, 0, -1.0]
    exp = orc.cost_volume(ref, nbrs, side, K, R, t, n, rho0, drho, 6, Ds=8)
    got = host(ctx.cost_volume(dev(ref), [dev(x) for x in nbrs], side, K, R, t, n, rho0, drho, 6),
               np.uint16)
    assert np.array_equal(got[..., :6], exp[..., :6])
    assert not got[7:-7, 8:-8, 2].any()


def _scene_cost(ctx, orc, sc, G, lo=None, D=None):
    D = G if D is None else D
    exp = orc.cost_volume(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho,
                          G, lo=lo, D=D)
    got = host(ctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t,
                               sc.plane_n, sc.rho_far, sc.drho, G,
                               lo=None if lo is None else dev(lo.astype(np.int32)), D=D), np.uint16)
    return got[..., :D], exp


def test_cost_volume_tiny_scene_vs_fp64(ctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("tiny_160x120_g64", 0)
    got, exp = _scene_cost(ctx, orc, sc, 64)
    diff = np.mean(got != exp)
    assert diff <= 1e-4, diff


def _blocky(g, H, W):
    """Piecewise-constant 6x6 blocks of a few grey levels (two of them one
    apart), saturated areas and one-pixel stripes: nearly every warped
    sample is a plateau or sits on an edge between equal-looking regions."""
    bs = 6
    levels = np.array([0, 0, 37, 100, 101, 180, 255, 255], np.uint8)
    blk = levels[g.integers(0, len(levels), ((H + bs - 1) // bs, (W + bs - 1) // bs))]
    img = np.kron(blk, np.ones((bs, bs), np.uint8))[:H, :W].copy()
    img[:, 3::17] = 101
    img[10:40, 20:90] = 255
    img[H - 30:H - 5, W - 80:W - 10] = 0
    return np.ascontiguousarray(img)


def test_cost_volume_plateau_rich_images_vs_fp64(ctx, orc):
    """Near ties everywhere: blocky images under general-position homographies
    give plateau ties, ties across saturated areas, and non-plateau samples
    near an integer at every block edge.  The census decides each comparison
    with the FP64 order (FP32 where the difference reaches 2^-14, else the
    plateau rules or the double-float recompute): the stage entry point's
    volume (global taps) and the estimate's level-0 volume (staged taps,
    packed interior path) against the oracle, at most 1e-4 differing."""
    from paper_2112_00821_b300 import fassmvs, synth
    sc = synth.make_frame("planes", 77, W=240, H=160, G0=64, n_left=2, n_right=2, want_gt=False)
    g = np.random.default_rng(77)
    sc.ref = _blocky(g, 160, 240)
    sc.nbrs = [_blocky(g, 160, 240) for _ in sc.nbrs]
    got, exp = _scene_cost(ctx, orc, sc, 64)
    frac = float(np.mean(got != exp))
    print("PARITY cost plateau-rich 240x160x64: differing %.3g (%d voxels)" % (frac, int(np.sum(got != exp))))
    assert frac <= 1e-4, frac
    c = fassmvs.Context(fassmvs.default_config(levels=1, D=[64], paths=8, variant=0, p1=24))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    c.debug_capture(0)
    c.estimate(dev(sc.ref), [dev(x) for x in sc.nbrs], fassmvs.planes_of(sc))
    vol, _ = c.debug_dump(0, "cost")
    c.sync()
    est = host(vol, np.uint16)[..., :64]
    c.close()
    frac = float(np.mean(est != exp))
    print("PARITY cost plateau-rich, estimate level 0: differing %.3g" % frac)
    assert frac <= 1e-4, frac


def test_cost_volume_points_behind_a_neighbour(ctx, orc):
    """A neighbour turned 75 degrees about the vertical axis sees part of
    every plane behind it (homogeneous w <= 0): those samples take the
    behind-the-camera position of the sampling reading and the views whose
    centre sample lies there are invalid.  Both the stage entry point (global
    taps) and the estimate's level-0 volume (staged taps, a box that cannot be
    planned for such pairs) against the oracle."""
    from paper_2112_00821_b300 import fassmvs, synth
    sc = synth.make_frame("planes", 81, W=120, H=90, G0=24, n_left=1, n_right=2)
    a = math.radians(75.0)
    R = np.array(sc.R, dtype=np.float64).copy()
    R[1] = [[math.cos(a), 0.0, math.sin(a)], [0.0, 1.0, 0.0], [-math.sin(a), 0.0, math.cos(a)]]
    sc.R = R
    # precondition: some pixel of some plane lies behind the turned view
    Ki = np.linalg.inv(sc.K)
    ys, xs = np.mgrid[0:90, 0:120]
    rays = np.stack([xs, ys, np.ones_like(xs)], -1).reshape(-1, 3) @ Ki.T
    behind = 0
    for g in (0, 23):
        X = rays / (sc.rho_far + g * sc.drho)
        behind += int(np.sum((X @ R[1].T + sc.t[1])[:, 2] <= 0))
    assert behind > 100
    got, exp = _scene_cost(ctx, orc, sc, 24)
    assert np.mean(got != exp) <= 1e-4
    c = fassmvs.Context(fassmvs.default_config(levels=1, D=[24], paths=8, variant=0, p1=24))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    c.debug_capture(0)
    c.estimate(dev(sc.ref), [dev(x) for x in sc.nbrs], fassmvs.planes_of(sc))
    vol, _ = c.debug_dump(0, "cost")
    c.sync()
    est = host(vol, np.uint16)[..., :24]
    c.close()
    assert np.mean(est != exp) <= 1e-4


@pytest.mark.parametrize("nl,nr", [(2, 3), (1, 0), (3, 1)])
def test_cost_volume_ragged_unequal_subsets_windows(ctx, orc, nl, nr):
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("planes", 5 + nl, W=75, H=53, G0=40, n_left=nl, n_right=nr)
    g = np.random.default_rng(9)
    lo = np.clip(np.cumsum(g.integers(-1, 2, (53, 75)), axis=1) // 4 + 10, 0, 40 - 16).astype(np.int32)
    got, exp = _scene_cost(ctx, orc, sc, 40, lo=lo, D=16)
    assert np.mean(got != exp) <= 1e-4


def test_cost_volume_fhd_sampled(ctx, orc):
    """Full 1920x1080 x 256 planes x 5 views volume, checked on 200,000
    voxels computed one by one by the oracle (image borders and the first /
    last plane included): at most 1e-4 of them may differ."""
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    got = ctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t,
                          sc.plane_n, sc.rho_far, sc.drho, 256)
    n = 200_000
    g = np.random.default_rng(1)
    xs = g.integers(0, 1920, n)
    ys = g.integers(0, 1080, n)
    gs = g.integers(0, 256, n)
    xs[:400] = np.r_[np.zeros(200, int), np.full(200, 1919)]
    ys[400:800] = np.r_[np.zeros(200, int), np.full(200, 1079)]
    gs[800:1200] = np.r_[np.zeros(200, int), np.full(200, 255)]
    exp = orc.cost_at(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho,
                      xs, ys, gs)
    gv = host(got[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda(),
                  torch.from_numpy(gs).cuda()], np.uint16)
    frac = float(np.mean(gv != exp))
    print("PARITY cost fhd sampled %d voxels: differing %.3g" % (n, frac))
    assert frac <= 1e-4, frac
    assert int(host(got, np.uint16).max()) <= 62 * 3


def test_cost_volume_fhd_every_voxel(ctx, orc):
    """Every voxel of the benchmark's 1080p frame (1920 x 1080 x 256 planes,
    5 views, 531 M voxels) against the FP64 oracle, band by band: at most
    1e-4 may differ."""
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    got = ctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t,
                          sc.plane_n, sc.rho_far, sc.drho, 256)
    vol = host(got, np.uint16)[..., :256]
    diff, maxd = 0, 0
    for y0 in range(0, 1080, 120):
        exp = orc.cost_band(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, 256,
                            y0, y0 + 120)
        band = vol[y0:y0 + 120]
        diff += int(np.sum(band != exp))
        maxd = max(maxd, int(np.abs(band.astype(int) - exp).max()))
    frac = diff / vol.size
    print("PARITY cost fhd 1920x1080x256, every voxel: %d differ (%.3g, max |diff| %d)" % (diff, frac, maxd))
    assert frac <= 1e-4, frac


def test_cost_volume_vga_scene_vs_fp64(ctx, orc):
    """The 640x480 random-planes frame (noise 2 DN, 2L + 2R views) over 128
    planes spanning its sweep: at most 1e-4 of the voxels may differ."""
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("vga_640x480_g512_l3", 0, want_gt=False)
    G = 128
    drho = sc.drho * (sc.G0 - 1) / (G - 1)
    exp = orc.cost_volume(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, drho, G)
    got = host(ctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t,
                               sc.plane_n, sc.rho_far, drho, G), np.uint16)[..., :G]
    frac = float(np.mean(got != exp))
    print("PARITY cost vga 640x480x128: differing %.3g" % frac)
    assert frac <= 1e-4, frac


# ------------------------------------------------------------------ SGM
def _sgm_case(ctx, orc, S, D, G, p1, lut=None, p2=0, lo=None, dI=None, img=None, paths=8, variant=0,
              dmax=8):
    H, W, _ = S.shape
    Ds = ((D + 7) // 8) * 8
    Sp = np.zeros((H, W, Ds), np.uint16)
    Sp[..., :D] = S
    exp = orc.sgm_aggregate(S, p1, p2=p2, lut=lut, lo=lo, dI=dI, img=img, paths=paths,
                            variant=variant, dmax=dmax)
    got = host(ctx.sgm_aggregate(dev(Sp), D, p1, p2=p2, lut=lut,
                                 lo=None if lo is None else dev(lo), dI=None if dI is None else dev(dI),
                                 img=None if img is None else dev(img), paths=paths, variant=variant,
                                 dmax=dmax), np.uint16)
    return got[..., :D], exp


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("paths", [8, 4])
def test_sgm_bit_exact_random(ctx, orc, variant, paths):
    g = np.random.default_rng(variant * 10 + paths)
    H, W, D, G = 37, 53, 24, 60
    S = g.integers(0, 63 * 2, (H, W, D)).astype(np.uint16)
    img = rand_img(g, H, W)
    lo = np.clip(np.cumsum(g.integers(-2, 3, (H, W)), axis=1) // 3 + 20, 0, G - D).astype(np.int32)
    dI = g.integers(-5, 6, (8, H, W)).astype(np.int8) if variant == 1 else None
    lut = orc.p2_table(20)
    got, exp = _sgm_case(ctx, orc, S, D, G, 20, lut=lut, lo=lo, dI=dI, img=img, paths=paths,
                         variant=variant, dmax=4)
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("D", [1, 7, 64, 256])
def test_sgm_bit_exact_plane_counts(ctx, orc, D):
    g = np.random.default_rng(D)
    H, W = 19, 23
    S = g.integers(0, 63, (H, W, D)).astype(np.uint16)
    got, exp = _sgm_case(ctx, orc, S, D, D, 10, p2=120)
    assert np.array_equal(got, exp)


def test_sgm_on_oracle_cost_volume(ctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("tiny_160x120_g64", 1)
    S = orc.cost_volume(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, 64)
    for variant in (0, 2):
        got, exp = _sgm_case(ctx, orc, S, 64, 64, 10, p2=120, variant=variant)
        assert np.array_equal(got, exp)


def test_sgm_path_gradient_fhd_vs_oracle(ctx, orc):
    """The benchmark's aggregation at full size: path-gradient SGM, 8 paths,
    the adaptive P2 table of the estimate (P1 = 24 n_max), on the whole
    1920 x 1080 finest-level cost volume (256 planes, 5 views) -- 1920-step
    horizontal lines, 1080-step vertical and diagonal ones -- against the
    oracle's aggregation of the same volume: bit-exact."""
    from paper_2112_00821_b300 import synth
    sc, cfg = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    S = ctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t,
                        sc.plane_n, sc.rho_far, sc.drho, 256)
    vol = np.ascontiguousarray(host(S, np.uint16)[..., :256])
    del S
    nmax = max(sum(1 for s in sc.side if s < 0), sum(1 for s in sc.side if s > 0))
    p1 = cfg["p1"] * nmax
    got, exp = _sgm_case(ctx, orc, vol, 256, 256, p1, lut=orc.p2_table(p1), img=np.ascontiguousarray(sc.ref),
                         paths=8, variant=2, dmax=8)
    diff = int(np.count_nonzero(got != exp))
    print("PARITY sgm path-gradient 1920x1080x256: %d of %d voxels differ" % (diff, got.size))
    assert diff == 0


def test_sgm_zero_penalties_full_size(ctx):
    """P1 = P2 = 0 gives paths * S exactly, at 1920 x 1080 x 256."""
    g = torch.Generator(device="cuda").manual_seed(0)
    S = torch.randint(0, 187, (1080, 1920, 256), dtype=torch.int16, device="cuda", generator=g)
    out = ctx.sgm_aggregate(S, 256, 0, p2=0, paths=8)
    assert torch.equal(out, S * 8)


# ------------------------------------------------------------------ WTA / median / normals
def test_wta_refine_parity(ctx, orc):
    g = np.random.default_rng(4)
    H, W, D, G = 45, 70, 32, 80
    Sb = g.integers(0, 3000, (H, W, D)).astype(np.uint16)
    Sb[3, 4, 5] = Sb[3, 4, 9] = 0                # tie: lowest slot wins
    lo = g.integers(0, G - D + 1, (H, W)).astype(np.int32)
    K = np.array([[300.0, 0, 34.5], [0, 300.0, 22.0], [0, 0, 1]])
    rho0, drho = 0.01, 0.0009
    d_exp, g_exp = orc.wta_refine(Sb, K, [0, 0, -1.0], rho0, drho, lo=lo)
    d_got, g_got = ctx.wta_refine(dev(Sb), D, K, [0, 0, -1.0], rho0, drho, G, lo=dev(lo))
    assert np.array_equal(host(g_got), g_exp)
    assert np.max(np.abs(host(d_got) - d_exp) / d_exp) < 1e-5


@pytest.mark.parametrize("H,W", [(64, 80), (7, 3), (1080, 1920)])
def test_median5_bit_exact(ctx, orc, H, W):
    g = np.random.default_rng(H)
    d = g.normal(20, 5, (H, W)).astype(np.float32)
    d[::7] = 3.0                                 # ties
    exp = orc.median5(d) if H * W < 1e5 else None
    got = host(ctx.median5(dev(d)))
    if exp is None:
        ys = g.integers(0, H, 2000)
        xs = g.integers(0, W, 2000)
        pad = np.pad(d, 2, mode="edge")
        exp_s = np.array([np.median(pad[y:y + 5, x:x + 5]) for y, x in zip(ys, xs)], np.float32)
        assert np.array_equal(got[ys, xs], exp_s)
    else:
        assert np.array_equal(got, exp)


def _angle_deg(a, b):
    c = np.clip(np.sum(a * b, -1) / np.maximum(np.linalg.norm(a, axis=-1) * np.linalg.norm(b, axis=-1),
                                                 1e-30), -1, 1)
    return np.degrees(np.arccos(c))


def test_normals_confidence_parity(ctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("tiny_160x120_g64", 2)
    d = sc.depth_gt.astype(np.float32)
    n_exp, raw_exp = orc.normals(d, sc.ref, sc.K)
    c_exp = orc.confidence(n_exp)
    n_got, raw_got, c_got = ctx.normals(dev(d), dev(sc.ref), sc.K)
    n_got, c_got = host(n_got), host(c_got)
    valid = np.linalg.norm(n_exp, axis=-1) > 0
    assert np.percentile(_angle_deg(n_got[valid], n_exp[valid]), 99.9) < 0.5
    assert np.max(np.abs(c_got - c_exp)) < 2e-3
    assert c_got.min() >= 0 and c_got.max() <= 1


# ------------------------------------------------------------------ window / dsn
def test_window_bit_exact(ctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("vga_640x480_g512_l3", 0)
    dc = orc.median5(sc.depth_gt[::2, ::2].astype(np.float32))
    K = sc.K
    G, D = 512, 128
    exp = orc.window(dc, 640, 480, K, sc.plane_n, sc.rho_far, sc.drho, G, D)
    got = host(ctx.window(dev(dc), 640, 480, K, sc.plane_n, sc.rho_far, sc.drho, G, D))
    assert np.array_equal(got, exp)
    assert exp.min() >= 0 and exp.max() <= G - D


def test_dsn_bit_exact(ctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("vga_640x480_g512_l3", 1)
    Kc = sc.K.copy()
    Kc[:2] /= 2.0
    dc = sc.depth_gt[::2, ::2].astype(np.float32)
    nc, _ = orc.normals(dc, sc.ref[::2, ::2], Kc)
    exp = orc.dsn(dc, nc, 640, 480, sc.K, sc.drho, dmax=8)
    got = host(ctx.dsn(dev(dc), dev(nc), 640, 480, sc.K, sc.drho, dmax=8))
    assert np.array_equal(got, exp)
    assert np.abs(exp).max() > 0


# ------------------------------------------------------------------ end to end
def _run_estimate(ctx_cfg, sc):
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.Context(ctx_cfg)
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    d, n, conf = c.estimate(dev(sc.ref), [dev(x) for x in sc.nbrs], fassmvs.planes_of(sc))
    c.sync()
    out = host(d), host(n), host(conf)
    c.close()
    return out


def _erode(m, r):
    out = m.copy()
    H, W = m.shape
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            sh = np.zeros_like(m)
            sh[max(dy, 0):H + min(dy, 0), max(dx, 0):W + min(dx, 0)] = \
                m[max(-dy, 0):H + min(-dy, 0), max(-dx, 0):W + min(-dx, 0)]
            out &= sh
    return out


@pytest.mark.parametrize("variant,levels", [(0, 1), (1, 3), (2, 3), (2, 2)])
def test_estimate_end_to_end(orc, variant, levels):
    """The whole estimate against the FP64 oracle's on non-occluded pixels
    (ground-truth visibility in every view, eroded by the 3-pixel reach of the
    median and the normal window): depth L1-rel <= 1e-3, the 99.9th percentile
    of the normal angle <= 0.5 degree, confidence within 2e-3 on average.  The
    numbers over all pixels are printed beside them."""
    from paper_2112_00821_b300 import fassmvs, synth
    if levels == 1:
        sc, _ = synth.workload("tiny_160x120_g64", 3)
        kw = dict(levels=1, D=[64], paths=8, variant=variant, p1=10, p2=120, adaptive_p2=0)
    else:
        sc = synth.make_frame("planes", 7 + variant, W=200, H=150, G0=128)
        kw = dict(levels=levels, D=[32, 32, 32], paths=8, variant=variant, p1=24, p2=0, adaptive_p2=1)
    cfg = fassmvs.default_config(**kw)
    d, n, conf = _run_estimate(cfg, sc)
    ocfg = orc.make_config(**kw)
    d_e, n_e, c_e = orc.estimate(sc, ocfg)
    rel = np.abs(d - d_e) / d_e
    vis = _erode(synth.visibility_mask(sc), 3) & (np.linalg.norm(n_e, axis=-1) > 0)
    ang = _angle_deg(n[vis], n_e[vis])
    cdiff = np.abs(conf - c_e)
    print("PARITY estimate variant %d levels %d: on %d non-occluded px depth L1-rel %.3g, normal angle "
          "p99.9 %.3g deg max %.3g deg, confidence mean abs %.3g; on all px depth L1-rel %.3g, "
          "differing depth %.3g, confidence mean abs %.3g"
          % (variant, levels, vis.sum(), np.mean(rel[vis]), np.percentile(ang, 99.9), ang.max(),
             np.mean(cdiff[vis]), np.mean(rel), np.mean(rel > 1e-5), np.mean(cdiff)))
    assert vis.mean() > 0.3
    assert np.mean(rel[vis]) <= 1e-3, np.mean(rel[vis])
    assert np.percentile(ang, 99.9) <= 0.5
    assert np.mean(cdiff[vis]) < 2e-3


def test_estimate_benchmark_frame_end_to_end(orc):
    """The benchmark's whole estimate (1920x1080, 5 views, 256 planes, 4
    levels with their windows, path-gradient SGM with the adaptive P2,
    winner-takes-all, median, normals, confidence) against the FP64 oracle's
    on non-occluded pixels: the same bars as at small sizes."""
    from paper_2112_00821_b300 import fassmvs, synth
    sc, base = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=True)
    kw = dict(levels=base["levels"], D=base["D"], paths=base["paths"], variant=base["variant"], p1=base["p1"],
              p2=base["p2"], adaptive_p2=base["adaptive_p2"])
    d, n, conf = _run_estimate(fassmvs.default_config(**kw), sc)
    d_e, n_e, c_e = orc.estimate(sc, orc.make_config(**kw))
    rel = np.abs(d - d_e) / d_e
    vis = _erode(synth.visibility_mask(sc), 3) & (np.linalg.norm(n_e, axis=-1) > 0)
    ang = _angle_deg(n[vis], n_e[vis])
    cdiff = np.abs(conf - c_e)
    print("PARITY estimate 1080p benchmark frame: on %d non-occluded px depth L1-rel %.3g, differing depth %.3g, "
          "normal angle p99.9 %.3g deg max %.3g deg, confidence mean abs %.3g"
          % (vis.sum(), np.mean(rel[vis]), np.mean(rel[vis] > 1e-5), np.percentile(ang, 99.9), ang.max(),
             np.mean(cdiff[vis])))
    assert vis.mean() > 0.5
    assert np.mean(rel[vis]) <= 1e-3, np.mean(rel[vis])
    assert np.percentile(ang, 99.9) <= 0.5
    assert np.mean(cdiff[vis]) < 2e-3


def test_estimate_equals_the_stage_entry_points_at_full_size(ctx):
    """The benchmark's frame at one level (1920x1080, 5 views, 256 planes,
    path-gradient SGM with the adaptive P2): the estimate, i.e. the batched
    cost kernel with TMA-staged view images, the 16-plane blocked volume and
    its relayout, and the aggregation's partial sums, equals the chain of stage
    entry points bit for bit.  Each stage entry point is checked against the
    oracle above."""
    import math
    from paper_2112_00821_b300 import fassmvs, synth
    sc, base = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    c = fassmvs.Context(fassmvs.default_config(**dict(base, levels=1, D=[256])))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    ref = dev(sc.ref)
    nbrs = [dev(x) for x in sc.nbrs]
    d, n, conf = c.estimate(ref, nbrs, fassmvs.planes_of(sc))
    nmax = max(sum(1 for s in sc.side if s < 0), sum(1 for s in sc.side if s > 0))
    p1 = base["p1"] * nmax
    lut = [min(65535, math.floor(p1 * (1.0 + 8.0 * math.exp(-i / 10.0)) + 0.5)) for i in range(256)]
    S = c.cost_volume(ref, nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, 256)
    Sb = c.sgm_aggregate(S, 256, p1, lut=lut, img=ref, paths=8, variant=2)
    dr, _ = c.wta_refine(Sb, 256, sc.K, sc.plane_n, sc.rho_far, sc.drho, 256)
    dm = c.median5(dr)
    nn, _, cc = c.normals(dm, ref, sc.K, n_plane=sc.plane_n)
    c.sync()
    assert torch.equal(d, dm)
    assert torch.equal(n, nn) and torch.equal(conf, cc)
    c.close()
