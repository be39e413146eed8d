"""The warped values the census reads (FASSMVS_DUMP_WARP, the cost kernel's own
sample tile) against the oracle's FP64 reading of Alg. 1's patch warping: the
bilinear value in lerp form at the exact position, not rounded.  The census
decides every comparison whose FP32 difference reaches 2^-14 by its FP32 sign
and the closer ones again in double-float; that is exact only if every FP32
value lies within 2^-15 (3.05e-5) of its FP64 value.  The kernel's
arithmetic bounds the error by 2.7e-5; measured here on every pixel of whole
1080p (plane, view) pairs, with staging (the estimate's kernel), and at a
windowed level of a 3-level estimate."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BOUND = 2.0 ** -15      # what the exact census needs (the derived bound is 2.7e-5)


def _check(orc, ctx, sc, level, pairs, K_level, imgs, planes, rho0, drho):
    from paper_2112_00821_b300 import fassmvs
    worst, n = 0.0, 0
    ref = torch.from_numpy(sc.ref).cuda()
    nbrs = [torch.from_numpy(x).cuda() for x in sc.nbrs]
    for g, k in pairs:
        ctx.debug_capture(level)
        ctx.debug_capture_warp(g, k)
        ctx.estimate(ref, nbrs, planes)
        ctx.sync()
        got, dims = ctx.debug_dump(level, "warp")
        got = got.cpu().numpy().astype(np.float64)
        Hm = orc.homography(K_level, sc.R[k], sc.t[k], sc.plane_n, 1.0 / (rho0 + g * drho))
        exp, _ = orc.warp_image(imgs[k], Hm)
        have = np.isfinite(got)
        d = np.abs(got[have] - (exp[have] - 128.0))
        print("PARITY warp level %d plane %d view %d: %d px, max |FP32 - FP64| %.3g grey levels"
              % (level, g, k, int(have.sum()), d.max()))
        assert have.sum() > 0
        worst = max(worst, float(d.max()))
        n += int(have.sum())
    ctx.debug_capture_warp(-1, -1)
    ctx.debug_capture(-1)
    return worst, n


def test_warped_values_of_whole_1080p_pairs(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import fassmvs, synth
    sc, _ = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    cfg = fassmvs.default_config(levels=1, D=[256], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    ctx = fassmvs.Context(cfg)
    ctx.set_cameras(sc.K, sc.R, sc.t, sc.side)
    worst, n = _check(orc, ctx, sc, 0, ((0, 0), (97, 2), (255, 4), (180, 1)), sc.K, sc.nbrs,
                      fassmvs.planes_of(sc), sc.rho_far, sc.drho)
    ctx.close()
    assert n >= 4 * 1920 * 1080 * 0.999     # every pixel of the level sweeps every plane
    assert worst <= BOUND, worst


def test_warped_values_at_a_windowed_level(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import fassmvs, synth
    sc, _ = synth.workload("vga_640x480_g512_l3", 0, want_gt=False)
    cfg = fassmvs.default_config(levels=3, D=[32, 32, 32], paths=8, variant=1, p1=24, p2=0, adaptive_p2=1)
    ctx = fassmvs.Context(cfg)
    ctx.set_cameras(sc.K, sc.R, sc.t, sc.side)
    # level 1: 320x240 with half the focal length and centre, pyramid images,
    # planes rho_far + g * 2 drho; windows of 32 of its 256 planes, so a pair
    # is sampled only where some pixel of the tile needs that plane
    imgs = [orc.pyramid_down(x) for x in sc.nbrs]
    K1 = np.array(sc.K, dtype=np.float64).copy()
    K1[0, 0] /= 2; K1[0, 1] /= 2; K1[0, 2] /= 2; K1[1, 1] /= 2; K1[1, 2] /= 2
    worst, n = _check(orc, ctx, sc, 1, ((100, 0), (140, 3)), K1, imgs, fassmvs.planes_of(sc), sc.rho_far,
                      2 * sc.drho)
    ctx.close()
    assert worst <= BOUND, worst
