"""Parity of the NCC 5x5 cost (the paper's selected matching cost, Sec. 3.4)
with the oracle: cost volumes voxel for voxel (same bar as the census: the
FP32 warp may move at most 1e-4 of the voxels; the window sums are exact
integers and the last steps follow the oracle's single-precision order),
sampled voxels of a full-size volume, the full estimate, and the batched
form against one estimate per frame."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.Context(fassmvs.default_config(cost=1))
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host16(t):
    return t.cpu().numpy().view(np.uint16)


def _scene_cost(nctx, orc, sc, G, lo=None, D=None):
    D = G if D is None else D
    exp = orc.cost_volume(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, G,
                          lo=lo, D=D, cost=1)
    got = _host16(nctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t,
                                   sc.plane_n, sc.rho_far, sc.drho, G,
                                   lo=None if lo is None else dev(lo.astype(np.int32)), D=D))
    return got[..., :D], exp


def test_ncc_cost_volume_tiny_scene(nctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("tiny_160x120_g64", 0)
    got, exp = _scene_cost(nctx, orc, sc, 64)
    print("PARITY ncc tiny 160x120x64: differing %.3g" % np.mean(got != exp))
    assert np.mean(got != exp) <= 1e-4, np.mean(got != exp)
    assert exp.max() > 200 and exp.min() == 0              # the whole cost range is exercised


@pytest.mark.parametrize("nl,nr", [(2, 3), (1, 0), (3, 1)])
def test_ncc_cost_volume_ragged_unequal_subsets_windows(nctx, orc, nl, nr):
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("planes", 5 + nl, W=75, H=53, G0=40, n_left=nl, n_right=nr)
    g = np.random.default_rng(9)
    lo = np.clip(np.cumsum(g.integers(-1, 2, (53, 75)), axis=1) // 4 + 10, 0, 40 - 16).astype(np.int32)
    got, exp = _scene_cost(nctx, orc, sc, 40, lo=lo, D=16)
    assert np.mean(got != exp) <= 1e-4


def test_ncc_cost_volume_flat_regions_and_invalid_views(nctx, orc):
    """A flat patch (zero variance) and views that leave the image cost 255."""
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("planes", 21, W=64, H=48, G0=24, n_left=1, n_right=1)
    sc.ref = sc.ref.copy()
    sc.ref[10:30, 10:30] = 128
    got, exp = _scene_cost(nctx, orc, sc, 24)
    assert np.mean(got != exp) <= 1e-4
    assert np.all(exp[14:26, 14:26] == 255)


def test_ncc_cost_volume_fhd_every_voxel(nctx, orc):
    """Every voxel of the 1080p benchmark frame's NCC cost volume (1920 x
    1080 x 256 planes, 5 views) against the FP64 oracle, band by band: the
    FP32 correlation can round a cost next to a .5 boundary the other way, so
    at most 1e-4 of the voxels may differ."""
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    got = nctx.cost_volume(dev(sc.ref), [dev(x) for x in sc.nbrs], sc.side, sc.K, sc.R, sc.t, sc.plane_n,
                           sc.rho_far, sc.drho, 256)
    vol = _host16(got)[..., :256]
    diff, maxd = 0, 0
    for y0 in range(0, 1080, 120):
        exp = orc.cost_band(sc.ref, sc.nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, 256,
                            y0, y0 + 120, cost=1)
        band = vol[y0:y0 + 120]
        diff += int(np.sum(band != exp))
        maxd = max(maxd, int(np.abs(band.astype(int) - exp).max()))
    frac = diff / vol.size
    print("PARITY ncc fhd 1920x1080x256, every voxel: %d differ (%.3g, max |diff| %d)" % (diff, frac, maxd))
    assert frac <= 1e-4, frac


@pytest.mark.parametrize("variant", [0, 2])
def test_ncc_estimate_end_to_end(orc, variant):
    from paper_2112_00821_b300 import fassmvs, synth
    sc = synth.make_frame("planes", 23 + variant, W=200, H=150, G0=128, n_left=2, n_right=2)
    kw = dict(levels=3, D=[32, 32, 32], paths=8, variant=variant, p1=100, p2=0, adaptive_p2=1, cost=1)
    c = fassmvs.Context(fassmvs.default_config(**kw))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    d, n, conf = c.estimate(dev(sc.ref), [dev(x) for x in sc.nbrs], fassmvs.planes_of(sc))
    c.sync()
    d = d.cpu().numpy()
    c.close()
    d_e, n_e, c_e = orc.estimate(sc, orc.make_config(**kw))
    rel = np.abs(d - d_e) / d_e
    print("PARITY ncc estimate variant %d: depth L1-rel %.3g, differing depth %.3g"
          % (variant, np.mean(rel), np.mean(rel > 1e-5)))
    assert np.mean(rel) <= 1e-3, np.mean(rel)


def test_ncc_batch_equals_one_estimate_per_frame():
    from paper_2112_00821_b300 import fassmvs, synth
    cfg = fassmvs.default_config(levels=3, D=[32, 32, 32], paths=8, variant=2, p1=100, p2=0, adaptive_p2=1,
                                 cost=1)
    scs = [synth.make_frame("planes", 30 + i, W=90 + 17 * i, H=70 + 5 * i, G0=64 + 32 * i, n_left=1 + i % 2,
                            n_right=2, want_gt=False) for i in range(3)]
    items = [dict(ref=dev(s.ref), nbrs=[dev(x) for x in s.nbrs], K=s.K, R=s.R, t=s.t, side=s.side,
                  planes=fassmvs.planes_of(s)) for s in scs]
    ctx = fassmvs.Context(cfg)
    got = ctx.estimate_batch(items)
    ctx.sync()
    for s, it, gq in zip(scs, items, got):
        c = fassmvs.Context(cfg)
        c.set_cameras(s.K, s.R, s.t, s.side)
        ref = c.estimate(it["ref"], it["nbrs"], it["planes"])
        c.sync()
        c.close()
        for x, y in zip(gq, ref):
            assert torch.equal(x, y)
    ctx.close()
