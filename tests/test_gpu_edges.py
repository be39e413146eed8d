"""Edge cases of the full estimate and the batched form against the oracle:
minimum image sizes, one plane, sixteen views, the 256-plane cap of the top
level, batches larger than one aggregation launch group, and the argument
checks of the ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(kw, sc):
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.Context(fassmvs.default_config(**kw))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    d, n, conf = c.estimate(torch.from_numpy(sc.ref).cuda(), [torch.from_numpy(x).cuda() for x in sc.nbrs],
                            fassmvs.planes_of(sc))
    c.sync()
    out = d.cpu().numpy(), n.cpu().numpy(), conf.cpu().numpy()
    c.close()
    return out


def _compare(orc, kw, sc, mean_rel=1e-3):
    d, n, c = _run(kw, sc)
    d_e, n_e, c_e = orc.estimate(sc, orc.make_config(**kw))
    rel = np.abs(d - d_e) / np.abs(d_e)
    assert np.all(np.isfinite(d))
    assert np.mean(rel) <= mean_rel, np.mean(rel)
    assert np.mean(np.abs(c - c_e)) < 2e-3
    return d, d_e


@pytest.mark.parametrize("W,H,levels", [(2, 2, 1), (5, 5, 3), (9, 3, 2), (57, 53, 1)])
def test_estimate_minimum_and_ragged_sizes(orc, W, H, levels):
    _need_gpu()
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("planes", 11, W=W, H=H, G0=32, n_left=1, n_right=1)
    kw = dict(levels=levels, D=[16, 16, 16], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    _compare(orc, kw, sc)


def test_estimate_single_plane(orc):
    _need_gpu()
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("planes", 12, W=96, H=72, G0=2, n_left=1, n_right=2)
    sc.G0 = 1                                      # the farthest plane alone
    kw = dict(levels=2, D=[1, 1], paths=8, variant=1, p1=24, p2=0, adaptive_p2=1)
    d, d_e = _compare(orc, kw, sc, mean_rel=1e-6)
    # one fronto plane: every depth is that plane's distance
    assert np.allclose(d, 1.0 / sc.rho_far, rtol=1e-5)


def test_estimate_sixteen_views(orc):
    _need_gpu()
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("planes", 13, W=80, H=60, G0=64, n_left=8, n_right=8)
    kw = dict(levels=2, D=[32, 32], paths=4, variant=0, p1=10, p2=120, adaptive_p2=0)
    _compare(orc, kw, sc)


def test_estimate_top_level_plane_cap(orc):
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs, synth
    # 2048 finest planes over 4 levels leave exactly 256 at the top (Sec. 3.2 cap)
    sc = synth.make_frame("planes", 14, W=72, H=64, G0=2048, n_left=1, n_right=1)
    kw = dict(levels=4, D=[16, 16, 16, 16], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    _compare(orc, kw, sc)
    sc.G0 = 2049                                   # 257 at the top: refused
    with pytest.raises(fassmvs.FassmvsError) as ei:
        _run(kw, sc)
    assert ei.value.status == fassmvs.EINVAL


def test_batch_larger_than_one_launch_group():
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs, synth
    kw = dict(levels=2, D=[24, 24], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    cfg = fassmvs.default_config(**kw)
    scs = [synth.make_frame("planes", 100 + i, W=48 + (i % 5) * 3, H=40 + (i % 3), G0=32 + 8 * (i % 4),
                            n_left=1 + i % 2, n_right=1 + (i // 2) % 2, want_gt=False) for i in range(40)]
    items = [dict(ref=torch.from_numpy(s.ref).cuda(), nbrs=[torch.from_numpy(x).cuda() for x in s.nbrs], K=s.K,
                  R=s.R, t=s.t, side=s.side, planes=fassmvs.planes_of(s)) for s in scs]
    ctx = fassmvs.Context(cfg)
    got = ctx.estimate_batch(items)
    ctx.sync()
    for s, it, g in zip(scs, items, got):
        c = fassmvs.Context(cfg)
        c.set_cameras(s.K, s.R, s.t, s.side)
        ref = c.estimate(it["ref"], it["nbrs"], it["planes"])
        c.sync()
        c.close()
        for x, y in zip(g, ref):
            assert torch.equal(x, y)
    ctx.close()


def test_estimate_rejects_bad_arguments():
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs, synth
    sc = synth.make_frame("planes", 15, W=64, H=48, G0=32, n_left=1, n_right=1, want_gt=False)
    c = fassmvs.Context(fassmvs.default_config(levels=3, D=[16, 16, 16]))
    ref = torch.from_numpy(sc.ref).cuda()
    nbrs = [torch.from_numpy(x).cuda() for x in sc.nbrs]
    with pytest.raises(fassmvs.FassmvsError):          # cameras not set
        c.estimate(ref, nbrs, fassmvs.planes_of(sc))
    K = sc.K.copy()
    K[2, 0] = 1.0
    with pytest.raises(fassmvs.FassmvsError):          # not an intrinsic matrix
        c.set_cameras(K, sc.R, sc.t, sc.side)
        c.estimate(ref, nbrs, fassmvs.planes_of(sc))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    with pytest.raises(fassmvs.FassmvsError):          # view count differs from the cameras
        c.estimate(ref, nbrs[:1], fassmvs.planes_of(sc))
    tiny = torch.zeros((3, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(fassmvs.FassmvsError):          # too small for 3 levels
        c.estimate(tiny, [tiny, tiny], fassmvs.planes_of(sc))
    p = fassmvs.planes_of(sc)
    p.drho = float("nan")
    with pytest.raises(fassmvs.FassmvsError) as ei:
        c.estimate(ref, nbrs, p)
    assert ei.value.status == fassmvs.EINVAL
    with pytest.raises(fassmvs.FassmvsError):          # bad configuration
        c.set_config(fassmvs.default_config(levels=9))
    # the context still works after every refusal
    d, n, conf = c.estimate(ref, nbrs, fassmvs.planes_of(sc))
    c.sync()
    assert torch.isfinite(d).all()
    c.close()
