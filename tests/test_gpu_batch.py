"""Batched form of the estimate (fassmvs_estimate_batch).

A batch shares launches across frames (one persistent cost kernel over the
(frame, tile, plane chunk) work items of every frame, one aggregation launch
per direction over the path lines of every frame), so each result must equal,
bit for bit, that of one fassmvs_estimate per frame; the per-frame estimate is
itself checked against the oracle in test_gpu_parity.py, and one batched frame
is checked against the oracle here as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _frames(seeds=(0, 1, 2, 3)):
    """Frames of mixed size, view count and plane count (ragged sizes
    included)."""
    from paper_2112_00821_b300 import synth
    return [
        synth.make_frame("planes", 40 + seeds[0], W=200, H=150, G0=128, n_left=2, n_right=2, want_gt=False),
        synth.make_frame("planes", 40 + seeds[1], W=131, H=97, G0=96, n_left=1, n_right=2, want_gt=False),
        synth.make_frame("city", 40 + seeds[2], W=240, H=136, G0=256, n_left=2, n_right=3, want_gt=False),
        synth.make_frame("tiny", 40 + seeds[3], W=160, H=120, G0=64, n_left=1, n_right=1),
    ]


def _item(sc):
    from paper_2112_00821_b300 import fassmvs
    return dict(ref=torch.from_numpy(sc.ref).cuda(), nbrs=[torch.from_numpy(x).cuda() for x in sc.nbrs],
                K=sc.K, R=sc.R, t=sc.t, side=sc.side, planes=fassmvs.planes_of(sc))


def _cfg(variant):
    from paper_2112_00821_b300 import fassmvs
    return fassmvs.default_config(levels=3, D=[32, 32, 32], paths=8, variant=variant, p1=24, p2=0,
                                  adaptive_p2=1)


def _single(cfg, items):
    from paper_2112_00821_b300 import fassmvs
    out = []
    for it in items:
        c = fassmvs.Context(cfg)
        c.set_cameras(it["K"], it["R"], it["t"], it["side"])
        out.append(c.estimate(it["ref"], it["nbrs"], it["planes"]))
        c.sync()
        c.close()
    return out


def _same(a, b):
    for (d0, n0, c0), (d1, n1, c1) in zip(a, b):
        assert torch.equal(d0, d1)
        assert torch.equal(n0, n1)
        assert torch.equal(c0, c1)


@pytest.mark.parametrize("variant", [1, 2])
def test_batch_equals_one_estimate_per_frame(variant):
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs
    items = [_item(sc) for sc in _frames()]
    cfg = _cfg(variant)
    ref = _single(cfg, items)
    ctx = fassmvs.Context(cfg)
    got = ctx.estimate_batch(items)
    ctx.sync()
    _same(got, ref)
    # a second call on the same context (scratch and staging reused) and a
    # call with the frames in another order
    got2 = ctx.estimate_batch(items[::-1])[::-1]
    ctx.sync()
    _same(got2, ref)
    ctx.close()


def synth_visible(sc, r=3):
    from paper_2112_00821_b300 import synth
    m = synth.visibility_mask(sc)
    out = m.copy()
    H, W = m.shape
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            sh = np.zeros_like(m)
            sh[max(dy, 0):H + min(dy, 0), max(dx, 0):W + min(dx, 0)] = \
                m[max(-dy, 0):H + min(-dy, 0), max(-dx, 0):W + min(-dx, 0)]
            out &= sh
    return out


def test_batched_frame_against_oracle(orc):
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs
    scs = _frames()
    items = [_item(sc) for sc in scs]
    kw = dict(levels=3, D=[32, 32, 32], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    ctx = fassmvs.Context(fassmvs.default_config(**kw))
    got = ctx.estimate_batch(items)
    ctx.sync()
    d = got[1][0].cpu().numpy()
    d_e, n_e, c_e = orc.estimate(scs[1], orc.make_config(**kw))
    rel = np.abs(d - d_e) / d_e
    # on pixels every view sees (ground-truth visibility, 3 px from occlusions)
    from paper_2112_00821_b300 import synth
    gt = synth.make_frame("planes", 41, W=131, H=97, G0=96, n_left=1, n_right=2, want_gt=True)
    assert np.array_equal(gt.ref, scs[1].ref)
    vis = synth_visible(gt)
    cdiff = np.abs(got[1][2].cpu().numpy() - c_e)
    print("PARITY batched frame: depth L1-rel %.3g on %d non-occluded px (%.3g on all), confidence %.3g (%.3g)"
          % (np.mean(rel[vis]), vis.sum(), np.mean(rel), np.mean(cdiff[vis]), np.mean(cdiff)))
    assert np.mean(rel[vis]) <= 1e-3, np.mean(rel[vis])
    assert np.mean(cdiff[vis]) < 2e-3
    ctx.close()


def test_graph_replay_matches_eager():
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs
    cfg = _cfg(2)
    A = [_item(sc) for sc in _frames((0, 1, 2, 3))]
    B = [_item(sc) for sc in _frames((5, 6, 7, 8))]       # same shapes, other scenes
    ref_a, ref_b = _single(cfg, A), _single(cfg, B)
    ctx = fassmvs.Context(cfg)
    ctx.set_graph(True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        first = ctx.estimate_batch(A)        # first run of these shapes: eager
        ga = ctx.estimate_batch(A)           # captured, instantiated, launched
        gb = ctx.estimate_batch(B)           # captured, executable graph updated
        gb2 = ctx.estimate_batch(B)
    s.synchronize()
    _same(first, ref_a)
    _same(ga, ref_a)
    _same(gb, ref_b)
    _same(gb2, ref_b)
    ctx.close()


def test_tuning_choices_do_not_change_results():
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs
    cfg = _cfg(2)
    items = [_item(sc) for sc in _frames()]
    ref = _single(cfg, items)
    ctx = fassmvs.Context(cfg)
    # sgm_parts -1 is the two-pass wavefront form (winner-takes-all fused)
    for chunk, cps, parts in ((8, 1, 1), (256, 2, 2), (48, 2, 4), (0, 1, 8), (0, 2, 0), (32, 0, 8), (0, 0, 0),
                              (0, 2, -1), (32, 0, -1)):
        ctx.set_tuning(chunk, cps, parts)
        got = ctx.estimate_batch(items)
        ctx.sync()
        _same(got, ref)
    chunk, cps, parts = ctx.autotune(items)
    assert chunk in (0, 64) and cps in (0, 1, 2) and parts in (-1, 0, 2, 4, 8)
    got = ctx.estimate_batch(items)
    ctx.sync()
    _same(got, ref)
    ctx.close()


def test_batch_rejects_bad_frames_by_index():
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs
    items = [_item(sc) for sc in _frames()[:2]]
    ctx = fassmvs.Context(_cfg(2))
    bad = dict(items[1])
    K = np.array(bad["K"], dtype=np.float64)
    K[2, 0] = 0.5                     # not an intrinsic matrix
    bad["K"] = K
    with pytest.raises(fassmvs.FassmvsError) as ei:
        ctx.estimate_batch([items[0], bad])
    assert ei.value.status == fassmvs.EINVAL and "frame 1" in str(ei.value)
    with pytest.raises(fassmvs.FassmvsError):
        ctx.set_tuning(-1, 2)
    with pytest.raises(fassmvs.FassmvsError):
        ctx.set_tuning(0, 2, 3)
    # the context stays usable
    ctx.estimate_batch(items)
    ctx.sync()
    ctx.close()


@pytest.mark.parametrize("cost", [0, 1])
def test_staging_of_the_view_images_changes_no_result(cost):
    """The cost kernel's TMA staging of the view images (levels whose rows
    are 16-byte aligned: 640x480 at every level, 240x136 and 160x120 at the
    finest) gives the volume of the global reads, bit for bit."""
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs, synth
    scs = _frames() + [synth.make_frame("planes", 47, W=640, H=480, G0=128, n_left=2, n_right=2, want_gt=False)]
    items = [_item(sc) for sc in scs]
    cfg = fassmvs.default_config(levels=3, D=[32, 32, 32], paths=8, variant=2, p1=100 if cost else 24, p2=0,
                                 adaptive_p2=1, cost=cost)
    ctx = fassmvs.Context(cfg)
    ctx.set_tuning(no_staging=0)
    staged = ctx.estimate_batch(items)
    ctx.sync()
    ctx.set_tuning(no_staging=1)
    plain = ctx.estimate_batch(items)
    ctx.sync()
    _same(staged, plain)
    ctx.close()


def test_staging_changes_no_result_at_full_size():
    """The benchmark's frame and configuration (1920x1080, 5 views, 256
    planes, 4 levels, path-gradient SGM): staged and global reads agree bit
    for bit; the unstaged volume itself is checked against the oracle on
    sampled voxels at this size in test_gpu_parity.py."""
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs, synth
    sc, base = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    items = [_item(sc)]
    ctx = fassmvs.Context(fassmvs.default_config(**base))
    ctx.set_tuning(no_staging=0)
    staged = ctx.estimate_batch(items)
    ctx.sync()
    ctx.set_tuning(no_staging=1)
    plain = ctx.estimate_batch(items)
    ctx.sync()
    _same(staged, plain)
    ctx.close()


def test_a_staged_wait_that_gives_up_is_reported_and_changes_no_result():
    """Failure detection without a fault: under the test hook the cost
    kernel's staging waits find nothing to wait for and give up at their
    bound; the kernel reads global memory instead, the outputs are those of
    a normal run, sync reports ETIMEOUT once, and the context stays usable."""
    _need_gpu()
    from paper_2112_00821_b300 import fassmvs
    items = [_item(sc) for sc in _frames()]
    ctx = fassmvs.Context(_cfg(2))
    ref = ctx.estimate_batch(items)
    ctx.sync()
    ctx.debug_inject(1)
    got = ctx.estimate_batch(items)
    with pytest.raises(fassmvs.FassmvsError) as ei:
        ctx.sync()
    assert ei.value.status == fassmvs.ETIMEOUT and "staged copy" in str(ei.value)
    _same(got, ref)
    ctx.debug_inject(0)
    again = ctx.estimate_batch(items)
    ctx.sync()
    _same(again, ref)
    ctx.close()
