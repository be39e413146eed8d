"""Post-filters of Sec. 2.6 against the oracle: the DoG texture mask (Alg. 3)
bit for bit (integer pipeline, connected components are unique), and the
geometric consistency check (Alg. 4) hit for hit (the same FP64 operations in
the same order on both sides)."""
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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _images():
    from paper_2112_00821_b300 import synth
    g = np.random.default_rng(51)
    island = np.full((97, 131), 100, np.uint8)
    island[20:60, 30:90] = g.integers(0, 256, (40, 60), dtype=np.uint8)
    island[80, 10] = 200                                     # an isolated speck
    island[85:87, 100:103] = 30                              # a small dark patch
    ramp = np.tile((np.arange(131) // 2).astype(np.uint8), (97, 1))
    return {
        "flat": np.full((40, 50), 90, np.uint8),
        "noise": g.integers(0, 256, (40, 50), dtype=np.uint8),
        "island": island,
        "ramp": ramp,
        "planes": synth.make_frame("planes", 52, W=200, H=150, G0=64, want_gt=False).ref,
        "tiny": synth.workload("tiny_160x120_g64", 1)[0].ref,
    }


@pytest.mark.parametrize("name", ["flat", "noise", "island", "ramp", "planes", "tiny"])
def test_dog_mask_bit_exact(ctx, orc, name):
    img = _images()[name]
    got = ctx.dog_filter(dev(img)).cpu().numpy()
    ctx.sync()
    assert np.array_equal(got, orc.dog_mask(img))


def test_dog_mask_full_size_and_applied(ctx, orc):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("fhd_1920x1080_g256_l4", 0, want_gt=False)
    ref = sc.ref.copy()
    ref[200:500, 300:800] = 250                              # an overexposed, textureless area
    sc.ref = ref
    g = np.random.default_rng(53)
    d = g.uniform(20, 300, sc.ref.shape).astype(np.float32)
    n = g.normal(size=sc.ref.shape + (3,)).astype(np.float32)
    c = g.uniform(0, 1, sc.ref.shape).astype(np.float32)
    dd, nn, cc = dev(d), dev(n), dev(c)
    mask = ctx.dog_filter(dev(sc.ref), dd, nn, cc).cpu().numpy()
    ctx.sync()
    exp = orc.dog_mask(sc.ref)
    assert np.array_equal(mask, exp)
    assert 0.05 < exp.mean() < 0.999                         # both outcomes occur
    assert not exp[250:450, 350:750].any() and exp[600:].mean() > 0.99
    d2, n2, c2 = orc.apply_mask(exp, d, n, c)
    assert np.array_equal(dd.cpu().numpy(), d2) and np.array_equal(nn.cpu().numpy(), n2)
    assert np.array_equal(cc.cpu().numpy(), c2)


def _gt_window(W=160, H=120, n=5, seed=3):
    """Ground-truth depth maps of the oblique city from 5 consecutive poses of
    a trajectory; relative poses from the centre frame to the others."""
    from paper_2112_00821_b300 import synth
    K, pose, _, _ = synth.trajectory_frames(n, W, H, seed, speed=2.0)
    f = 0.9375 * W
    quads = synth._oblique_city_quads(seed, f, 45.0, 60.0, zmax=300.0)
    maps = []
    for i in range(n):
        R, t = pose(i)
        _, depth, _, _ = synth.render_view(quads, K, R, t, W, H, return_gt=True)
        maps.append(depth.astype(np.float32))
    r = n // 2
    Rr, tr = pose(r)
    Rs, ts, others = [], [], []
    for k in range(n):
        if k == r:
            continue
        Rk, tk = pose(k)
        Rrel = Rk @ Rr.T
        Rs.append(Rrel)
        ts.append(tk - Rrel @ tr)
        others.append(maps[k])
    return K, maps[r], others, np.stack(Rs), np.stack(ts)


@pytest.mark.parametrize("eta_r,eta_h", [(10.0, 3), (0.5, 4), (2.0, 1)])
def test_geometric_hits_bit_exact(ctx, orc, eta_r, eta_h):
    K, dref, others, R, t = _gt_window()
    g = np.random.default_rng(54)
    noisy = dref.copy()
    noisy[g.random(dref.shape) < 0.05] *= 0.6                # outliers
    noisy[:4] = 0.0                                          # invalid rows
    d = dev(noisy)
    nrm = dev(np.ones(dref.shape + (3,), np.float32))
    cf = dev(np.ones(dref.shape, np.float32))
    hits = ctx.geo_filter(d, K, [dev(x) for x in others], R, t, normal=nrm, conf=cf, eta_r=eta_r,
                          eta_h=eta_h).cpu().numpy()
    ctx.sync()
    exp = orc.geo_hits(noisy, K, others, R, t, eta_r=eta_r)
    assert np.array_equal(hits, exp)
    keep = exp >= eta_h
    assert np.array_equal(d.cpu().numpy(), np.where(keep, noisy, 0.0).astype(np.float32))
    assert np.array_equal(cf.cpu().numpy(), keep.astype(np.float32))
    if eta_r == 10.0:
        # the ground truth is consistent: nearly every valid inner pixel keeps
        # its estimate
        assert keep[10:-10, 10:-10].mean() > 0.8
