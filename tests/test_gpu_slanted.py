"""Slanted (non-fronto) sweeps against the oracle (Sec. 2.2.2, Alg. 2): the
surface-normal index jumps under a tilted sweep normal bit for bit, and full
estimates whose sweep normal is tilted and whose planes come from the bounding
planes and the cross-ratio list, on the random-planes frame and on the
oblique city swept with planes parallel to the ground."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


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


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("nv", [[0, -0.5, -1.0], [0.3, 0.2, -1.0]])
def test_dsn_slanted_sweep_bit_exact(ctx, orc, nv):
    from paper_2112_00821_b300 import synth
    sc, _ = synth.workload("vga_640x480_g512_l3", 1)
    Kc = sc.K.copy()
    Kc[:2] /= 2.0
    dc = sc.depth_gt[::2, ::2].astype(np.float32)
    nc, _ = orc.normals(dc, sc.ref[::2, ::2], Kc)
    m = _unit(nv)
    exp = orc.dsn(dc, nc, 640, 480, sc.K, sc.drho, dmax=8, n=m)
    got = ctx.dsn(dev(dc), dev(nc), 640, 480, sc.K, sc.drho, dmax=8, n=m).cpu().numpy()
    ctx.sync()
    assert np.array_equal(got, exp)
    assert np.abs(exp).max() > 0


def _slant(sc, n, d_min, d_max):
    """Sweep sc with normal n over the frustum between depths d_min, d_max,
    planes from the cross-ratio list of its cameras."""
    from paper_2112_00821_b300 import fassmvs
    H, W = sc.ref.shape
    lo, hi = fassmvs.plane_bounds(sc.K, W, H, n, d_min, d_max)
    _, _, uni = fassmvs.cross_ratio_planes(sc.K, W, H, sc.R, sc.t, n, lo, hi)
    sc.plane_n = np.asarray(n, float)
    sc.rho_far, sc.drho, sc.G0 = uni.rho_far, uni.drho, uni.G0
    return sc


def _compare(orc, sc, kw):
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.Context(fassmvs.default_config(**kw))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    d, n, conf = (x.cpu().numpy() for x in c.estimate(dev(sc.ref), [dev(x) for x in sc.nbrs],
                                                         fassmvs.planes_of(sc)))
    c.sync()
    c.close()
    d_e, n_e, c_e = orc.estimate(sc, orc.make_config(**kw))
    assert (d_e > 0).mean() > 0.99
    rel = np.abs(d - d_e) / d_e
    assert np.mean(rel) <= 1e-3, np.mean(rel)
    valid = (np.linalg.norm(n_e, axis=-1) > 0) & (rel < 1e-4)
    cosang = np.clip(np.sum(n[valid] * n_e[valid], -1), -1, 1)
    assert np.median(np.degrees(np.arccos(cosang))) <= 0.5
    assert np.mean(np.abs(conf - c_e)) < 2e-3
    return d_e


@pytest.mark.parametrize("variant,nv", [(0, [0, -0.5, -1.0]), (1, [0.3, 0.2, -1.0]), (2, [0, -0.5, -1.0]),
                                        (1, [0, 0, -1.0])])
def test_slanted_estimate_end_to_end(orc, variant, nv):
    from paper_2112_00821_b300 import synth
    sc = _slant(synth.make_frame("planes", 41 + variant, W=320, H=240, want_gt=False), _unit(nv), 5.4, 31.5)
    assert sc.G0 >= 54
    _compare(orc, sc, dict(levels=2, D=[16, 16], paths=8, variant=variant, p1=24, p2=0, adaptive_p2=1))


@pytest.mark.parametrize("cost", [0, 1])
def test_ground_parallel_sweep_on_the_oblique_city(orc, cost):
    """Planes parallel to the ground of the 45 deg oblique view (n = world up
    in the camera frame); the ground itself is one plane of the sweep."""
    from paper_2112_00821_b300 import synth
    sc = synth.make_frame("city", 5, W=320, H=180, want_gt=True)
    gt = sc.depth_gt
    sc = _slant(sc, synth._pitch_up(45.0), 20.0, 300.0)
    p1 = 100 if cost else 24
    d_e = _compare(orc, sc, dict(levels=3, D=[32, 32, 32], paths=8, variant=0, p1=p1, p2=0, adaptive_p2=1,
                                 cost=cost))
    # and it is a sensible depth map of the scene
    ok = gt > 0
    assert np.median(np.abs(d_e[ok] - gt[ok]) / gt[ok]) < 0.05
