"""Plane selection of Sec. 2.2.2 through the C-ABI (host-side FP64 geometry,
no device work, so these run without a GPU): the bounding planes and the
cross-ratio plane list of Alg. 2 against the oracle, the uniform
inverse-distance sweep the estimate takes, and the error cases."""
import math

import numpy as np
import pytest


def _rot(axis, deg):
    a = math.radians(deg)
    ax = np.asarray(axis, float) / np.linalg.norm(axis)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(a) * Kx + (1 - math.cos(a)) * Kx @ Kx


def _K(W, H, f):
    return np.array([[f, 0, (W - 1) / 2], [0, f, (H - 1) / 2], [0, 0, 1.0]])


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


POSES = {
    "stereo": (np.eye(3)[None], np.array([[-0.5, 0.0, 0.0]]), 5.0, 50.0),
    "two_sided": (np.stack([_rot([0, 1, 0], -5), _rot([0, 1, 0], 8)]),
                  np.array([[-0.4, 0.05, 0.1], [0.9, -0.1, 0.2]]), 4.0, 40.0),
    "forward": (np.stack([_rot([1, 0, 0], 3)]), np.array([[0.3, 0.0, -2.0]]), 5.0, 60.0),
    "oblique": (np.stack([_rot([1, 0.2, 0], 4), _rot([0.3, 1, 0], -6)]),
                np.array([[-0.7, 0.3, -0.2], [0.5, 0.6, 0.4]]), 6.0, 80.0),
}
NORMALS = [[0, 0, -1.0], [0, -0.5, -1.0], [0.3, 0.2, -1.0], [0.0, -1.0, -0.6]]


@pytest.fixture(scope="module")
def fm():
    from paper_2112_00821_b300 import build, fassmvs
    build.build()
    return fassmvs


@pytest.mark.parametrize("nv", NORMALS)
def test_bounds_match_the_oracle(fm, orc, nv):
    K, n = _K(320, 240, 300.0), _unit(nv)
    got = fm.plane_bounds(K, 320, 240, n, 3.0, 45.0)
    exp = orc.plane_bounds(K, 320, 240, n, 3.0, 45.0)
    assert np.allclose(got, exp, rtol=1e-14, atol=0)


@pytest.mark.parametrize("pose", sorted(POSES))
@pytest.mark.parametrize("nv", NORMALS[:3])
def test_cross_ratio_list_matches_the_oracle(fm, orc, pose, nv):
    W, H, f = 320, 240, 300.0
    R, t, dmin, dmax = POSES[pose]
    K, n = _K(W, H, f), _unit(nv)
    lo, hi = orc.plane_bounds(K, W, H, n, dmin, dmax)
    exp, k_exp = orc.cross_ratio_planes(K, W, H, R, t, n, lo, hi)
    got, k, uni = fm.cross_ratio_planes(K, W, H, R, t, n, lo, hi)
    assert k == k_exp and len(got) == len(exp) > 10
    assert np.allclose(got, exp, rtol=1e-11, atol=0)
    assert got[-1] == lo
    # the uniform sweep, from 1/delta_max until delta_min is reached, at most
    # as coarse as the list's whole-pixel steps
    inv = 1.0 / exp
    assert uni.rho_far == 1.0 / hi
    assert uni.drho <= np.diff(inv)[:-1].min() * (1 + 1e-12)
    assert tuple(uni.n) == tuple(n)
    last = uni.rho_far + (uni.G0 - 1) * uni.drho
    assert last == pytest.approx(1.0 / lo, rel=1e-12)
    assert uni.G0 >= len(exp) - 1
    # by direct projection, no step of the uniform sweep moves p_ref (the
    # corner with the longest segment) in camera k by more than a pixel
    rho = uni.rho_far + np.arange(uni.G0) * uni.drho
    segs, steps = [], []
    for v in (0, H - 1):
        for u in (0, W - 1):
            ray = np.linalg.solve(K, [u, v, 1.0])
            X = ray[None] * (-(1.0 / rho) / (ray @ n))[:, None]
            x = (X @ R[k].T + t[k]) @ K.T
            x = x[:, :2] / x[:, 2:]
            segs.append(np.hypot(*(x[-1] - x[0])))
            steps.append(np.hypot(*np.diff(x, axis=0).T).max())
    assert 0.9 < steps[int(np.argmax(segs))] <= 1.0 + 1e-9


def test_uniform_sweep_of_rectified_stereo_is_the_list(fm):
    """For a rectified pair the list is already uniform in 1/delta."""
    W, H, f, b = 64, 48, 400.0, 0.5
    d, k, uni = fm.cross_ratio_planes(_K(W, H, f), W, H, np.eye(3)[None], [[-b, 0, 0]], [0, 0, -1.0], 5.0, 50.0)
    assert uni.G0 == len(d) == 37
    assert uni.drho == pytest.approx(1.0 / (f * b), rel=1e-12)
    assert np.allclose(uni.rho_far + np.arange(37) * uni.drho, 1.0 / d, rtol=1e-12, atol=0)


def test_count_only_and_capacity(fm):
    from paper_2112_00821_b300.fassmvs import FassmvsError
    K = _K(64, 48, 400.0)
    with pytest.raises(FassmvsError):
        fm.cross_ratio_planes(K, 64, 48, np.eye(3)[None], [[-0.5, 0, 0]], [0, 0, -1.0], 5.0, 50.0, max_planes=10)


@pytest.mark.parametrize("case", ["behind", "miss", "not_unit", "order"])
def test_errors(fm, case):
    from paper_2112_00821_b300.fassmvs import FassmvsError
    K = _K(64, 48, 60.0)
    args = dict(R=np.eye(3)[None], t=[[0.3, 0, -1.0]], n=[0, 0, -1.0], lo=5.0, hi=60.0)
    if case == "behind":
        args["t"] = [[0.3, 0, -6.0]]                              # C_k at z = 6, in front of nothing
    elif case == "miss":
        args["n"] = [1.0, 0, 0]
    elif case == "not_unit":
        args["n"] = [0, 0, -2.0]
    else:
        args["lo"], args["hi"] = 60.0, 5.0
    with pytest.raises(FassmvsError):
        fm.cross_ratio_planes(K, 64, 48, args["R"], args["t"], args["n"], args["lo"], args["hi"])
    if case in ("miss", "not_unit"):
        with pytest.raises(FassmvsError):
            fm.plane_bounds(K, 64, 48, args["n"], 5.0, 60.0)
