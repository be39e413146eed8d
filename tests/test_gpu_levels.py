"""Every stage inside the batched estimate, level by level, against the
oracle: the intermediates the estimate captured at each pyramid level
(fassmvs_debug_capture / fassmvs_debug_dump) are checked against the oracle's
step fed with the same inputs.  The window comes from the coarser level's
captured depth; the surface-normal jumps from its depth and normals; the cost
volume from the level's pyramid images and the captured window; the
aggregation from the captured volume; the winner-takes-all from the captured
aggregate; the median and normals from the captured depths."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _host(t):
    return t.cpu().numpy()


def _angle_deg(a, b):
    c = np.clip(np.sum(a * b, -1) / np.maximum(np.linalg.norm(a, axis=-1) * np.linalg.norm(b, axis=-1), 1e-30),
                -1, 1)
    return np.degrees(np.arccos(c))


@pytest.mark.parametrize("variant,cost", [(1, 0), (2, 0), (1, 1)])
def test_each_level_of_the_estimate_against_the_oracle(orc, variant, cost):
    from paper_2112_00821_b300 import fassmvs, synth
    sc = synth.make_frame("planes", 61 + variant, W=200, H=150, G0=128, n_left=2, n_right=2)
    L, Dcfg, p1 = 3, 32, (100 if cost else 24)
    cfg = fassmvs.default_config(levels=L, D=[Dcfg] * L, paths=8, variant=variant, p1=p1, p2=0, adaptive_p2=1,
                                 cost=cost)
    ctx = fassmvs.Context(cfg)
    ctx.set_cameras(sc.K, sc.R, sc.t, sc.side)
    ref = torch.from_numpy(sc.ref).cuda()
    nbrs = [torch.from_numpy(x).cuda() for x in sc.nbrs]
    P1 = p1 * max(sum(1 for s in sc.side if s < 0), sum(1 for s in sc.side if s > 0))
    lut = orc.p2_table(P1)
    imgs = [[sc.ref] + list(sc.nbrs)]
    for _ in range(1, L):
        imgs.append([orc.pyramid_down(x) for x in imgs[-1]])
    got = {}
    for l in range(L - 1, -1, -1):
        ctx.debug_capture(l)
        ctx.estimate(ref, nbrs, fassmvs.planes_of(sc))
        ctx.sync()
        # every intermediate but the warped tile, which a chosen pair fills
        got[l] = {w: _host(ctx.debug_dump(l, w)[0]) for w in fassmvs.Context.DUMPS if w != "warp"}
        got[l]["dims"] = ctx.debug_dump(l, "cost")[1]
    ctx.debug_capture(-1)
    ctx.close()
    for l in range(L - 1, -1, -1):
        g, dm = got[l], got[l]["dims"]
        W, H, D, Ds, G = dm["W"], dm["H"], dm["D"], dm["Ds"], dm["G"]
        s = float(1 << l)
        Kl = sc.K.copy()
        Kl[0, :] /= s
        Kl[1, :] /= s
        drho = sc.drho * s
        assert G == (sc.G0 - 1) // (1 << l) + 1 and D == (G if l == L - 1 else min(Dcfg, G))
        lo = g["window"]
        if l < L - 1:
            # window and surface-normal jumps from the coarser level's results
            dc, nc = got[l + 1]["depth"], got[l + 1]["normal"]
            assert np.array_equal(lo, orc.window(dc, W, H, Kl, sc.plane_n, sc.rho_far, drho, G, D))
            if variant == 1:
                assert np.array_equal(g["dsn"], orc.dsn(dc, nc, W, H, Kl, drho, dmax=8, n=sc.plane_n))
        else:
            assert not lo.any()
        lo_arg = lo if l < L - 1 else None
        dI = g["dsn"] if variant == 1 else None
        # cost volume: the FP32 warp may move at most 1e-4 of the voxels
        S = g["cost"].view(np.uint16)[..., :D]
        S_exp = orc.cost_volume(imgs[l][0], imgs[l][1:], sc.side, Kl, sc.R, sc.t, sc.plane_n, sc.rho_far, drho, G,
                                lo=lo_arg, D=D, cost=cost)
        assert np.mean(S != S_exp) <= 1e-4, (l, np.mean(S != S_exp))
        # aggregation of the captured volume: bit for bit
        A_exp = orc.sgm_aggregate(np.ascontiguousarray(S), P1, lut=lut, lo=lo_arg, dI=dI, img=imgs[l][0], paths=8,
                                  variant=variant, D=D, G=G)
        A = g["agg"].view(np.uint16)[..., :D]
        assert np.array_equal(A, A_exp), l
        # winner-takes-all + refinement of the captured aggregate
        d_exp, w_exp = orc.wta_refine(np.ascontiguousarray(A), Kl, sc.plane_n, sc.rho_far, drho, lo=lo_arg)
        assert np.array_equal(g["argmin"], w_exp)
        assert np.max(np.abs(g["depth_raw"] - d_exp) / d_exp) < 1e-5
        # median of the captured raw depth, normals of the captured depth
        assert np.array_equal(g["depth"], orc.median5(g["depth_raw"]))
        n_exp, _ = orc.normals(g["depth"], imgs[l][0], Kl)
        valid = np.linalg.norm(n_exp, axis=-1) > 0
        assert np.percentile(_angle_deg(g["normal"][valid], n_exp[valid]), 99.9) < 0.5


def test_capture_arguments():
    from paper_2112_00821_b300 import fassmvs
    ctx = fassmvs.Context(fassmvs.default_config(levels=2, D=[32, 32]))
    with pytest.raises(fassmvs.FassmvsError):
        ctx.debug_capture(2)
    ctx.debug_capture(1)
    with pytest.raises(fassmvs.FassmvsError):          # nothing captured yet
        ctx.debug_dump(1, "cost")
    ctx.close()
