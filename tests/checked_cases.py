"""The cases the bounds-checked build runs (tests/test_gpu_checked.py): ragged
and minimum sizes, one plane, sixteen views, windows, both costs, 8 and 4
paths, every SGM variant and aggregation form, the batched form with mixed
frames, and the stage entry points.  Run as a script with the library chosen
by FASSMVS_CHECKED; writes every output to the .npz file named on the command
line and prints "CASES OK" once fassmvs_sync has returned without a recorded
check (it raises otherwise)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _frames():
    from paper_2112_00821_b300 import synth
    return [
        ("min2x2", synth.make_frame("planes", 11, W=2, H=2, G0=32, n_left=1, n_right=1)),
        ("ragged9x3", synth.make_frame("planes", 11, W=9, H=3, G0=32, n_left=1, n_right=1)),
        ("ragged57x53", synth.make_frame("planes", 11, W=57, H=53, G0=32, n_left=1, n_right=1)),
        ("ragged131x97", synth.make_frame("planes", 41, W=131, H=97, G0=96, n_left=1, n_right=2)),
        ("city240x136", synth.make_frame("city", 42, W=240, H=136, G0=256, n_left=2, n_right=3)),
        ("sixteen", synth.make_frame("planes", 13, W=64, H=48, G0=32, n_left=8, n_right=8)),
    ]


def main(out_path):
    import torch
    from paper_2112_00821_b300 import fassmvs
    out = {}
    frames = _frames()

    def item(sc):
        return dict(ref=torch.from_numpy(sc.ref).cuda(), nbrs=[torch.from_numpy(x).cuda() for x in sc.nbrs],
                    K=sc.K, R=sc.R, t=sc.t, side=sc.side, planes=fassmvs.planes_of(sc))

    configs = [
        ("pg8", dict(levels=3, D=[16, 16, 16], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1), (0, 2, 0)),
        ("sn4", dict(levels=2, D=[24, 24], paths=4, variant=1, p1=24, p2=0, adaptive_p2=1), (8, 1, 2)),
        ("pw8_fixed_p2", dict(levels=1, D=[32], paths=8, variant=0, p1=10, p2=120, adaptive_p2=0), (0, 0, 4)),
        ("ncc_pg8", dict(levels=2, D=[16, 16], paths=8, variant=2, p1=40, p2=0, adaptive_p2=1, cost=1),
         (0, 2, 0)),
        ("twopass_pg8", dict(levels=3, D=[16, 16, 16], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1),
         (0, 2, -1)),
        ("twopass_sn4", dict(levels=2, D=[24, 24], paths=4, variant=1, p1=24, p2=0, adaptive_p2=1),
         (0, 2, -1)),
    ]
    for cname, kw, tune in configs:
        # one estimate per frame, then the batch of all frames at once
        L = kw["levels"]
        fits = [(f, sc) for f, sc in frames if ((sc.W - 1) >> (L - 1)) + 1 >= 2 and ((sc.H - 1) >> (L - 1)) + 1 >= 2]
        for fname, sc in fits:
            c = fassmvs.Context(fassmvs.default_config(**kw))
            c.set_tuning(*tune)
            c.set_cameras(sc.K, sc.R, sc.t, sc.side)
            d, n, conf = c.estimate(torch.from_numpy(sc.ref).cuda(),
                                    [torch.from_numpy(x).cuda() for x in sc.nbrs], fassmvs.planes_of(sc))
            c.sync()
            out["%s/%s/depth" % (cname, fname)] = d.cpu().numpy()
            out["%s/%s/normal" % (cname, fname)] = n.cpu().numpy()
            c.close()
        c = fassmvs.Context(fassmvs.default_config(**kw))
        c.set_tuning(*tune)
        batch = fits
        res = c.estimate_batch([item(sc) for _, sc in batch])
        c.sync()
        for (fname, _), (d, n, conf) in zip(batch, res):
            out["%s/batch/%s/depth" % (cname, fname)] = d.cpu().numpy()
        c.close()

    # stage entry points at a ragged size
    g = np.random.default_rng(5)
    H, W, D, G = 19, 23, 7, 20
    S = torch.from_numpy(g.integers(0, 120, (H, W, 8)).astype(np.int16)).cuda()
    lo = torch.from_numpy(np.clip(np.cumsum(g.integers(-2, 3, (H, W)), axis=1) // 3 + 6, 0, G - D)
                          .astype(np.int32)).cuda()
    img = torch.from_numpy(g.integers(0, 256, (H, W)).astype(np.uint8)).cuda()
    ctx = fassmvs.Context()
    for variant in (0, 1, 2):
        dI = torch.from_numpy(g.integers(-3, 4, (8, H, W)).astype(np.int8)).cuda() if variant == 1 else None
        Sb = ctx.sgm_aggregate(S, D, 20, lut=np.arange(256, dtype=np.uint16) // 4 + 20, lo=lo, dI=dI, img=img,
                               paths=8, variant=variant, dmax=4)
        ctx.sync()
        out["stage/sgm%d" % variant] = Sb.cpu().numpy()
    sc = frames[2][1]
    vol = ctx.cost_volume(torch.from_numpy(sc.ref).cuda(), [torch.from_numpy(x).cuda() for x in sc.nbrs],
                          sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, 32)
    ctx.sync()
    out["stage/cost"] = vol.cpu().numpy()
    ctx.close()
    np.savez(out_path, **out)
    print("CASES OK", len(out))


if __name__ == "__main__":
    main(sys.argv[1])
