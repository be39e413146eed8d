"""Runs one stage of the hot path on a synthetic oblique-city frame, for
profiling a single kernel (ncu -k ...) or timing it with CUDA events.

  python -m paper_2112_00821_b300.profile_stage --stage cost|sgm|both|estimate \
      [--W 960 --H 540 --planes 256 --views 5 --reps 2 --variant 2 --sgm-parts 0]

cost / sgm: the single-level stage entry points (cost_kernel, sgm_dir_kernel).
estimate: the full 4-level estimate (the kernels the benchmark runs:
cost_batch_kernel, sgm_batch_dir_kernel, ...), one untimed warm-up call then
`reps` timed calls, with the stage timers.

Prints one JSON line with the per-launch time of the stage(s) (CUDA events on
the launching stream, after one untimed launch).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--stage", default="both", choices=["cost", "sgm", "both", "estimate"])
    p.add_argument("--W", type=int, default=960)
    p.add_argument("--H", type=int, default=540)
    p.add_argument("--planes", type=int, default=256)
    p.add_argument("--views", type=int, default=5)
    p.add_argument("--variant", type=int, default=2)
    p.add_argument("--paths", type=int, default=8)
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cost", type=int, default=0, help="0 census 9x7, 1 NCC 5x5 (estimate stage)")
    p.add_argument("--sgm-parts", type=int, default=0,
                   help="aggregation form of the estimate stage: 0 automatic, -1 two-pass, 1/2/4/8 partial sums")
    a = p.parse_args()

    import numpy as np
    import torch
    from paper_2112_00821_b300 import fassmvs, synth

    nl = a.views // 2
    sc = synth.make_frame("city", a.seed, W=a.W, H=a.H, G0=a.planes, n_left=nl, n_right=a.views - nl,
                          want_gt=False)
    if a.stage == "estimate":
        cfg = fassmvs.default_config(levels=4, D=[256] * 4, paths=a.paths, variant=a.variant,
                                     p1=100 if a.cost else 24, p2=0, adaptive_p2=1, cost=a.cost)
        ctx = fassmvs.Context(cfg)
        ctx.set_tuning(0, 2, a.sgm_parts)
        ctx.set_cameras(sc.K, sc.R, sc.t, sc.side)
        ref = torch.from_numpy(sc.ref).cuda()
        nbrs = [torch.from_numpy(x).cuda() for x in sc.nbrs]
        pl = fassmvs.planes_of(sc)
        ctx.estimate(ref, nbrs, pl)
        torch.cuda.synchronize()
        ctx.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            ctx.estimate(ref, nbrs, pl)
        e1.record()
        torch.cuda.synchronize()
        st = ctx.profile_read()
        out = {"W": a.W, "H": a.H, "planes": a.planes, "views": a.views, "levels": 4,
               "ms": round(e0.elapsed_time(e1) / a.reps, 3),
               "stage_ms": {k: round(v[0] / a.reps, 3) for k, v in st.items()}}
        print(json.dumps(out))
        ctx.close()
        return
    ctx = fassmvs.Context()
    G = D = a.planes
    Ds = ((D + 7) // 8) * 8
    ref = torch.from_numpy(sc.ref).cuda()
    nbrs = [torch.from_numpy(x).cuda() for x in sc.nbrs]
    S = torch.zeros((a.H, a.W, Ds), dtype=torch.int16, device="cuda")
    Sb = torch.zeros_like(S)
    nmax = max(nl, a.views - nl)
    p1 = 24 * nmax
    lut = np.floor(p1 * (1.0 + 8.0 * np.exp(-np.arange(256) / 10.0)) + 0.5).astype(np.uint16)
    dI = torch.zeros((8, a.H, a.W), dtype=torch.int8, device="cuda") if a.variant == 1 else None

    def cost():
        ctx.cost_volume(ref, nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, G, D=D,
                        Ds=Ds, out=S)

    def sgm():
        ctx.sgm_aggregate(S, D, p1, lut=lut, img=ref, dI=dI, paths=a.paths, variant=a.variant, out=Sb)

    out = {"W": a.W, "H": a.H, "planes": a.planes, "views": a.views}
    stages = [("cost", cost), ("sgm", sgm)]
    cost()
    torch.cuda.synchronize()
    for name, fn in stages:
        if a.stage not in (name, "both"):
            continue
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name + "_ms"] = e0.elapsed_time(e1) / a.reps
    vox = a.W * a.H * a.planes
    out["voxels"] = vox
    if "cost_ms" in out:
        out["cost_Gvoxel_views_per_s"] = vox * a.views / out["cost_ms"] / 1e6
    if "sgm_ms" in out:
        out["sgm_algo_GBs"] = 4.0 * vox / out["sgm_ms"] / 1e6
    print(json.dumps(out))
    ctx.close()


if __name__ == "__main__":
    main()
