"""No kernel writes outside the caller's buffers: every output of the
estimate, the batched estimate and the stage entry points is a slice of a
larger buffer whose guard bands (on both sides) hold a pattern, at ragged
sizes and pitches; the bands must come back unchanged.  (compute-sanitizer is
not available here; this checks the write side of the index arithmetic on the
buffers the caller owns.)"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

GUARD_BYTES = 16 * 257          # on each side: 16-byte aligned (as volumes must be), not 256-byte aligned


def _guarded(shape, dtype):
    n = int(np.prod(shape))
    fill = {torch.float32: -12345.5, torch.int16: 0x5A5A, torch.int64: 0x5A5A5A5A5A5A5A5A,
            torch.int32: 0x5A5A5A5A, torch.uint8: 0xA5, torch.int8: 0x5A}[dtype]
    g = GUARD_BYTES // torch.empty((), dtype=dtype).element_size()
    buf = torch.full((n + 2 * g,), fill, dtype=dtype, device="cuda")
    return buf, buf[g:g + n].view(shape), fill


def _intact(buf, n, fill):
    torch.cuda.synchronize()
    g = (buf.numel() - n) // 2
    head, tail = buf[:g], buf[g + n:]
    return bool((head == fill).all()) and bool((tail == fill).all())


def _frame(W, H, seed, G0=48):
    from paper_2112_00821_b300 import synth
    return synth.make_frame("planes", seed, W=W, H=H, G0=G0, n_left=1, n_right=2, want_gt=False)


@pytest.mark.parametrize("W,H,levels", [(37, 23, 1), (131, 97, 3), (200, 7, 1), (96, 130, 2)])
def test_estimate_writes_only_its_outputs(W, H, levels):
    from paper_2112_00821_b300 import fassmvs
    sc = _frame(W, H, 70 + W)
    cfg = fassmvs.default_config(levels=levels, D=[16] * levels, paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    ctx = fassmvs.Context(cfg)
    ctx.set_cameras(sc.K, sc.R, sc.t, sc.side)
    # images at a wider pitch, the outputs inside guarded buffers
    pitch = W + 13
    def strided(img):
        big = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
        big[:, :W] = torch.from_numpy(img).cuda()
        return big[:, :W]
    ref = strided(sc.ref)
    nbrs = [strided(x) for x in sc.nbrs]
    outs = [_guarded((H, W), torch.float32), _guarded((H, W, 3), torch.float32), _guarded((H, W), torch.float32)]
    ctx.estimate(ref, nbrs, fassmvs.planes_of(sc), *[o[1] for o in outs])
    ctx.sync()
    for buf, view, fill in outs:
        assert _intact(buf, view.numel(), fill)
        assert not (view == fill).any()                  # every output element was written
    ctx.close()


def test_batched_estimate_writes_only_its_outputs():
    from paper_2112_00821_b300 import fassmvs
    scs = [_frame(37, 23, 80), _frame(131, 97, 81), _frame(64, 48, 82)]
    cfg = fassmvs.default_config(levels=2, D=[16, 16], paths=8, variant=1, p1=24, p2=0, adaptive_p2=1)
    ctx = fassmvs.Context(cfg)
    items, guards = [], []
    for sc in scs:
        H, W = sc.ref.shape
        o = [_guarded((H, W), torch.float32), _guarded((H, W, 3), torch.float32), _guarded((H, W), torch.float32)]
        guards += o
        items.append(dict(ref=torch.from_numpy(sc.ref).cuda(), nbrs=[torch.from_numpy(x).cuda() for x in sc.nbrs],
                          K=sc.K, R=sc.R, t=sc.t, side=sc.side, planes=fassmvs.planes_of(sc),
                          depth=o[0][1], normal=o[1][1], conf=o[2][1]))
    ctx.estimate_batch(items)
    ctx.sync()
    for buf, view, fill in guards:
        assert _intact(buf, view.numel(), fill)
    ctx.close()


@pytest.mark.parametrize("W,H", [(37, 23), (129, 61)])
def test_stage_entry_points_write_only_their_outputs(W, H):
    from paper_2112_00821_b300 import fassmvs
    sc = _frame(W, H, 90 + W)
    ctx = fassmvs.Context()
    ref = torch.from_numpy(sc.ref).cuda()
    nbrs = [torch.from_numpy(x).cuda() for x in sc.nbrs]
    G, D = 40, 24
    Ds = 32
    lo = torch.from_numpy(np.random.default_rng(3).integers(0, G - D + 1, (H, W)).astype(np.int32)).cuda()
    S = _guarded((H, W, Ds), torch.int16)
    ctx.cost_volume(ref, nbrs, sc.side, sc.K, sc.R, sc.t, sc.plane_n, sc.rho_far, sc.drho, G, lo=lo, D=D, Ds=Ds,
                    out=S[1])
    Sb = _guarded((H, W, Ds), torch.int16)
    ctx.sgm_aggregate(S[1], D, 48, p2=96, lo=lo, img=ref, paths=8, variant=2, out=Sb[1])
    pyr = _guarded(((H + 1) // 2, (W + 1) // 2), torch.uint8)
    ctx.pyramid_down(ref, out=pyr[1])
    cen = _guarded((H, W), torch.int64)
    ctx.census(ref, out=cen[1])
    ctx.sync()
    for buf, view, fill in (S, Sb, pyr, cen):
        assert _intact(buf, view.numel(), fill)
    ctx.close()
