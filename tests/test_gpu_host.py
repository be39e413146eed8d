"""The estimate from host images to host maps (fassmvs_estimate_host and its
pipelined form) equals the estimate on device copies of the same images, bit
for bit: page-locked and pageable host memory, a row pitch wider than the
image, a width that is not a multiple of 16 (the device copies are padded to
16-byte rows), and sequences of frames whose copies overlap the kernels,
with a change of image size inside the sequence."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def scene():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import synth
    return synth.make_frame("planes", 61, W=203, H=141, G0=64, n_left=2, n_right=1)


def _ctx(sc):
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.Context(fassmvs.default_config(levels=2, D=[32, 32], paths=8, variant=2, p1=24, p2=0,
                                               adaptive_p2=1))
    c.set_cameras(sc.K, sc.R, sc.t, sc.side)
    return c


def _device_estimate(c, sc):
    from paper_2112_00821_b300 import fassmvs
    d, n, cf = c.estimate(torch.from_numpy(sc.ref).cuda(), [torch.from_numpy(x).cuda() for x in sc.nbrs],
                          fassmvs.planes_of(sc))
    c.sync()
    return d.cpu(), n.cpu(), cf.cpu()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("pad", [0, 13])
def test_host_estimate_equals_device_estimate(scene, pinned, pad):
    from paper_2112_00821_b300 import fassmvs
    sc = scene
    c = _ctx(sc)
    exp = _device_estimate(c, sc)

    def host(a):
        H, W = a.shape
        buf = torch.zeros((H, W + pad), dtype=torch.uint8)
        buf[:, :W] = torch.from_numpy(a)
        if pinned:
            buf = buf.pin_memory()
        return buf[:, :W]

    ref = host(sc.ref)
    nbrs = [host(x) for x in sc.nbrs]
    assert ref.stride(0) == sc.ref.shape[1] + pad
    got = c.estimate_host(ref, nbrs, fassmvs.planes_of(sc))
    for g, e in zip(got, exp):
        assert g.device.type == "cpu"
        assert torch.equal(g, e)
    # again into caller buffers (the device copies are reused)
    outs = tuple(torch.full_like(e, -1.0) for e in exp)
    c.estimate_host(ref, nbrs, fassmvs.planes_of(sc), *outs)
    for g, e in zip(outs, exp):
        assert torch.equal(g, e)
    c.close()


def test_host_estimate_rejects_bad_arguments(scene):
    from paper_2112_00821_b300 import fassmvs
    sc = scene
    c = _ctx(sc)
    ref = torch.from_numpy(sc.ref)
    nbrs = [torch.from_numpy(x) for x in sc.nbrs]
    with pytest.raises(RuntimeError):
        c.estimate_host(ref, nbrs[:-1], fassmvs.planes_of(sc))          # view count differs from the cameras
    with pytest.raises(ValueError):
        c.estimate_host(ref.cuda(), nbrs, fassmvs.planes_of(sc))        # device tensors are not host images
    c.close()


def test_pipelined_sequence_equals_one_estimate_per_frame():
    """Four frames through the pipelined call (two device slots, so the third
    and fourth reuse them), a fifth of another size, then one sync."""
    from paper_2112_00821_b300 import fassmvs, synth
    scs = [synth.make_frame("planes", 70 + i, W=203, H=141, G0=64, n_left=2, n_right=1) for i in range(4)]
    scs.append(synth.make_frame("planes", 75, W=160, H=120, G0=64, n_left=2, n_right=1))
    exp = []
    for sc in scs:
        c = _ctx(sc)
        exp.append(_device_estimate(c, sc))
        c.close()
    c = _ctx(scs[0])
    outs = []
    for sc in scs:
        c.set_cameras(sc.K, sc.R, sc.t, sc.side)
        ref = torch.from_numpy(sc.ref).pin_memory()
        nbrs = [torch.from_numpy(x).pin_memory() for x in sc.nbrs]
        H, W = sc.ref.shape
        o = (torch.empty((H, W)).pin_memory(), torch.empty((H, W, 3)).pin_memory(), torch.empty((H, W)).pin_memory())
        c.estimate_host(ref, nbrs, fassmvs.planes_of(sc), *o, wait=False)
        del ref, nbrs                      # the images have been copied when the call returns
        outs.append(o)
    c.sync()
    for o, e in zip(outs, exp):
        for g, x in zip(o, e):
            assert torch.equal(g, x)
    c.close()
