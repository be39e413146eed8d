"""Serving form (fassmvs_server_*): continuous batching must not change any
result, admission must keep the device memory within the budget, and the
host-side failure modes (a request that can never fit, a request not admitted
before its deadline, a cancelled request, a frame that does not fit, an unknown
frame) must be reported as statuses without disturbing the other requests.
The post-filters of Sec. 2.6 run in the server equal the standalone ones."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_CFG = dict(levels=3, D=[32, 32, 32], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def streams():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import serve
    return serve.make_streams(sizes=((320, 180), (416, 234)), n_frames=26, seed=3, device="cuda")


def _cfg():
    from paper_2112_00821_b300 import fassmvs
    return fassmvs.default_config(**_CFG)


def _serve_all_at_once(streams, scfg):
    """Every frame pushed first, then every request submitted in one go, so
    that requests queue behind the running ones and share batches whatever the
    speed of the kernels; returns the server statistics and the outputs."""
    from paper_2112_00821_b300 import fassmvs, serve
    srv = fassmvs.Server(_cfg(), scfg)
    for s in streams:
        for k in range(len(s.frames)):
            R, t = s.poses[k]
            srv.push_frame(s.fid(k), s.frames[k], s.K, R, t)
    outs, rid = {}, 0
    for si, s in enumerate(streams):
        for j, (r, idx, G0) in enumerate(s.reqs):
            o = tuple(serve._pinned(shp) for shp in ((s.H, s.W), (s.H, s.W, 3), (s.H, s.W)))
            srv.submit(rid, s.fid(r), [s.fid(k) for k in idx], serve._planes(G0), *o)
            outs[(si, j)] = o
            rid += 1
    done = 0
    for _ in range(600):
        for r in srv.poll(64, 100):
            assert r["status"] == fassmvs.OK
            done += 1
        if done == rid:
            break
    assert done == rid
    st = srv.stats()
    srv.close()
    return st, outs


def test_each_result_is_the_same_alone_and_in_the_mix(streams):
    from paper_2112_00821_b300 import fassmvs, serve
    scfg = fassmvs.server_config(lanes=2, max_batch=3, mem_budget=4 << 30, tuning=(0, 2, 4),
                                 tuning_overlap=(16, 0, 4), overlap_queue=1)
    st, outs = _serve_all_at_once(streams, scfg)
    assert st["max_batch_seen"] > 1                    # requests really shared batches
    assert st["overlapped"] > 0                        # and batches ran next to each other
    n_checked = 0
    for (si, j), o in outs.items():
        s = streams[si]
        r, idx, G0 = s.reqs[j]
        alone = fassmvs.Server(_cfg(), fassmvs.server_config(lanes=1, max_batch=1, mem_budget=1 << 30,
                                                              tuning=(0, 2, 4), tuning_overlap=(0, 2, 4)))
        for k in sorted(idx + [r]):
            R, t = s.poses[k]
            alone.push_frame(s.fid(k), s.frames[k], s.K, R, t)
        a = tuple(torch.empty_like(x).pin_memory() for x in o)
        alone.submit(7, s.fid(r), [s.fid(k) for k in idx], serve._planes(G0), *a)
        res = alone.poll(4, 60000)
        alone.close()
        assert len(res) == 1 and res[0]["status"] == fassmvs.OK
        for x, y in zip(o, a):
            assert torch.equal(x, y)
        n_checked += 1
    assert n_checked == sum(len(s.reqs) for s in streams)


def test_served_results_match_the_plain_estimate(streams):
    from paper_2112_00821_b300 import fassmvs, serve
    scfg = fassmvs.server_config(lanes=2, max_batch=4, mem_budget=4 << 30)
    _, so = serve.run_server(streams, _cfg(), scfg, fps=None, keep=True)
    _, po = serve.run_plain(streams, _cfg(), fps=None, keep=True)
    # the plain form forms the relative poses in the server's order of FP64
    # operations, so the two give the same cameras and the same maps, bit for bit
    for key in so:
        for x, y in zip(so[key], po[key]):
            assert torch.equal(x, y), key


def test_two_pass_aggregation_serves_the_same_maps(streams):
    """The two-pass wavefront aggregation (sgm_parts -1) on two lanes whose
    batches overlap gives the maps of the plain per-direction estimate."""
    from paper_2112_00821_b300 import fassmvs, serve
    scfg = fassmvs.server_config(lanes=2, max_batch=3, mem_budget=4 << 30, tuning=(0, 2, -1),
                                 tuning_overlap=(32, 0, -1), overlap_queue=1)
    res, so = serve.run_server(streams, _cfg(), scfg, fps=None, keep=True)
    assert res["server"]["completed"] == sum(len(s.reqs) for s in streams)
    _, po = serve.run_plain(streams, _cfg(), fps=None, keep=True)
    for key in so:
        for x, y in zip(so[key], po[key]):
            assert torch.equal(x, y), key


def test_admission_keeps_memory_within_the_budget(streams):
    from paper_2112_00821_b300 import fassmvs, serve
    # room for the resident frames and about two requests of the larger stream
    scfg = fassmvs.server_config(lanes=3, max_batch=4, mem_budget=48 << 20, tuning=(0, 2, 2),
                                 tuning_overlap=(32, 0, 2))
    res = serve.run_server(streams, _cfg(), scfg, fps=None)
    st = res["server"]
    assert st["completed"] == sum(len(s.reqs) for s in streams)
    assert st["peak_bytes"] <= st["capacity"]


def _one_frame_server(budget, deadline_ms=0):
    from paper_2112_00821_b300 import fassmvs
    return fassmvs.Server(_cfg(), fassmvs.server_config(lanes=1, max_batch=1, mem_budget=budget,
                                                        deadline_ms=deadline_ms))


def _push(srv, s, ks):
    for k in ks:
        R, t = s.poses[k]
        srv.push_frame(s.fid(k), s.frames[k], s.K, R, t)


def _outs(s):
    return tuple(torch.empty(sh, dtype=torch.float32, device="cuda")
                 for sh in ((s.H, s.W), (s.H, s.W, 3), (s.H, s.W)))


def test_request_larger_than_the_budget_is_rejected(streams):
    from paper_2112_00821_b300 import fassmvs, serve
    s = streams[1]
    srv = _one_frame_server(8 << 20)
    r, idx, G0 = s.reqs[1]
    _push(srv, s, sorted(idx + [r]))
    with pytest.raises(fassmvs.FassmvsError) as ei:
        srv.submit(1, s.fid(r), [s.fid(k) for k in idx], serve._planes(G0), *_outs(s))
    assert ei.value.status == fassmvs.ENOMEM
    srv.close()


def _need_bytes(s, req, cfg):
    """Frame bytes and scratch bytes of one request, measured on a roomy
    server."""
    from paper_2112_00821_b300 import fassmvs, serve
    r, idx, G0 = req
    probe = fassmvs.Server(cfg, fassmvs.server_config(lanes=1, max_batch=1, mem_budget=32 << 30))
    _push(probe, s, sorted(idx + [r]))
    before = probe.stats()["bytes_in_use"]
    probe.submit(1, s.fid(r), [s.fid(k) for k in idx], serve._planes(G0), *_outs(s))
    assert probe.poll(4, 60000)[0]["status"] == fassmvs.OK
    need = probe.stats()["peak_bytes"] - before
    probe.close()
    return before, need


def test_request_that_can_never_fit_is_refused(streams):
    from paper_2112_00821_b300 import fassmvs, serve
    s = streams[1]
    r, idx, G0 = s.reqs[1]
    before, need = _need_bytes(s, s.reqs[1], _cfg())
    # fits the budget on its own but never next to its own resident frames,
    # with nothing else in flight: refused at once, not left waiting
    srv = _one_frame_server(before + need - 4096)
    _push(srv, s, sorted(idx + [r]))
    srv.submit(2, s.fid(r), [s.fid(k) for k in idx], serve._planes(G0), *_outs(s))
    got = srv.poll(4, 60000)
    assert len(got) == 1 and got[0]["status"] == fassmvs.ENOMEM and got[0]["batch_size"] == 0
    assert srv.stats()["failed"] == 1 and srv.stats()["queued"] == 0
    srv.close()


def test_request_not_admitted_before_its_deadline_times_out():
    from paper_2112_00821_b300 import fassmvs, serve
    # a 1080p keyframe with 256 planes everywhere runs for tens of ms; a
    # second one waits for its memory and passes its 2 ms deadline meanwhile
    s = serve.make_streams(sizes=((1920, 1080),), n_frames=5, seed=5, device="cuda")[0]
    r, idx, _ = s.reqs[0]
    req = (r, idx, 256)
    cfg = fassmvs.default_config(levels=3, D=[256, 256, 256], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    before, need = _need_bytes(s, req, cfg)
    srv = fassmvs.Server(cfg, fassmvs.server_config(lanes=2, max_batch=1, mem_budget=before + need + need // 2,
                                                    deadline_ms=2))
    _push(srv, s, sorted(idx + [r]))
    for q in (1, 2):
        srv.submit(q, s.fid(r), [s.fid(k) for k in idx], serve._planes(256), *_outs(s))
    got = {}
    for _ in range(10):
        for x in srv.poll(4, 60000):
            got[x["id"]] = x
        if len(got) == 2:
            break
    assert got[1]["status"] == fassmvs.OK and got[1]["batch_size"] == 1
    assert got[2]["status"] == fassmvs.ETIMEOUT and got[2]["batch_size"] == 0
    assert got[2]["t_done_ns"] - got[2]["t_submit_ns"] >= 2_000_000
    assert got[2]["t_done_ns"] < got[1]["t_done_ns"]
    srv.close()


def test_frames_beyond_the_budget_are_refused_until_memory_returns(streams):
    from paper_2112_00821_b300 import fassmvs
    s = streams[0]
    per = s.W * s.H * 4 // 3 + 4096
    srv = _one_frame_server(3 * per)       # two or three frames fit
    pushed = []
    with pytest.raises(fassmvs.FassmvsError) as ei:
        for k in range(10):
            _push(srv, s, [k])
            pushed.append(k)
    assert ei.value.status == fassmvs.EBUSY and 1 <= len(pushed) < 10
    srv.release_frame(s.fid(pushed[0]))
    _push(srv, s, [len(pushed)])
    srv.close()


def test_unknown_frames_are_rejected(streams):
    from paper_2112_00821_b300 import fassmvs, serve
    s = streams[0]
    srv = _one_frame_server(1 << 30)
    _push(srv, s, [0, 1])
    with pytest.raises(fassmvs.FassmvsError) as ei:
        srv.submit(1, s.fid(0), [s.fid(1), s.fid(5)], serve._planes(64), *_outs(s))
    assert ei.value.status == fassmvs.EINVAL and "not resident" in str(ei.value)
    with pytest.raises(fassmvs.FassmvsError):
        srv.release_frame(s.fid(9))
    srv.close()


def test_cancelled_request_completes_at_once_and_the_others_are_unchanged():
    import time
    from paper_2112_00821_b300 import fassmvs, serve
    s = serve.make_streams(sizes=((1920, 1080),), n_frames=5, seed=5, device="cuda")[0]
    r, idx, _ = s.reqs[0]
    cfg = fassmvs.default_config(levels=3, D=[256, 256, 256], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
    srv = fassmvs.Server(cfg, fassmvs.server_config(lanes=1, max_batch=1, mem_budget=40 << 30))
    _push(srv, s, sorted(idx + [r]))
    outs = {q: _outs(s) for q in (1, 2, 3)}
    srv.submit(1, s.fid(r), [s.fid(k) for k in idx], serve._planes(256), *outs[1])
    t0 = time.monotonic()
    while srv.stats()["batches"] < 1 and time.monotonic() - t0 < 30:
        time.sleep(0.0005)
    for q in (2, 3):
        srv.submit(q, s.fid(r), [s.fid(k) for k in idx], serve._planes(256), *outs[q])
    assert srv.cancel(2) is True
    try:
        running = srv.cancel(1)                 # the blocker is on the device: it cannot be withdrawn
        assert running is False
    except fassmvs.FassmvsError as e:           # unless it already finished
        assert e.status == fassmvs.EINVAL
    with pytest.raises(fassmvs.FassmvsError) as ei:
        srv.cancel(99)
    assert ei.value.status == fassmvs.EINVAL
    got = {}
    t0 = time.monotonic()
    while len(got) < 3 and time.monotonic() - t0 < 60:
        for x in srv.poll(4, 1000):
            got[x["id"]] = x
    assert got[2]["status"] == fassmvs.ECANCELED and got[2]["batch_size"] == 0
    assert got[2]["t_done_ns"] < got[1]["t_done_ns"]
    assert got[1]["status"] == fassmvs.OK and got[3]["status"] == fassmvs.OK
    torch.cuda.synchronize()
    for x, y in zip(outs[1], outs[3]):
        assert torch.equal(x, y)
    st = srv.stats()
    assert st["completed"] == 2 and st["failed"] == 1 and st["queued"] == 0
    srv.close()


def _rel_pose(Rr, tr, Rk, tk):
    """Reference -> k from world -> camera poses, in the server's order of
    operations (so that the FP64 consistency test sees identical inputs)."""
    RrT = [[float(Rr[j][i]) for j in range(3)] for i in range(3)]
    R = [[0.0] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            v = 0.0
            for m in range(3):
                v += float(Rk[i][m]) * RrT[m][j]
            R[i][j] = v
    t = []
    for i in range(3):
        v = float(tk[i])
        for m in range(3):
            v -= R[i][m] * float(tr[m])
        t.append(v)
    return np.array(R), np.array(t)


def test_post_filters_in_the_server_equal_the_standalone_filters(streams):
    """DoG mask (Alg. 3) and geometric consistency (Alg. 4) run by the server
    on a request's outputs equal the standalone filters applied to the same
    request served unfiltered, the partner being an earlier request's kept
    depth map; kept maps are given back by release_depth."""
    import time
    from paper_2112_00821_b300 import fassmvs, serve
    s = streams[0]
    (r1, idx1, G1), (r2, idx2, G2) = s.reqs[0], s.reqs[1]
    srv = fassmvs.Server(_cfg(), fassmvs.server_config(lanes=1, max_batch=1, mem_budget=2 << 30))
    _push(srv, s, sorted(set(idx1 + idx2 + [r1, r2])))
    flat = s.frames[r1].copy()
    flat[40:120, 100:220] = 128                          # an untextured patch for the DoG mask
    R1, t1 = s.poses[r1]
    srv.push_frame(9001, flat, s.K, R1, t1)
    o = {q: _outs(s) for q in (1, 2, 3, 4)}
    got = {}

    def run(q, ref, idx, G, **kw):
        srv.submit(q, ref, [s.fid(k) for k in idx], serve._planes(G), *o[q], **kw)
        t0 = time.monotonic()
        while q not in got and time.monotonic() - t0 < 60:
            for x in srv.poll(4, 1000):
                got[x["id"]] = x
        assert got[q]["status"] == fassmvs.OK, got[q]

    run(1, 9001, idx1, G1, postfilter=fassmvs.POST_KEEP)
    run(2, s.fid(r2), idx2, G2, postfilter=fassmvs.POST_KEEP)
    run(3, 9001, idx1, G1, postfilter=fassmvs.POST_DOG)
    run(4, s.fid(r2), idx2, G2, postfilter=fassmvs.POST_DOG | fassmvs.POST_GEO, geo_ids=[1], geo_eta_r=1.0,
        geo_eta_h=1)
    torch.cuda.synchronize()
    ctx = fassmvs.Context(_cfg())
    e3 = [x.clone() for x in o[1]]
    mask = ctx.dog_filter(torch.from_numpy(flat).cuda(), *e3)
    e4 = [x.clone() for x in o[2]]
    ctx.dog_filter(torch.from_numpy(s.frames[r2]).cuda(), *e4)
    R21, t21 = _rel_pose(*s.poses[r2], R1, t1)          # request 2's reference -> request 1's
    hits = ctx.geo_filter(e4[0], s.K, [o[1][0]], R21[None], t21[None], normal=e4[1], conf=e4[2], eta_r=1.0,
                          eta_h=1)
    ctx.sync()
    for x, y in zip(o[3], e3):
        assert torch.equal(x, y)
    for x, y in zip(o[4], e4):
        assert torch.equal(x, y)
    assert not mask[60:100, 120:200].any()                # the filters did act
    assert (hits == 0).any() and (o[4][0] == 0).sum() > (o[2][0] == 0).sum()
    ctx.close()
    with pytest.raises(fassmvs.FassmvsError) as ei:      # only kept maps can be partners
        srv.submit(5, s.fid(r2), [s.fid(k) for k in idx2], serve._planes(G2), *_outs(s),
                   postfilter=fassmvs.POST_GEO, geo_ids=[3])
    assert ei.value.status == fassmvs.EINVAL
    before = srv.stats()["bytes_in_use"]
    srv.release_depth(1)
    srv.release_depth(2)
    assert srv.stats()["bytes_in_use"] < before
    with pytest.raises(fassmvs.FassmvsError):
        srv.release_depth(1)
    srv.close()


def test_post_filters_with_host_outputs(streams):
    """With pinned host outputs the filters act on the server's device copy
    before it is copied back: the result equals the device-output request's."""
    import time
    from paper_2112_00821_b300 import fassmvs, serve
    s = streams[1]
    r, idx, G0 = s.reqs[2]
    srv = fassmvs.Server(_cfg(), fassmvs.server_config(lanes=1, max_batch=1, mem_budget=2 << 30))
    _push(srv, s, sorted(idx + [r]))
    dev_o = _outs(s)
    host_o = tuple(torch.empty_like(x, device="cpu").pin_memory() for x in dev_o)
    got = {}
    for q, o in ((1, dev_o), (2, host_o)):
        srv.submit(q, s.fid(r), [s.fid(k) for k in idx], serve._planes(G0), *o, postfilter=fassmvs.POST_DOG)
        t0 = time.monotonic()
        while q not in got and time.monotonic() - t0 < 60:
            for x in srv.poll(4, 1000):
                got[x["id"]] = x
        assert got[q]["status"] == fassmvs.OK
    torch.cuda.synchronize()
    for x, y in zip(dev_o, host_o):
        assert torch.equal(x.cpu(), y)
    srv.close()
