"""Simulated UAV video streams and two ways of serving their keyframes.

* serving form: fassmvs.Server (frames resident on the device with their
  pyramids, admission by device memory, continuous batching over lanes);
* plain per-frame form: one fassmvs_estimate per keyframe, in arrival order,
  each waited for before the next starts.

A stream is a seeded oblique-city trajectory at a fixed frame rate; every
`every`-th frame is a keyframe whose request names 4-6 frames around it and a
plane count, and becomes ready when its last frame has arrived.  Latency is
measured from that scheduled moment (on the monotonic clock the server's
timestamps use) to the result being in host memory, so time a driver spends
blocked is counted, not hidden.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import fassmvs, synth


class Stream:
    """One camera: rendered frames, world -> camera poses, keyframe requests
    (ref index, neighbour indices, plane count), frame ids offset by id_base."""

    def __init__(self, W, H, n_frames, seed, id_base=0, every=5, device=None, phase=0.0):
        K, pose, render, reqs = synth.trajectory_frames(n_frames, W, H, seed, every=every, device=device)
        self.W, self.H, self.K = W, H, K
        self.frames = [render(i) for i in range(n_frames)]
        self.poses = [pose(i) for i in range(n_frames)]
        self.reqs = reqs
        self.id_base = id_base
        self.phase = phase          # arrival offset in frame periods

    def fid(self, i):
        return self.id_base + i


def subset(streams, n_req):
    """Shallow copies keeping the first n_req keyframe requests of each
    stream and the frames they need (for warm-up runs)."""
    out = []
    for s in streams:
        c = Stream.__new__(Stream)
        c.__dict__.update(s.__dict__)
        c.reqs = s.reqs[:n_req]
        last = max(max(idx + [r]) for r, idx, G0 in c.reqs)
        c.frames = s.frames[:last + 1]
        c.poses = s.poses[:last + 1]
        out.append(c)
    return out


def make_streams(sizes=((1920, 1080), (2720, 1530)), n_frames=150, seed=0, device=None, every=5):
    """Cameras of the given sizes flying interleaved (arrivals offset by a
    fraction of the frame period)."""
    return [Stream(W, H, n_frames, seed + 17 * k, id_base=1_000_000 * k, every=every, device=device,
                   phase=k / len(sizes)) for k, (W, H) in enumerate(sizes)]


def _events(streams, fps):
    """Frame arrivals in time order: (t, stream index, frame index, [requests
    that become ready])."""
    ev = []
    for si, s in enumerate(streams):
        last = {}
        for j, (r, idx, G0) in enumerate(s.reqs):
            last.setdefault(max(idx + [r]), []).append(j)
        for i in range(len(s.frames)):
            t = (i + s.phase) / fps if fps else 0.0
            ev.append((t, si, i, last.get(i, [])))
    ev.sort(key=lambda e: (e[0], e[1], e[2]))
    return ev


def _planes(G0):
    p = fassmvs.Planes()
    p.n = (fassmvs.C.c_double * 3)(0.0, 0.0, -1.0)
    p.rho_far, p.drho = synth.city_sweep(G0)
    p.G0 = int(G0)
    return p


def _last_use(s):
    lu = {}
    for j, (r, idx, G0) in enumerate(s.reqs):
        for i in idx + [r]:
            lu[i] = max(lu.get(i, -1), j)
    return lu


def relative_pose(Rr, tr, Rk, tk):
    """Reference -> view k pose from two world -> camera poses,
    X_k = R_k R_r^T X_r + (t_k - R_k R_r^T t_r), summed in the order the
    server forms it (plain FP64 products and sums, no fused multiply-add), so
    that one estimate per keyframe and the server get identical cameras."""
    Rr = [[float(v) for v in row] for row in np.asarray(Rr, np.float64)]
    Rk_ = [[float(v) for v in row] for row in np.asarray(Rk, np.float64)]
    R = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            v = 0.0
            for m in range(3):
                v += Rk_[i][m] * Rr[j][m]          # (R_k R_r^T)_ij
            R[i, j] = v
    t = np.zeros(3)
    for i in range(3):
        v = float(tk[i])
        for m in range(3):
            v -= float(R[i, m]) * float(tr[m])
        t[i] = v
    return R, t


def _pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float32, pin_memory=True)


def run_server(streams, cfg, scfg, fps=30.0, keep=False, wait_s=300.0, post=0, eta_r=10.0, eta_h=1):
    """Serves the streams through one fassmvs.Server.  fps=None: every frame
    is available at once (throughput).  post > 0: every keyframe also gets the
    DoG mask and the geometric consistency check against the kept depth maps
    of the last `post` completed keyframes of its stream (a sliding window;
    older maps are given back).  Returns a summary dict and, with keep, the
    outputs per (stream, request).  Raises if a frame stays refused or results
    stay out for longer than the bounds."""
    srv = fassmvs.Server(cfg, scfg)
    lat, outs, pend = [], {}, {}
    last_use = [_last_use(s) for s in streams]
    window = [[] for _ in streams]          # completed keyframes with kept depth maps, oldest first
    n_req = sum(len(s.reqs) for s in streams)
    t0 = time.monotonic_ns()

    def drain(timeout_ms=0):
        for r in srv.poll(64, timeout_ms):
            key, t_ready = pend.pop(r["id"])
            if r["status"] != fassmvs.OK:
                raise fassmvs.FassmvsError(r["status"], "request %d failed" % r["id"])
            lat.append((r["t_done_ns"] - t_ready) * 1e-9)
            if post:
                w = window[key[0]]
                w.append(r["id"])
                while len(w) > post:
                    srv.release_depth(w.pop(0))

    rid = 0
    for t, si, i, ready in _events(streams, fps):
        s = streams[si]
        while fps and time.monotonic_ns() - t0 < t * 1e9:
            drain(0)
            time.sleep(0.0002)
        for attempt in range(2001):
            try:
                R, tv = s.poses[i]
                srv.push_frame(s.fid(i), s.frames[i], s.K, R, tv)
                break
            except fassmvs.FassmvsError as e:
                if e.status != fassmvs.EBUSY or attempt == 2000:
                    raise
                drain(5)
        for j in ready:
            r, idx, G0 = s.reqs[j]
            o = (_pinned((s.H, s.W)), _pinned((s.H, s.W, 3)), _pinned((s.H, s.W)))
            kw = {}
            if post:
                part = window[si][-post:]
                kw = dict(postfilter=fassmvs.POST_KEEP | fassmvs.POST_DOG | (fassmvs.POST_GEO if part else 0),
                          geo_ids=part, geo_eta_r=eta_r, geo_eta_h=min(eta_h, len(part)))
            srv.submit(rid, s.fid(r), [s.fid(k) for k in idx], _planes(G0), *o, **kw)
            pend[rid] = ((si, j), t0 + int(t * 1e9))
            if keep:
                outs[(si, j)] = o
            rid += 1
            for k in idx + [r]:
                if last_use[si].get(k) == j:
                    srv.release_frame(s.fid(k))
        if i not in last_use[si]:
            srv.release_frame(s.fid(i))
        drain(0)
    t_give_up = time.monotonic_ns() + int(wait_s * 1e9)
    while pend:
        if time.monotonic_ns() > t_give_up:
            raise TimeoutError("%d requests still pending after %.0f s" % (len(pend), wait_s))
        drain(50)
    t_end = time.monotonic_ns()
    st = srv.stats()
    srv.close()
    n_frames = sum(len(s.frames) for s in streams)
    res = _summary(lat, n_req, n_frames, (t_end - t0) * 1e-9)
    res["server"] = {k: st[k] for k in ("capacity", "peak_bytes", "batches", "max_batch_seen", "overlapped",
                                        "completed")}
    return (res, outs) if keep else res


def run_plain(streams, cfg, fps=30.0, keep=False):
    """One fassmvs_estimate per keyframe in arrival order (frames uploaded on
    arrival and kept on the device; the estimate rebuilds the pyramids)."""
    import torch
    ctx = fassmvs.Context(cfg)
    dev = {}
    queue, lat, outs = [], [], {}
    n_req = sum(len(s.reqs) for s in streams)
    t0 = time.monotonic_ns()
    evs = _events(streams, fps)
    e = 0
    done = 0
    while done < n_req:
        now = (time.monotonic_ns() - t0) * 1e-9
        while e < len(evs) and (not fps or evs[e][0] <= now):
            t, si, i, ready = evs[e]
            dev[(si, i)] = torch.from_numpy(streams[si].frames[i]).cuda()
            for j in ready:
                queue.append((si, j, t0 + int(t * 1e9)))
            e += 1
        if not queue:
            time.sleep(0.0002)
            continue
        si, j, t_ready = queue.pop(0)
        s = streams[si]
        r, idx, G0 = s.reqs[j]
        Rr, tr = s.poses[r]
        Rs, ts, side = [], [], []
        for k in idx:
            Rk, tk = s.poses[k]
            Rrel, trel = relative_pose(Rr, tr, Rk, tk)
            Rs.append(Rrel)
            ts.append(trel)
            side.append(-1 if k < r else 1)
        ctx.set_cameras(s.K, np.stack(Rs), np.stack(ts), np.array(side, np.int8))
        d, n, c = ctx.estimate(dev[(si, r)], [dev[(si, k)] for k in idx], _planes(G0))
        o = (_pinned((s.H, s.W)), _pinned((s.H, s.W, 3)), _pinned((s.H, s.W)))
        o[0].copy_(d, non_blocking=True)
        o[1].copy_(n, non_blocking=True)
        o[2].copy_(c, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        lat.append((time.monotonic_ns() - t_ready) * 1e-9)
        if keep:
            outs[(si, j)] = o
        done += 1
    t_end = time.monotonic_ns()
    ctx.close()
    n_frames = sum(len(s.frames) for s in streams)
    res = _summary(lat, n_req, n_frames, (t_end - t0) * 1e-9)
    return (res, outs) if keep else res


def _summary(lat, n_req, n_frames, wall):
    a = np.sort(np.asarray(lat)) * 1e3
    q = lambda p: float(a[min(len(a) - 1, int(math.ceil(p / 100.0 * len(a))) - 1)]) if len(a) else None
    return {"keyframes": n_req, "frames": n_frames, "wall_s": round(wall, 3),
            "keyframes_per_s": round(n_req / wall, 2), "frames_per_s": round(n_frames / wall, 2),
            "latency_ms": {"p50": round(q(50), 2), "p99": round(q(99), 2), "mean": round(float(a.mean()), 2),
                           "max": round(float(a.max()), 2)}}
