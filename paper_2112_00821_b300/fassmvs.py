"""Thin ctypes binding of libfassmvs.so (see include/fassmvs.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch provides device memory and the current stream.  There
is no CPU fallback: if the library is missing or no CUDA device is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FASSMVS_CHECKED=1 loads the bounds-checked build (same ABI; a failed check
# makes fassmvs_sync return FASSMVS_EINTERNAL)
LIB_PATH = os.path.join(_HERE, "libfassmvs_checked.so" if os.environ.get("FASSMVS_CHECKED") == "1"
                        else "libfassmvs.so")
_lib = None

OK, EINVAL, ENOMEM, EBUSY, ETIMEOUT, ECUDA, EINTERNAL, ECANCELED = range(8)
_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EBUSY", 4: "ETIMEOUT", 5: "ECUDA", 6: "EINTERNAL",
          7: "ECANCELED"}


class FassmvsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_NAMES.get(status, status), msg))
        self.status = status


class Planes(C.Structure):
    _fields_ = [("n", C.c_double * 3), ("rho_far", C.c_double), ("drho", C.c_double),
                ("G0", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("levels", C.c_int32), ("D", C.c_int32 * 8), ("paths", C.c_int32),
                ("variant", C.c_int32), ("p1", C.c_int32), ("p2", C.c_int32),
                ("adaptive_p2", C.c_int32), ("alpha", C.c_float), ("beta", C.c_float),
                ("median5", C.c_int32), ("normal_radius", C.c_int32), ("normal_beta", C.c_float),
                ("rho_deg", C.c_float), ("dmax", C.c_int32), ("cost", C.c_int32)]


class Frame(C.Structure):
    _fields_ = [("ref", C.c_void_p), ("nbrs", C.c_void_p), ("W", C.c_int32), ("H", C.c_int32),
                ("pitch", C.c_int32), ("n_nb", C.c_int32), ("K", C.c_void_p), ("R", C.c_void_p),
                ("t", C.c_void_p), ("side", C.c_void_p), ("planes", Planes), ("depth", C.c_void_p),
                ("normal", C.c_void_p), ("conf", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("chunk_planes", C.c_int32), ("ctas_per_sm", C.c_int32), ("sgm_parts", C.c_int32),
                ("no_staging", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("max_batch", C.c_int32), ("mem_budget", C.c_size_t),
                ("deadline_ms", C.c_int32), ("overlap_queue", C.c_int32), ("tuning", Tuning),
                ("tuning_overlap", Tuning)]


POST_DOG, POST_GEO, POST_KEEP = 1, 2, 4


class Request(C.Structure):
    _fields_ = [("id", C.c_int64), ("ref", C.c_int64), ("nbrs", C.c_void_p), ("n_nb", C.c_int32),
                ("planes", Planes), ("depth", C.c_void_p), ("normal", C.c_void_p), ("conf", C.c_void_p),
                ("host_outputs", C.c_int32), ("postfilter", C.c_int32), ("geo_n", C.c_int32),
                ("geo_ids", C.c_int64 * 4), ("geo_eta_r", C.c_double), ("geo_eta_h", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("batch_size", C.c_int32),
                ("t_submit_ns", C.c_int64), ("t_admit_ns", C.c_int64), ("t_launch_ns", C.c_int64),
                ("t_done_ns", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("capacity", "bytes_in_use", "peak_bytes", "frames", "resident_frames",
                                         "submitted", "completed", "failed", "queued", "batches",
                                         "max_batch_seen", "overlapped")]


class SgmParams(C.Structure):
    _fields_ = [("paths", C.c_int32), ("variant", C.c_int32), ("p1", C.c_int32),
                ("p2", C.c_int32), ("dmax", C.c_int32), ("p2_lut", C.c_void_p)]


_VP = C.c_void_p
_SIGS = {
    "fassmvs_config_default": [_VP],
    "fassmvs_create": [_VP, C.c_int, C.c_size_t, _VP],
    "fassmvs_destroy": [_VP],
    "fassmvs_set_config": [_VP, _VP],
    "fassmvs_set_cameras": [_VP, _VP, C.c_int, _VP, _VP, _VP],
    "fassmvs_estimate": [_VP, _VP, C.c_int, C.c_int, C.c_int, _VP, C.c_int, _VP, _VP, _VP, _VP, _VP],
    "fassmvs_estimate_host": [_VP, _VP, C.c_int, C.c_int, C.c_int, _VP, C.c_int, _VP, _VP, _VP, _VP, _VP],
    "fassmvs_estimate_host_async": [_VP, _VP, C.c_int, C.c_int, C.c_int, _VP, C.c_int, _VP, _VP, _VP, _VP, _VP],
    "fassmvs_pyramid_down": [_VP, _VP, C.c_int, C.c_int, _VP, _VP],
    "fassmvs_census": [_VP, _VP, C.c_int, C.c_int, _VP, _VP],
    "fassmvs_cost_volume": [_VP, _VP, _VP, C.c_int, _VP, C.c_int, C.c_int, _VP, _VP, _VP, _VP,
                            C.c_double, C.c_double, C.c_int, _VP, C.c_int, C.c_int, _VP, _VP],
    "fassmvs_sgm_aggregate": [_VP, _VP, _VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP,
                              _VP, _VP],
    "fassmvs_wta_refine": [_VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double,
                           C.c_double, C.c_int, _VP, _VP, _VP],
    "fassmvs_wta_refine_noalloc": [_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double,
                                   C.c_double, C.c_int, _VP, _VP, _VP],
    "fassmvs_median5": [_VP, _VP, C.c_int, C.c_int, _VP, _VP],
    "fassmvs_normals": [_VP, _VP, _VP, C.c_int, C.c_int, _VP, C.c_int, C.c_float, _VP, _VP, _VP,
                        C.c_float, _VP, _VP],
    "fassmvs_window": [_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double,
                       C.c_double, C.c_int, C.c_int, _VP, _VP],
    "fassmvs_dsn": [_VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double, C.c_int,
                    _VP, _VP],
    "fassmvs_estimate_batch": [_VP, _VP, C.c_int, _VP],
    "fassmvs_set_graph": [_VP, C.c_int],
    "fassmvs_set_tuning": [_VP, _VP],
    "fassmvs_autotune": [_VP, _VP, C.c_int, _VP, _VP],
    "fassmvs_server_config_default": [_VP],
    "fassmvs_server_create": [_VP, _VP, C.c_int, _VP],
    "fassmvs_server_destroy": [_VP],
    "fassmvs_server_push_frame": [_VP, C.c_int64, _VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP],
    "fassmvs_server_release_frame": [_VP, C.c_int64],
    "fassmvs_server_submit": [_VP, _VP],
    "fassmvs_server_cancel": [_VP, C.c_int64],
    "fassmvs_server_release_depth": [_VP, C.c_int64],
    "fassmvs_server_poll": [_VP, _VP, C.c_int, _VP, C.c_int],
    "fassmvs_server_get_stats": [_VP, _VP],
    "fassmvs_server_last_error": [_VP],
    "fassmvs_debug_inject": [_VP, C.c_int],
    "fassmvs_debug_capture": [_VP, C.c_int],
    "fassmvs_debug_capture_warp": [_VP, C.c_int, C.c_int],
    "fassmvs_debug_dump": [_VP, C.c_int, C.c_int, _VP, C.c_size_t, _VP, _VP],
    "fassmvs_plane_bounds": [_VP, C.c_int, C.c_int, _VP, C.c_double, C.c_double, _VP, _VP],
    "fassmvs_cross_ratio_planes": [_VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, C.c_double, C.c_double, C.c_int,
                                   _VP, _VP, _VP, _VP],
    "fassmvs_dog_filter": [_VP, _VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, _VP, _VP],
    "fassmvs_geo_filter": [_VP, _VP, _VP, _VP, C.c_int, C.c_int, _VP, C.c_int, _VP, _VP, _VP, C.c_double, C.c_int,
                           _VP, _VP],
    "fassmvs_profile_enable": [_VP, C.c_int],
    "fassmvs_profile_read": [_VP, _VP, _VP, C.c_int],
    "fassmvs_sync": [_VP],
    "fassmvs_last_error": [_VP],
    "fassmvs_launch_count": [_VP],
}
EXPORTS = tuple(_SIGS)


def lib():
    """Load the in-tree library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built; run paper_2112_00821_b300/build.py"
                              % os.path.basename(LIB_PATH))
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.fassmvs_destroy.restype = None
        L.fassmvs_server_destroy.restype = None
        L.fassmvs_server_config_default.restype = None
        L.fassmvs_server_last_error.restype = C.c_char_p
        L.fassmvs_last_error.restype = C.c_char_p
        L.fassmvs_launch_count.restype = C.c_uint64
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dbl(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if n is not None and a.size != n:
        raise ValueError("expected %d values" % n)
    return a, a.ctypes.data_as(C.c_void_p)


def default_config(**kw):
    c = Config()
    lib().fassmvs_config_default(C.byref(c))
    for k, v in kw.items():
        if k == "D":
            v = list(v) + [256] * (8 - len(v))
            c.D = (C.c_int32 * 8)(*v)
        else:
            setattr(c, k, v)
    return c


class Context:
    """A fassmvs_ctx on one CUDA device (torch's current device by default)."""

    def __init__(self, cfg=None, device=None, mem_budget=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("fassmvs needs a CUDA device; there is no CPU fallback")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._h = C.c_void_p()
        cfg = cfg if cfg is not None else default_config()
        self._check(lib().fassmvs_create(C.byref(cfg), self.device, mem_budget, C.byref(self._h)),
                    ctx=False)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().fassmvs_destroy(h)
            self._h = C.c_void_p()

    __del__ = close

    def _check(self, st, ctx=True):
        if st != OK:
            msg = lib().fassmvs_last_error(self._h if ctx else None)
            raise FassmvsError(st, (msg or b"").decode())

    # ------------------------------------------------------------ full path
    def set_config(self, cfg):
        self._check(lib().fassmvs_set_config(self._h, C.byref(cfg)))

    def set_cameras(self, K, R, t, side):
        R = np.asarray(R, dtype=np.float64)
        V = R.shape[0]
        k_, kp = _dbl(K, 9)
        r_, rp = _dbl(R, 9 * V)
        t_, tp = _dbl(t, 3 * V)
        s_ = np.ascontiguousarray(side, dtype=np.int8)
        self._check(lib().fassmvs_set_cameras(self._h, kp, V, rp, tp, s_.ctypes.data_as(C.c_void_p)))

    def estimate(self, ref, nbrs, planes, depth=None, normal=None, conf=None):
        import torch
        H, W = ref.shape
        pitch = ref.stride(0)
        for x in nbrs:
            if x.shape != ref.shape or x.stride(0) != pitch or x.dtype != torch.uint8:
                raise ValueError("neighbours must match the reference layout")
        dev = ref.device
        depth = depth if depth is not None else torch.empty((H, W), dtype=torch.float32, device=dev)
        normal = normal if normal is not None else torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        conf = conf if conf is not None else torch.empty((H, W), dtype=torch.float32, device=dev)
        arr = (C.c_void_p * len(nbrs))(*[x.data_ptr() for x in nbrs])
        self._check(lib().fassmvs_estimate(self._h, _ptr(ref), W, H, pitch, arr, len(nbrs),
                                           C.byref(planes), _ptr(depth), _ptr(normal), _ptr(conf),
                                           _stream()))
        return depth, normal, conf

    def estimate_host(self, ref, nbrs, planes, depth=None, normal=None, conf=None, wait=True):
        """The estimate from host images to host maps: ref and nbrs are CPU
        uint8 tensors (page-locked or not) of one layout; depth / normal / conf
        are CPU float32 tensors (allocated here when absent).  wait: return
        once the maps are in them (fassmvs_estimate_host); otherwise once the
        images are copied, the maps following by the next sync() or waiting
        call (fassmvs_estimate_host_async)."""
        import torch
        H, W = ref.shape
        pitch = ref.stride(0)
        for x in [ref] + list(nbrs):
            if x.device.type != "cpu" or x.dtype != torch.uint8 or x.shape != ref.shape or x.stride(0) != pitch \
                    or x.stride(1) != 1:
                raise ValueError("images must be CPU uint8 tensors of one row layout")
        depth = depth if depth is not None else torch.empty((H, W), dtype=torch.float32)
        normal = normal if normal is not None else torch.empty((H, W, 3), dtype=torch.float32)
        conf = conf if conf is not None else torch.empty((H, W), dtype=torch.float32)
        for t, shp in ((depth, (H, W)), (normal, (H, W, 3)), (conf, (H, W))):
            if t.device.type != "cpu" or t.dtype != torch.float32 or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError("outputs must be contiguous CPU float32 tensors of the map shapes")
        arr = (C.c_void_p * len(nbrs))(*[x.data_ptr() for x in nbrs])
        fn = lib().fassmvs_estimate_host if wait else lib().fassmvs_estimate_host_async
        self._check(fn(self._h, C.c_void_p(ref.data_ptr()), W, H, pitch, arr, len(nbrs), C.byref(planes),
                       C.c_void_p(depth.data_ptr()), C.c_void_p(normal.data_ptr()), C.c_void_p(conf.data_ptr()),
                       _stream()))
        return depth, normal, conf

    # ------------------------------------------------------------ batched form
    @staticmethod
    def _frames(items):
        """fassmvs_frame array of `items`: dicts with ref, nbrs, K, R, t, side,
        planes (a Planes) and optional depth / normal / conf tensors (allocated
        here when absent).  Returns (array, keep-alive list, outputs)."""
        import torch
        arr = (Frame * len(items))()
        keep, outs = [], []
        for i, it in enumerate(items):
            ref, nbrs = it["ref"], it["nbrs"]
            H, W = ref.shape
            pitch = ref.stride(0)
            for x in nbrs:
                if x.shape != ref.shape or x.stride(0) != pitch or x.dtype != torch.uint8:
                    raise ValueError("neighbours must match the reference layout")
            V = len(nbrs)
            dev = ref.device
            depth = it.get("depth")
            depth = depth if depth is not None else torch.empty((H, W), dtype=torch.float32, device=dev)
            normal = it.get("normal")
            normal = normal if normal is not None else torch.empty((H, W, 3), dtype=torch.float32, device=dev)
            conf = it.get("conf")
            conf = conf if conf is not None else torch.empty((H, W), dtype=torch.float32, device=dev)
            nb = (C.c_void_p * V)(*[x.data_ptr() for x in nbrs])
            k_, kp = _dbl(it["K"], 9)
            r_, rp = _dbl(it["R"], 9 * V)
            t_, tp = _dbl(it["t"], 3 * V)
            s_ = np.ascontiguousarray(it["side"], dtype=np.int8)
            if s_.size != V:
                raise ValueError("one side per neighbour")
            keep += [nb, k_, r_, t_, s_]
            f = arr[i]
            f.ref = ref.data_ptr()
            f.nbrs = C.cast(nb, C.c_void_p)
            f.W, f.H, f.pitch, f.n_nb = W, H, pitch, V
            f.K, f.R, f.t = kp, rp, tp
            f.side = s_.ctypes.data_as(C.c_void_p)
            f.planes = it["planes"]
            f.depth, f.normal, f.conf = depth.data_ptr(), normal.data_ptr(), conf.data_ptr()
            outs.append((depth, normal, conf))
        return arr, keep, outs

    def estimate_batch(self, items):
        """fassmvs_estimate_batch; returns [(depth, normal, conf)] per frame."""
        arr, keep, outs = self._frames(items)
        self._check(lib().fassmvs_estimate_batch(self._h, arr, len(items), _stream()))
        return outs

    def set_graph(self, on=True):
        self._check(lib().fassmvs_set_graph(self._h, 1 if on else 0))

    def set_tuning(self, chunk_planes=0, ctas_per_sm=2, sgm_parts=0, no_staging=0):
        t = Tuning(int(chunk_planes), int(ctas_per_sm), int(sgm_parts), int(no_staging))
        self._check(lib().fassmvs_set_tuning(self._h, C.byref(t)))

    def autotune(self, items):
        """Times the work decompositions on this batch; returns the chosen
        (chunk_planes, ctas_per_sm, sgm_parts), kept for batches of the same
        shapes."""
        arr, keep, outs = self._frames(items)
        t = Tuning()
        self._check(lib().fassmvs_autotune(self._h, arr, len(items), _stream(), C.byref(t)))
        return t.chunk_planes, t.ctas_per_sm, t.sgm_parts

    def sync(self):
        self._check(lib().fassmvs_sync(self._h))

    # ------------------------------------------------------------ post-filters
    def dog_filter(self, ref, depth=None, normal=None, conf=None):
        """Alg. 3: returns the texture mask (uint8 tensor); depth / normal /
        conf (if given) are zeroed in place where it is 0."""
        import torch
        H, W = ref.shape
        mask = torch.empty((H, W), dtype=torch.uint8, device=ref.device)
        self._check(lib().fassmvs_dog_filter(self._h, _ptr(ref), W, H, ref.stride(0), _ptr(depth), _ptr(normal),
                                             _ptr(conf), _ptr(mask), _stream()))
        return mask

    def geo_filter(self, depth, K, depths, R, t, normal=None, conf=None, eta_r=10.0, eta_h=3):
        """Alg. 4 in place on depth (and normal / conf); returns the hit counts."""
        import torch
        H, W = depth.shape
        hits = torch.empty((H, W), dtype=torch.uint8, device=depth.device)
        n = len(depths)
        arr = (C.c_void_p * max(1, n))(*[x.data_ptr() for x in depths])
        k_, kp = _dbl(K, 9)
        r_, rp = _dbl(np.asarray(R, np.float64).reshape(-1), 9 * n) if n else (None, None)
        t_, tp = _dbl(np.asarray(t, np.float64).reshape(-1), 3 * n) if n else (None, None)
        self._check(lib().fassmvs_geo_filter(self._h, _ptr(depth), _ptr(normal), _ptr(conf), W, H, kp, n, arr, rp,
                                             tp, float(eta_r), int(eta_h), _ptr(hits), _stream()))
        return hits

    STAGES = ("pyramid", "census", "cost", "sgm", "wta", "median", "normals", "window", "relayout")

    DUMPS = ("cost", "window", "dsn", "agg", "argmin", "depth_raw", "depth", "normal", "warp")

    def debug_capture(self, level):
        """The next estimates keep the intermediates of pyramid level `level`
        (frame 0); -1 turns capturing off."""
        self._check(lib().fassmvs_debug_capture(self._h, int(level)))

    def debug_capture_warp(self, plane, view):
        """The captures keep the warped values (minus 128) of this (plane of
        the level's list, neighbour view) pair, dumped as "warp"; -1, -1: none."""
        self._check(lib().fassmvs_debug_capture_warp(self._h, int(plane), int(view)))

    def debug_dump(self, level, what):
        """One captured intermediate (a name of DUMPS) as a CUDA tensor:
        cost / agg uint16 (H, W, Ds) viewed as int16, window / argmin int32
        (H, W), dsn int8 (8, H, W), depth_raw / depth float32 (H, W), normal
        float32 (H, W, 3), warp float32 (H, W)."""
        import torch
        w = self.DUMPS.index(what)
        dims = (C.c_int32 * 5)()
        nb = C.c_size_t()
        self._check(lib().fassmvs_debug_dump(self._h, int(level), w, None, 0, C.byref(nb), dims))
        W, H, D, Ds, G = list(dims)
        shape, dt = {0: ((H, W, Ds), torch.int16), 1: ((H, W), torch.int32), 2: ((8, H, W), torch.int8),
                     3: ((H, W, Ds), torch.int16), 4: ((H, W), torch.int32), 5: ((H, W), torch.float32),
                     6: ((H, W), torch.float32), 7: ((H, W, 3), torch.float32), 8: ((H, W), torch.float32)}[w]
        out = torch.empty(shape, dtype=dt, device="cuda")
        self._check(lib().fassmvs_debug_dump(self._h, int(level), w, _ptr(out), nb.value, None, None))
        return out, dict(W=W, H=H, D=D, Ds=Ds, G=G)

    def debug_inject(self, mode):
        """Test hook: 1 makes the cost kernel's staged waits give up (results
        unchanged, the next sync reports ETIMEOUT); 0 turns it off."""
        self._check(lib().fassmvs_debug_inject(self._h, int(mode)))

    def profile(self, on=True):
        self._check(lib().fassmvs_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset=True):
        """{stage: (total ms, stage launches)} accumulated since the last reset."""
        ms = (C.c_double * len(self.STAGES))()
        cnt = (C.c_uint64 * len(self.STAGES))()
        self._check(lib().fassmvs_profile_read(self._h, ms, cnt, 1 if reset else 0))
        return {n: (ms[i], int(cnt[i])) for i, n in enumerate(self.STAGES)}

    @staticmethod
    def launch_count():
        return int(lib().fassmvs_launch_count(None))

    # ------------------------------------------------------------ stages
    def pyramid_down(self, img, out=None):
        import torch
        H, W = img.shape
        out = out if out is not None else torch.empty(((H + 1) // 2, (W + 1) // 2), dtype=torch.uint8,
                                                      device=img.device)
        self._check(lib().fassmvs_pyramid_down(self._h, _ptr(img), W, H, _ptr(out), _stream()))
        return out

    def census(self, img, out=None):
        import torch
        H, W = img.shape
        out = out if out is not None else torch.empty((H, W), dtype=torch.int64, device=img.device)
        self._check(lib().fassmvs_census(self._h, _ptr(img), W, H, _ptr(out), _stream()))
        return out

    def cost_volume(self, ref, nbrs, side, K, R, t, n, rho0, drho, G, lo=None, D=None, Ds=None,
                    out=None):
        import torch
        H, W = ref.shape
        D = G if D is None else D
        Ds = ((D + 7) // 8) * 8 if Ds is None else Ds
        V = len(nbrs)
        out = out if out is not None else torch.zeros((H, W, Ds), dtype=torch.int16, device=ref.device)
        arr = (C.c_void_p * V)(*[x.data_ptr() for x in nbrs])
        s_ = np.ascontiguousarray(side, dtype=np.int8)
        k_, kp = _dbl(K, 9)
        r_, rp = _dbl(R, 9 * V)
        t_, tp = _dbl(t, 3 * V)
        n_, npp = _dbl(n, 3)
        self._check(lib().fassmvs_cost_volume(self._h, _ptr(ref), arr, V, s_.ctypes.data_as(C.c_void_p),
                                              W, H, kp, rp, tp, npp, rho0, drho, int(G), _ptr(lo),
                                              int(D), int(Ds), _ptr(out), _stream()))
        return out

    def sgm_aggregate(self, S, D, p1, p2=0, lut=None, lo=None, dI=None, img=None, paths=8,
                      variant=0, dmax=8, out=None):
        import torch
        H, W, Ds = S.shape
        out = out if out is not None else torch.zeros_like(S)
        lut_a = None
        if lut is not None:
            lut_a = np.ascontiguousarray(lut, dtype=np.uint16)
        prm = SgmParams(paths, variant, int(p1), int(p2), int(dmax),
                        None if lut_a is None else lut_a.ctypes.data)
        self._check(lib().fassmvs_sgm_aggregate(self._h, _ptr(S), _ptr(lo), _ptr(dI), _ptr(img), W, H,
                                                int(D), Ds, C.byref(prm), _ptr(out), _stream()))
        return out

    def wta_refine(self, Sbar, D, K, n, rho0, drho, G, lo=None):
        import torch
        H, W, Ds = Sbar.shape
        depth = torch.empty((H, W), dtype=torch.float32, device=Sbar.device)
        gwin = torch.empty((H, W), dtype=torch.int32, device=Sbar.device)
        k_, kp = _dbl(K, 9)
        n_, npp = _dbl(n, 3)
        self._check(lib().fassmvs_wta_refine(self._h, _ptr(Sbar), _ptr(lo), W, H, int(D), Ds, kp, npp,
                                             rho0, drho, int(G), _ptr(depth), _ptr(gwin), _stream()))
        return depth, gwin

    def median5(self, d):
        import torch
        H, W = d.shape
        out = torch.empty_like(d)
        self._check(lib().fassmvs_median5(self._h, _ptr(d), W, H, _ptr(out), _stream()))
        return out

    def normals(self, depth, img, K, radius=2, beta=10.0, n_plane=(0.0, 0.0, -1.0), rho_deg=60.0,
                with_conf=True):
        import torch
        H, W = depth.shape
        normal = torch.empty((H, W, 3), dtype=torch.float32, device=depth.device)
        raw = torch.empty((H, W, 3), dtype=torch.float32, device=depth.device)
        conf = torch.empty((H, W), dtype=torch.float32, device=depth.device) if with_conf else None
        k_, kp = _dbl(K, 9)
        n_, npp = _dbl(n_plane, 3)
        self._check(lib().fassmvs_normals(self._h, _ptr(depth), _ptr(img), W, H, kp, int(radius),
                                          float(beta), _ptr(normal), _ptr(raw), npp, float(rho_deg),
                                          _ptr(conf), _stream()))
        return normal, raw, conf

    def window(self, dc, W, H, K, n, rho0, drho, G, D):
        import torch
        Hc, Wc = dc.shape
        lo = torch.empty((H, W), dtype=torch.int32, device=dc.device)
        k_, kp = _dbl(K, 9)
        n_, npp = _dbl(n, 3)
        self._check(lib().fassmvs_window(self._h, _ptr(dc), Wc, Hc, W, H, kp, npp, rho0, drho, int(G),
                                         int(D), _ptr(lo), _stream()))
        return lo

    def dsn(self, dc, nc, W, H, K, drho, dmax=8, n=(0.0, 0.0, -1.0)):
        import torch
        Hc, Wc = dc.shape
        out = torch.empty((8, H, W), dtype=torch.int8, device=dc.device)
        k_, kp = _dbl(K, 9)
        n_, np_ = _dbl(n, 3)
        self._check(lib().fassmvs_dsn(self._h, _ptr(dc), _ptr(nc), Wc, Hc, W, H, kp, np_, drho, int(dmax),
                                      _ptr(out), _stream()))
        return out


def server_config(**kw):
    c = ServerConfig()
    lib().fassmvs_server_config_default(C.byref(c))
    for k, v in kw.items():
        if k in ("tuning", "tuning_overlap"):
            setattr(c, k, Tuning(*v))
        else:
            setattr(c, k, v)
    return c


class Server:
    """A fassmvs_server: resident frames, admission by device memory,
    continuous batching over lanes (see include/fassmvs.h)."""

    def __init__(self, cfg=None, scfg=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("fassmvs needs a CUDA device; there is no CPU fallback")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._h = C.c_void_p()
        cfg = cfg if cfg is not None else default_config()
        scfg = scfg if scfg is not None else server_config()
        self._check(lib().fassmvs_server_create(C.byref(cfg), C.byref(scfg), self.device, C.byref(self._h)),
                    own=False)
        self._keep = {}

    def _check(self, st, own=True):
        if st != OK:
            msg = lib().fassmvs_server_last_error(self._h if own else None)
            raise FassmvsError(st, (msg or b"").decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().fassmvs_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    __del__ = close

    def push_frame(self, fid, img, K, R, t):
        """img: (H, W) uint8 numpy array (host); R, t: world -> camera."""
        img = np.ascontiguousarray(img, dtype=np.uint8)
        H, W = img.shape
        k_, kp = _dbl(K, 9)
        r_, rp = _dbl(R, 9)
        t_, tp = _dbl(t, 3)
        self._check(lib().fassmvs_server_push_frame(self._h, int(fid), img.ctypes.data_as(C.c_void_p), W, H,
                                                    img.strides[0], kp, rp, tp))

    def release_frame(self, fid):
        self._check(lib().fassmvs_server_release_frame(self._h, int(fid)))

    def submit(self, rid, ref, nbrs, planes, depth, normal, conf, postfilter=0, geo_ids=(), geo_eta_r=10.0,
               geo_eta_h=3):
        """Outputs: pinned host tensors (copied back) or CUDA tensors.
        postfilter: POST_DOG | POST_GEO | POST_KEEP; geo_ids: earlier requests
        with kept depth maps (POST_GEO)."""
        host = not depth.is_cuda
        nb = (C.c_int64 * len(nbrs))(*[int(x) for x in nbrs])
        gi = list(geo_ids)
        if len(gi) > 4:
            raise ValueError("at most 4 consistency partners")
        rq = Request(int(rid), int(ref), C.cast(nb, C.c_void_p), len(nbrs), planes, depth.data_ptr(),
                     normal.data_ptr(), conf.data_ptr(), 1 if host else 0, int(postfilter), len(gi),
                     (C.c_int64 * 4)(*(gi + [0] * (4 - len(gi)))), float(geo_eta_r), int(geo_eta_h))
        self._check(lib().fassmvs_server_submit(self._h, C.byref(rq)))
        self._keep[int(rid)] = (depth, normal, conf)

    def release_depth(self, rid):
        """Gives back the depth map kept for request rid (POST_KEEP)."""
        self._check(lib().fassmvs_server_release_depth(self._h, int(rid)))

    def cancel(self, rid):
        """Withdraws a request not launched yet (its result comes with status
        ECANCELED); False when it is already running (it completes normally)."""
        st = lib().fassmvs_server_cancel(self._h, int(rid))
        if st == EBUSY:
            return False
        self._check(st)
        return True

    def poll(self, max_results=64, timeout_ms=0):
        """Completed results: list of dicts (id, status, batch_size, times in ns)."""
        out = (Result * max_results)()
        n = C.c_int()
        self._check(lib().fassmvs_server_poll(self._h, out, max_results, C.byref(n), int(timeout_ms)))
        res = []
        for i in range(n.value):
            r = out[i]
            self._keep.pop(int(r.id), None)
            res.append(dict(id=r.id, status=r.status, batch_size=r.batch_size, t_submit_ns=r.t_submit_ns,
                            t_admit_ns=r.t_admit_ns, t_launch_ns=r.t_launch_ns, t_done_ns=r.t_done_ns))
        return res

    def stats(self):
        st = ServerStats()
        self._check(lib().fassmvs_server_get_stats(self._h, C.byref(st)))
        return {n: int(getattr(st, n)) for n, _ in ServerStats._fields_}


def wta_refine_noalloc(Sbar, D, K, n, rho0, drho, G, lo=None, depth=None, gwin=None):
    """fassmvs_wta_refine_noalloc on the current device: no context and no
    device allocation inside the library (pass depth / gwin to avoid torch
    allocating them here)."""
    import torch
    H, W, Ds = Sbar.shape
    dev = Sbar.device
    if dev.type != "cuda":
        raise ValueError("Sbar must be a CUDA tensor")
    depth = depth if depth is not None else torch.empty((H, W), dtype=torch.float32, device=dev)
    gwin = gwin if gwin is not None else torch.empty((H, W), dtype=torch.int32, device=dev)
    for name, t in (("Sbar", Sbar), ("lo", lo), ("depth", depth), ("gwin", gwin)):
        if t is not None and (t.device != dev or not t.is_contiguous()):
            raise ValueError("%s must be a contiguous tensor on %s" % (name, dev))
    k_, kp = _dbl(K, 9)
    n_, npp = _dbl(n, 3)
    # the library runs on the current device and stream: make them Sbar's
    with torch.cuda.device(dev):
        st = lib().fassmvs_wta_refine_noalloc(_ptr(Sbar), _ptr(lo), W, H, int(D), Ds, kp, npp, rho0, drho,
                                              int(G), _ptr(depth), _ptr(gwin), _stream())
    if st != OK:
        raise FassmvsError(st, (lib().fassmvs_last_error(None) or b"").decode())
    return depth, gwin


def plane_bounds(K, W, H, n, d_min, d_max):
    """(delta_min, delta_max) of planes with normal n enclosing the reference
    frustum between depths d_min and d_max (host computation, no device)."""
    k_, kp = _dbl(K, 9)
    n_, np_ = _dbl(n, 3)
    lo, hi = C.c_double(), C.c_double()
    st = lib().fassmvs_plane_bounds(kp, int(W), int(H), np_, float(d_min), float(d_max), C.byref(lo), C.byref(hi))
    if st != OK:
        raise FassmvsError(st, (lib().fassmvs_last_error(None) or b"").decode())
    return lo.value, hi.value


def cross_ratio_planes(K, W, H, R, t, n, delta_min, delta_max, max_planes=4096):
    """Alg. 2 plane distances (far to near), the index of camera k, and the
    uniform inverse-distance Planes the estimate takes (host computation, no
    device).  R: (n, 3, 3), t: (n, 3), reference -> camera."""
    R = np.ascontiguousarray(np.asarray(R, np.float64).reshape(-1, 9))
    t = np.ascontiguousarray(np.asarray(t, np.float64).reshape(-1, 3))
    if R.shape[0] != t.shape[0]:
        raise ValueError("R and t disagree on the camera count")
    k_, kp = _dbl(K, 9)
    n_, np_ = _dbl(n, 3)
    out = np.zeros(max_planes, np.float64)
    cnt, cam = C.c_int(), C.c_int(-1)
    uni = Planes()
    st = lib().fassmvs_cross_ratio_planes(kp, int(W), int(H), R.shape[0], R.ctypes.data_as(C.c_void_p),
                                          t.ctypes.data_as(C.c_void_p), np_, float(delta_min), float(delta_max),
                                          int(max_planes), out.ctypes.data_as(C.c_void_p), C.byref(cnt),
                                          C.byref(cam), C.byref(uni))
    if st != OK:
        raise FassmvsError(st, (lib().fassmvs_last_error(None) or b"").decode())
    return out[:cnt.value].copy(), cam.value, uni


def planes_of(scene):
    """fassmvs_planes of a synth.Scene."""
    p = Planes()
    p.n = (C.c_double * 3)(*[float(v) for v in scene.plane_n])
    p.rho_far = float(scene.rho_far)
    p.drho = float(scene.drho)
    p.G0 = int(scene.G0)
    return p

