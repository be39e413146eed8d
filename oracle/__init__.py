"""CPU oracle for the FaSS-MVS hot path -- test infrastructure only.

Plain FP64 C (``fassmvs_oracle.c``) restating each step of the paper, loaded
with ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the product path never does.  It
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fassmvs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction, IEEE arithmetic)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", *CFLAGS, "-o", _LIB, _SRC, "-lm"])
    return _LIB


class SgmParams(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("D", C.c_int32), ("Ds", C.c_int32),
                ("G", C.c_int32), ("paths", C.c_int32), ("variant", C.c_int32),
                ("p1", C.c_int32), ("p2", C.c_int32), ("dmax", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("levels", C.c_int32), ("D", C.c_int32 * 8), ("paths", C.c_int32),
                ("variant", C.c_int32), ("p1", C.c_int32), ("p2", C.c_int32),
                ("adaptive_p2", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double),
                ("median5", C.c_int32), ("normal_radius", C.c_int32), ("normal_beta", C.c_double),
                ("rho_deg", C.c_double), ("dmax", C.c_int32), ("cost", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _lib.or_hamming.restype = C.c_int
        _lib.or_lr_combine.restype = C.c_uint16
        _lib.or_parabola_vertex.restype = C.c_double
        _lib.or_parabola_vertex.argtypes = [C.c_double] * 6
        _lib.or_warp_sample.restype = C.c_double
        _lib.or_cost_volume.restype = C.c_int
        _lib.or_cost_band.restype = C.c_int
        _lib.or_ncc_window.restype = C.c_int
        _lib.or_sgm_aggregate.restype = C.c_int
        _lib.or_estimate.restype = C.c_int
        _lib.or_plane_bounds.restype = C.c_int
        _lib.or_cross_ratio_planes.restype = C.c_int
        _lib.or_threads.restype = C.c_int
        _lib.or_threads.argtypes = [C.c_int]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def pyr_weights():
    w = np.zeros(3, np.int32)
    lib().or_pyr_weights(_p(w))
    return w


def pyramid_down(img):
    img = _c(img, np.uint8)
    H, W = img.shape
    out = np.zeros(((H + 1) // 2, (W + 1) // 2), np.uint8)
    lib().or_pyramid_down(_p(img), W, H, _p(out))
    return out


def census(img):
    img = _c(img, np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.uint64)
    lib().or_census_u8(_p(img), W, H, _p(out))
    return out


def hamming(a, b):
    return lib().or_hamming(C.c_uint64(int(a)), C.c_uint64(int(b)))


def homography(K, R, t, n, delta):
    Hm = np.zeros(9, np.float64)
    lib().or_homography(_p(_c(K, np.float64)), _p(_c(R, np.float64)), _p(_c(t, np.float64)),
                        _p(_c(n, np.float64)), C.c_double(delta), _p(Hm))
    return Hm.reshape(3, 3)


def warp_image(img, Hm):
    """Alg. 1 warp of a whole image: FP64 lerp-form bilinear values (not
    rounded) and whether each position lies on the image grid."""
    img = _c(img, np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.float64)
    val = np.zeros((H, W), np.uint8)
    lib().or_warp_image(_p(img), W, H, _p(_c(Hm, np.float64).ravel()), _p(out), _p(val))
    return out, val.astype(bool)


def lr_combine(sL, nL, sR, nR):
    return lib().or_lr_combine(C.c_uint32(sL), nL, C.c_uint32(sR), nR)


def ncc_window(a, b):
    """NCC cost of two 5x5 windows (reference grey levels, warped real
    values), reading of Sec. 2.2.1 in fassmvs_oracle.c."""
    a = _c(np.asarray(a, np.float64).ravel(), np.float64)
    b = _c(np.asarray(b, np.float64).ravel(), np.float64)
    assert a.size == 25 and b.size == 25
    return lib().or_ncc_window(_p(a), _p(b))


def cost_volume(ref, nbrs, side, K, R, t, n, rho0, drho, G, lo=None, D=None, Ds=None, cost=0):
    ref = _c(ref, np.uint8)
    H, W = ref.shape
    V = len(nbrs)
    nb = [_c(x, np.uint8) for x in nbrs]
    arr = (C.c_void_p * V)(*[x.ctypes.data for x in nb])
    D = G if D is None else D
    Ds = D if Ds is None else Ds
    S = np.zeros((H, W, Ds), np.uint16)
    lo_a = None if lo is None else _c(lo, np.int32)
    rc = lib().or_cost_volume(_p(ref), arr, V, _p(_c(side, np.int8)), W, H, _p(_c(K, np.float64)),
                              _p(_c(R, np.float64)), _p(_c(t, np.float64)), _p(_c(n, np.float64)),
                              C.c_double(rho0), C.c_double(drho), G,
                              None if lo_a is None else _p(lo_a), D, Ds, int(cost), _p(S))
    if rc != 0:
        raise ValueError("or_cost_volume rc=%d" % rc)
    return S


def cost_band(ref, nbrs, side, K, R, t, n, rho0, drho, G, y0, y1, lo=None, D=None, Ds=None, cost=0):
    """Rows y0 .. y1 - 1 of the cost volume (warps of the rows they reach)."""
    ref = _c(ref, np.uint8)
    H, W = ref.shape
    V = len(nbrs)
    nb = [_c(x, np.uint8) for x in nbrs]
    arr = (C.c_void_p * V)(*[x.ctypes.data for x in nb])
    D = G if D is None else D
    Ds = D if Ds is None else Ds
    S = np.zeros((y1 - y0, W, Ds), np.uint16)
    lo_a = None if lo is None else _c(lo, np.int32)
    rc = lib().or_cost_band(_p(ref), arr, V, _p(_c(side, np.int8)), W, H, _p(_c(K, np.float64)),
                            _p(_c(R, np.float64)), _p(_c(t, np.float64)), _p(_c(n, np.float64)),
                            C.c_double(rho0), C.c_double(drho), G,
                            None if lo_a is None else _p(lo_a), D, Ds, int(cost), int(y0), int(y1), _p(S))
    if rc != 0:
        raise ValueError("or_cost_band rc=%d" % rc)
    return S


def cost_at(ref, nbrs, side, K, R, t, n, rho0, drho, xs, ys, gs, cost=0):
    ref = _c(ref, np.uint8)
    H, W = ref.shape
    V = len(nbrs)
    nb = [_c(x, np.uint8) for x in nbrs]
    arr = (C.c_void_p * V)(*[x.ctypes.data for x in nb])
    xs, ys, gs = (_c(a, np.int32) for a in (xs, ys, gs))
    out = np.zeros(xs.size, np.uint16)
    lib().or_cost_at(_p(ref), arr, V, _p(_c(side, np.int8)), W, H, _p(_c(K, np.float64)),
                     _p(_c(R, np.float64)), _p(_c(t, np.float64)), _p(_c(n, np.float64)),
                     C.c_double(rho0), C.c_double(drho), int(xs.size), _p(xs), _p(ys), _p(gs), int(cost),
                     _p(out))
    return out


def p2_table(p1, alpha=8.0, beta=10.0):
    lut = np.zeros(256, np.uint16)
    lib().or_p2_table(int(p1), C.c_double(alpha), C.c_double(beta), _p(lut))
    return lut


def sgm_aggregate(S, p1, p2=0, lut=None, lo=None, dI=None, img=None, paths=8, variant=0, dmax=8,
                  D=None, G=None):
    S = _c(S, np.uint16)
    H, W, Ds = S.shape
    D = Ds if D is None else D
    P = SgmParams(W, H, D, Ds, G or D, paths, variant, int(p1), int(p2), int(dmax))
    Sb = np.zeros_like(S)
    args = [_p(S), None if lo is None else _p(_c(lo, np.int32)),
            None if dI is None else _p(_c(dI, np.int8)),
            None if img is None else _p(_c(img, np.uint8)),
            None if lut is None else _p(_c(lut, np.uint16)), C.byref(P), _p(Sb)]
    rc = lib().or_sgm_aggregate(*args)
    if rc != 0:
        raise OverflowError("aggregated cost exceeds 16 bits")
    return Sb


def sgm_path(S, r, p1, p2=0, lut=None, lo=None, dI=None, img=None, variant=0, dmax=8, D=None):
    S = _c(S, np.uint16)
    H, W, Ds = S.shape
    D = Ds if D is None else D
    P = SgmParams(W, H, D, Ds, D, 8, variant, int(p1), int(p2), int(dmax))
    L = np.zeros((H, W, D), np.uint32)
    lib().or_sgm_path(_p(S), None if lo is None else _p(_c(lo, np.int32)),
                      None if dI is None else _p(_c(dI, np.int8)),
                      None if img is None else _p(_c(img, np.uint8)),
                      None if lut is None else _p(_c(lut, np.uint16)), C.byref(P), int(r), _p(L))
    return L


def path_dir(r):
    dx, dy = C.c_int(), C.c_int()
    lib().or_path_dir(int(r), C.byref(dx), C.byref(dy))
    return dx.value, dy.value


def parabola_vertex(xm, cm, x0, c0, xp, cp):
    return lib().or_parabola_vertex(xm, cm, x0, c0, xp, cp)


def wta_refine(Sbar, K, n, rho0, drho, lo=None, D=None):
    Sbar = _c(Sbar, np.uint16)
    H, W, Ds = Sbar.shape
    D = Ds if D is None else D
    depth = np.zeros((H, W), np.float32)
    g = np.zeros((H, W), np.int32)
    lib().or_wta_refine(_p(Sbar), None if lo is None else _p(_c(lo, np.int32)), W, H, D, Ds,
                        _p(_c(K, np.float64)), _p(_c(n, np.float64)), C.c_double(rho0),
                        C.c_double(drho), _p(depth), _p(g))
    return depth, g


def median5(d):
    d = _c(d, np.float32)
    H, W = d.shape
    out = np.zeros_like(d)
    lib().or_median5(_p(d), W, H, _p(out))
    return out


def normals(depth, img, K, radius=2, beta=10.0):
    depth = _c(depth, np.float32)
    H, W = depth.shape
    out = np.zeros((H, W, 3), np.float32)
    raw = np.zeros((H, W, 3), np.float32)
    lib().or_normals(_p(depth), _p(_c(img, np.uint8)), W, H, _p(_c(K, np.float64)), int(radius),
                     C.c_double(beta), _p(out), _p(raw))
    return out, raw


def normals_smooth(raw, img, radius=2, beta=10.0):
    """Eq. normal-smooth + Eq. normal on a given raw normal field (H, W, 3)."""
    raw = _c(raw, np.float64)
    H, W, _ = raw.shape
    out = np.zeros((H, W, 3), np.float32)
    lib().or_normals_smooth(_p(raw), _p(_c(img, np.uint8)), W, H, int(radius), C.c_double(beta), _p(out))
    return out


def confidence(normal, nPi=(0.0, 0.0, -1.0), rho_deg=60.0):
    normal = _c(normal, np.float32)
    H, W, _ = normal.shape
    out = np.zeros((H, W), np.float32)
    lib().or_confidence(_p(normal), W, H, _p(_c(nPi, np.float64)), C.c_double(rho_deg), _p(out))
    return out


def window(dc, W, H, K, n, rho0, drho, G, D):
    dc = _c(dc, np.float32)
    Hc, Wc = dc.shape
    lo = np.zeros((H, W), np.int32)
    lib().or_window(_p(dc), Wc, Hc, W, H, _p(_c(K, np.float64)), _p(_c(n, np.float64)),
                    C.c_double(rho0), C.c_double(drho), int(G), int(D), _p(lo))
    return lo


def dsn(dc, nc, W, H, K, drho, dmax=8, n=(0.0, 0.0, -1.0)):
    """Eq. sgm-smooth-sn index jumps; n is the sweep normal."""
    dc = _c(dc, np.float32)
    nc = _c(nc, np.float32)
    Hc, Wc = dc.shape
    out = np.zeros((8, H, W), np.int8)
    lib().or_dsn(_p(dc), _p(nc), Wc, Hc, W, H, _p(_c(K, np.float64)), _p(_c(n, np.float64)), C.c_double(drho),
                 int(dmax), _p(out))
    return out


def plane_bounds(K, W, H, n, d_min, d_max):
    """(delta_min, delta_max) of the bounding planes (Sec. 2.2.2)."""
    out = np.zeros(2, np.float64)
    rc = lib().or_plane_bounds(_p(_c(K, np.float64)), int(W), int(H), _p(_c(n, np.float64)), C.c_double(d_min),
                               C.c_double(d_max), _p(out))
    if rc != 0:
        raise ValueError("or_plane_bounds rc=%d" % rc)
    return float(out[0]), float(out[1])


def cross_ratio_planes(K, W, H, R, t, n, delta_min, delta_max, maxn=100000):
    """Alg. 2 plane distances, far to near, and the index of camera k."""
    R = _c(np.asarray(R, np.float64).reshape(-1, 9), np.float64)
    t = _c(np.asarray(t, np.float64).reshape(-1, 3), np.float64)
    out = np.zeros(maxn, np.float64)
    k = C.c_int(-1)
    m = lib().or_cross_ratio_planes(_p(_c(K, np.float64)), int(W), int(H), R.shape[0], _p(R), _p(t),
                                    _p(_c(n, np.float64)), C.c_double(delta_min), C.c_double(delta_max), int(maxn),
                                    _p(out), C.byref(k))
    if m < 0:
        raise ValueError("or_cross_ratio_planes rc=%d" % m)
    return out[:m].copy(), k.value


def dog_weights():
    w = np.zeros(7, np.int32)
    lib().or_dog_weights(_p(w))
    return w


def speckle(mask, val, minsize):
    m = _c(mask, np.uint8).copy()
    H, W = m.shape
    lib().or_speckle(_p(m), W, H, int(val), int(minsize))
    return m


def dog_mask(img):
    """Alg. 3 mask of a reference image: 1 where the texture suffices."""
    img = _c(img, np.uint8)
    H, W = img.shape
    m = np.zeros((H, W), np.uint8)
    lib().or_dog_mask(_p(img), W, H, _p(m))
    return m


def apply_mask(mask, depth, normal, conf):
    d, n, c = (_c(a, np.float32).copy() for a in (depth, normal, conf))
    H, W = d.shape
    lib().or_apply_mask(_p(_c(mask, np.uint8)), W, H, _p(d), _p(n), _p(c))
    return d, n, c


def geo_hits(dref, K, dks, R, t, eta_r=10.0):
    """Alg. 4 hit counts of a reference depth map against neighbour maps
    (R, t: reference -> neighbour)."""
    dref = _c(dref, np.float32)
    H, W = dref.shape
    dk = [_c(x, np.float32) for x in dks]
    arr = (C.c_void_p * max(1, len(dk)))(*[x.ctypes.data for x in dk])
    hits = np.zeros((H, W), np.uint8)
    rc = lib().or_geo_hits(_p(dref), W, H, _p(_c(K, np.float64)), len(dk), arr,
                           _p(_c(np.asarray(R, np.float64).reshape(-1, 9), np.float64)),
                           _p(_c(np.asarray(t, np.float64).reshape(-1, 3), np.float64)), C.c_double(eta_r), _p(hits))
    if rc != 0:
        raise ValueError("or_geo_hits rc=%d" % rc)
    return hits


def make_config(levels=1, D=(64,), paths=8, variant=0, p1=10, p2=120, adaptive_p2=0, alpha=8.0,
                beta=10.0, median5=1, normal_radius=2, normal_beta=10.0, rho_deg=60.0, dmax=8, cost=0):
    Dl = (C.c_int32 * 8)(*(list(D) + [0] * (8 - len(D))))
    return Config(levels, Dl, paths, variant, p1, p2, adaptive_p2, alpha, beta, median5,
                  normal_radius, normal_beta, rho_deg, dmax, cost)


def estimate(scene, cfg):
    """Full hierarchical estimate of a synth.Scene with an oracle Config."""
    H, W = scene.ref.shape
    nb = [_c(x, np.uint8) for x in scene.nbrs]
    arr = (C.c_void_p * len(nb))(*[x.ctypes.data for x in nb])
    depth = np.zeros((H, W), np.float32)
    normal = np.zeros((H, W, 3), np.float32)
    conf = np.zeros((H, W), np.float32)
    ref = _c(scene.ref, np.uint8)
    rc = lib().or_estimate(C.byref(cfg), _p(ref), arr, len(nb), _p(_c(scene.side, np.int8)), W, H,
                           _p(_c(scene.K, np.float64)), _p(_c(scene.R, np.float64)),
                           _p(_c(scene.t, np.float64)), _p(_c(scene.plane_n, np.float64)),
                           C.c_double(scene.rho_far), C.c_double(scene.drho), int(scene.G0),
                           _p(depth), _p(normal), _p(conf))
    if rc != 0:
        raise ValueError("or_estimate rc=%d" % rc)
    return depth, normal, conf


def threads(n=0):
    """Thread count of the oracle's parallel loops (timing only); n >= 1 sets
    it.  Returns the count in force."""
    return int(lib().or_threads(int(n)))
