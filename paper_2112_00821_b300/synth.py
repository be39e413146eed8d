"""Seeded synthetic multi-view scenes for the plane-sweep / SGM hot path.

This module is the input generator shared by the tests, the benchmark and the
smoke check. It holds none of the method's arithmetic: it ray-casts textured
planar quads from pinhole cameras on the CPU (numpy), and returns the images,
the camera calibration, the relative poses of the neighbour views, the plane
sweep parameters and the ground-truth depth / normal maps of the reference.

Conventions (FaSS-MVS Sec. 2.1 and Eq. homography):
  * every pose is given relative to the reference camera, whose frame is the
    world frame; a neighbour k maps a reference-frame point X to its own frame
    as X_k = R_k X + t_k;
  * images are row-major uint8 (H, W); pixel centres sit at integer (x, y);
  * K = [[f, 0, cx], [0, f, cy], [0, 0, 1]] with cx = (W-1)/2, cy = (H-1)/2;
  * depth is the z coordinate in the reference frame; normals are unit vectors
    in the reference frame that face the camera (n . X < 0).
The sweep planes are fronto-parallel (n = (0, 0, -1)) and uniform in inverse
depth between the near and far bounds (Sec. 2.2.3: the cross-ratio rule leads
to inverse-depth sampling): 1/delta_g = rho_far + g * drho, g = 0 farthest.

Textures are 3-octave value noise with lattice values drawn from
numpy.random.Generator(PCG64(seed)) and smoothstep interpolation; the base
lattice cell projects to at least 4 px.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Quad", "Frame", "Scene", "render_view", "make_scene", "make_frame",
    "WORKLOADS", "workload", "box_quads", "trajectory_frames", "BATCH_SIZES", "batch_frames",
    "render_view_torch", "city_sweep",
]


# --------------------------------------------------------------------------
# geometry helpers (scene construction only)
# --------------------------------------------------------------------------

def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def _look_at(center, target):
    """Rotation whose rows are the camera axes (x right, y down, z forward) in
    the reference frame, for a camera at `center` looking at `target`; the
    reference camera itself is the identity."""
    z = _unit(np.asarray(target, dtype=np.float64) - np.asarray(center, dtype=np.float64))
    x = _unit(np.cross(np.array([0.0, 1.0, 0.0]), z))
    y = np.cross(z, x)
    return np.stack([x, y, z])


def _pitch_up(pitch_deg):
    """World 'up' in the frame of a camera pitched down by pitch_deg."""
    a = np.deg2rad(pitch_deg)
    return np.array([0.0, -math.cos(a), -math.sin(a)])


@dataclass
class Quad:
    """A textured planar patch origin + s*au + t*av, s in su, t in tv
    (unbounded when a bound is infinite). au, av are orthonormal."""
    origin: np.ndarray
    au: np.ndarray
    av: np.ndarray
    su: tuple = (-math.inf, math.inf)
    tv: tuple = (-math.inf, math.inf)
    cell: float = 1.0
    tex_seed: int = 0
    contrast: float = 1.6

    @property
    def normal(self):
        return _unit(np.cross(self.au, self.av))


def _quad(origin, au, av, su, tv, cell, tex_seed, contrast=1.6):
    au = _unit(au)
    av = np.asarray(av, dtype=np.float64)
    av = _unit(av - np.dot(av, au) * au)
    return Quad(np.asarray(origin, dtype=np.float64), au, av, tuple(su), tuple(tv),
                float(cell), int(tex_seed), float(contrast))


def box_quads(center_xz, half_w, half_d, height, ground_y_at, up, cell, seed0):
    """Five quads (roof and four walls) of an axis-aligned box standing on the
    ground; `ground_y_at(x, z)` returns the ground point below (x, z) and `up`
    is the unit up vector of the world in the reference frame."""
    up = _unit(up)
    # horizontal axes orthogonal to up
    ex = _unit(np.array([1.0, 0.0, 0.0]) - np.dot([1.0, 0.0, 0.0], up) * up)
    ez = _unit(np.cross(ex, up))
    base = ground_y_at(*center_xz)
    top = base + height * up
    quads = [_quad(top, ex, ez, (-half_w, half_w), (-half_d, half_d), cell, seed0)]
    for k, (ax, hw, off) in enumerate(((ex, half_w, ez * half_d), (ex, half_w, -ez * half_d),
                                       (ez, half_d, ex * half_w), (ez, half_d, -ex * half_w))):
        o = base + off + 0.5 * height * up
        quads.append(_quad(o, ax, up, (-hw, hw), (-0.5 * height, 0.5 * height), cell, seed0 + 1 + k))
    return quads


# --------------------------------------------------------------------------
# value-noise texture
# --------------------------------------------------------------------------

class _Noise:
    def __init__(self, seed):
        g = np.random.Generator(np.random.PCG64(seed))
        self.perm = g.permutation(256).astype(np.int64)
        self.vals = g.integers(0, 256, size=256, dtype=np.int64).astype(np.float64)

    def lattice(self, i, j):
        return self.vals[self.perm[(self.perm[i & 255] + j) & 255]]

    def octave(self, s, t):
        i0 = np.floor(s).astype(np.int64)
        j0 = np.floor(t).astype(np.int64)
        fs = s - i0
        ft = t - j0
        ws = fs * fs * (3.0 - 2.0 * fs)
        wt = ft * ft * (3.0 - 2.0 * ft)
        a = self.lattice(i0, j0)
        b = self.lattice(i0 + 1, j0)
        c = self.lattice(i0, j0 + 1)
        d = self.lattice(i0 + 1, j0 + 1)
        top = a + ws * (b - a)
        bot = c + ws * (d - c)
        return top + wt * (bot - top)

    def __call__(self, s, t):
        v = 0.60 * self.octave(s, t) + 0.25 * self.octave(2.0 * s + 17.3, 2.0 * t + 5.1) \
            + 0.15 * self.octave(4.0 * s + 3.7, 4.0 * t + 29.9)
        return v


# --------------------------------------------------------------------------
# rendering
# --------------------------------------------------------------------------

def _bbox(q, K, R, t, W, H):
    """Pixel bounding box (y0, y1, x0, x1) of a bounded quad seen by a camera,
    the whole image when the quad is unbounded or crosses the camera plane."""
    if not (math.isfinite(q.su[0]) and math.isfinite(q.tv[0])):
        return 0, H, 0, W
    cs = [q.origin + a * q.au + b * q.av for a in q.su for b in q.tv]
    Xc = np.stack(cs) @ R.T + t
    if np.any(Xc[:, 2] <= 1e-6):
        return 0, H, 0, W
    u = K[0, 0] * Xc[:, 0] / Xc[:, 2] + K[0, 2]
    v = K[1, 1] * Xc[:, 1] / Xc[:, 2] + K[1, 2]
    x0 = max(0, int(math.floor(u.min())) - 1)
    x1 = min(W, int(math.ceil(u.max())) + 2)
    y0 = max(0, int(math.floor(v.min())) - 1)
    y1 = min(H, int(math.ceil(v.max())) + 2)
    return y0, y1, x0, x1


def render_view(quads, K, R, t, W, H, noise_sigma=0.0, noise_seed=None, return_gt=False):
    """Ray-cast pixel centres of a camera X_cam = R X_ref + t.

    Returns the uint8 image, and with return_gt the depth (z in the camera
    frame), the unit normal in the camera frame (facing the camera) and the
    index of the quad hit per pixel."""
    K = np.asarray(K, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    C = -R.T @ t
    xs, ys = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    Kinv = np.linalg.inv(K)
    dc = np.stack([xs, ys, np.ones_like(xs)], axis=-1) @ Kinv.T      # camera-frame ray, z = 1
    dref = dc @ R                                                    # = (R^T dc) per pixel
    best = np.full((H, W), np.inf)
    who = np.full((H, W), -1, dtype=np.int64)
    for qi, q in enumerate(quads):
        y0, y1, x0, x1 = _bbox(q, K, R, t, W, H)
        if y0 >= y1 or x0 >= x1:
            continue
        n = q.normal
        dsub = dref[y0:y1, x0:x1]
        denom = dsub @ n
        num = float(np.dot(n, q.origin - C))
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = num / denom
        bsub = best[y0:y1, x0:x1]
        ok = np.isfinite(lam) & (lam > 1e-9) & (lam < bsub)
        if not np.any(ok):
            continue
        if math.isfinite(q.su[0]) or math.isfinite(q.tv[0]):
            P = C + lam[..., None] * dsub
            rel = P - q.origin
            s = rel @ q.au
            tt = rel @ q.av
            ok &= (s >= q.su[0]) & (s <= q.su[1]) & (tt >= q.tv[0]) & (tt <= q.tv[1])
        best[y0:y1, x0:x1] = np.where(ok, lam, bsub)
        who[y0:y1, x0:x1] = np.where(ok, qi, who[y0:y1, x0:x1])
    if np.any(who < 0):
        raise ValueError("scene has rays that hit nothing; add a backdrop quad")
    img = np.zeros((H, W), dtype=np.float64)
    for qi, q in enumerate(quads):
        m = who == qi
        if not np.any(m):
            continue
        P = C + best[m][:, None] * dref[m]
        rel = P - q.origin
        s = (rel @ q.au) / q.cell
        tt = (rel @ q.av) / q.cell
        v = _Noise(q.tex_seed)(s, tt)
        img[m] = 128.0 + q.contrast * (v - 128.0)
    if noise_sigma > 0:
        g = np.random.Generator(np.random.PCG64(noise_seed))
        img = img + g.normal(0.0, noise_sigma, size=img.shape)
    img8 = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    if not return_gt:
        return img8
    depth = best.astype(np.float64)                     # ray param == z_cam since dc_z == 1
    normals = np.zeros((H, W, 3), dtype=np.float64)
    for qi, q in enumerate(quads):
        m = who == qi
        if not np.any(m):
            continue
        nc = R @ q.normal
        P = depth[m][:, None] * dc[m]
        flip = (P @ nc) > 0
        nn = np.where(flip[:, None], -nc[None, :], nc[None, :])
        normals[m] = nn
    return img8, depth, normals, who


def render_view_torch(quads, K, R, t, W, H, device="cuda"):
    """render_view (image only, no noise) with torch tensors on `device`, for
    long synthetic streams; the same ray cast and texture in FP64, returned
    as a uint8 numpy array."""
    import torch
    dt = torch.float64
    Kn = np.asarray(K, dtype=np.float64)
    Rn = np.asarray(R, dtype=np.float64)
    tn = np.asarray(t, dtype=np.float64)
    C = torch.as_tensor(-Rn.T @ tn, dtype=dt, device=device)
    ys, xs = torch.meshgrid(torch.arange(H, dtype=dt, device=device), torch.arange(W, dtype=dt, device=device),
                            indexing="ij")
    Kinv = torch.as_tensor(np.linalg.inv(Kn), dtype=dt, device=device)
    dc = torch.stack([xs, ys, torch.ones_like(xs)], dim=-1) @ Kinv.T
    dref = dc @ torch.as_tensor(Rn, dtype=dt, device=device)
    best = torch.full((H, W), math.inf, dtype=dt, device=device)
    who = torch.full((H, W), -1, dtype=torch.int64, device=device)
    for qi, q in enumerate(quads):
        y0, y1, x0, x1 = _bbox(q, Kn, Rn, tn, W, H)
        if y0 >= y1 or x0 >= x1:
            continue
        n = torch.as_tensor(q.normal, dtype=dt, device=device)
        dsub = dref[y0:y1, x0:x1]
        denom = dsub @ n
        num = float(np.dot(q.normal, q.origin - (-Rn.T @ tn)))
        lam = num / denom
        bsub = best[y0:y1, x0:x1]
        ok = torch.isfinite(lam) & (lam > 1e-9) & (lam < bsub)
        if math.isfinite(q.su[0]) or math.isfinite(q.tv[0]):
            rel = C + lam[..., None] * dsub - torch.as_tensor(q.origin, dtype=dt, device=device)
            s = rel @ torch.as_tensor(q.au, dtype=dt, device=device)
            tt = rel @ torch.as_tensor(q.av, dtype=dt, device=device)
            ok &= (s >= q.su[0]) & (s <= q.su[1]) & (tt >= q.tv[0]) & (tt <= q.tv[1])
        best[y0:y1, x0:x1] = torch.where(ok, lam, bsub)
        who[y0:y1, x0:x1] = torch.where(ok, torch.full_like(who[y0:y1, x0:x1], qi), who[y0:y1, x0:x1])
    if bool((who < 0).any()):
        raise ValueError("scene has rays that hit nothing; add a backdrop quad")
    img = torch.zeros((H, W), dtype=dt, device=device)
    for qi, q in enumerate(quads):
        m = who == qi
        if not bool(m.any()):
            continue
        P = C + best[m][:, None] * dref[m]
        rel = P - torch.as_tensor(q.origin, dtype=dt, device=device)
        s = (rel @ torch.as_tensor(q.au, dtype=dt, device=device)) / q.cell
        tt = (rel @ torch.as_tensor(q.av, dtype=dt, device=device)) / q.cell
        nz = _Noise(q.tex_seed)
        perm = torch.as_tensor(nz.perm, device=device)
        vals = torch.as_tensor(nz.vals, dtype=dt, device=device)

        def octave(a, b):
            i0 = torch.floor(a).to(torch.int64)
            j0 = torch.floor(b).to(torch.int64)
            fa = a - i0
            fb = b - j0
            wa = fa * fa * (3.0 - 2.0 * fa)
            wb = fb * fb * (3.0 - 2.0 * fb)

            def lat(i, j):
                return vals[perm[(perm[i & 255] + j) & 255]]
            top = lat(i0, j0) + wa * (lat(i0 + 1, j0) - lat(i0, j0))
            bot = lat(i0, j0 + 1) + wa * (lat(i0 + 1, j0 + 1) - lat(i0, j0 + 1))
            return top + wb * (bot - top)
        v = 0.60 * octave(s, tt) + 0.25 * octave(2.0 * s + 17.3, 2.0 * tt + 5.1) \
            + 0.15 * octave(4.0 * s + 3.7, 4.0 * tt + 29.9)
        img[m] = 128.0 + q.contrast * (v - 128.0)
    return torch.clamp(torch.round(img), 0, 255).to(torch.uint8).cpu().numpy()


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

@dataclass
class Scene:
    """One reference frame with its neighbour bundle and sweep parameters."""
    W: int
    H: int
    K: np.ndarray                 # 3x3 float64
    ref: np.ndarray               # (H, W) uint8
    nbrs: list                    # list of (H, W) uint8
    R: np.ndarray                 # (V, 3, 3) float64, ref -> neighbour
    t: np.ndarray                 # (V, 3) float64
    side: np.ndarray              # (V,) int8, -1 left (k < ref), +1 right
    plane_n: np.ndarray           # (3,) sweep plane normal
    rho_far: float                # inverse depth of plane 0 (farthest)
    drho: float                   # inverse-depth step between finest planes
    G0: int                       # planes in the finest list
    depth_gt: np.ndarray = None   # (H, W) float64
    normal_gt: np.ndarray = None  # (H, W, 3) float64
    meta: dict = field(default_factory=dict)

    @property
    def n_views(self):
        return len(self.nbrs)

    def plane_depth(self, g):
        return 1.0 / (self.rho_far + g * self.drho)


def _K(W, H, f):
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


def _sweep(d_near, d_far, G0):
    rho_far = 1.0 / d_far
    rho_near = 1.0 / d_near
    return rho_far, (rho_near - rho_far) / (G0 - 1)


def make_scene(quads, W, H, f, centers, targets, sides, G0, d_near, d_far, seed,
               noise_sigma=0.0, jitter_deg=0.3, want_gt=True, meta=None):
    """Render the reference (identity pose) and the neighbours whose centres
    (reference frame) look at `targets`; small seeded roll/pitch jitter keeps
    the relative rotations generic."""
    g = np.random.Generator(np.random.PCG64(seed + 7919))
    K = _K(W, H, f)
    I3 = np.eye(3)
    if want_gt:
        ref, depth, normal, _ = render_view(quads, K, I3, np.zeros(3), W, H, noise_sigma,
                                            seed * 131 + 1, return_gt=True)
    else:
        ref = render_view(quads, K, I3, np.zeros(3), W, H, noise_sigma, seed * 131 + 1)
        depth = normal = None
    nbrs, Rs, ts = [], [], []
    for k, (c, tg) in enumerate(zip(centers, targets)):
        Rk = _look_at(c, tg)
        j = np.deg2rad(jitter_deg)
        Rk = _rot_z(g.uniform(-j, j)) @ _rot_x(g.uniform(-j, j)) @ Rk
        tk = -Rk @ np.asarray(c, dtype=np.float64)
        nbrs.append(render_view(quads, K, Rk, tk, W, H, noise_sigma, seed * 131 + 2 + k))
        Rs.append(Rk)
        ts.append(tk)
    rho_far, drho = _sweep(d_near, d_far, G0)
    meta = dict(meta or {})
    meta["quads"] = quads
    return Scene(W, H, K, ref, nbrs, np.stack(Rs), np.stack(ts), np.asarray(sides, dtype=np.int8),
                 np.array([0.0, 0.0, -1.0]), rho_far, drho, G0, depth, normal, meta)


def visibility_mask(sc, rel_tol=1e-2):
    """Ground-truth visibility of the reference pixels of a rendered scene:
    True where the surface point seen by the reference pixel is also the one
    seen by every neighbour at its projection (inside the image, in front of
    the camera, its depth there within rel_tol of the neighbour's rendered
    depth).  Scene geometry only: occluded and out-of-view pixels are False."""
    quads = sc.meta["quads"]
    H, W = sc.H, sc.W
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    rays = np.stack([xs, ys, np.ones_like(xs)], -1) @ np.linalg.inv(sc.K).T
    X = rays * sc.depth_gt[..., None]
    vis = np.ones((H, W), bool)
    for k in range(sc.n_views):
        _, dk, _, _ = render_view(quads, sc.K, sc.R[k], sc.t[k], W, H, return_gt=True)
        Xk = X @ sc.R[k].T + sc.t[k]
        z = Xk[..., 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = sc.K[0, 0] * Xk[..., 0] / z + sc.K[0, 2]
            v = sc.K[1, 1] * Xk[..., 1] / z + sc.K[1, 2]
        ok = (z > 0) & (u >= 0) & (u <= W - 1) & (v >= 0) & (v <= H - 1)
        ui = np.clip(np.rint(np.where(ok, u, 0)), 0, W - 1).astype(int)
        vi = np.clip(np.rint(np.where(ok, v, 0)), 0, H - 1).astype(int)
        ok &= np.abs(dk[vi, ui] - z) <= rel_tol * np.abs(z)
        vis &= ok
    return vis


# --- recipes --------------------------------------------------------------

def _tiny_quads(seed, f, zc=20.0):
    """Ground seen from a camera pitched down 30 degrees (the optical axis
    meets it at depth zc), two slanted facades standing on it, and a far
    backdrop (reference frame: x right, y down, z forward)."""
    g = np.random.Generator(np.random.PCG64(seed))
    cell = 8.0 * zc / f
    up = _pitch_up(30.0)
    ex = np.array([1.0, 0.0, 0.0])
    fwd = np.cross(up, ex)
    ground_o = np.array([0.0, 0.0, zc])
    quads = [_quad(ground_o, ex, fwd, (-1e9, 1e9), (-1e9, 1e9), cell, int(g.integers(1 << 30)))]
    for s in (-1.0, 1.0):
        yaw = np.deg2rad(s * g.uniform(20.0, 35.0))
        a = math.cos(yaw) * ex + math.sin(yaw) * fwd
        hgt = g.uniform(3.0, 5.0)
        o = ground_o + s * g.uniform(1.5, 3.0) * ex - g.uniform(0.0, 3.0) * fwd + 0.5 * hgt * up
        quads.append(_quad(o, a, up, (-2.0, 2.0), (-0.5 * hgt, 0.5 * hgt), cell * 0.8,
                           int(g.integers(1 << 30))))
    quads.append(_quad(np.array([0.0, 0.0, 2.0 * zc]), ex, [0, 1, 0], (-1e9, 1e9), (-1e9, 1e9),
                       cell * 2.0, int(g.integers(1 << 30))))
    return quads


def _random_plane_quads(seed, f, n_planes, zmin, zmax, W, H):
    g = np.random.Generator(np.random.PCG64(seed))
    zc = 0.5 * (zmin + zmax)
    cell = 7.0 * zc / f
    quads = []
    # ground (slanted) and backdrop so every ray hits something
    up = _pitch_up(35.0)
    quads.append(_quad(np.array([0.0, 0.0, 0.9 * zmax]), [1, 0, 0], np.cross(up, [1, 0, 0]),
                       (-1e9, 1e9), (-1e9, 1e9), cell, int(g.integers(1 << 30))))
    quads.append(_quad(np.array([0.0, 0.0, zmax]), [1, 0, 0], [0, 1, 0], (-1e9, 1e9), (-1e9, 1e9),
                       cell * 2.5, int(g.integers(1 << 30))))
    fovx = (W / 2.0) / f
    fovy = (H / 2.0) / f
    for _ in range(n_planes):
        z = g.uniform(zmin * 1.15, zmax * 0.8)
        cx = g.uniform(-0.8, 0.8) * fovx * z
        cy = g.uniform(-0.8, 0.8) * fovy * z
        # random orientation within 55 degrees of facing the camera
        tilt = np.deg2rad(g.uniform(0.0, 55.0))
        az = g.uniform(0.0, 2.0 * np.pi)
        n = np.array([math.sin(tilt) * math.cos(az), math.sin(tilt) * math.sin(az), -math.cos(tilt)])
        a = _unit(np.cross(n, [0.0, 1.0, 0.0]) if abs(n[1]) < 0.9 else np.cross(n, [1.0, 0.0, 0.0]))
        b = _unit(np.cross(n, a))
        size = g.uniform(0.12, 0.3) * fovx * z
        quads.append(_quad([cx, cy, z], a, b, (-size, size), (-0.7 * size, 0.7 * size),
                           cell * g.uniform(0.6, 1.0), int(g.integers(1 << 30))))
    return quads


def _oblique_city_quads(seed, f, tilt_deg=45.0, height=60.0, n_boxes=14, zmax=300.0):
    """Ground plane seen at `tilt_deg` from a camera `height` metres above it,
    with box buildings and a far backdrop (reference frame)."""
    g = np.random.Generator(np.random.PCG64(seed))
    up = _pitch_up(tilt_deg)
    # ground point below the camera: -height * up
    ground_o = -height * up
    fwd = np.cross(up, np.array([1.0, 0.0, 0.0]))   # horizontal, away from the camera
    cell_ground = 8.0 * (height * 1.4) / f
    quads = [_quad(ground_o, [1, 0, 0], fwd, (-1e9, 1e9), (-1e9, 1e9), cell_ground, int(g.integers(1 << 30)))]

    def ground_at(x, d):
        return ground_o + x * np.array([1.0, 0.0, 0.0]) + d * fwd

    for _ in range(n_boxes):
        d = g.uniform(height * 0.7, height * 1.9)
        x = g.uniform(-0.45, 0.45) * math.hypot(d, height)
        hw = g.uniform(4.0, 10.0)
        hd = g.uniform(4.0, 10.0)
        hgt = g.uniform(6.0, 0.45 * height)
        quads += box_quads((x, d), hw, hd, hgt, ground_at, up, cell_ground * 0.6, int(g.integers(1 << 30)))
    quads.append(_quad(np.array([0.0, 0.0, zmax * 0.95]), [1, 0, 0], [0, 1, 0], (-1e9, 1e9), (-1e9, 1e9),
                       cell_ground * 3.0, int(g.integers(1 << 30))))
    return quads


def _bundle(n_left, n_right, base, target_z, seed, yjit=0.15):
    """Camera centres along x (flight direction) with a slight seeded vertical
    offset, converging on (0, 0, target_z)."""
    g = np.random.Generator(np.random.PCG64(seed + 104729))
    centers, targets, sides = [], [], []
    offs = [-(n_left - i) for i in range(n_left)] + [i + 1 for i in range(n_right)]
    for o in offs:
        c = np.array([o * base, g.uniform(-yjit, yjit) * base, g.uniform(-0.1, 0.1) * base])
        centers.append(c)
        targets.append(np.array([0.0, 0.0, target_z]))
        sides.append(-1 if o < 0 else 1)
    return centers, targets, sides


WORKLOADS = {
    # name: description (sizes in the name are the reference resolution)
    "tiny_160x120_g64": "160x120, 1L+1R views, 3 textured planes + backdrop, 64 planes, 1 level, "
                        "P1=10 P2=120 fixed, plane-wise SGM, 8 paths",
    "vga_640x480_g512_l3": "640x480, 2L+2R views, 8-20 random planes, noise 2 DN, 3 levels, "
                           "G0=512 D=128, surface-normal SGM, adaptive P2",
    "fhd_1920x1080_g256_l4": "1920x1080, 45 deg oblique city, 2L+3R views, depth 20-300 m, "
                             "4 levels, G0=256 D=256, path-gradient SGM, 8 paths",
    "planes_1600x1200_g512_l3": "1600x1200, 8-20 random planes, noise 2 DN, 2L+2R views, 3 levels, "
                                "G0=512 D=128 (128 at the top), SGM variant / paths as run",
}


def make_frame(kind, seed, W=None, H=None, G0=None, n_left=None, n_right=None, want_gt=True, base_frac=None):
    """Build one reference frame of the given scene kind (base_frac: the
    camera spacing as a fraction of the mean scene depth, "planes" only)."""
    if kind == "tiny":
        W = W or 160
        H = H or 120
        f = 150.0 * W / 160.0
        zc = 20.0
        quads = _tiny_quads(seed, f, zc)
        base = 0.035 * zc
        c, tg, s = _bundle(n_left or 1, n_right or 1, base, zc, seed)
        sc = make_scene(quads, W, H, f, c, tg, s, G0 or 64, 1.0, 2.0, seed, want_gt=True)
        # sweep range from the rendered GT: [0.9 d_min, 1.1 d_max]
        dmin = float(sc.depth_gt.min())
        dmax = float(sc.depth_gt.max())
        sc.rho_far, sc.drho = _sweep(0.9 * dmin, 1.1 * dmax, sc.G0)
        return sc
    if kind == "planes":
        W = W or 640
        H = H or 480
        f = 0.9375 * W
        g = np.random.Generator(np.random.PCG64(seed + 11))
        n_planes = int(g.integers(8, 21))
        zmin, zmax = 6.0, 30.0
        quads = _random_plane_quads(seed, f, n_planes, zmin, zmax, W, H)
        base = (0.03 if base_frac is None else base_frac) * 0.5 * (zmin + zmax)
        c, tg, s = _bundle(n_left or 2, n_right or 2, base, 0.5 * (zmin + zmax), seed)
        sc = make_scene(quads, W, H, f, c, tg, s, G0 or 512, 0.9 * zmin, 1.05 * zmax, seed,
                        noise_sigma=2.0, want_gt=want_gt, meta={"n_planes": n_planes})
        return sc
    if kind == "city":
        W = W or 1920
        H = H or 1080
        f = 0.9375 * W
        height = 60.0
        quads = _oblique_city_quads(seed, f, 45.0, height, zmax=300.0)
        base = 0.03 * height * 1.5
        c, tg, s = _bundle(n_left or 2, n_right or 3, base, height * 1.5, seed)
        sc = make_scene(quads, W, H, f, c, tg, s, G0 or 256, 20.0, 300.0, seed,
                        want_gt=want_gt)
        return sc
    raise ValueError(kind)


def workload(name, seed=0, want_gt=True):
    """Named workloads (see WORKLOADS): returns (scene, estimation settings)."""
    if name == "tiny_160x120_g64":
        sc = make_frame("tiny", seed)
        cfg = dict(levels=1, D=[64], paths=8, variant=0, p1=10, p2=120, adaptive_p2=0)
        return sc, cfg
    if name == "vga_640x480_g512_l3":
        sc = make_frame("planes", seed, want_gt=want_gt)
        cfg = dict(levels=3, D=[128, 128, 128], paths=8, variant=1, p1=24, p2=0, adaptive_p2=1)
        return sc, cfg
    if name == "fhd_1920x1080_g256_l4":
        sc = make_frame("city", seed, want_gt=want_gt)
        cfg = dict(levels=4, D=[256, 256, 256, 256], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
        return sc, cfg
    if name == "planes_1600x1200_g512_l3":
        sc = make_frame("planes", seed, W=1600, H=1200, G0=512, n_left=2, n_right=2, want_gt=want_gt)
        cfg = dict(levels=3, D=[128, 128, 128], paths=8, variant=2, p1=24, p2=0, adaptive_p2=1)
        return sc, cfg
    raise KeyError(name)


BATCH_SIZES = ((640, 480), (1280, 720), (1920, 1080), (2720, 1530))


def batch_frames(seed=0, n=16):
    """The mixed batch: n reference frames whose sizes are drawn from
    BATCH_SIZES, plane counts from 64..256 (multiples of 32) and neighbour
    counts from 3..6, all of the 45 deg oblique city (depth 20-300 m).

    Frames of one size share the images of one rendered bundle (3 left + 3
    right views): a frame with n_nb neighbours takes the n_nb // 2 nearest left
    and the rest nearest right views of it, and its own plane list.  This keeps
    the rendering at one bundle per size; the estimates of two such frames
    differ through their views and planes."""
    g = np.random.Generator(np.random.PCG64(seed + 271))
    picks = [(int(g.integers(0, len(BATCH_SIZES))), int(g.integers(2, 9)) * 32, int(g.integers(3, 7)))
             for _ in range(n)]
    bundles = {}
    out = []
    for si, G0, nn in picks:
        if si not in bundles:
            W, H = BATCH_SIZES[si]
            bundles[si] = make_frame("city", 7 * seed + si, W=W, H=H, G0=256, n_left=3, n_right=3,
                                     want_gt=False)
        b = bundles[si]
        nl = nn // 2
        nr = nn - nl
        idx = list(range(3 - nl, 3)) + list(range(3, 3 + nr))
        rho_far, drho = _sweep(20.0, 300.0, G0)
        out.append(Scene(b.W, b.H, b.K, b.ref, [b.nbrs[i] for i in idx], b.R[idx].copy(), b.t[idx].copy(),
                         b.side[idx].copy(), b.plane_n.copy(), rho_far, drho, G0,
                         meta={"size_class": si, "bundle_views": idx}))
    return out


def city_sweep(G0):
    """(rho_far, drho) of G0 fronto planes uniform in inverse depth over the
    oblique city's 20-300 m."""
    return _sweep(20.0, 300.0, G0)


def trajectory_frames(n_frames, W, H, seed, speed=0.6, every=5, n_nb=(4, 6), G0=(128, 256), device=None):
    """A simulated 30 fps UAV pass over the oblique city: camera centres move
    along x by `speed` metres per frame. Returns the list of keyframe requests
    (reference index, neighbour indices, plane count) and a render callback
    rendering frame i (uint8) in the frame of frame 0's camera (with torch on
    `device` when given)."""
    f = 0.9375 * W
    height = 60.0
    quads = _oblique_city_quads(seed, f, 45.0, height, zmax=300.0)
    K = _K(W, H, f)
    g = np.random.Generator(np.random.PCG64(seed + 3))

    def pose(i):
        c = np.array([i * speed, 0.05 * math.sin(0.1 * i), 0.0])
        R = _rot_z(np.deg2rad(0.2 * math.sin(0.07 * i))) @ np.eye(3)
        return R, -R @ c

    def render(i):
        R, t = pose(i)
        if device is not None:
            return render_view_torch(quads, K, R, t, W, H, device)
        return render_view(quads, K, R, t, W, H)

    reqs = []
    for r in range(0, n_frames, every):
        nn = int(g.integers(n_nb[0], n_nb[1] + 1))
        nl = nn // 2
        nr = nn - nl
        lo = max(0, r - nl)
        hi = min(n_frames - 1, r + nr)
        idx = [i for i in range(lo, hi + 1) if i != r]
        reqs.append((r, idx, int(g.choice(np.array(G0)))))
    return K, pose, render, reqs
