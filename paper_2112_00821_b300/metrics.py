"""Error measures of Sec. 3.2 for depth and normal maps (host side, numpy).

Evaluation helpers, not part of the estimate: L1-abs and L1-rel (Eq. l1abs,
l1rel) over the pixels V where both maps are valid; the accuracy and
completeness scores Acc_theta, Cpl_theta (Eq. acc, cpl), which count the
pixels of V whose ratio max(d_est/d_gt, d_gt/d_est) is below theta and divide
by the valid estimates E or the valid ground truth G respectively; their
harmonic mean F_theta (Eq. fscore); and the mean angular error of normals
(AAE, stated in the paper's source but not used in its tables).  A depth is
valid when it is finite and > 0; a normal when its norm is > 0.
"""
from __future__ import annotations

import numpy as np


def _valid(d):
    d = np.asarray(d, np.float64)
    return np.isfinite(d) & (d > 0)


def _both(est, gt):
    est = np.asarray(est, np.float64)
    gt = np.asarray(gt, np.float64)
    if est.shape != gt.shape:
        raise ValueError("shape mismatch")
    e, g = _valid(est), _valid(gt)
    return est, gt, e, g, e & g


def l1_abs(est, gt):
    est, gt, _, _, v = _both(est, gt)
    return float(np.abs(est[v] - gt[v]).mean()) if v.any() else float("nan")


def l1_rel(est, gt):
    est, gt, _, _, v = _both(est, gt)
    return float((np.abs(est[v] - gt[v]) / gt[v]).mean()) if v.any() else float("nan")


def _hits(est, gt, v, theta):
    r = np.maximum(est[v] / gt[v], gt[v] / est[v])
    return int(np.count_nonzero(r < theta))


def acc(est, gt, theta):
    est, gt, e, _, v = _both(est, gt)
    n = int(np.count_nonzero(e))
    return _hits(est, gt, v, theta) / n if n else float("nan")


def cpl(est, gt, theta):
    est, gt, _, g, v = _both(est, gt)
    n = int(np.count_nonzero(g))
    return _hits(est, gt, v, theta) / n if n else float("nan")


def fscore(est, gt, theta):
    a, c = acc(est, gt, theta), cpl(est, gt, theta)
    return 2.0 * a * c / (a + c) if a + c > 0 else 0.0


def aae_deg(n_est, n_gt):
    """Mean angle (degrees) between normal maps [..., 3] over the pixels
    where both are non-zero."""
    a = np.asarray(n_est, np.float64)
    b = np.asarray(n_gt, np.float64)
    na, nb = np.linalg.norm(a, axis=-1), np.linalg.norm(b, axis=-1)
    v = (na > 0) & (nb > 0)
    if not v.any():
        return float("nan")
    c = np.clip(np.sum(a[v] * b[v], -1) / (na[v] * nb[v]), -1.0, 1.0)
    return float(np.degrees(np.arccos(c)).mean())


def depth_report(est, gt, thetas=(1.05, 1.25)):
    out = {"l1_abs": l1_abs(est, gt), "l1_rel": l1_rel(est, gt)}
    for t in thetas:
        out["acc_%g" % t] = acc(est, gt, t)
        out["cpl_%g" % t] = cpl(est, gt, t)
        out["f_%g" % t] = fscore(est, gt, t)
    return out
