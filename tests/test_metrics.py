"""The error measures of Sec. 3.2 on hand-computed maps."""
import math

import numpy as np
import pytest

from paper_2112_00821_b300 import metrics as M


def _maps():
    gt = np.array([[10.0, 20.0, 0.0], [40.0, 50.0, 60.0]])
    est = np.array([[11.0, 0.0, 30.0], [40.0, 75.0, np.nan]])
    return est, gt


def test_l1_over_pixels_valid_in_both():
    est, gt = _maps()                                      # V = {(0,0), (1,0), (1,1)}
    assert M.l1_abs(est, gt) == pytest.approx((1 + 0 + 25) / 3)
    assert M.l1_rel(est, gt) == pytest.approx((0.1 + 0 + 0.5) / 3)


def test_accuracy_completeness_and_f():
    est, gt = _maps()
    # ratios on V: 1.1, 1.0, 1.5; E = 4 valid estimates, G = 5 valid GT pixels
    assert M.acc(est, gt, 1.25) == pytest.approx(2 / 4)
    assert M.cpl(est, gt, 1.25) == pytest.approx(2 / 5)
    assert M.acc(est, gt, 1.05) == pytest.approx(1 / 4)
    assert M.fscore(est, gt, 1.25) == pytest.approx(2 * 0.5 * 0.4 / 0.9)
    assert M.acc(est, gt, 1.0) == 0.0 and M.fscore(est, gt, 1.0) == 0.0


def test_perfect_and_symmetric_ratio():
    gt = np.random.default_rng(1).uniform(5, 50, (7, 9))
    r = M.depth_report(gt, gt)
    assert r["l1_abs"] == 0 and r["l1_rel"] == 0 and r["f_1.05"] == 1.0
    # over- and under-estimates by the same factor count alike
    assert M.acc(gt * 1.2, gt, 1.25) == M.acc(gt / 1.2, gt, 1.25) == 1.0


def test_aae():
    a = np.array([[[0, 0, -1.0], [1, 0, 0], [0, 0, 0]]])
    b = np.array([[[0, 0, -2.0], [0, 1, 0], [1, 0, 0]]])
    assert M.aae_deg(a, b) == pytest.approx(45.0)
    c = np.array([[[math.sin(0.1), 0, -math.cos(0.1)]]])
    assert M.aae_deg(c, np.array([[[0, 0, -1.0]]])) == pytest.approx(math.degrees(0.1))
