"""Constants the paper fixes (tests/golden/paper_constants.json, each with
its passage) against the library's configuration defaults and the oracle's
behaviour.  The top-level cap of 256 planes is pinned on the GPU
(test_gpu_edges.py::test_estimate_top_level_plane_cap)."""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = {k: v["value"] for k, v in json.load(open(os.path.join(HERE, "golden", "paper_constants.json"))).items()
        if not k.startswith("_")}


@pytest.fixture(scope="module")
def fm():
    from paper_2112_00821_b300 import build, fassmvs
    build.build()
    return fassmvs


def test_library_defaults_are_the_papers(fm):
    c = fm.default_config()
    assert c.alpha == GOLD["adaptive_p2_alpha"] and c.beta == GOLD["adaptive_p2_beta"]
    assert c.p1 == GOLD["census_phi1"] and c.cost == 0 and c.paths == GOLD["sgm_paths"]
    # a served request names up to |Psi| - 1 other maps for the consistency check
    assert len(fm.Request().geo_ids) == GOLD["geo_window"] - 1


def test_oracle_adaptive_p2_follows_the_papers_alpha_and_beta(orc):
    p1 = GOLD["ncc_phi1"]
    lut = orc.p2_table(p1)
    a, b = GOLD["adaptive_p2_alpha"], GOLD["adaptive_p2_beta"]
    assert lut[0] == p1 * (1 + a)
    for d in (1, 10, 37, 255):
        assert abs(int(lut[d]) - p1 * (1 + a * math.exp(-d / b))) <= 0.5


def test_oracle_census_window_is_9x7(orc):
    """A bright centre over a dark 9x7 neighbourhood sets every comparison
    bit: 9 * 7 - 1 of them, which fit one 64-bit word."""
    w, h = GOLD["census_window"]
    img = np.zeros((21, 21), np.uint8)
    img[10, 10] = 255
    c = int(orc.census(img)[10, 10])
    assert bin(c).count("1") == w * h - 1 and c < (1 << 64)
    img[10 - h // 2 - 1, 10] = 0                       # outside the window: no effect
    assert int(orc.census(img)[10, 10]) == c


def test_oracle_ncc_window_and_range(orc):
    n = GOLD["ncc_window"][0] * GOLD["ncc_window"][1]
    g = np.random.default_rng(5)
    a = g.integers(0, 256, n)
    assert orc.ncc_window(a, a) == 0                                # perfect correlation
    assert orc.ncc_window(a, 255 - a) == GOLD["ncc_max_cost"]       # anti-correlated: truncated


def test_geometric_filter_defaults_are_the_papers(orc, fm):
    import inspect
    sig = inspect.signature(orc.geo_hits)
    assert sig.parameters["eta_r"].default == GOLD["geo_eta_r"]
    bsig = inspect.signature(fm.Context.geo_filter)
    assert bsig.parameters["eta_r"].default == GOLD["geo_eta_r"]
    assert bsig.parameters["eta_h"].default == GOLD["geo_eta_h"]


def test_fronto_normal_bounds_are_the_depth_range(fm):
    K = np.array([[100.0, 0, 31.5], [0, 100.0, 23.5], [0, 0, 1]])
    assert fm.plane_bounds(K, 64, 48, GOLD["fronto_normal"], 4.0, 40.0) == (4.0, 40.0)
