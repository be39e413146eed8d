"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/fassmvs.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fassmvs.h")).read()
    return sorted(set(re.findall(r"FASSMVS_API\s+[\w\s\*]+?\b(fassmvs_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fassmvs_create", "fassmvs_set_cameras", "fassmvs_estimate", "fassmvs_sgm_aggregate",
              "fassmvs_cost_volume", "fassmvs_destroy", "fassmvs_sync", "fassmvs_last_error"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2112_00821_b300 import build, fassmvs
    build.build()
    lib = ctypes.CDLL(build.LIB)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) == set(fassmvs.EXPORTS)


def test_binding_fails_loudly_without_a_device():
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2112_00821_b300 import fassmvs
    with pytest.raises(RuntimeError):
        fassmvs.Context()


def test_default_config_and_error_text_without_a_device():
    from paper_2112_00821_b300 import fassmvs
    c = fassmvs.default_config()
    assert c.levels == 1 and c.paths == 8 and c.p1 == 24 and abs(c.alpha - 8) < 1e-6
    lib = fassmvs.lib()
    h = ctypes.c_void_p()
    bad = fassmvs.default_config(levels=9)
    st = lib.fassmvs_create(ctypes.byref(bad), 0, 0, ctypes.byref(h))
    assert st == fassmvs.EINVAL
    assert b"levels" in lib.fassmvs_last_error(None)
