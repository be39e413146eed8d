"""The bounds-checked build (libfassmvs_checked.so, -DFASSMVS_CHECKED): every
index the kernels form into shared and global memory is tested before the
access, a failure is recorded with its site and the access skipped, and
fassmvs_sync then returns FASSMVS_EINTERNAL.  Runs the cases of
tests/checked_cases.py (ragged and minimum sizes, both costs, every SGM variant
and aggregation form, batches, stage entry points) once with the checked build
and once with the default build, each in its own process (a process loads one
library): the checked run must record no check, and both must give the same
bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(tmp_path, checked):
    out = os.path.join(str(tmp_path), "checked.npz" if checked else "default.npz")
    env = dict(os.environ, FASSMVS_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "CASES OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(out)


def test_checked_build_records_no_check_and_changes_no_result(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00821_b300 import build
    if not os.path.exists(build.LIB_CHECKED):
        build.build(checked=True)
    a = _run(tmp_path, checked=True)
    b = _run(tmp_path, checked=False)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
