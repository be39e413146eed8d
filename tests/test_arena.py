"""The serving form's host-side allocator (csrc/arena.h) on the CPU: a
randomised run of allocations (low best-fit and high) and frees checks
alignment, bounds, disjointness, exact accounting and coalescing."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_arena_allocator(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "arena_check")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-Wall", "-o", exe, os.path.join(HERE, "arena_check.cpp")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"
