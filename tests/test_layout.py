"""The column pass's per-warp shared-memory layout, checked on the host: the
layout code (paper_2511_09753_gb300/csrc/colpass_shape.cuh) is compiled with
g++ into a checker that walks every pass kind, value size, cap 1..80 and
row width 1..40 and verifies that each buffer lies inside the warp's bytes
and that buffers which are live at the same time never overlap.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_09753_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "helpers", "layout_check.cpp")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_layout_buffers_in_bounds_and_disjoint(tmp_path):
    inc = _cuda_include()
    if not shutil.which("g++") or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "layout_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", inc, "-o", exe, SRC],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    assert "violations 0" in r.stdout
