"""The float64 exp / expm1 pair of the plain form (Cody-Waite reduction plus
a degree-13 Taylor series), built for the host from the same header the
kernels include, held to 2 ulp of long-double expl / expm1l over y in
[-760, 0] (about 4e6 points, including both sides of every reduction
boundary), with (0, -1) below the normal range and exact results at y = 0
and y = -1e-300."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exp_pair_error_bound(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "expd_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_1706_07476_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "c", "expd_check.cpp"), "-o", str(exe), "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
