"""The float64 helpers of the plain form.  The exp / expm1 pair (Tang's table-driven
reduction with 2048 entries, a degree-4 Taylor series), built for the host from
the same header the kernels include: e^y held to 0.6 ulp and e^y - 1 to 2 ulp
of long-double expl / expm1l over y in [-760, 0] (about 2.3e7 points,
including both sides of reduction boundaries, each with the float32
estimate of y the kernels pass and one float32 ulp either side), (0, -1)
below the normal range, exact results at y = 0 and y = -1e-300; the exact
float32 product (integer significand product) bit for bit the float64
product, zero and subnormal factors included; and the table's rows against
2^(j/2048) from exact decimal arithmetic.  The reciprocal of a float32
(float32 estimate plus a third-order Newton-Raphson step) equal to the
rounded float64 quotient on 2.1e6 normal float32 inputs."""
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
    exe = tmp_path / "math64_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_1706_07476_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "c", "math64_check.cpp"), "-o", str(exe), "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr


def test_exp2_table_is_exact():
    """Every kExp2Tab row is (nearest float64 to 2^(j/2048), nearest float64
    to the remainder), checked against 2^(j/2048) from exact decimal
    arithmetic written here, and head + tail is within 2^-104 of it."""
    import re
    from decimal import Decimal, getcontext
    src = open(os.path.join(ROOT, "paper_1706_07476_gb300", "csrc", "vrc_exp2_table.h")).read()
    body = src[src.index("kExp2Tab[2048][2] = {"):]
    body = body[:body.index("};")]
    rows = re.findall(r"\{\s*([-0-9a-fx.p+]+)\s*,\s*([-0-9a-fx.p+]+)\s*\}", body)
    assert len(rows) == 2048
    getcontext().prec = 60
    for j, (h, l) in enumerate(rows):
        hi, lo = float.fromhex(h), float.fromhex(l)
        exact = Decimal(2) ** (Decimal(j) / 2048)
        assert hi == float(exact), j
        assert lo == float(exact - Decimal(hi)), j
        assert abs(Decimal(hi) + Decimal(lo) - exact) <= exact * Decimal(2) ** -104, j
