"""The C-ABI library loads and exports every symbol include/vrc.h declares,
and rejects bad arguments with the documented codes (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1706_07476_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(vrc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for core in ("vrc_create_mesh", "vrc_load_xs", "vrc_cast_rays", "vrc_read_tally"):
        assert core in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True)
    exported = set(re.findall(r" T (vrc_\w+)", out.stdout))
    assert set(_declared_symbols()) <= exported


def test_c_driver_error_codes(lib_path, tmp_path):
    exe = tmp_path / "abi_errors"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "abi_errors.c"), "-o", str(exe),
                           lib_path, f"-Wl,-rpath,{os.path.dirname(lib_path)}", "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr + r.stdout


def test_python_binding_argument_errors(lib_path):
    from paper_1706_07476_gb300 import vrc
    import vrc_workloads as W
    p = W.uniform_small(n=4, n_rays=8)
    with pytest.raises(vrc.VrcError) as ei:
        vrc.vrc_create_mesh(p.mesh, 1)  # ids 0..1 but only 1 material
    assert ei.value.code == vrc.VRC_ERR_ARG
    with pytest.raises(vrc.VrcError):
        vrc.vrc_create_mesh(p.mesh, 2, group_edges=np.array([1.0, 1.0]))
    with pytest.raises(TypeError):
        vrc.vrc_default_options(nonsense=1)
    o = vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, block=128)
    assert o.form == 1 and o.block == 128
