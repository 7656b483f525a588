"""The oracle's pins have teeth: each planted mistake fails at least one pin.

Every mutant is a textual edit of a private copy of the oracle's C source,
compiled into a temporary library and swapped in for the duration of the
check (CPU only).  The committed oracle source is never modified.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import pytest

import oracle
from tests import helpers as H
from tests import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "vrc_oracle.c")

MUTANTS = {
    "drop_attenuation": ("return wt * exp(-tau) * path;", "return wt * path;"),
    "expm1_sign": ("-expm1(-sig * l) / sig", "expm1(sig * l) / sig"),
    "transposed_spacing": ("return lo[k] + (double)j * h[k];",
                           "return lo[k] + (double)j * h[(k + 1) % 3];"),
    "boundary_off_by_one": ("tn[k] = (plane(m, k, idx[k] + 1) - p[k]) / d[k];",
                            "tn[k] = (plane(m, k, idx[k] + 2) - p[k]) / d[k];"),
    "interp_wrong_end": ("S[lo] + (e - E[lo]) * (S[hi] - S[lo])", "S[lo] + (E[hi] - e) * (S[hi] - S[lo])"),
    "tau_not_accumulated": ("tau += sg * lens[s];", ""),
    "no_vacuum_clip": ("if (ta > a) a = ta;", ""),
    "wrong_group_bin": ("if (edges[mid] <= e) lo = mid; else hi = mid;",
                        "if (edges[mid] < e) lo = mid; else hi = mid;"),
    "rect_edge_index_shift": ("if (e) return e[j];", "if (e) return e[j > 0 ? j - 1 : 0];"),
    "rect_locate_as_uniform": ("  if (!e) {\n    const double lo[3]", "  if (1) {\n    const double lo[3]"),
}


def _pins():
    cases = H.golden_cases()
    checks = [lambda c=c: P.test_golden_closed_forms(c) for c in cases]
    checks += [P.test_sigma_linlin_matches_numpy_interp, P.test_homogeneous_total_is_eq1_closed_form,
               P.test_void_scores_geometric_chord, P.test_telescoping_invariant,
               P.test_start_outside_equals_start_at_entry, P.test_group_edges,
               P.test_brute_force_quadrature_tiny_meshes, P.test_rect_void_chords_are_cell_widths,
               P.test_rect_axis_aligned_per_cell_scores, P.test_rect_inserted_plane_additivity,
               P.test_rect_dda_matches_brute_force_traversal]
    return checks


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-pthread", "-ffp-contract=off", "-o", str(so), str(path), "-lm"])
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    real = oracle._load()
    lib = ctypes.CDLL(_build_mutant(tmp_path, name))
    for fn in ("orc_sigma_t", "orc_group", "orc_trace_dda", "orc_trace_brute", "orc_ray_segments",
               "orc_cast", "orc_hardware_threads"):
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
        getattr(lib, fn).restype = getattr(real, fn).restype
    monkeypatch.setattr(oracle, "_lib", lib)
    failed = []
    for chk in _pins():
        try:
            chk()
        except AssertionError:
            failed.append(chk)
    assert failed, f"mutant {name} survived every pin"
