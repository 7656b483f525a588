"""Test-side helpers: golden-case loading and the tally comparison metric."""
from __future__ import annotations

import json
import math
import os

import numpy as np

import vrc_workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Cells whose oracle tally is below this (in units of weight x cm) are outside
# the relative-error parity set; they are checked with an absolute bound.
PARITY_FLOOR = 1e-30


def golden_cases(name: str = "closed_forms.json"):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)["cases"]


def golden_problem(case) -> W.Problem:
    m = case["mesh"]
    nx, ny, nz = m["n"]
    mat = np.asarray(m["material"], np.uint8).reshape(nz, ny, nx)
    mesh = W.Mesh(nx, ny, nz, *[float(v) for v in m["origin"]],
                  *[float(v) for v in m["spacing"]], mat)
    tables = [None if t is None else (np.asarray(t[0], np.float64), np.asarray(t[1], np.float64))
              for t in case["tables"]]
    edges = None if case["group_edges"] is None else np.asarray(case["group_edges"], np.float64)
    r = np.asarray(case["rays"], np.float64)
    for v in r.reshape(-1):  # every field must be exact in float32
        assert float(np.float32(v)) == v
    rays = W.make_rays(*[r[:, k].astype(np.float32) for k in range(8)])
    return W.Problem(case["name"], mesh, tables, edges, rays)


def golden_expected(case, problem) -> np.ndarray:
    out = np.zeros(problem.tally_size, np.float64)
    for k, expr in case["expected"].items():
        out[int(k)] = eval(expr, {"math": math})  # noqa: S307 - fixture expressions
    return out


def rel_err_report(ref: np.ndarray, got: np.ndarray, floor: float = PARITY_FLOOR):
    """Eq. 7 relative difference |ref - got| / ref over cells with ref >= floor.

    Returns dict(max_rel, mean_rel, n_cells, max_abs_below, n_below) where the
    last two cover cells below the floor (absolute error, count).
    """
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    sel = np.abs(ref) >= floor
    if sel.any():
        rel = np.abs(ref[sel] - got[sel]) / np.abs(ref[sel])
        max_rel, mean_rel = float(rel.max()), float(rel.mean())
        worst = int(np.flatnonzero(sel)[int(np.argmax(rel))])
    else:
        max_rel, mean_rel, worst = 0.0, 0.0, -1
    below = ~sel
    max_abs_below = float(np.abs(got[below] - ref[below]).max()) if below.any() else 0.0
    return dict(max_rel=max_rel, mean_rel=mean_rel, n_cells=int(sel.sum()), worst=worst,
                max_abs_below=max_abs_below, n_below=int(below.sum()))
