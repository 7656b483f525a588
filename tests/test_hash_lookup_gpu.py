"""The hashed cross-section lookup (Sec. 3: Brown's hash on the log-energy
grid, then lin-lin interpolation), checked ray by ray.

The GPU looks Sigma_t up on the union of all materials' grids: a log2 hash
bin gives a bracket of grid intervals, a bounded fix-up and a binary search
then pick the interval E[i] <= E < E[i+1].  A wrong interval shows up as a
wrong Sigma_t wherever the table is not one straight line across both
intervals.  This test puts one ray in its own cell for every energy that can
expose a wrong bracket:

- every union-grid point, and the float32 values one ulp below and above it;
- the midpoint of every union-grid interval;
- every edge of the hash bins, for every bin count the library can choose
  (powers of two from 64 to 4,096 over [log2 E_first, log2 E_last]), and one
  ulp below and above it: the float32 log2 of an energy on a bin edge may
  round into the neighbouring bin;
- energies below, at and above the ends of every material's table (each
  material clamps to its own end values).

Three materials with different grids (log-spaced over the full range; a
narrower range; jittered spacing) make the union grid irregular.  Each ray
crosses exactly one cell, 20 cm long, so its score wt (1 - e^{-Sigma l}) /
Sigma moves by at least 0.69 of any relative change of Sigma.  Every cell is
compared with the FP64 oracle, which uses a plain binary search on each
material's own grid.  The bound per ray is 1e-6 relative plus what the
single-precision interpolation itself may lose with the right bracket:
Sigma = a + f (b - a) in float32 from float32 table values a, b at the
interval ends carries an error up to about 2^-24 (|a| + |b| + 3 |b - a| +
Sigma) (on a steep resonance flank, where a or b is far above Sigma, this
reaches 1e-5 relative).  For nine rays in ten the bound stays at 1e-6 or
just above, far below what a neighbouring interval gives on these tables.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

L_CELL = 20.0


def _tables():
    rng = np.random.default_rng(11)
    a = W.xs_table(rng, 2000, 20)
    E, S = W.xs_table(rng, 1500, 15, e_min=1e-3, e_max=1e6)
    b = (E, S)
    # jittered log spacing, its own resonances
    lg = np.sort(rng.uniform(math.log10(W.E_MIN_EV), math.log10(W.E_MAX_EV), 997))
    Ej = np.unique(10.0 ** lg)
    Sj = 0.5 + 3.0 / np.sqrt(Ej)
    for _ in range(10):
        er = 10.0 ** rng.uniform(0.0, 5.0)
        Sj = Sj + 10.0 ** rng.uniform(0, 3) / (1.0 + ((Ej - er) / (er * 10.0 ** rng.uniform(-3, -1.5))) ** 2)
    return [a, b, (Ej, Sj)]


def _energies(tables):
    U = np.unique(np.concatenate([t[0] for t in tables]))
    pts = U.astype(np.float32)
    up = np.nextafter(pts, np.float32(np.inf))
    dn = np.nextafter(pts, np.float32(0))
    mid = (0.5 * (U[:-1] + U[1:])).astype(np.float32)
    l2a, l2b = math.log2(U[0]), math.log2(U[-1])
    edges = []
    for nh in (64, 128, 256, 512, 1024, 2048, 4096):
        inv_bw = np.float32(nh / (l2b - l2a))
        b = np.arange(nh + 1, dtype=np.float64)
        e = np.exp2(np.float64(np.float32(l2a)) + b / np.float64(inv_bw)).astype(np.float32)
        edges += [e, np.nextafter(e, np.float32(np.inf)), np.nextafter(e, np.float32(0))]
    ends = []
    for E, _ in tables:
        for v in (E[0], E[-1]):
            f = np.float32(v)
            ends += [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(0))]
    ends += [np.float32(1e-6), np.float32(5e7)]
    allE = np.concatenate([pts, up, dn, mid, *edges, np.array(ends, np.float32)])
    allE = allE[np.isfinite(allE) & (allE > 0)]
    return np.unique(allE)


def _problem():
    tables = _tables()
    E = _energies(tables)
    n_e, n_m = len(E), len(tables)
    mat = np.repeat(np.arange(n_m, dtype=np.uint8), n_e).reshape(n_m, 1, n_e)
    mesh = W.Mesh(n_e, 1, n_m, 0.0, 0.0, 0.0, 1.0, L_CELL, 1.0, mat)
    ix = np.tile(np.arange(n_e), n_m)
    iz = np.repeat(np.arange(n_m), n_e)
    n = n_e * n_m
    rays = W.make_rays((ix + 0.5).astype(np.float32), np.zeros(n, np.float32),
                       (iz + 0.5).astype(np.float32), np.zeros(n, np.float32),
                       np.ones(n, np.float32), np.zeros(n, np.float32),
                       np.tile(E, n_m).astype(np.float32), np.ones(n, np.float32))
    return W.Problem("hash_lookup", mesh, tables, None, rays)


def _interp_bound(prob):
    """Per ray: the relative error float32 lin-lin interpolation may carry
    with the right bracket, 2^-24 (|a| + |b| + 3 |b - a| + Sigma) / Sigma,
    with a, b the material's values at the ends of the ray's interval of the
    union grid (float64, from the tables)."""
    U = np.unique(np.concatenate([t[0] for t in prob.tables]))
    n_e = prob.mesh.nx
    E = prob.rays["E"][:n_e].astype(np.float64)
    i = np.clip(np.searchsorted(U, E, side="right") - 1, 0, len(U) - 2)
    out = []
    for Et, St in prob.tables:
        a, b, s = np.interp(U[i], Et, St), np.interp(U[i + 1], Et, St), np.interp(E, Et, St)
        out.append(2.0 ** -24 * (np.abs(a) + np.abs(b) + 3 * np.abs(b - a) + s) / s)
    return np.concatenate(out)


@pytest.fixture(scope="module")
def lookup_case():
    prob = _problem()
    want, st = oracle.cast(prob)
    return prob, want, st


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_hash_bracket_per_ray(vrc, lookup_case, form):
    prob, want, st = lookup_case
    # every ray crosses exactly its own cell, 20 cm
    assert st["segments"] == prob.n_rays
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form, sort=0))
    try:
        vrc.vrc_cast_rays(ctx, prob.rays)
        rc, stats = vrc.vrc_sync(ctx)
        got, _ = vrc.vrc_read_tally(ctx)
    finally:
        ctx.close()
    assert rc == vrc.VRC_OK and stats["segments"] == st["segments"]
    assert np.all(want > 0)
    rel = np.abs(got - want) / want
    bound = 1e-6 + _interp_bound(prob)
    assert np.mean(bound <= 1.5e-6) > 0.9
    worst = int(np.argmax(rel / bound))
    n_e = prob.mesh.nx
    print(f"form={form}: {prob.n_rays} rays, max rel {rel.max():.3e}, worst against its bound "
          f"{rel[worst]:.3e} <= {bound[worst]:.3e} at material {worst // n_e}, E={prob.rays['E'][worst]!r}")
    assert np.all(rel <= bound), (rel[worst], bound[worst], worst, prob.rays["E"][worst])


def test_hash_case_is_sensitive_to_a_wrong_bracket(lookup_case):
    """The bound above catches a neighbouring interval: at the interval
    midpoints of every material's table, interpolating from the next
    interval instead (as a bracket off by one would) moves the score by more
    than 2e-6 (above the typical per-ray bound of 1.2e-6) for over 80 % of
    the energies (the rest lie where the table is nearly straight across
    both intervals)."""
    prob, want, _ = lookup_case
    for E0, S0 in prob.tables:
        mid = 0.5 * (E0[1:-2] + E0[2:-1])
        k = np.arange(1, len(E0) - 2)
        exact = S0[k] + (mid - E0[k]) * (S0[k + 1] - S0[k]) / (E0[k + 1] - E0[k])
        wrong = S0[k + 1] + (mid - E0[k + 1]) * (S0[k + 2] - S0[k + 1]) / (E0[k + 2] - E0[k + 1])

        def score(s):
            return -np.expm1(-np.minimum(s * L_CELL, 700.0)) / s

        d = np.abs(score(wrong) - score(exact)) / score(exact)
        assert np.mean(d > 2e-6) > 0.8, np.mean(d > 2e-6)
