"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these retypes the oracle's own formulas: each expected value comes
from a closed form (Eq. 1, Eq. 3), from a hand-derived golden case, from an
invariant (telescoping, mesh refinement, translation, ray order), from an
independent brute-force quadrature of the attenuation integral (Eq. 2), or
from a library routine (numpy.interp for lin-lin interpolation).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H


def _const_table(sig):
    return (np.array([W.E_MIN_EV, W.E_MAX_EV]), np.array([sig, sig]))


def _rays(p, d, E, wt):
    p = np.asarray(p, np.float32).reshape(-1, 3)
    d = np.asarray(d, np.float32).reshape(-1, 3)
    n = p.shape[0]
    E = np.broadcast_to(np.asarray(E, np.float32), (n,))
    wt = np.broadcast_to(np.asarray(wt, np.float32), (n,))
    return W.make_rays(p[:, 0], p[:, 1], p[:, 2], d[:, 0], d[:, 1], d[:, 2], E, wt)


def _mesh(n, origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0), material=None, rng=None, nmat=1):
    nx, ny, nz = n
    if material is None:
        material = (np.zeros((nz, ny, nx), np.uint8) if rng is None
                    else rng.integers(0, nmat, size=(nz, ny, nx)).astype(np.uint8))
    return W.Mesh(nx, ny, nz, *origin, *spacing, np.asarray(material, np.uint8))


# ---------------------------------------------------------------- golden

@pytest.mark.parametrize("case", H.golden_cases(), ids=lambda c: c["name"])
def test_golden_closed_forms(case):
    prob = H.golden_problem(case)
    got, _ = oracle.cast(prob, nthreads=1)
    want = H.golden_expected(case, prob)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- cross sections

def test_sigma_linlin_matches_numpy_interp():
    rng = np.random.default_rng(11)
    E, S = W.xs_table(rng, 500, 7)
    es = np.concatenate([E, 0.5 * (E[1:] + E[:-1]), np.exp(rng.uniform(-14, 18, 2000)),
                         [E[0] * 0.5, E[-1] * 2.0, E[0], E[-1]]])
    want = np.interp(es, E, S)  # library lin-lin with end clamping
    got = np.array([oracle.sigma_t(E, S, e) for e in es])
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


def test_sigma_table_points_midpoints_and_clamp():
    E = np.array([1.0, 2.0, 4.0, 8.0])
    S = np.array([3.0, 1.0, 7.0, 2.0])
    for e, s in zip(E, S):
        assert oracle.sigma_t(E, S, e) == s
    for i in range(3):
        assert oracle.sigma_t(E, S, 0.5 * (E[i] + E[i + 1])) == pytest.approx(
            0.5 * (S[i] + S[i + 1]), rel=1e-15)
    assert oracle.sigma_t(E, S, 0.1) == 3.0
    assert oracle.sigma_t(E, S, 100.0) == 2.0
    assert oracle.sigma_t(E[:0], S[:0], 5.0) == 0.0  # void


def test_group_edges():
    edges = np.array([1.0, 10.0, 100.0, 1000.0])
    assert oracle.group(edges, 1.0) == 0
    assert oracle.group(edges, 9.999) == 0
    assert oracle.group(edges, 10.0) == 1
    assert oracle.group(edges, 999.0) == 2
    assert oracle.group(edges, 1000.0) == 2
    assert oracle.group(edges, 0.999) == -1
    assert oracle.group(edges, 1000.5) == -1
    assert oracle.group(None, 123.0) == 0


# ---------------------------------------------------------------- closed forms

def test_homogeneous_total_is_eq1_closed_form():
    """One material everywhere: the per-cell scores of a ray sum to
    w (1 - exp(-Sigma L)) / Sigma with L the distance to the box exit (Eq. 1)."""
    rng = np.random.default_rng(5)
    mesh = _mesh((7, 5, 6), origin=(-1.5, 2.0, 0.25), spacing=(0.5, 1.25, 0.75))
    lo, hi = np.array(mesh.lo), np.array(mesh.hi)
    sig = 0.37
    for _ in range(40):
        p = lo + (hi - lo) * rng.random(3)
        d = rng.normal(size=3)
        p32, d32 = p.astype(np.float32), d.astype(np.float32)
        prob = W.Problem("h", mesh, [_const_table(sig)], None, _rays(p32, d32, 1.0, 1.75))
        tal, st = oracle.cast(prob, nthreads=1)
        pp, dd = p32.astype(np.float64), d32.astype(np.float64)
        dd = dd / np.linalg.norm(dd)
        L = min(((hi[k] if dd[k] > 0 else lo[k]) - pp[k]) / dd[k] for k in range(3) if dd[k] != 0)
        assert tal.sum() == pytest.approx(1.75 * (1 - math.exp(-sig * L)) / sig, rel=1e-12)


def test_axis_aligned_per_cell_scores():
    """Ray along +x from x=x0 (the float32 nearest 0.3): cell i entered at
    t_i = i - x0 (i >= 1) with l_i = 1; score w exp(-Sigma t_i)(1 -
    exp(-Sigma l_i))/Sigma (Eq. 3)."""
    mesh = _mesh((5, 1, 1))
    sig = 0.8
    x0 = float(np.float32(0.3))
    prob = W.Problem("ax", mesh, [_const_table(sig)], None,
                     _rays([x0, 0.5, 0.5], [1, 0, 0], 1.0, 2.0))
    tal, _ = oracle.cast(prob, nthreads=1)
    want = [2.0 * (1 - math.exp(-sig * (1 - x0))) / sig]
    for i in range(1, 5):
        want.append(2.0 * math.exp(-sig * (i - x0)) * (1 - math.exp(-sig)) / sig)
    np.testing.assert_allclose(tal, want, rtol=1e-13)


def test_void_scores_geometric_chord():
    """In void the expected track length is the chord length itself."""
    rng = np.random.default_rng(6)
    mesh = _mesh((6, 6, 6))
    # axis-aligned rays through cell centres: chord 1 per cell, 0.5 in the start cell
    prob = W.Problem("v", mesh, [None], None, _rays([2.5, 3.5, 4.5], [0, -1, 0], 1.0, 3.0))
    tal, _ = oracle.cast(prob, nthreads=1)
    tal = tal.reshape(6, 6, 6)
    assert tal[4, 3, 2] == pytest.approx(1.5, rel=1e-15)
    for iy in range(3):
        assert tal[4, iy, 2] == pytest.approx(3.0, rel=1e-15)
    assert tal.sum() == pytest.approx(3.0 * 3.5, rel=1e-15)
    # random rays: total = w * L
    for _ in range(30):
        p = (6 * rng.random(3)).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32)
        prob = W.Problem("v", mesh, [None], None, _rays(p, d, 1.0, 1.0))
        tal, _ = oracle.cast(prob, nthreads=1)
        dd = d.astype(np.float64) / np.linalg.norm(d.astype(np.float64))
        pp = p.astype(np.float64)
        L = min(((6.0 if dd[k] > 0 else 0.0) - pp[k]) / dd[k] for k in range(3) if dd[k] != 0)
        assert tal.sum() == pytest.approx(L, rel=1e-12)


# ---------------------------------------------------------------- invariants

def _hetero_problem(rng, n=(6, 5, 4), nmat=4, n_rays=400, void=True, spacing=(1.0, 0.7, 1.3)):
    mesh = _mesh(n, origin=(0.5, -1.0, 2.0), spacing=spacing, rng=rng, nmat=nmat)
    tables = [W.xs_table(rng, 60, 3, peak_lo=0.1, peak_hi=3.0) for _ in range(nmat)]
    if void:
        tables[0] = None
    lo, hi = np.array(mesh.lo), np.array(mesh.hi)
    pos = (lo + (hi - lo) * rng.random((n_rays, 3))).astype(np.float32)
    d = rng.normal(size=(n_rays, 3)).astype(np.float32)
    E = W.log_uniform(rng, n_rays)
    wt = rng.lognormal(0, 0.5, n_rays).astype(np.float32)
    rays = W.make_rays(pos[:, 0], pos[:, 1], pos[:, 2], d[:, 0], d[:, 1], d[:, 2], E, wt)
    return W.Problem("het", mesh, tables, None, rays)


def test_telescoping_invariant():
    """sum_i Sigma_i s_i = w (1 - exp(-tau_exit)) for every ray (Eq. 4 summed
    along the ray telescopes), with tau_exit = sum_i Sigma_i l_i."""
    rng = np.random.default_rng(7)
    prob = _hetero_problem(rng, n_rays=200)
    for i in range(prob.n_rays):
        seg = oracle.ray_segments(prob, i)
        if len(seg["lens"]) == 0:
            continue
        tau = float(np.sum(seg["sigma"] * seg["lens"]))
        lhs = float(np.sum(seg["sigma"] * seg["score"]))
        void_part = seg["sigma"] == 0
        wt = float(prob.rays["wt"][i])
        assert lhs == pytest.approx(wt * -math.expm1(-tau), rel=1e-12, abs=1e-300)
        # void segments: score is the attenuated chord
        att = np.exp(-np.concatenate([[0.0], np.cumsum(seg["sigma"] * seg["lens"])[:-1]]))
        np.testing.assert_allclose(seg["score"][void_part],
                                   wt * att[void_part] * seg["lens"][void_part],
                                   rtol=1e-13)


def test_mesh_refinement_additivity():
    """Splitting every cell into 2x2x2 same-material sub-cells leaves the summed
    score of each parent cell unchanged."""
    rng = np.random.default_rng(8)
    prob = _hetero_problem(rng, n=(4, 3, 5), n_rays=300, spacing=(1.0, 1.0, 1.0))
    m = prob.mesh
    fine_mat = m.material.repeat(2, 0).repeat(2, 1).repeat(2, 2)
    fine = W.Mesh(2 * m.nx, 2 * m.ny, 2 * m.nz, m.x0, m.y0, m.z0, m.dx / 2, m.dy / 2, m.dz / 2,
                  fine_mat)
    coarse, _ = oracle.cast(prob, nthreads=1)
    ft, _ = oracle.cast(W.Problem("f", fine, prob.tables, None, prob.rays), nthreads=1)
    ft = ft.reshape(2 * m.nz, 2 * m.ny, 2 * m.nx)
    folded = ft.reshape(m.nz, 2, m.ny, 2, m.nx, 2).sum(axis=(1, 3, 5)).reshape(-1)
    np.testing.assert_allclose(folded, coarse, rtol=1e-11, atol=1e-300)


def test_translation_by_whole_cells():
    rng = np.random.default_rng(9)
    prob = _hetero_problem(rng, n_rays=300, spacing=(1.0, 0.5, 2.0))
    base, _ = oracle.cast(prob, nthreads=1)
    m = prob.mesh
    shift = np.array([3 * m.dx, -2 * m.dy, 5 * m.dz])
    mesh2 = W.Mesh(m.nx, m.ny, m.nz, m.x0 + shift[0], m.y0 + shift[1], m.z0 + shift[2], m.dx, m.dy,
                   m.dz, m.material)
    r = dict(prob.rays)
    for k, key in enumerate("xyz"):
        r[key] = (r[key].astype(np.float64) + shift[k]).astype(np.float32)
    # shifted float32 positions may round: compare against the rounded-back rays
    back = dict(prob.rays)
    for k, key in enumerate("xyz"):
        back[key] = (r[key].astype(np.float64) - shift[k]).astype(np.float32)
    base, _ = oracle.cast(prob, nthreads=1, rays=back)
    moved, _ = oracle.cast(W.Problem("t", mesh2, prob.tables, None, r), nthreads=1)
    np.testing.assert_allclose(moved, base, rtol=1e-9, atol=1e-12)


def test_ray_order_and_threads_do_not_matter():
    rng = np.random.default_rng(10)
    prob = _hetero_problem(rng, n_rays=5000)
    a, sa = oracle.cast(prob, nthreads=1)
    perm = rng.permutation(prob.n_rays)
    b, _ = oracle.cast(W.take_rays(prob, perm), nthreads=1)
    c, sc = oracle.cast(prob, nthreads=4)
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(c, a, rtol=1e-12, atol=1e-300)
    assert sa["segments"] == sc["segments"]


def test_start_outside_equals_start_at_entry():
    """Vacuum outside the mesh: a ray started before the mesh scores like the
    same ray started on the entry face."""
    mesh = _mesh((4, 4, 4), rng=np.random.default_rng(3), nmat=2)
    tables = [_const_table(0.3), _const_table(1.1)]
    d = np.array([0.5, 0.25, 1.0])
    entry = np.array([1.0, 1.5, 0.0])
    outside = entry - 2.0 * d
    a, _ = oracle.cast(W.Problem("o", mesh, tables, None, _rays(outside, d, 1.0, 1.0)), nthreads=1)
    b, _ = oracle.cast(W.Problem("o", mesh, tables, None, _rays(entry, d, 1.0, 1.0)), nthreads=1)
    np.testing.assert_allclose(a, b, rtol=1e-13)
    assert a.sum() > 0


def test_degenerate_rays_score_nothing():
    mesh = _mesh((3, 3, 3))
    rays = _rays([[1.5, 1.5, 1.5]] * 6,
                 [[0, 0, 0], [1, 0, 0], [1, 0, 0], [1, 0, 0], [1, 0, 0], [-1, 0, 0]],
                 [1.0, np.nan, -1.0, 0.0, 1.0, 1.0], [1.0, 1.0, 1.0, 1.0, np.inf, 1.0])
    rays["x"][5] = -0.5  # outside, pointing away
    tal, st = oracle.cast(W.Problem("d", mesh, [_const_table(1.0)], None, rays), nthreads=1)
    assert tal.sum() == 0.0
    assert st["rejected"] == 5 and st["segments"] == 0


# ---------------------------------------------------------------- traversal

def test_dda_matches_brute_force_traversal():
    """The grid walk's positive-length segments equal the sorted plane-crossing
    traversal's, cell for cell, to 1e-12 cm."""
    rng = np.random.default_rng(12)
    meshes = [_mesh((5, 7, 3), origin=(-2.0, 0.5, 1.0), spacing=(0.3, 1.1, 2.0)),
              _mesh((16, 16, 16)), _mesh((1, 9, 2), spacing=(0.039375, 0.039375, 5.0))]
    n_checked = 0
    for mesh in meshes:
        lo, hi = np.array(mesh.lo), np.array(mesh.hi)
        ext = hi - lo
        for i in range(3000):
            p = lo - 0.3 * ext + 1.6 * ext * rng.random(3)
            d = rng.normal(size=3)
            if i % 10 == 0:
                d[rng.integers(0, 3)] = 0.0  # axis-parallel components
            if i % 37 == 0:  # start exactly on a grid plane
                k = rng.integers(0, 3)
                p[k] = lo[k] + rng.integers(0, mesh.material.shape[2 - k] + 1) * (ext[k] / mesh.material.shape[2 - k])
            nrm = np.linalg.norm(d)
            if nrm == 0:
                continue
            d = d / nrm
            c1, t1, l1 = oracle.trace_dda(mesh, p, d)
            keep = l1 > 0
            c2, t2, l2 = oracle.trace_brute(mesh, p, d)
            assert np.array_equal(c1[keep], c2), (p, d)
            np.testing.assert_allclose(l1[keep], l2, rtol=0, atol=1e-12)
            np.testing.assert_allclose(t1[keep], t2, rtol=0, atol=1e-12)
            n_checked += int(keep.sum())
    assert n_checked > 10000


# ---------------------------------------------------------------- quadrature

def _quadrature_tally(prob, h_rel=1e-4):
    """Independent brute force: per ray, sort all plane crossings, classify each
    interval midpoint by floor (outside the box = vacuum), get sigma from
    numpy.interp, and integrate w exp(-tau(s)) over each interval with a
    midpoint rule of step <= h_rel * min spacing (and sigma * step <= 3e-4, so
    the rule's relative error (sigma h)^2/24 stays below 4e-9), accumulating
    tau by the same rule.  Returns the tally."""
    m = prob.mesh
    lo = np.array(m.lo)
    h = np.array([m.dx, m.dy, m.dz])
    n = np.array([m.nx, m.ny, m.nz])
    hi = lo + n * h
    step = h_rel * h.min()
    tally = np.zeros(prob.tally_size)
    r = prob.rays
    for i in range(prob.n_rays):
        p = np.array([r["x"][i], r["y"][i], r["z"][i]], np.float64)
        d = np.array([r["u"][i], r["v"][i], r["w"][i]], np.float64)
        d /= np.linalg.norm(d)
        E, wt = float(r["E"][i]), float(r["wt"][i])
        sig = [0.0 if t is None else float(np.interp(E, t[0], t[1])) for t in prob.tables]
        ts = [0.0]
        for k in range(3):
            if d[k] != 0:
                tk = (lo[k] + np.arange(n[k] + 1) * h[k] - p[k]) / d[k]
                ts.extend(tk[tk > 0])
        far = np.max(np.linalg.norm(np.stack([lo, hi]) - p, axis=1)) * 2 + 1
        ts.append(far)
        ts = np.unique(np.array(ts))
        tau = 0.0
        for a, b in zip(ts[:-1], ts[1:]):
            mid = p + 0.5 * (a + b) * d
            if np.any(mid < lo) or np.any(mid >= hi):
                continue  # vacuum
            idx = np.floor((mid - lo) / h).astype(int)
            cell = (idx[2] * m.ny + idx[1]) * m.nx + idx[0]
            s = sig[m.material.reshape(-1)[cell]]
            hs = step if s == 0 else min(step, 3e-4 / s)
            k = max(1, int(math.ceil((b - a) / hs)))
            hh = (b - a) / k
            mids = (np.arange(k) + 0.5) * hh
            tally[cell] += wt * float(np.sum(np.exp(-(tau + s * mids)))) * hh
            tau += s * (b - a)
    return tally


def test_brute_force_quadrature_tiny_meshes():
    rng = np.random.default_rng(13)
    for n in [(2, 2, 2), (3, 2, 4), (4, 4, 4)]:
        mesh = _mesh(n, origin=(0.25, -0.5, 1.0), spacing=(1.0, 0.75, 0.5), rng=rng, nmat=3)
        tables = [None, W.xs_table(rng, 40, 2, peak_lo=0.1, peak_hi=2.0),
                  (np.array([1e-5, 1.0, 2e7]), np.array([2.5, 0.4, 1.2]))]
        lo, hi = np.array(mesh.lo), np.array(mesh.hi)
        k = 12
        pos = lo - 0.2 * (hi - lo) + 1.4 * (hi - lo) * rng.random((k, 3))
        d = rng.normal(size=(k, 3))
        E = W.log_uniform(rng, k)
        rays = W.make_rays(pos[:, 0].astype(np.float32), pos[:, 1].astype(np.float32),
                           pos[:, 2].astype(np.float32), d[:, 0].astype(np.float32),
                           d[:, 1].astype(np.float32), d[:, 2].astype(np.float32), E,
                           rng.lognormal(0, 0.5, k).astype(np.float32))
        prob = W.Problem("q", mesh, tables, None, rays)
        got, _ = oracle.cast(prob, nthreads=1)
        want = _quadrature_tally(prob)
        assert got.sum() > 0
        np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-12)


# ---------------------------------------------------------------- workloads

def test_uniform_workload_segment_count_and_scale():
    """The 32^3 parity workload: about 2.9e6 positive-length segments for 2^17
    rays (22 per ray) and no rejected or overflowing rays."""
    prob = W.uniform_small()
    tal, st = oracle.cast(prob)
    assert st["rejected"] == 0 and st["overflow"] == 0
    assert 2.7e6 < st["segments"] < 3.1e6
    assert np.all(tal > 0)


def test_batch_moments_closed_forms():
    """Two batches: sigma = |t1 - t2| (B/(B-1) (t1^2 + t2^2 - (t1+t2)^2/2) =
    (t1 - t2)^2); equal batches: sigma = 0; one batch: sigma = 0."""
    t1 = np.array([1.0, 3.0, 0.0, 2.5])
    t2 = np.array([2.0, 3.0, 5.0, 0.5])
    total, sig = oracle.batch_moments([t1, t2])
    np.testing.assert_allclose(total, t1 + t2)
    np.testing.assert_allclose(sig, np.abs(t1 - t2), rtol=1e-14, atol=1e-14)
    total, sig = oracle.batch_moments([t1, t1, t1])
    np.testing.assert_allclose(sig, 0.0, atol=1e-14)
    _, sig = oracle.batch_moments([t1])
    assert not sig.any()
    # sigma scales with sqrt(B) for B copies of the same two-valued spread
    a, b = np.array([1.0]), np.array([3.0])
    _, s4 = oracle.batch_moments([a, b, a, b])
    assert s4[0] == pytest.approx(np.sqrt(4 / 3 * (20 - 64 / 4)), rel=1e-14)


def test_point_detector_closed_forms():
    """Homogeneous medium: exp(-Sigma R)/(4 pi R^2) per unit weight; void: the
    bare 1/(4 pi R^2); a detector outside the mesh sees only the chord inside
    (vacuum outside); groups route by energy."""
    mesh = _mesh((4, 4, 4))
    sig = 0.7
    ev = _rays([[1.25, 2.0, 2.5], [3.5, 0.5, 0.5]], [[1, 0, 0], [0, 1, 0]], [1.0, 1e6], [2.0, 0.5])
    det = np.array([[3.0, 2.0, 2.5], [1.0, 3.0, 3.0]])
    prob = W.Problem("pd", mesh, [_const_table(sig)], np.array([1e-5, 10.0, 2e7]), ev)
    got = oracle.point_detector(prob, det)
    p = np.stack([ev["x"], ev["y"], ev["z"]], 1).astype(np.float64)
    want = np.zeros((2, 2))
    for i, g in enumerate([0, 1]):
        for k in range(2):
            R = np.linalg.norm(det[k] - p[i])
            want[k, g] += float(ev["wt"][i]) * np.exp(-sig * R) / (4 * np.pi * R * R)
    np.testing.assert_allclose(got, want, rtol=1e-13)
    # void: no attenuation
    vprob = W.Problem("pdv", mesh, [None], None, ev)
    got = oracle.point_detector(vprob, det)
    R = np.linalg.norm(det[None, :, :] - p[:, None, :], axis=2)
    np.testing.assert_allclose(got[:, 0], (ev["wt"].astype(np.float64)[:, None] / (4 * np.pi * R ** 2)).sum(0),
                               rtol=1e-13)
    # detector 2 cm beyond the +x face: attenuation only over the 4 - 1.25 cm inside
    far = np.array([[6.0, 2.0, 2.5]])
    one = W.Problem("pdf", mesh, [_const_table(sig)], None, W.take_rays(prob, [0]).rays)
    got = oracle.point_detector(one, far)
    R = 6.0 - 1.25
    assert got[0, 0] == pytest.approx(2.0 * np.exp(-sig * (4.0 - 1.25)) / (4 * np.pi * R * R), rel=1e-13)


def test_history_moments_closed_form():
    """Void 4x1x1 mesh, rays along +x from x = 0.5: chord 0.5 in cell 0 and 1
    in cells 1..3, times wt.  History 7 has two rays (wt 1 and 2), history 3
    one ray (wt 1), and one more history has no ray (N = 3).  Then
    x_7 = 3 l, x_3 = l per cell, S1 = 4 l, S2 = 10 l^2 and
    sigma^2 = 3/2 (10 - 16/3) l^2 = 7 l^2.  Squaring ray by ray instead of
    history by history would give S2 = 6 l^2 and sigma = l."""
    mesh = _mesh((4, 1, 1))
    ev = _rays([[0.5, 0.5, 0.5]] * 3, [[1, 0, 0]] * 3, 1.0, [1.0, 2.0, 1.0])
    prob = W.Problem("hist", mesh, [None], None, ev)
    l = np.array([0.5, 1.0, 1.0, 1.0])
    total, sig, s2 = oracle.history_moments(prob, np.array([7, 7, 3], np.uint32), 3)
    np.testing.assert_allclose(total, 4 * l, rtol=1e-15)
    np.testing.assert_allclose(s2, 10 * l * l, rtol=1e-15)
    np.testing.assert_allclose(sig, np.sqrt(7.0) * l, rtol=1e-14)
    # the same rays with N = 2 (no empty history): sigma^2 = 2 (10 - 8) l^2
    _, sig2, _ = oracle.history_moments(prob, np.array([7, 7, 3], np.uint32), 2)
    np.testing.assert_allclose(sig2, 2.0 * l, rtol=1e-14)
    # ray order and id values do not matter, only which rays share an id
    perm = [2, 0, 1]
    rays = {k: v[perm] for k, v in ev.items()}
    _, sig3, _ = oracle.history_moments(prob, np.array([1, 9, 9], np.uint32), 3, rays=rays)
    np.testing.assert_allclose(sig3, sig, rtol=1e-15)
    with pytest.raises(ValueError):
        oracle.history_moments(prob, np.array([1, 2, 3], np.uint32), 2)


# ------------------------------------------------- rectilinear (graded) meshes

def _rect(xe, ye, ze, material=None, rng=None, nmat=1):
    xe, ye, ze = (np.asarray(e, np.float64) for e in (xe, ye, ze))
    shape = (len(ze) - 1, len(ye) - 1, len(xe) - 1)
    if material is None:
        material = (np.zeros(shape, np.uint8) if rng is None
                    else rng.integers(0, nmat, size=shape).astype(np.uint8))
    return W.RectMesh(xe, ye, ze, np.asarray(material, np.uint8))


def _random_edges(rng, n, lo=-1.0):
    return lo + np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 2.0, n))])


def test_rect_uniform_edges_equal_uniform_mesh():
    """Edges x0 + j dx reproduce the uniform mesh's tally."""
    rng = np.random.default_rng(31)
    prob = _hetero_problem(rng, n=(5, 4, 3), n_rays=400, spacing=(0.7, 1.3, 0.9))
    m = prob.mesh
    rect = W.RectMesh(m.x0 + np.arange(m.nx + 1) * m.dx, m.y0 + np.arange(m.ny + 1) * m.dy,
                      m.z0 + np.arange(m.nz + 1) * m.dz, m.material)
    want, st0 = oracle.cast(prob, nthreads=1)
    got, st1 = oracle.cast(W.Problem("r", rect, prob.tables, None, prob.rays), nthreads=1)
    assert st0["segments"] == st1["segments"]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-300)


def test_rect_void_chords_are_cell_widths():
    """Void graded mesh, axis-aligned rays: every crossed cell scores wt times
    its own width (the start cell from the start point)."""
    xe, ye, ze = [0.0, 0.5, 0.7, 1.5, 3.0], [0.0, 1.0, 2.5], [0.0, 0.25, 1.0]
    mesh = _rect(xe, ye, ze)
    x0 = float(np.float32(0.2))
    prob = W.Problem("rv", mesh, [None], None,
                     _rays([[x0, 0.5, 0.5], [1.0, 2.0, 0.1]], [[1, 0, 0], [0, -1, 0]], 1.0, [2.0, 3.0]))
    tal, _ = oracle.cast(prob, nthreads=1)
    tal = tal.reshape(2, 2, 4)
    want = np.zeros((2, 2, 4))
    want[1, 0, :] = 2.0 * np.diff(xe)
    want[1, 0, 0] = 2.0 * (0.5 - x0)
    want[0, 1, 2] = 3.0 * (2.0 - 1.0)
    want[0, 0, 2] = 3.0 * 1.0
    np.testing.assert_allclose(tal, want, rtol=1e-15, atol=0)


def test_rect_axis_aligned_per_cell_scores():
    """Homogeneous graded mesh, ray along +x: cell i is entered at
    t_i = max(x_i - x_s, 0) with length l_i = x_{i+1} - max(x_i, x_s), and
    scores wt exp(-Sigma t_i)(1 - exp(-Sigma l_i))/Sigma (Eq. 4)."""
    rng = np.random.default_rng(32)
    xe = _random_edges(rng, 9)
    mesh = _rect(xe, [0.0, 1.0], [0.0, 1.0])
    sig = 0.8
    xs = float(np.float32(xe[0] + 0.3 * (xe[1] - xe[0])))
    prob = W.Problem("ra", mesh, [_const_table(sig)], None, _rays([xs, 0.5, 0.5], [1, 0, 0], 1.0, 2.0))
    tal, _ = oracle.cast(prob, nthreads=1)
    t = np.maximum(xe[:-1] - xs, 0.0)
    l = xe[1:] - np.maximum(xe[:-1], xs)
    np.testing.assert_allclose(tal, 2.0 * np.exp(-sig * t) * -np.expm1(-sig * l) / sig, rtol=1e-13)


def test_rect_dda_matches_brute_force_traversal():
    """Graded meshes: the grid walk's positive-length segments equal the
    sorted plane-crossing traversal's, cell for cell, to 1e-12 cm."""
    rng = np.random.default_rng(33)
    meshes = [_rect(_random_edges(rng, 6), _random_edges(rng, 4, -3.0), _random_edges(rng, 5, 2.0)),
              _rect(W.graded_edges(8, 0.06, 1.5, 1.0, 3.0), W.graded_edges(4, 0.2, 1.3, 0.7, 2.0),
                    [0.0, 20.0, 40.0])]
    n_checked = 0
    for mesh in meshes:
        lo, hi = np.array(mesh.lo), np.array(mesh.hi)
        ext = hi - lo
        edges = (mesh.xe, mesh.ye, mesh.ze)
        for i in range(3000):
            p = lo - 0.3 * ext + 1.6 * ext * rng.random(3)
            d = rng.normal(size=3)
            if i % 10 == 0:
                d[rng.integers(0, 3)] = 0.0
            if i % 37 == 0:  # start exactly on a plane
                k = rng.integers(0, 3)
                p[k] = edges[k][rng.integers(0, len(edges[k]))]
            nrm = np.linalg.norm(d)
            if nrm == 0:
                continue
            d = d / nrm
            c1, t1, l1 = oracle.trace_dda(mesh, p, d)
            keep = l1 > 0
            c2, t2, l2 = oracle.trace_brute(mesh, p, d)
            assert np.array_equal(c1[keep], c2), (p, d)
            np.testing.assert_allclose(l1[keep], l2, rtol=0, atol=1e-12)
            np.testing.assert_allclose(t1[keep], t2, rtol=0, atol=1e-12)
            n_checked += int(keep.sum())
    assert n_checked > 10000


def test_rect_inserted_plane_additivity():
    """Inserting a plane inside a column of cells (same material on both
    sides) splits their scores and leaves every sum unchanged."""
    rng = np.random.default_rng(34)
    prob = _hetero_problem(rng, n=(4, 3, 3), n_rays=300, spacing=(1.0, 1.0, 1.0))
    m = prob.mesh
    xe = m.x0 + np.arange(m.nx + 1) * m.dx
    ye = m.y0 + np.arange(m.ny + 1) * m.dy
    ze = m.z0 + np.arange(m.nz + 1) * m.dz
    cut = xe[1] + 0.37 * m.dx
    xs = np.concatenate([xe[:2], [cut], xe[2:]])
    mat = np.concatenate([m.material[:, :, :2], m.material[:, :, 1:2], m.material[:, :, 2:]], axis=2)
    split = W.RectMesh(xs, ye, ze, mat)
    coarse, _ = oracle.cast(prob, nthreads=1)
    fine, _ = oracle.cast(W.Problem("s", split, prob.tables, None, prob.rays), nthreads=1)
    fine = fine.reshape(m.nz, m.ny, m.nx + 1)
    folded = np.concatenate([fine[:, :, :1], fine[:, :, 1:2] + fine[:, :, 2:3], fine[:, :, 3:]], axis=2)
    np.testing.assert_allclose(folded.reshape(-1), coarse, rtol=1e-11, atol=1e-300)
    assert np.count_nonzero(fine[:, :, 2]) > 0


def test_rect_telescoping_invariant():
    """sum_i Sigma_i s_i = w (1 - exp(-tau_exit)) along every ray of a random
    graded mesh."""
    rng = np.random.default_rng(35)
    mesh = _rect(_random_edges(rng, 7), _random_edges(rng, 5), _random_edges(rng, 6), rng=rng, nmat=3)
    tables = [None] + [W.xs_table(rng, 60, 3, peak_lo=0.1, peak_hi=3.0) for _ in range(2)]
    lo, hi = np.array(mesh.lo), np.array(mesh.hi)
    n = 150
    pos = (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    rays = W.make_rays(pos[:, 0], pos[:, 1], pos[:, 2], d[:, 0], d[:, 1], d[:, 2],
                       W.log_uniform(rng, n), np.ones(n, np.float32))
    prob = W.Problem("rt", mesh, tables, None, rays)
    checked = 0
    for i in range(n):
        seg = oracle.ray_segments(prob, i)
        if len(seg["lens"]) == 0:
            continue
        tau = float(np.sum(seg["sigma"] * seg["lens"]))
        assert float(np.sum(seg["sigma"] * seg["score"])) == pytest.approx(-math.expm1(-tau), rel=1e-12,
                                                                           abs=1e-300)
        checked += 1
    assert checked > 100
