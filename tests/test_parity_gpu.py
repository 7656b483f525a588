"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance: the plain form and the FP32 form must both match the oracle to
<= 1e-4 relative per (group, cell) wherever the oracle tally is >= 1e-30
(the Eq. 7 relative difference; cells below that floor are held to an
absolute 1e-28).  The floating-point budget behind 1e-4: float32 cross
sections and path lengths (2^-24 each), float32 exponentials (a few ulp) and,
in the FP32 form, a compensated float32 optical depth: a few 1e-7 per score,
far below 1e-4; the margin covers cells whose only contributions are short
corner clips, where the double-float crossing parameters (about 2^-46
relative) dominate.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
ABS_BELOW = 1e-28
FORMS = {"plain": 0, "fp32": 1}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _device_rays(torch, rays):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}


def run_gpu(vrc, torch, prob, form, rays=None, on_device=True, options=None, batches=1):
    opts = options or vrc.vrc_default_options(form=form)
    ctx = vrc.context_for(prob, opts)
    try:
        rays = prob.rays if rays is None else rays
        n = len(rays["x"])
        for b in range(batches):
            sl = slice(n * b // batches, n * (b + 1) // batches)
            part = {k: v[sl] for k, v in rays.items()}
            if on_device:
                part = _device_rays(torch, part)
            stream = torch.cuda.current_stream()
            vrc.vrc_cast_rays(ctx, part, stream=stream)
        rc, stats = vrc.vrc_sync(ctx, torch.cuda.current_stream())
        tally, rc2 = vrc.vrc_read_tally(ctx)
        assert rc == rc2
        return tally, rc, stats
    finally:
        ctx.close()


def assert_parity(want, got, tol=REL_TOL):
    rep = H.rel_err_report(want, got)
    assert rep["max_rel"] <= tol, rep
    assert rep["max_abs_below"] <= ABS_BELOW, rep
    return rep


# ---------------------------------------------------------------- golden cases

@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("case", H.golden_cases(), ids=lambda c: c["name"])
def test_golden_closed_forms_gpu(vrc, torch_cuda, case, form):
    prob = H.golden_problem(case)
    want = H.golden_expected(case, prob)
    got, rc, _ = run_gpu(vrc, torch_cuda, prob, FORMS[form])
    assert rc == vrc.VRC_OK
    nz = want != 0
    # float32 lengths and sigma (2^-24 each); the FP32 form adds float32
    # exponentials (expf within 2 ulp) and a difference of two of them
    np.testing.assert_allclose(got[nz], want[nz], rtol=1e-6 if form == "plain" else 2e-6)
    assert np.all(np.abs(got[~nz]) <= 1e-12)


# ---------------------------------------------------------------- workloads

@pytest.fixture(scope="module")
def uniform32():
    prob = W.uniform_small()  # 32^3, 2 materials, 2^17 rays, seed 0 (full size)
    want, st = oracle.cast(prob)
    return prob, want, st


@pytest.mark.parametrize("form", sorted(FORMS))
def test_uniform32_full_vs_oracle(vrc, torch_cuda, uniform32, form):
    prob, want, st = uniform32
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form])
    assert rc == vrc.VRC_OK
    assert stats["rays"] == prob.n_rays and stats["rejected"] == 0 and stats["overflow"] == 0
    assert stats["segments"] == st["segments"]
    rep = assert_parity(want, got)
    assert rep["n_cells"] == prob.tally_size


@pytest.fixture(scope="module")
def slab_small():
    prob = W.slab_room(seed=1, n=48, n_rays=1 << 16, n_points=2000, n_resonances=40)
    want, st = oracle.cast(prob)
    return prob, want, st


@pytest.mark.parametrize("form", sorted(FORMS))
def test_slab_groups_vs_oracle(vrc, torch_cuda, slab_small, form):
    prob, want, st = slab_small
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form])
    assert rc == vrc.VRC_OK
    assert stats["segments"] == st["segments"]
    assert_parity(want, got)


@pytest.fixture(scope="module")
def lattice_small():
    prob = W.pin_lattice(seed=2, pins=3, cells_per_pin=32, nz=6, n_rays=1 << 15, n_points=2000,
                         n_resonances=40)
    want, st = oracle.cast(prob)
    return prob, want, st


@pytest.mark.parametrize("form", sorted(FORMS))
def test_pin_lattice_vs_oracle(vrc, torch_cuda, lattice_small, form):
    prob, want, st = lattice_small
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form])
    assert rc == vrc.VRC_OK
    assert stats["segments"] == st["segments"]
    assert_parity(want, got)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_ragged_mesh_and_offsets(vrc, torch_cuda, form):
    """Non-cubic mesh, non-unit and unequal spacings, shifted origin, rays
    starting inside and outside the box, a ragged ray count."""
    rng = np.random.default_rng(21)
    nx, ny, nz = 37, 5, 19
    mat = rng.integers(0, 5, size=(nz, ny, nx)).astype(np.uint8)
    mesh = W.Mesh(nx, ny, nz, -3.25, 11.0, 0.125, 0.3, 2.5, 0.0625, mat)
    tables = [W.xs_table(rng, 300, 4, peak_lo=0.1, peak_hi=30.0) for _ in range(5)]
    tables[2] = None
    n = 10007
    lo, hi = np.array(mesh.lo), np.array(mesh.hi)
    pos = lo - 0.3 * (hi - lo) + 1.6 * (hi - lo) * rng.random((n, 3))
    d = rng.normal(size=(n, 3))
    rays = W.make_rays(*(pos[:, k].astype(np.float32) for k in range(3)),
                       *(d[:, k].astype(np.float32) for k in range(3)), W.log_uniform(rng, n),
                       rng.lognormal(0, 0.5, n).astype(np.float32))
    prob = W.Problem("ragged", mesh, tables, W.log_group_edges(3, 1e-3, 1e6), rays)
    want, st = oracle.cast(prob)
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form])
    assert rc == vrc.VRC_OK
    assert stats["segments"] == st["segments"]
    assert_parity(want, got)


# ---------------------------------------------------------------- edge cases

def _tiny():
    rng = np.random.default_rng(3)
    mat = rng.integers(0, 2, size=(4, 4, 4)).astype(np.uint8)
    mesh = W.Mesh(4, 4, 4, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat)
    return mesh, [W.xs_table(rng, 50, 2), None]


def test_empty_batch_is_noop(vrc, torch_cuda):
    mesh, tables = _tiny()
    prob = W.Problem("e", mesh, tables, None, W.make_rays(*([np.zeros(0, np.float32)] * 8)))
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, 0)
    assert rc == vrc.VRC_OK and stats["rays"] == 0 and not got.any()


def test_bad_rays_are_reported_and_skipped(vrc, torch_cuda):
    mesh, tables = _tiny()
    rng = np.random.default_rng(4)
    n = 64
    pos = (4 * rng.random((n, 3))).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    E = W.log_uniform(rng, n)
    wt = np.ones(n, np.float32)
    rays = W.make_rays(pos[:, 0], pos[:, 1], pos[:, 2], d[:, 0], d[:, 1], d[:, 2], E, wt)
    rays["x"][3] = np.nan
    rays["u"][5] = rays["v"][5] = rays["w"][5] = 0.0
    rays["E"][7] = -1.0
    rays["wt"][9] = np.inf
    prob = W.Problem("bad", mesh, tables, None, rays)
    want, st = oracle.cast(prob)
    assert st["rejected"] == 4
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, 0)
    assert rc == vrc.VRC_ERR_NONFINITE
    assert stats["rejected"] == 4 and stats["rays"] == n
    assert_parity(want, got)


def test_host_rays_equal_device_rays_and_batches_accumulate(vrc, torch_cuda, uniform32):
    prob, want, _ = uniform32
    a, _, sa = run_gpu(vrc, torch_cuda, prob, 0, on_device=False)
    b, _, sb = run_gpu(vrc, torch_cuda, prob, 0, on_device=True, batches=7)
    assert sa["segments"] == sb["segments"]
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_reset_per_volume_and_device_pointer(vrc, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(8)
    mat = np.zeros((3, 3, 3), np.uint8)
    mesh = W.Mesh(3, 3, 3, 0.0, 0.0, 0.0, 0.5, 2.0, 0.25, mat)
    prob = W.Problem("v", mesh, [W.xs_table(rng, 30, 1)], None,
                     W.make_rays(*(np.full(5, c, np.float32) for c in (0.7, 3.1, 0.3)),
                                 *(np.full(5, c, np.float32) for c in (0.3, -0.2, 1.0)),
                                 np.full(5, 2.0, np.float32), np.full(5, 1.5, np.float32)))
    want, _ = oracle.cast(prob)
    ctx = vrc.context_for(prob)
    try:
        vrc.vrc_cast_rays(ctx, _device_rays(torch, prob.rays))
        raw, rc = vrc.vrc_read_tally(ctx)
        pv, rc2 = vrc.vrc_read_tally(ctx, flags=vrc.VRC_PER_VOLUME)
        assert rc == rc2 == vrc.VRC_OK
        np.testing.assert_allclose(raw, want, rtol=1e-6)
        np.testing.assert_allclose(pv, want / (0.5 * 2.0 * 0.25), rtol=1e-6)
        ptr = vrc.vrc_tally_device_ptr(ctx)
        assert ptr != 0
        vrc.vrc_reset_tally(ctx)
        again, _ = vrc.vrc_read_tally(ctx)
        assert not again.any()
        _, stats = vrc.vrc_sync(ctx)
        assert stats["segments"] == 0
    finally:
        ctx.close()


def test_missing_table_is_state_error(vrc, torch_cuda):
    mesh, tables = _tiny()
    ctx = vrc.vrc_create_mesh(mesh, 2)
    try:
        vrc.vrc_load_xs(ctx, 0, *tables[0])  # material 1 is used but never loaded
        rays = W.make_rays(*(np.full(1, 0.5, np.float32) for _ in range(3)),
                           np.ones(1, np.float32), np.zeros(1, np.float32),
                           np.zeros(1, np.float32), np.ones(1, np.float32), np.ones(1, np.float32))
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_cast_rays(ctx, rays)
        assert ei.value.code == vrc.VRC_ERR_STATE
    finally:
        ctx.close()


def test_ray_starting_on_faces_and_parallel_to_planes(vrc, torch_cuda):
    """Starts exactly on grid planes, directions with zero components, a ray
    sliding along a face, and rays that only clip a corner."""
    mesh, tables = _tiny()
    P = [(1.0, 2.0, 3.0), (0.0, 0.5, 0.5), (4.0, 0.5, 0.5), (2.0, 2.0, 0.25), (0.5, 0.5, 0.5),
         (1.0, 1.0, 1.0), (3.999, 0.001, 2.5)]
    D = [(1, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 0, 1), (0, 1, 1), (1, 1, 1), (1, -1, 0.001)]
    n = len(P)
    rays = W.make_rays(*(np.array([p[k] for p in P], np.float32) for k in range(3)),
                       *(np.array([d[k] for d in D], np.float32) for k in range(3)),
                       np.full(n, 3.0, np.float32), np.ones(n, np.float32))
    prob = W.Problem("faces", mesh, tables, None, rays)
    want, st = oracle.cast(prob)
    for form in (0, 1):
        got, rc, stats = run_gpu(vrc, torch_cuda, prob, form)
        assert rc == vrc.VRC_OK
        assert_parity(want, got, tol=1e-5)


# ---------------------------------------------------------------- ray sort

@pytest.mark.parametrize("form", sorted(FORMS))
def test_sort_on_off_same_tally(vrc, torch_cuda, slab_small, form):
    """Sorting by (group, crossed cells) changes only the float64 summation
    order of the tally."""
    prob, want, st = slab_small
    a, rc_a, sa = run_gpu(vrc, torch_cuda, prob, FORMS[form],
                          options=vrc.vrc_default_options(form=FORMS[form], sort=0))
    b, rc_b, sb = run_gpu(vrc, torch_cuda, prob, FORMS[form],
                          options=vrc.vrc_default_options(form=FORMS[form], sort=1,
                                                          sort_len_buckets=17))
    assert rc_a == rc_b == vrc.VRC_OK
    assert sa["segments"] == sb["segments"] == st["segments"]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-300)
    assert_parity(want, b)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_ray_assignment_same_tally(vrc, torch_cuda, slab_small, form):
    """How the cast hands rays to warps (interleaved rounds, or chunks of 32,
    64 or 2048 sorted rays from a counter) changes only the float64
    summation order: every ray's scores are the same bits in each loop, so
    the tallies agree to rounding of the sums and the segment counts
    exactly."""
    prob, want, st = slab_small
    out = {}
    for rpw in (-1, 32, 64, 2048):
        t, rc, sx = run_gpu(vrc, torch_cuda, prob, FORMS[form],
                            options=vrc.vrc_default_options(form=FORMS[form], sort=1, rays_per_warp=rpw))
        assert rc == vrc.VRC_OK
        assert sx["segments"] == st["segments"] and sx["rays"] == prob.n_rays
        out[rpw] = t
    for rpw in (32, 64, 2048):
        np.testing.assert_allclose(out[rpw], out[-1], rtol=1e-12, atol=1e-300)
    assert_parity(want, out[32])


def test_sort_with_rejected_and_out_of_group_rays(vrc, torch_cuda):
    """Rejected rays and rays outside every group land in the last key and are
    still reported; a ragged count that is not a multiple of the chunk."""
    rng = np.random.default_rng(31)
    mat = rng.integers(0, 3, size=(9, 7, 11)).astype(np.uint8)
    mesh = W.Mesh(11, 7, 9, 0.5, -2.0, 1.0, 0.9, 1.7, 0.6, mat)
    tables = [W.xs_table(rng, 200, 3), None, W.xs_table(rng, 150, 2)]
    n = 20011
    lo, hi = np.array(mesh.lo), np.array(mesh.hi)
    pos = lo - 0.2 * (hi - lo) + 1.4 * (hi - lo) * rng.random((n, 3))
    d = rng.normal(size=(n, 3))
    rays = W.make_rays(*(pos[:, k].astype(np.float32) for k in range(3)),
                       *(d[:, k].astype(np.float32) for k in range(3)),
                       W.log_uniform(rng, n, 1e-6, 1e8), np.ones(n, np.float32))
    bad = rng.choice(n, 50, replace=False)
    rays["w"][bad[:25]] = np.nan
    rays["E"][bad[25:]] = 0.0
    edges = W.log_group_edges(5, 1e-4, 1e7)  # some energies fall outside
    prob = W.Problem("sortmix", mesh, tables, edges, rays)
    want, st = oracle.cast(prob)
    for sort in (0, 1):
        got, rc, stats = run_gpu(vrc, torch_cuda, prob, 1,
                                 options=vrc.vrc_default_options(form=1, sort=sort))
        assert rc == vrc.VRC_ERR_NONFINITE
        assert stats["rejected"] == 50 and stats["rays"] == n
        assert stats["segments"] == st["segments"]
        assert_parity(want, got)


def test_plain_form_keeps_float64_range_deep_in_attenuation(vrc, torch_cuda):
    """Rays along +x through 200 cells of flat Sigma = 2.5 /cm, weights up to
    3e38: cell i's Eq. 4 score is wt e^{-Sigma (i - x0)} (1 - e^{-Sigma})/Sigma
    down to optical depth 500 (2e-179 for the largest weight), far past the
    float32 underflow at depth 104.  The plain form must hold every cell to
    the closed form at 1e-11 (about 2 ulp per factor over 200 factors); the
    ray count (37) leaves a partial warp."""
    n_cells, sig = 200, 2.5
    mat = np.zeros((1, 1, n_cells), np.uint8)
    mesh = W.Mesh(n_cells, 1, 1, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, mat)
    table = (np.array([1e-5, 2e7]), np.array([sig, sig]))
    n = 37
    x0 = np.float32(0.25)
    wt = (np.float32(3e38) / np.float32(2.0) ** np.arange(n, dtype=np.float32)).astype(np.float32)
    f = lambda v: np.full(n, v, np.float32)  # noqa: E731
    rays = W.make_rays(f(x0), f(0.5), f(0.5), f(1.0), f(0.0), f(0.0), f(1.0e3), wt)
    prob = W.Problem("deep", mesh, [table], None, rays)
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS["plain"])
    assert rc == vrc.VRC_OK and stats["segments"] == n * n_cells
    tau_in = sig * (np.arange(n_cells) - float(x0))
    tau_in[0] = 0.0
    length = np.ones(n_cells)
    length[0] = 1.0 - float(x0)
    per_unit = np.exp(-tau_in) * -np.expm1(-sig * length) / sig
    want = per_unit * wt.astype(np.float64).sum()
    assert want[-1] > 1e-190
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=0)
    fp32, _, _ = run_gpu(vrc, torch_cuda, prob, FORMS["fp32"])
    assert not fp32[60:].any()  # the float32 form underflows past depth ~104


@pytest.mark.parametrize("block", [32, 96, 224])
@pytest.mark.parametrize("form", sorted(FORMS))
def test_block_sizes_vs_oracle(vrc, torch_cuda, uniform32, form, block):
    """Other thread-block shapes of the cast: one warp, and odd warp counts
    per block (the plain form's per-warp queues are carved from the block's
    shared memory by warp index)."""
    prob, want, st = uniform32
    opts = vrc.vrc_default_options(form=FORMS[form], block=block)
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form], options=opts)
    assert rc == vrc.VRC_OK
    assert stats["segments"] == st["segments"]
    assert_parity(want, got)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_weight_extremes_vs_oracle(vrc, torch_cuda, uniform32, form):
    """Weights are only a factor of Eq. 4: negative weights give the negated
    tally, zero weights score nothing, and weights from 1e-30 to 1e30 scale
    their rays' scores, all as in the oracle."""
    prob, _, st = uniform32
    n = prob.n_rays
    rng = np.random.default_rng(31)
    wt = (10.0 ** rng.uniform(-30, 30, n)).astype(np.float32)
    wt[rng.random(n) < 0.1] = 0.0
    wt = -wt
    rays = dict(prob.rays, wt=wt)
    p2 = W.Problem("weights", prob.mesh, prob.tables, prob.group_edges, rays)
    want, st2 = oracle.cast(p2)
    assert st2["segments"] == st["segments"]
    got, rc, stats = run_gpu(vrc, torch_cuda, p2, FORMS[form])
    assert rc == vrc.VRC_OK and stats["segments"] == st["segments"]
    assert (want <= 0).all() and want.min() < -1e20
    assert_parity(want, got)
