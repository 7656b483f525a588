"""Rectilinear (non-uniform Cartesian) meshes: CUDA path vs the FP64 oracle,
cell by cell, through the C ABI.  Same bar as the uniform mesh: <= 1e-4
relative per (group, cell) where the oracle tally is >= 1e-30, and the same
positive-length segment count."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H
from tests.test_parity_gpu import FORMS, assert_parity, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _graded():
    return W.graded_assembly(seed=5, pins=4, reflector=8.0, nz=5, height=100.0, n_rays=40000,
                             n_points=500, n_resonances=8)


def _random_rect(seed, n=(9, 7, 6), nmat=4, n_rays=20000, groups=3):
    """Random plane positions (widths 0.05..2 cm), random materials (0 void),
    starts uniform over a box 20% larger than the mesh, one in 25 placed
    exactly on a plane, one in 10 axis-parallel."""
    rng = np.random.default_rng(seed)
    edges = [lo + np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 2.0, k))])
             for lo, k in zip((-1.0, 0.5, 3.0), n)]
    mat = rng.integers(0, nmat, size=(n[2], n[1], n[0])).astype(np.uint8)
    mesh = W.RectMesh(*edges, mat)
    tables = [None] + [W.xs_table(rng, 200, 4) for _ in range(nmat - 1)]
    lo, hi = np.array(mesh.lo), np.array(mesh.hi)
    ext = hi - lo
    pos = lo - 0.1 * ext + 1.2 * ext * rng.random((n_rays, 3))
    on_plane = np.flatnonzero(np.arange(n_rays) % 25 == 0)
    for i in on_plane:
        k = rng.integers(0, 3)
        pos[i, k] = edges[k][rng.integers(0, len(edges[k]))]
    d = rng.normal(size=(n_rays, 3))
    par = np.flatnonzero(np.arange(n_rays) % 10 == 3)
    d[par, rng.integers(0, 3, par.size)] = 0.0
    pos = pos.astype(np.float32)
    d = d.astype(np.float32)
    rays = W.make_rays(pos[:, 0], pos[:, 1], pos[:, 2], d[:, 0], d[:, 1], d[:, 2],
                       W.log_uniform(rng, n_rays), rng.lognormal(0, 0.5, n_rays).astype(np.float32))
    return W.Problem("rect", mesh, tables, W.log_group_edges(groups), rays)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_graded_assembly_parity(vrc, torch_cuda, form):
    prob = _graded()
    want, st = oracle.cast(prob)
    for on_device in (True, False):
        got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form], on_device=on_device)
        assert rc == vrc.VRC_OK
        rep = assert_parity(want, got)
        assert stats["segments"] == st["segments"]
    print(f"graded {prob.mesh.nx}x{prob.mesh.ny}x{prob.mesh.nz} form={form}: max rel {rep['max_rel']:.2e}, "
          f"{st['segments']} segments")


@pytest.mark.parametrize("form", sorted(FORMS))
def test_random_rect_parity(vrc, torch_cuda, form):
    prob = _random_rect(41)
    want, st = oracle.cast(prob)
    got, rc, stats = run_gpu(vrc, torch_cuda, prob, FORMS[form])
    assert rc == vrc.VRC_OK
    rep = assert_parity(want, got)
    assert stats["segments"] == st["segments"]
    print(f"random rect form={form}: max rel {rep['max_rel']:.2e}")


def test_rect_uniform_edges_match_uniform_mesh(vrc, torch_cuda):
    """Edges x0 + j dx: the rectilinear walk reproduces the uniform walk."""
    prob = W.slab_room(seed=3, n=20, n_rays=20000, n_points=300, n_resonances=4, n_groups=2)
    m = prob.mesh
    rect = W.RectMesh(m.x0 + np.arange(m.nx + 1) * m.dx, m.y0 + np.arange(m.ny + 1) * m.dy,
                      m.z0 + np.arange(m.nz + 1) * m.dz, m.material)
    rprob = W.Problem("r", rect, prob.tables, prob.group_edges, prob.rays)
    a, _, sa = run_gpu(vrc, torch_cuda, prob, 1)
    b, _, sb = run_gpu(vrc, torch_cuda, rprob, 1)
    assert sa["segments"] == sb["segments"]
    assert H.rel_err_report(a, b)["max_rel"] <= 1e-5


def test_rect_per_volume(vrc, torch_cuda):
    prob = _random_rect(42, n_rays=4000)
    m = prob.mesh
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=0))
    try:
        vrc.vrc_cast_rays(ctx, prob.rays)
        raw, _ = vrc.vrc_read_tally(ctx)
        per, _ = vrc.vrc_read_tally(ctx, flags=vrc.VRC_PER_VOLUME)
        vol = (np.diff(m.ze)[:, None, None] * np.diff(m.ye)[None, :, None]
               * np.diff(m.xe)[None, None, :]).reshape(-1)
        np.testing.assert_allclose(per, raw / np.tile(vol, prob.n_groups), rtol=1e-14, atol=0)
    finally:
        ctx.close()


def test_rect_history_moments(vrc, torch_cuda):
    """Per-history moments on a rectilinear mesh (the table bound uses the
    plane positions)."""
    prob = _random_rect(43, n_rays=3000, groups=2)
    rng = np.random.default_rng(44)
    hist = rng.integers(0, 400, prob.n_rays).astype(np.uint32)
    N = 450
    want_total, want_sigma, _ = oracle.history_moments(prob, hist, N)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=1))
    try:
        vrc.vrc_moments_enable(ctx, vrc.VRC_MOMENTS_HISTORY)
        vrc.vrc_cast_histories(ctx, prob.rays, hist, N)
        total, sigma, samples = vrc.vrc_moments_read(ctx)
        assert samples == N
        assert H.rel_err_report(want_total, total)["max_rel"] <= 1e-4
        big = (want_sigma > 1e-2 * want_total) & (want_total >= 1e-30)
        assert big.sum() > 100
        assert np.max(np.abs(sigma[big] - want_sigma[big]) / want_sigma[big]) <= 1e-3
    finally:
        ctx.close()


def test_rect_unsupported_forms_refuse(vrc, torch_cuda):
    prob = _random_rect(45, n_rays=100)
    ctx = vrc.context_for(prob)
    try:
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_detector_flux(ctx, prob.rays, np.array([[0.0, 1.0, 4.0]]))
        assert ei.value.code == vrc.VRC_ERR_ARG
        dev = {k: torch_cuda.from_numpy(v).cuda() for k, v in prob.rays.items()}
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_cast_batched([ctx], [dev])
        assert ei.value.code == vrc.VRC_ERR_ARG
    finally:
        ctx.close()
