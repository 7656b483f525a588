"""Allocation failures through the C ABI, injected on the host.

vrc_debug_fail_alloc makes a chosen device or pinned-host allocation of the
library fail as if the GPU were out of memory, without asking the driver,
so no GPU is ever short of memory or faulted.  Each test makes the first,
second, ... allocation of one call fail in turn until the call succeeds.
Every failing call must return VRC_ERR_OOM, leave no device memory behind,
and leave the library usable: the call that finally succeeds, and the
casts after it, give the oracle's tally.  One test also provokes a genuine
failure, a tally larger than the device's memory, and then casts on a
small mesh: the failed cudaMalloc must not be reported later as the error
of an unrelated launch.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

LEAK_TOL = 4 << 20  # bytes lost at most: below the smallest large buffer here (the 32 MiB tally)


def _free(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _walk(vrc, call, max_allocs=64):
    """Runs call() with allocation k failing, k = 0, 1, ..., until it
    succeeds.  Returns (number of failures, the successful result)."""
    for k in range(max_allocs):
        vrc.vrc_debug_fail_alloc(k)
        try:
            res = call()
        except vrc.VrcError as e:
            assert e.code == vrc.VRC_ERR_OOM, (k, e)
            continue
        finally:
            vrc.vrc_debug_fail_alloc(-1)
        return k, res
    raise AssertionError(f"the call still failed with {max_allocs} allocations allowed")


def _problem(n_rays=20000):
    return W.slab_room(seed=1, n=64, n_rays=n_rays, n_points=1500, n_resonances=30)


def test_create_mesh_fails_cleanly_at_every_allocation(vrc):
    import torch
    prob = _problem()
    want, st = oracle.cast(prob)
    with vrc.context_for(prob) as warm:  # module loading and first-use costs outside the count
        vrc.vrc_cast_rays(warm, prob.rays)
        vrc.vrc_sync(warm)
    free0 = _free(torch)
    fails, ctx = _walk(vrc, lambda: vrc.vrc_create_mesh(prob.mesh, prob.n_materials, prob.group_edges))
    assert fails >= 2, fails  # at least the material array and the tally
    assert free0 - _free(torch) <= LEAK_TOL + 8 * ctx.tally_size  # only the live context's tally
    try:
        for m, t in enumerate(prob.tables):
            vrc.vrc_load_xs(ctx, m, *((None, None) if t is None else t))
        vrc.vrc_cast_rays(ctx, prob.rays)
        rc, stats = vrc.vrc_sync(ctx)
        got, _ = vrc.vrc_read_tally(ctx)
        assert rc == vrc.VRC_OK and stats["segments"] == st["segments"]
        assert H.rel_err_report(want, got)["max_rel"] <= 1e-4
    finally:
        ctx.close()
    assert free0 - _free(torch) <= LEAK_TOL


@pytest.mark.parametrize("where", ["device", "host", "host_chunked"])
def test_failed_cast_adds_nothing(vrc, where):
    """A cast whose allocation fails (cross-section tables, sort scratch, ray
    staging, upload slots) adds nothing; the next identical cast gives the
    oracle's tally.  host_chunked is a host batch above 2^22 rays, uploaded
    and cast in chunks: every buffer of every chunk is sized before the
    first chunk is cast."""
    import torch
    prob = _problem(n_rays=(1 << 22) + 4096 if where == "host_chunked" else 20000)
    want, st = oracle.cast(prob)
    rays = ({k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()} if where == "device"
            else prob.rays)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, sort=1))
    try:
        def cast():
            vrc.vrc_cast_rays(ctx, rays)
            return vrc.vrc_sync(ctx)

        zero = np.zeros(ctx.tally_size)
        for k in range(64):
            vrc.vrc_debug_fail_alloc(k)
            try:
                rc, stats = cast()
            except vrc.VrcError as e:
                assert e.code == vrc.VRC_ERR_OOM, (k, e)
                rc2, s2 = vrc.vrc_sync(ctx)
                assert rc2 == vrc.VRC_OK and s2["segments"] == 0 and s2["rays"] == 0, (k, s2)
                np.testing.assert_array_equal(vrc.vrc_read_tally(ctx)[0], zero)
                continue
            finally:
                vrc.vrc_debug_fail_alloc(-1)
            break
        else:
            raise AssertionError("the cast never succeeded")
        assert k >= 2, k  # the tables and the sort scratch at least
        got, _ = vrc.vrc_read_tally(ctx)
        assert rc == vrc.VRC_OK and stats["segments"] == st["segments"]
        assert H.rel_err_report(want, got)["max_rel"] <= 1e-4
    finally:
        ctx.close()


def test_surrogate_training_fails_cleanly(vrc):
    prob = W.surrogate_mesh(seed=4, n=16, n_rays=1 << 14, n_materials=4, n_points=2000,
                            n_resonances=20)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32))
    try:
        opts = vrc.vrc_default_surrogate_options(steps=200, tol=0.05)
        fails, rep = _walk(vrc, lambda: vrc.vrc_train_surrogate(ctx, opts))
        assert fails >= 1 and rep["bins"] > 0, (fails, rep)
        # the trained network is in place and a surrogate cast runs
        vrc.vrc_set_xs_mode(ctx, vrc.VRC_XS_SURROGATE)
        vrc.vrc_cast_rays(ctx, prob.rays)
        rc, stats = vrc.vrc_sync(ctx)
        assert rc == vrc.VRC_OK and stats["rays"] == prob.n_rays
    finally:
        ctx.close()


def test_batch_plan_and_stream_buffers_fail_cleanly(vrc):
    import torch
    probs = W.batched_problems(seed=3, n_problems=3, side_lo=16, side_hi=24, rays_lo=2e3, rays_hi=5e3)
    rays = [{k: torch.from_numpy(v).cuda() for k, v in p.rays.items()} for p in probs]
    ctxs = [vrc.context_for(p) for p in probs]
    try:
        for c, p in zip(ctxs, probs):  # tables on the device before the plan's walk
            vrc.vrc_cast_rays(c, W.take_rays(p, slice(0, 1)).rays)
            vrc.vrc_sync(c)
            vrc.vrc_reset_tally(c)
        fails, batch = _walk(vrc, lambda: vrc.vrc_batch_create(ctxs, rays))
        assert fails >= 1, fails
        try:
            vrc.vrc_batch_launch(batch)
            torch.cuda.synchronize()
        finally:
            batch.close()
        for c, p in zip(ctxs, probs):
            want, st = oracle.cast(p)
            rc, stats = vrc.vrc_sync(c)
            got, _ = vrc.vrc_read_tally(c)
            assert rc == vrc.VRC_OK and stats["segments"] == st["segments"]
            assert H.rel_err_report(want, got)["max_rel"] <= 1e-4
        fails, rs = _walk(vrc, lambda: vrc.RayStream(ctxs[0], capacity=1024, n_buffers=2))
        assert fails >= 1, fails  # the pinned and device buffers
        rs.close()
    finally:
        for c in ctxs:
            c.close()


def test_genuine_out_of_memory_then_small_cast(vrc):
    """A 360^3 mesh with 1,024 groups asks for a 382 GB tally, more than the
    device has: VRC_ERR_OOM, nothing created; a small cast then succeeds."""
    import torch
    n, groups = 360, 1024
    free0 = _free(torch)
    assert 8 * n ** 3 * groups > torch.cuda.mem_get_info()[1]
    mesh = W.Mesh(n, n, n, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, np.zeros((n, n, n), np.uint8))
    with pytest.raises(vrc.VrcError) as ei:
        vrc.vrc_create_mesh(mesh, 1, W.log_group_edges(groups))
    assert ei.value.code == vrc.VRC_ERR_OOM, ei.value
    # nothing kept (the driver may even hand back memory it had cached)
    assert free0 - _free(torch) <= LEAK_TOL
    prob = _problem(n_rays=4096)
    want, st = oracle.cast(prob)
    with vrc.context_for(prob) as ctx:
        vrc.vrc_cast_rays(ctx, prob.rays)
        rc, stats = vrc.vrc_sync(ctx)
        got, _ = vrc.vrc_read_tally(ctx)
    assert rc == vrc.VRC_OK and stats["segments"] == st["segments"]
    assert H.rel_err_report(want, got)["max_rel"] <= 1e-4


def test_history_moments_and_detectors_fail_cleanly(vrc):
    """Per-history moments and point detectors with every allocation of a
    first call failing in turn: a failed call folds nothing into the moments
    and counts none of its histories; the call that succeeds gives the
    oracle's per-history totals and detector flux."""
    prob = W.slab_room(seed=9, n=16, n_rays=6000, n_points=400, n_resonances=6, n_groups=3)
    rng = np.random.default_rng(10)
    N = 2000
    hist = rng.integers(0, N, size=prob.n_rays).astype(np.uint32)
    want_total, _, _ = oracle.history_moments(prob, hist, N)
    det = np.array([[8.3, 7.7, 9.1], [2.0, 3.0, 4.0]])
    want_flux = oracle.point_detector(prob, det)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, sort=1))
    try:
        vrc.vrc_moments_enable(ctx, vrc.VRC_MOMENTS_HISTORY)
        fails, _ = _walk(vrc, lambda: vrc.vrc_cast_histories(ctx, prob.rays, hist, N))
        assert fails >= 1, fails
        total, _, samples = vrc.vrc_moments_read(ctx)
        assert samples == N
        assert H.rel_err_report(want_total, total)["max_rel"] <= 1e-4
        fails, got = _walk(vrc, lambda: vrc.vrc_detector_flux(ctx, prob.rays, det))
        assert fails >= 1, fails
        sel = want_flux > 0
        assert (np.abs(got[sel] - want_flux[sel]) / want_flux[sel]).max() <= 1e-4
    finally:
        ctx.close()
