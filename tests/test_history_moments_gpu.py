"""Per-history tally moments (the standard deviation behind Eqs. 5 and 8)
against the oracle's literal per-history sums: total and sigma per cell, with
history ids scattered through the ray order, histories without rays, and the
histories split over two calls (host rays, then device rays)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

EMPTY = 40  # histories without rays


def _histories(n_rays, seed):
    """History ids: run lengths 1..24 (rays per history), then ray order and
    id values shuffled so a history's rays are not contiguous."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(1, 25, size=n_rays)
    ids = np.repeat(np.arange(lengths.size), lengths)[:n_rays]
    n_hist = int(ids.max()) + 1
    relabel = rng.permutation(np.arange(n_hist, dtype=np.uint32) * 7919 + 11)
    return relabel[ids][rng.permutation(n_rays)].astype(np.uint32), n_hist


def _sigma_bound(s1, s2, want_sigma, n_with_rays, N):
    """|sigma' - sigma| bound when every history score x_h carries an error
    d_h <= 1e-4 x_h + 1e-30 (scores are >= 0): propagated through
    var = N/(N-1) (sum x_h^2 - S1^2/N)."""
    eps, tiny = 1e-4, 1e-30
    sum_xd = eps * s2 + tiny * s1
    sum_dd = eps * eps * s2 + 2 * eps * tiny * s1 + n_with_rays * tiny * tiny
    sum_d = eps * s1 + n_with_rays * tiny
    dv = (N / (N - 1.0)) * (2 * sum_xd + sum_dd + 2 * s1 * sum_d / N + sum_d * sum_d / N)
    return np.minimum(dv / np.maximum(want_sigma, 1e-300), np.sqrt(dv))


@pytest.mark.parametrize("sort", [0, 1], ids=["unsorted", "sorted"])
@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_history_moments_match_oracle(vrc, form, sort):
    import torch
    prob = W.slab_room(seed=9, n=16, n_rays=12000, n_points=400, n_resonances=6, n_groups=3)
    hist, n_hist = _histories(prob.n_rays, seed=10)
    N = n_hist + EMPTY
    want_total, want_sigma, want_s2 = oracle.history_moments(prob, hist, N)

    # two calls: histories with an even id, then the rest (each complete)
    first = np.flatnonzero(hist % 2 == 0)
    second = np.flatnonzero(hist % 2 == 1)
    n_first = len(np.unique(hist[first]))
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form, sort=sort))
    try:
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_cast_histories(ctx, prob.rays, hist, N)
        assert ei.value.code == vrc.VRC_ERR_STATE
        vrc.vrc_moments_enable(ctx, vrc.VRC_MOMENTS_HISTORY)
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_moments_fold(ctx)
        assert ei.value.code == vrc.VRC_ERR_STATE
        host = {k: np.ascontiguousarray(v[first]) for k, v in prob.rays.items()}
        vrc.vrc_cast_histories(ctx, host, hist[first], n_first + EMPTY)
        dev = {k: torch.from_numpy(np.ascontiguousarray(v[second])).cuda() for k, v in prob.rays.items()}
        hdev = torch.from_numpy(hist[second].view(np.int32).copy()).cuda()
        vrc.vrc_cast_histories(ctx, dev, hdev, N - n_first - EMPTY)
        vrc.vrc_cast_histories(ctx, W.take_rays(prob, []).rays, np.zeros(0, np.uint32), 0)
        total, sigma, samples = vrc.vrc_moments_read(ctx)
        rc, stats = vrc.vrc_sync(ctx)
        assert rc == 0 and stats["rejected"] == 0
        assert samples == N
        tally, _ = vrc.vrc_read_tally(ctx)
        assert not tally.any()  # scores go to the moments only

        assert H.rel_err_report(want_total, total)["max_rel"] <= 1e-4
        bound = _sigma_bound(want_total, want_s2, want_sigma, n_hist, N)
        err = np.abs(sigma - want_sigma)
        assert np.all(err <= bound + 1e-12 * want_sigma), (err - bound).max()
        big = (want_sigma > 1e-2 * want_total) & (want_total >= 1e-30)
        assert big.sum() > 1000
        rel = err[big] / want_sigma[big]
        print(f"history sigma form={form} sort={sort}: max rel {rel.max():.2e} over {int(big.sum())} cells")
        assert rel.max() <= 1e-3
    finally:
        ctx.close()


def test_history_moments_one_ray_histories_equal_batches(vrc):
    """With one ray per history the per-history moments are the batch moments
    of one-ray batches: the same S1, S2 and count through both modes."""
    import torch
    prob = W.slab_room(seed=11, n=12, n_rays=64, n_points=300, n_resonances=4, n_groups=2)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=1, sort=0))
    try:
        vrc.vrc_moments_enable(ctx, vrc.VRC_MOMENTS_HISTORY)
        vrc.vrc_cast_histories(ctx, prob.rays, np.arange(prob.n_rays, dtype=np.uint32), prob.n_rays)
        t_h, s_h, n_h = vrc.vrc_moments_read(ctx)
        vrc.vrc_moments_enable(ctx, vrc.VRC_MOMENTS_BATCH)
        for i in range(prob.n_rays):
            one = W.take_rays(prob, [i]).rays
            vrc.vrc_cast_rays(ctx, {k: torch.from_numpy(v).cuda() for k, v in one.items()})
            vrc.vrc_moments_fold(ctx)
        t_b, s_b, n_b = vrc.vrc_moments_read(ctx)
        assert n_h == n_b == prob.n_rays
        np.testing.assert_allclose(t_h, t_b, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(s_h, s_b, rtol=1e-9, atol=1e-300)
    finally:
        ctx.close()
