"""Tally statistics by batches (the sigma of Eqs. 5 and 8) against the
oracle's batch moments of the same batches of rays."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_batch_moments_match_oracle(vrc):
    import torch
    prob = W.slab_room(seed=5, n=24, n_rays=36000, n_points=500, n_resonances=8, n_groups=3)
    B = 6
    parts = [W.take_rays(prob, slice(prob.n_rays * b // B, prob.n_rays * (b + 1) // B)) for b in range(B)]
    batch = [oracle.cast(p)[0] for p in parts]
    want_total, want_sigma = oracle.batch_moments(batch)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=1))
    try:
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_moments_fold(ctx)
        assert ei.value.code == vrc.VRC_ERR_STATE
        vrc.vrc_moments_enable(ctx)
        for p in parts:
            vrc.vrc_cast_rays(ctx, {k: torch.from_numpy(v).cuda() for k, v in p.rays.items()})
            vrc.vrc_moments_fold(ctx)
        total, sigma, batches = vrc.vrc_moments_read(ctx)
        assert batches == B
        left, _ = vrc.vrc_read_tally(ctx)
        assert not left.any()  # every fold clears the tally
        assert H.rel_err_report(want_total, total)["max_rel"] <= 1e-4
        # sigma: each GPU batch tally t_b' carries |t_b' - t_b| <= d_b with
        # d_b = 1e-4 |t_b| + 1e-30 (the per-cell parity bar; below 1e-30 the
        # FP32 form may underflow to 0).  Propagated through
        # var = B/(B-1) (sum t_b^2 - total^2/B) this bounds |var' - var| by
        # dv below, and |sigma' - sigma| <= min(dv / sigma, sqrt(dv)).
        T = np.asarray(batch)
        d = 1e-4 * np.abs(T) + 1e-30
        sd = d.sum(axis=0)
        dv = (B / (B - 1.0)) * (2 * np.sum(np.abs(T) * d, axis=0) + np.sum(d * d, axis=0)
                                + 2 * np.abs(want_total) * sd / B + sd * sd / B)
        bound = np.minimum(dv / np.maximum(want_sigma, 1e-300), np.sqrt(dv))
        err = np.abs(sigma - want_sigma)
        assert np.all(err <= bound + 1e-12 * want_sigma), (err - bound).max()
        # where the spread is a sizeable part of the total the bound is tight
        big = (want_sigma > 1e-2 * np.abs(want_total)) & (np.abs(want_total) >= 1e-30)
        assert big.sum() > 1000
        rel = err[big] / want_sigma[big]
        print(f"batch sigma: max rel {rel.max():.2e} over {int(big.sum())} cells")
        assert rel.max() <= 1e-3, rel.max()
        assert np.all(sigma >= 0)
    finally:
        ctx.close()
