"""Host ray batches of more than 2^22 rays take the pipelined path of
vrc_cast_rays (chunks of 2^21, then up to 2^24 rays): chunk i+1 uploads
while chunk i is sorted and cast.  Its tally must equal the device-array
cast of the same rays up to float64 summation order, with the same segment
count, also when the call is repeated (the staging slots are reused across
calls)."""
from __future__ import annotations

import numpy as np
import pytest

import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", [1, 0], ids=["fp32", "plain"])
def test_pipelined_host_cast_equals_device_cast(vrc, form):
    import torch
    n = (1 << 24) + (1 << 21) + 12345  # three chunks (2^21, 2^24, ragged), both slots used
    prob = W.slab_room(seed=12, n=32, n_rays=n, n_points=300, n_resonances=6, n_groups=3)
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in prob.rays.items()}
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form))
    try:
        vrc.vrc_cast_rays(ctx, dev)
        rc, sd = vrc.vrc_sync(ctx)
        want, _ = vrc.vrc_read_tally(ctx)
        for rays in (pinned, prob.rays):  # pinned torch tensors, then pageable numpy
            vrc.vrc_reset_tally(ctx)
            vrc.vrc_cast_rays(ctx, rays)
            vrc.vrc_cast_rays(ctx, rays)  # the slots are reused by the next call
            rc2, sh = vrc.vrc_sync(ctx)
            got, _ = vrc.vrc_read_tally(ctx)
            assert rc == rc2 == vrc.VRC_OK
            assert sh["segments"] == 2 * sd["segments"] and sh["rays"] == 2 * n
            rep = H.rel_err_report(2 * want, got)
            assert rep["max_rel"] <= 1e-12, rep
    finally:
        ctx.close()
