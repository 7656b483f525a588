"""Device rays produced on a torch stream other than the library's: the
binding makes the library stream wait for the producer (and keeps the
tensors alive until the cast has read them).  The producer stream first
sleeps on the GPU, then writes the rays into buffers holding poison (NaN):
a cast that did not wait would read the poison and report non-finite rays
or a different tally."""
from __future__ import annotations

import numpy as np
import pytest

import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_cast_waits_for_the_producer_stream(vrc):
    import torch
    prob = W.slab_room(seed=16, n=24, n_rays=50000, n_points=200, n_resonances=4, n_groups=2)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=1))
    try:
        vrc.vrc_cast_rays(ctx, {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()})
        rc, ref_stats = vrc.vrc_sync(ctx)
        want, _ = vrc.vrc_read_tally(ctx)
        assert rc == vrc.VRC_OK
        vrc.vrc_reset_tally(ctx)
        producer = torch.cuda.Stream()
        host = {k: torch.from_numpy(v).pin_memory() for k, v in prob.rays.items()}
        dev = {k: torch.full((prob.n_rays,), float("nan"), device="cuda") for k in prob.rays}
        torch.cuda.synchronize()
        with torch.cuda.stream(producer):
            torch.cuda._sleep(50_000_000)  # about 25 ms of GPU time before the data lands
            for k in dev:
                dev[k].copy_(host[k], non_blocking=True)
            vrc.vrc_cast_rays(ctx, dev)  # the library's own stream (stream=None)
        rc, stats = vrc.vrc_sync(ctx)
        got, _ = vrc.vrc_read_tally(ctx)
        assert rc == vrc.VRC_OK, rc
        assert stats["rejected"] == 0 and stats["segments"] == ref_stats["segments"]
        assert H.rel_err_report(want, got)["max_rel"] <= 1e-12
    finally:
        ctx.close()
