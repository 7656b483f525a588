"""options.stop_at_zero: a walk ends once the ray's transmitted fraction is
exactly 0.  Every later Eq. 4 score would be +0, so the tally equals the
full walk's up to float64 summation order; only the segment counter (walked
segments) is smaller.  Uniform and rectilinear meshes, both forms."""
from __future__ import annotations

import numpy as np
import pytest

import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _cast(vrc, torch, prob, **opts):
    ctx = vrc.context_for(prob, vrc.vrc_default_options(**opts))
    try:
        vrc.vrc_cast_rays(ctx, {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()})
        rc, st = vrc.vrc_sync(ctx)
        tally, _ = vrc.vrc_read_tally(ctx)
        assert rc == vrc.VRC_OK
        return tally, st
    finally:
        ctx.close()


@pytest.mark.parametrize("mesh", ["uniform", "graded"])
@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_stop_at_zero_keeps_the_tally(vrc, form, mesh):
    import torch
    if mesh == "uniform":
        prob = W.slab_room(seed=13, n=48, n_rays=200000, n_points=400, n_resonances=20, n_groups=3)
    else:
        prob = W.graded_assembly(seed=14, pins=4, reflector=8.0, n_rays=100000, n_points=400,
                                 n_resonances=20)
    full, sf = _cast(vrc, torch, prob, form=form)
    stop, ss = _cast(vrc, torch, prob, form=form, stop_at_zero=1)
    assert ss["rays"] == sf["rays"] and ss["rejected"] == sf["rejected"] == 0
    assert ss["segments"] < sf["segments"]  # the workload has rays that go dark
    rep = H.rel_err_report(full, stop, floor=1e-300)
    assert rep["max_rel"] <= 1e-12, rep
    assert np.array_equal(full == 0, stop == 0)
    print(f"stop_at_zero {mesh} form={form}: {ss['segments']} of {sf['segments']} segments walked")


def test_stop_at_zero_void_walks_everything(vrc):
    """In void the transmitted fraction stays 1: every ray is walked to the exit."""
    import torch
    prob = W.slab_room(seed=15, n=24, n_rays=20000, n_points=100, n_resonances=2, n_groups=1)
    prob = W.Problem("void", prob.mesh, [None] * prob.n_materials, None, prob.rays)
    full, sf = _cast(vrc, torch, prob, form=1)
    stop, ss = _cast(vrc, torch, prob, form=1, stop_at_zero=1)
    assert ss["segments"] == sf["segments"]
    assert H.rel_err_report(full, stop)["max_rel"] <= 1e-12
