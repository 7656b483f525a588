"""Next-event (point-detector) estimator against the FP64 oracle: flux at
detector points inside the mesh, on a cell face and outside the box, per
energy group, from device and host rays."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sort", [0, 1], ids=["input_order", "sorted"])
@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_detector_flux_vs_oracle(vrc, form, sort):
    import torch
    prob = W.slab_room(seed=7, n=20, n_rays=20000, n_points=600, n_resonances=8, n_groups=3)
    det = np.array([[10.3, 9.7, 11.1], [5.0, 5.0, 5.0], [25.0, 10.0, 10.0], [-3.0, 30.0, 4.0]])
    want = oracle.point_detector(prob, det)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form, sort=sort))
    try:
        dev = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
        got = vrc.vrc_detector_flux(ctx, dev, det)
        host = vrc.vrc_detector_flux(ctx, prob.rays, det)
        assert got.shape == want.shape
        sel = want > 0
        rel = np.abs(got[sel] - want[sel]) / want[sel]
        print(f"detectors form={form} sort={sort}: max rel {rel.max():.2e}")
        assert rel.max() <= 1e-4, rel.max()
        np.testing.assert_allclose(host, got, rtol=1e-12)
        tally, _ = vrc.vrc_read_tally(ctx)
        assert not tally.any()  # the tally is untouched
    finally:
        ctx.close()
