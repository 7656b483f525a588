"""Streaming ray buffers (Sec. 3: the CPU fills a buffer, the GPU casts it
while the CPU keeps going): buffers streamed through vrc_stream, including a
partial last one and more submits than buffers, give the tally of one direct
cast of the same rays, and that tally matches the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu
FIELDS = ("x", "y", "z", "u", "v", "w", "E", "wt")


@pytest.mark.parametrize("n_buffers,capacity", [(2, 5000), (3, 7001)])
def test_streamed_buffers_equal_one_cast(vrc, n_buffers, capacity):
    prob = W.slab_room(seed=1, n=40, n_rays=40000, n_points=800, n_resonances=10, n_groups=4)
    want, st = oracle.cast(prob)
    opts = vrc.vrc_default_options(form=1, sort=0)
    direct = vrc.context_for(prob, opts)
    streamed = vrc.context_for(prob, opts)
    rs = vrc.RayStream(streamed, capacity, n_buffers)
    try:
        vrc.vrc_cast_rays(direct, prob.rays)
        a, _ = vrc.vrc_read_tally(direct)
        records = np.stack([prob.rays[k] for k in FIELDS], axis=1)
        for lo in range(0, prob.n_rays, capacity):
            part = records[lo:lo + capacity]
            buf = rs.acquire()
            buf[:len(part)] = part
            rs.submit(len(part))
        rs.finish()
        b, rc = vrc.vrc_read_tally(streamed)
        _, stats = vrc.vrc_sync(streamed)
        assert rc == vrc.VRC_OK and stats["rays"] == prob.n_rays
        assert stats["segments"] == st["segments"]
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-300)
        assert H.rel_err_report(want, b)["max_rel"] <= 1e-4
    finally:
        rs.close()
        direct.close()
        streamed.close()


def test_stream_argument_errors(vrc):
    prob = W.slab_room(seed=1, n=8, n_rays=16, n_points=50, n_resonances=2)
    ctx = vrc.context_for(prob)
    try:
        with pytest.raises(vrc.VrcError) as ei:
            vrc.RayStream(ctx, 1000, 1)
        assert ei.value.code == vrc.VRC_ERR_ARG
        rs = vrc.RayStream(ctx, 100, 2)
        with pytest.raises(vrc.VrcError) as ei:
            rs.submit(10)  # nothing acquired
        assert ei.value.code == vrc.VRC_ERR_STATE
        rs.acquire()
        with pytest.raises(vrc.VrcError):
            rs.submit(101)
        rs.close()
    finally:
        ctx.close()
