"""Parity at full size, in the launch configuration the benchmark times.

The 256^3 slab workload (2^24 rays, 16 groups, 2 GiB tally) and the 544x544x64
pin lattice (2^24 rays) are cast by the CUDA path with default options and
compared cell by cell with the multithreaded FP64 oracle over the whole
tally (Eq. 7 relative difference, cells with oracle tally >= 1e-30), and the
GPU's segment count with the oracle's.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


def _run(vrc, torch, prob, form):
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form))
    try:
        rays = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
        s = torch.cuda.current_stream()
        vrc.vrc_cast_rays(ctx, rays, stream=s)
        rc, stats = vrc.vrc_sync(ctx, s)
        tally, _ = vrc.vrc_read_tally(ctx, stream=s)
        del rays
        return tally, rc, stats
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def slab_full():
    prob = W.slab_room(seed=1)
    want, st = oracle.cast(prob)
    return prob, want, st


@pytest.fixture(scope="module")
def lattice_full():
    prob = W.pin_lattice(seed=2)
    want, st = oracle.cast(prob)
    return prob, want, st


@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_slab256_full_size(vrc, slab_full, form):
    import torch
    prob, want, st = slab_full
    got, rc, stats = _run(vrc, torch, prob, form)
    rep = H.rel_err_report(want, got)
    print(f"slab256 form={form}: rc={rc} {stats} oracle={st} {rep}")
    assert rc == vrc.VRC_OK
    assert stats["rays"] == prob.n_rays and stats["overflow"] == 0
    assert stats["segments"] == st["segments"], (stats, st)
    assert rep["max_rel"] <= REL_TOL, rep
    assert rep["max_abs_below"] <= 1e-28, rep


@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_pin_lattice_full_size(vrc, lattice_full, form):
    import torch
    prob, want, st = lattice_full
    got, rc, stats = _run(vrc, torch, prob, form)
    rep = H.rel_err_report(want, got)
    print(f"lattice form={form}: rc={rc} {stats} oracle={st} {rep}")
    assert rc == vrc.VRC_OK
    assert stats["segments"] == st["segments"], (stats, st)
    assert rep["max_rel"] <= REL_TOL, rep
    assert rep["max_abs_below"] <= 1e-28, rep
