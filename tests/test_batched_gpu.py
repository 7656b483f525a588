"""Batched form: many problems in one persistent launch, each problem's tally
against the FP64 oracle (same tolerance as the single-problem parity tests)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import vrc_workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
FIELDS = ("x", "y", "z", "u", "v", "w", "E", "wt")


@pytest.fixture(scope="module")
def small_batch():
    probs = W.batched_problems(seed=3, n_problems=40, side_lo=6, side_hi=30, rays_lo=50,
                               rays_hi=20000, n_points=300, n_resonances=3)
    # a few problems with groups, void and bad rays, to cover the general path
    rng = np.random.default_rng(9)
    probs[3].group_edges = W.log_group_edges(4)
    probs[5].tables[0] = None
    probs[7].rays["E"][:3] = -1.0
    probs[8] = W.take_rays(probs[8], slice(0, 0))  # an empty problem
    want = [oracle.cast(p) for p in probs]
    return probs, want


def _run(vrc, torch, probs, form, bopts, launches=1):
    ctxs = [vrc.context_for(p, vrc.vrc_default_options(form=form)) for p in probs]
    rays = [{k: torch.from_numpy(p.rays[k]).cuda() for k in FIELDS} for p in probs]
    try:
        batch = vrc.vrc_batch_create(ctxs, rays, bopts)
        s = torch.cuda.Stream()
        for _ in range(launches):
            vrc.vrc_batch_launch(batch, stream=s)
        s.synchronize()
        out = []
        for c in ctxs:
            rc, stats = vrc.vrc_sync(c)
            tally, _ = vrc.vrc_read_tally(c)
            out.append((tally, rc, stats))
        batch.close()
        return out
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
@pytest.mark.parametrize("sort,graph,chunk,rpw", [(16, 1, 0, 0), (0, 1, 512, 0), (4, 0, 128, 0),
                                                   (16, 1, 0, 32), (0, 0, 512, 128)],
                         ids=["sorted-graph", "unsorted-graph", "sorted-nograph", "sorted-graph-warp32",
                              "unsorted-nograph-warp128"])
def test_batched_problems_vs_oracle(vrc, small_batch, form, sort, graph, chunk, rpw):
    import torch
    probs, want = small_batch
    opts = vrc.vrc_default_batch_options(sort_len_buckets=sort, use_graph=graph, chunk=chunk,
                                         rays_per_warp=rpw)
    res = _run(vrc, torch, probs, form, opts)
    for p, (prob, (wt, st), (got, rc, stats)) in enumerate(zip(probs, want, res)):
        assert stats["rays"] == prob.n_rays, p
        assert stats["segments"] == st["segments"], p
        assert stats["rejected"] == st["rejected"], p
        assert rc == (vrc.VRC_ERR_NONFINITE if st["rejected"] else vrc.VRC_OK), p
        rep = H.rel_err_report(wt, got)
        assert rep["max_rel"] <= REL_TOL, (p, rep)
        assert rep["max_abs_below"] <= 1e-28, (p, rep)


def test_batched_repeated_launches_accumulate(vrc, small_batch):
    import torch
    probs, want = small_batch
    res = _run(vrc, torch, probs, 1, vrc.vrc_default_batch_options(), launches=3)
    for (wt, st), (got, rc, stats) in zip(want, res):
        assert stats["segments"] == 3 * st["segments"]
        rep = H.rel_err_report(3 * wt, got)
        assert rep["max_rel"] <= REL_TOL


def test_cast_batched_one_shot_equals_separate_casts(vrc, small_batch):
    import torch
    probs, want = small_batch
    ctxs = [vrc.context_for(p, vrc.vrc_default_options(form=1)) for p in probs]
    rays = [{k: torch.from_numpy(p.rays[k]).cuda() for k in FIELDS} for p in probs]
    try:
        vrc.vrc_cast_batched(ctxs, rays)
        for c, (wt, st) in zip(ctxs, want):
            got, _ = vrc.vrc_read_tally(c)
            assert H.rel_err_report(wt, got)["max_rel"] <= REL_TOL
    finally:
        for c in ctxs:
            c.close()


def test_batch_rejects_mixed_forms_and_host_rays(vrc, small_batch):
    import torch
    probs, _ = small_batch
    a = vrc.context_for(probs[0], vrc.vrc_default_options(form=0))
    b = vrc.context_for(probs[1], vrc.vrc_default_options(form=1))
    try:
        dev = [{k: torch.from_numpy(p.rays[k]).cuda() for k in FIELDS} for p in probs[:2]]
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_batch_create([a, b], dev)
        assert ei.value.code == vrc.VRC_ERR_ARG
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_batch_create([a], [probs[0].rays])
        assert ei.value.code == vrc.VRC_ERR_ARG
    finally:
        a.close()
        b.close()


def test_full_size_batched_sampled_problems(vrc):
    """The 1,024-problem workload (about 1.5e8 rays) in the launch
    configuration the batched benchmark times; 24 problems spread over the
    size range are checked cell by cell against the oracle, and every
    problem's ray count."""
    import torch
    probs = W.batched_problems(seed=3)
    ctxs = [vrc.context_for(p, vrc.vrc_default_options(form=1)) for p in probs]
    rays = [{k: torch.from_numpy(p.rays[k]).cuda() for k in FIELDS} for p in probs]
    try:
        batch = vrc.vrc_batch_create(ctxs, rays)
        vrc.vrc_batch_launch(batch)
        torch.cuda.synchronize()
        batch.close()
        sizes = np.array([p.mesh.nx * p.n_rays for p in probs])
        pick = np.argsort(sizes)[np.linspace(0, len(probs) - 1, 24).astype(int)]
        for i, c in enumerate(ctxs):
            rc, stats = vrc.vrc_sync(c)
            assert rc == vrc.VRC_OK and stats["rays"] == probs[i].n_rays
        for i in pick:
            want, st = oracle.cast(probs[i])
            got, _ = vrc.vrc_read_tally(ctxs[i])
            _, stats = vrc.vrc_sync(ctxs[i])
            assert stats["segments"] == st["segments"], i
            rep = H.rel_err_report(want, got)
            assert rep["max_rel"] <= REL_TOL, (i, rep)
    finally:
        for c in ctxs:
            c.close()
