"""vrc_sort_rays_static: the ray sort without any allocation.

Some callers may not allocate device memory once their run has started (a
transport code that gives all free device memory to its own pool at
start-up, or one whose batch loop must not pay cudaMalloc's device-wide
synchronisation).  For them libvrc keeps the sort's scratch in a fixed
device array.  This test calls that entry point through the C ABI on two
batches in a row and checks each result against the allocating path:
the output is a permutation of the input in group order, and casting it with
sorting off gives vrc_cast_rays' sorted tally to the tolerance the sort
tests use.  It also checks the promise itself: once the first call on the
device has done its set-up, a second call leaves the device's free memory
(as the driver reports it) unchanged.  It sits in its own file, collected
last, and passes both alone in a fresh process and after the other tests.
"""
from __future__ import annotations

import numpy as np
import pytest

import vrc_workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "u", "v", "w", "E", "wt")


def _cast(vrc, torch, prob, rays_dev, sort, stream):
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, sort=sort))
    try:
        vrc.vrc_cast_rays(ctx, rays_dev, stream=stream)
        rc, stats = vrc.vrc_sync(ctx, stream)
        tally, _ = vrc.vrc_read_tally(ctx, stream=stream)
        assert rc == vrc.VRC_OK
        return tally, stats
    finally:
        ctx.close()


def test_static_sort_matches_allocating_path_twice_in_a_row(vrc):
    import torch
    stream = torch.cuda.Stream()
    n = 150_000
    prob = W.slab_room(seed=1, n=40, n_rays=2 * n, n_points=1500, n_resonances=30)
    sorter = vrc.context_for(prob)  # mesh box and groups of the sort key
    try:
        # every input and output of both calls exists before the first call,
        # so that between the two free-memory readings only the second call runs
        parts = [W.take_rays(prob, sl) for sl in (slice(0, n), slice(n, 2 * n))]
        devs = [{k: torch.from_numpy(p.rays[k]).cuda() for k in FIELDS} for p in parts]
        outs = [torch.full((8 * n,), float("nan"), dtype=torch.float32, device="cuda") for _ in parts]
        torch.cuda.synchronize()
        vrc.vrc_sort_rays_static(sorter, devs[0], outs[0], stream=stream)
        stream.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        vrc.vrc_sort_rays_static(sorter, devs[1], outs[1], stream=stream)
        stream.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert free_after == free_before, (free_before, free_after)

        for call in range(2):
            part, dev, out = parts[call], devs[call], outs[call]
            got = out.view(8, n).cpu().numpy()

            # a permutation of the input rays
            a = np.stack([part.rays[k] for k in FIELDS], axis=1)
            b = got.T.copy()
            assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])]), call
            # energy groups in ascending order
            edges = prob.group_edges
            g = np.clip(np.searchsorted(edges, got[6].astype(np.float64), side="right") - 1,
                        0, len(edges) - 2)
            assert np.all(np.diff(g) >= 0), call

            # cast of the statically sorted rays (sorting off) against the
            # allocating path's sorted cast of the original rays
            sorted_dev = {k: out.view(8, n)[i].contiguous() for i, k in enumerate(FIELDS)}
            t_static, s_static = _cast(vrc, torch, part, sorted_dev, 0, stream)
            t_alloc, s_alloc = _cast(vrc, torch, part, dev, 1, stream)
            assert s_static["segments"] == s_alloc["segments"], call
            np.testing.assert_allclose(t_static, t_alloc, rtol=1e-12, atol=1e-300)
    finally:
        sorter.close()


def test_static_sort_rejects_what_does_not_fit(vrc):
    import torch
    prob = W.slab_room(seed=1, n=16, n_rays=8, n_points=100, n_resonances=2)
    ctx = vrc.context_for(prob)
    try:
        big = (1 << 18) + 1
        dev = {k: torch.zeros(big, dtype=torch.float32, device="cuda") for k in FIELDS}
        out = torch.empty(8 * big, dtype=torch.float32, device="cuda")
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_sort_rays_static(ctx, dev, out)
        assert ei.value.code == vrc.VRC_ERR_ARG and "262144" in str(ei.value)
        host = {k: np.zeros(4, np.float32) for k in FIELDS}
        with pytest.raises(vrc.VrcError) as ei:
            vrc.vrc_sort_rays_static(ctx, host, out)
        assert ei.value.code == vrc.VRC_ERR_ARG
    finally:
        ctx.close()
