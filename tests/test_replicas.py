"""The N > 1 path on CPU: two gloo ranks each cast (with the oracle, on the
host) their shard of a batch and sum their tallies; the result equals the
one-rank tally of the whole batch.  Also checks the benchmark's cross-rank
timing reduction (max of the ranks' times, sum of their segments)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import vrc_workloads as W
from paper_1706_07476_gb300.replicas import allreduce_tally, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    return W.slab_room(seed=1, n=20, n_rays=3001, n_points=300, n_resonances=5, n_groups=3)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        part = W.take_rays(prob, shard(prob.n_rays, rank, world))
        tally, st = oracle.cast(part, nthreads=1)
        t = torch.from_numpy(tally)
        allreduce_tally(t)
        seg = torch.tensor([float(st["segments"])], dtype=torch.float64)
        dist.all_reduce(seg, op=dist.ReduceOp.SUM)
        elapsed = torch.tensor([0.5 + rank], dtype=torch.float64)
        dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
        if rank == 0:
            np.save(out, t.numpy())
            np.save(out + ".meta.npy", np.array([seg.item(), elapsed.item()]))
    finally:
        dist.destroy_process_group()


def test_shards_cover_the_batch():
    for n in (0, 1, 7, 3001):
        for world in (1, 2, 3, 8):
            idx = np.concatenate([np.arange(n)[shard(n, r, world)] for r in range(world)])
            assert np.array_equal(idx, np.arange(n))
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def test_two_gloo_ranks_sum_to_the_whole_batch(tmp_path):
    out = str(tmp_path / "tally.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    seg, elapsed = np.load(out + ".meta.npy")
    prob = _problem()
    want, st = oracle.cast(prob, nthreads=1)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
    assert seg == st["segments"]
    assert elapsed == 1.5  # the slowest rank's time


@pytest.mark.gpu
def test_device_tally_view_and_single_rank_reduce(vrc):
    """The device tally wrapped for torch.distributed is the library's tally."""
    from paper_1706_07476_gb300.replicas import device_tally
    prob = _problem()
    ctx = vrc.context_for(prob)
    try:
        vrc.vrc_cast_rays(ctx, prob.rays)
        host, _ = vrc.vrc_read_tally(ctx)
        dev = device_tally(vrc, ctx)
        assert dev.dtype == torch.float64 and dev.numel() == prob.tally_size
        allreduce_tally(dev)  # one rank: identity
        np.testing.assert_array_equal(dev.cpu().numpy(), host)
    finally:
        ctx.close()
