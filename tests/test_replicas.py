"""The N > 1 path: two gloo ranks each cast their shard of a batch and sum
their tallies; the result equals the one-rank tally of the whole batch.  On
CPU the ranks cast with the oracle (and the benchmark's cross-rank timing
reduction is checked: max of the ranks' times, sum of their segments); on
the GPU two replica processes share the one GPU and cast with libvrc."""
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


def _gpu_worker(rank, world, port, out, form):
    """One replica: casts its shard through libvrc on cuda:0, reads its tally
    to the host and sums it with the other ranks' over gloo."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from paper_1706_07476_gb300 import vrc
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _gpu_problem()
        part = W.take_rays(prob, shard(prob.n_rays, rank, world))
        ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form))
        try:
            dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in part.rays.items()}
            vrc.vrc_cast_rays(ctx, dev)
            rc, st = vrc.vrc_sync(ctx)
            host, _ = vrc.vrc_read_tally(ctx)
        finally:
            ctx.close()
        t = torch.from_numpy(host)
        allreduce_tally(t)
        seg = torch.tensor([float(st["segments"]), float(rc != vrc.VRC_OK)], dtype=torch.float64)
        dist.all_reduce(seg, op=dist.ReduceOp.SUM)
        if rank == 0:
            np.save(out, t.numpy())
            np.save(out + ".meta.npy", seg.numpy())
    finally:
        dist.destroy_process_group()


def _gpu_problem():
    return W.slab_room(seed=5, n=32, n_rays=1 << 16, n_points=500, n_resonances=8, n_groups=2)


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1], ids=["plain", "fp32"])
def test_two_replicas_through_libvrc_sum_to_the_whole_batch(vrc, tmp_path, form):
    """Two processes on the one GPU, each a replica that casts its shard with
    the library (their kernels never wait on each other: the only exchange
    is the host-side gloo sum after both casts), reproduce the single cast
    of the whole batch to float64 summation order and the oracle to 1e-4."""
    out = str(tmp_path / "tally.npy")
    port = _free_port()
    mp.start_processes(_gpu_worker, args=(2, port, out, form), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    seg, bad = np.load(out + ".meta.npy")
    prob = _gpu_problem()
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form))
    try:
        vrc.vrc_cast_rays(ctx, {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()})
        rc, st = vrc.vrc_sync(ctx)
        whole, _ = vrc.vrc_read_tally(ctx)
    finally:
        ctx.close()
    assert bad == 0 and rc == vrc.VRC_OK
    assert seg == st["segments"]
    np.testing.assert_allclose(got, whole, rtol=1e-12, atol=1e-300)
    want, sto = oracle.cast(prob)
    assert st["segments"] == sto["segments"]
    sel = want >= 1e-30
    assert np.max(np.abs(got[sel] - want[sel]) / want[sel]) <= 1e-4
