"""The autotuner's search and cache on the CPU, with the GPU timing replaced
by a planted cost function.

The coordinate descent must find the planted minimum of a separable cost
over the cast's launch options (sort buckets, threads per block, rays per
warp), leave the winning options set on the context, and store them under a
key made of the GPU name and the configuration class; a second call with the
cache on must return the stored choice without timing anything.
"""
from __future__ import annotations

import types

import numpy as np
import pytest

import vrc_workloads as W

autotune = pytest.importorskip("paper_1706_07476_gb300.autotune")


class FakeVrc:
    """Stands in for the binding: records options, casts nothing."""

    def __init__(self):
        self.current = None
        self.casts = 0

    def vrc_default_options(self, **kw):
        return dict(kw)

    def vrc_set_options(self, ctx, o):
        self.current = dict(o)

    def vrc_cast_rays(self, ctx, rays, stream=None):
        self.casts += 1

    def vrc_default_batch_options(self, **kw):
        return dict(kw)

    def vrc_batch_create(self, ctxs, rays, o):
        self.current = dict(o)
        return types.SimpleNamespace(close=lambda: None)

    def vrc_batch_launch(self, batch, stream=None):
        self.casts += 1


def fake_torch(name):
    cuda = types.SimpleNamespace(get_device_name=lambda i: name, current_device=lambda: 0)
    return types.SimpleNamespace(cuda=cuda)


PLANT = {"sort_len_buckets": 32, "block": 128, "rays_per_warp": 512}


def planted_cost(opts):
    """Separable, minimal at PLANT; every other value costs more."""
    ms = 10.0
    for k, best in PLANT.items():
        ms += 0.0 if opts[k] == best else 1.0 + abs(np.log2(abs(opts[k]) + 1) - np.log2(abs(best) + 1))
    return ms


def test_descent_finds_planted_minimum_and_caches(monkeypatch, tmp_path):
    fake = FakeVrc()
    monkeypatch.setattr(autotune, "vrc", fake)
    monkeypatch.setenv("VRC_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    prob = W.uniform_small(seed=0, n=16, n_rays=256)
    timed = []

    def timer(fn):
        fn()
        ms = planted_cost(fake.current)
        timed.append((dict(fake.current), ms))
        return ms

    best, ms, table = autotune.tune_cast(fake_torch("GPU-A"), prob, object(), {}, form=1, timer=timer)
    assert {k: best[k] for k in PLANT} == PLANT
    assert ms == pytest.approx(10.0)
    assert {k: fake.current[k] for k in PLANT} == PLANT  # left set on the context
    assert fake.current["form"] == 1 and fake.current["sort"] == 1
    # every axis was swept, the rays-per-warp axis included
    swept = {k: {o[k] for o, _ in table} for k in autotune.CAST_SPACE}
    for k, values in autotune.CAST_SPACE.items():
        assert set(values) <= swept[k], k
    assert len(timed) == len(table)

    # the cache: keyed by GPU name and configuration class
    import json
    data = json.loads((tmp_path / "cache.json").read_text())
    key = "GPU-A|" + autotune.cast_class(prob, 1)
    assert list(data) == [key] and data[key]["options"] == best

    # a second call hits the cache and times nothing
    n_before = len(timed)
    best2, ms2, table2 = autotune.tune_cast(fake_torch("GPU-A"), prob, object(), {}, form=1, timer=timer)
    assert best2 == best and ms2 == ms and table2 == [] and len(timed) == n_before
    assert {k: fake.current[k] for k in PLANT} == PLANT

    # another GPU name, another form or another configuration class is a miss
    autotune.tune_cast(fake_torch("GPU-B"), prob, object(), {}, form=1, timer=timer)
    assert len(timed) > n_before
    other = W.uniform_small(seed=0, n=64, n_rays=256)
    assert autotune.cast_class(other, 1) != autotune.cast_class(prob, 1)
    assert autotune.cast_class(prob, 0) != autotune.cast_class(prob, 1)
    data = json.loads((tmp_path / "cache.json").read_text())
    assert set(data) == {key, "GPU-B|" + autotune.cast_class(prob, 1)}


def test_descent_holds_the_best_values_found_so_far():
    """Coordinate descent on a cost where the best value of the second axis
    depends on the first: each axis is swept holding the best so far."""
    space = {"a": [1, 2, 3], "b": [10, 20, 30]}
    cost = lambda o: (o["a"] - 3) ** 2 + 0.01 * (o["b"] - 10 * o["a"]) ** 2  # noqa: E731
    best, ms, table = autotune._descend(space, {"a": 1, "b": 10}, cost)
    # a = 2 wins at b = 10; b is then swept at a = 2 (at a = 1 it would stay 10)
    assert best == {"a": 2, "b": 20} and ms == pytest.approx(1.0)
    assert table[0] == ({"a": 1, "b": 10}, cost({"a": 1, "b": 10}))
    assert len(table) == 1 + 2 + 2


def test_batched_descent_with_planted_minimum(monkeypatch, tmp_path):
    fake = FakeVrc()
    monkeypatch.setattr(autotune, "vrc", fake)
    monkeypatch.setenv("VRC_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    plant = {"sort_len_buckets": 8, "chunk": 4096, "block": 128, "rays_per_warp": 32}

    def timer(fn):
        fn()
        return 1.0 + sum(fake.current[k] != v for k, v in plant.items())

    probs = [W.uniform_small(seed=s, n=16, n_rays=64) for s in range(3)]
    best, ms, _ = autotune.tune_batched(fake_torch("GPU-A"), probs, [], [], form=1, timer=timer)
    assert best == plant and ms == 1.0
