"""Launch-shape autotuner for the cast and the batched form.

Sweeps the options that set the launch shape (threads per block, rays per
warp, rays per work item, sort granularity), times each candidate with CUDA
events on the launching stream, and caches the best choice per GPU name and
configuration class in a JSON file (``$VRC_AUTOTUNE_CACHE``, default
``~/.cache/vrc_autotune.json``).  The sweep is a coordinate descent: one
option at a time, holding the best values found so far.

Tuning only changes how the same work is scheduled: every candidate casts
every ray and produces the same tally up to float64 summation order.
"""
from __future__ import annotations

import json
import math
import os
import time

from paper_1706_07476_gb300 import vrc



def cache_path() -> str:
    return os.environ.get("VRC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "vrc_autotune.json"))

# rays_per_warp (batched): 0 interleaved within a work item; R > 0, each
# warp takes R rays at a time from the item's shared counter
BATCH_SPACE = {
    "sort_len_buckets": [0, 8, 16, 32],
    "chunk": [1024, 2048, 4096, 8192],
    "block": [128, 256],
    "rays_per_warp": [0, 32, 128],
}
# rays_per_warp: -1 interleaved assignment; R > 0, each warp takes R
# consecutive sorted rays at a time from a device counter
CAST_SPACE = {
    "sort_len_buckets": [8, 32, 64, 128, 256],
    "block": [128, 256],
    "rays_per_warp": [-1, 32, 64, 128, 512, 2048],
}
CAST_DEFAULT = {"sort_len_buckets": 256, "block": 256, "rays_per_warp": 32}


def _gpu_name(torch) -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    data = _load_cache()
    data[key] = value
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _pow2_bucket(x: float) -> int:
    return int(round(math.log2(max(x, 1.0))))


def batched_class(problems, form: int) -> str:
    n = len(problems)
    rays = sum(p.n_rays for p in problems)
    side = sum(p.mesh.nx + p.mesh.ny + p.mesh.nz for p in problems) / max(n, 1) / 3
    return f"batched|form{form}|p{_pow2_bucket(n)}|r{_pow2_bucket(rays)}|s{_pow2_bucket(side)}"


def cast_class(problem, form: int) -> str:
    m = problem.mesh
    return (f"cast|form{form}|c{_pow2_bucket(m.ncells)}|g{problem.n_groups}|"
            f"r{_pow2_bucket(problem.n_rays)}")


def _time_events(torch, fn, stream, reps):
    fn()  # warm-up
    stream.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _descend(space, default, measure):
    best = dict(default)
    table = []
    best_ms = measure(best)
    table.append((dict(best), best_ms))
    for key, values in space.items():
        for v in values:
            if v == best.get(key):
                continue
            cand = dict(best)
            cand[key] = v
            ms = measure(cand)
            table.append((dict(cand), ms))
            if ms < best_ms:
                best, best_ms = cand, ms
    return best, best_ms, table


def tune_batched(torch, problems, ctxs, rays_list, form: int, reps: int = 2, use_cache=True,
                 timer=None):
    """Best vrc_batch_options fields for this batch (dict), ms, and the sweep
    table.  timer(fn) -> ms as in tune_cast."""
    key = f"{_gpu_name(torch)}|{batched_class(problems, form)}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit["options"], hit["ms"], []
    stream = torch.cuda.Stream() if timer is None else None
    if timer is None:
        timer = lambda fn: _time_events(torch, fn, stream, reps)  # noqa: E731

    def measure(opts):
        o = vrc.vrc_default_batch_options(**opts)
        batch = vrc.vrc_batch_create(ctxs, rays_list, o)
        try:
            return timer(lambda: vrc.vrc_batch_launch(batch, stream=stream))
        finally:
            if stream is not None:
                stream.synchronize()
            batch.close()

    best, ms, table = _descend(BATCH_SPACE, {"sort_len_buckets": 16, "chunk": 2048, "block": 256,
                                             "rays_per_warp": 0}, measure)
    _store(key, {"options": best, "ms": ms, "when": time.time()})
    return best, ms, table


def tune_cast(torch, problem, ctx, dev_rays, form: int, reps: int = 2, use_cache=True, timer=None):
    """Best vrc_options fields (sort buckets, block, rays per warp) for one
    problem's casts; leaves them set on ctx.  timer(fn) -> ms times one call
    (default: the best of `reps` CUDA-event timings after a warm-up)."""
    key = f"{_gpu_name(torch)}|{cast_class(problem, form)}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            vrc.vrc_set_options(ctx, vrc.vrc_default_options(form=form, sort=1, **hit["options"]))
            return hit["options"], hit["ms"], []
    if timer is None:
        stream = torch.cuda.Stream()
        timer = lambda fn: _time_events(torch, fn, stream, reps)  # noqa: E731
    else:
        stream = None

    def measure(opts):
        vrc.vrc_set_options(ctx, vrc.vrc_default_options(form=form, sort=1, **opts))
        return timer(lambda: vrc.vrc_cast_rays(ctx, dev_rays, stream=stream))

    best, ms, table = _descend(CAST_SPACE, CAST_DEFAULT, measure)
    vrc.vrc_set_options(ctx, vrc.vrc_default_options(form=form, sort=1, **best))
    _store(key, {"options": best, "ms": ms, "when": time.time()})
    return best, ms, table
