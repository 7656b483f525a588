#!/usr/bin/env python3
"""Throughput of the VRC cast on GB300: ray-cell segments per second.

One step casts one batch of 2^24 synthetic rays through the 256^3 slab mesh
(8 materials with 20,000-point tables, 16 energy groups) into the
device-resident tally: the whole hot path (cross-section lookup, grid walk,
Eq. 4 score, tally update) in libvrc's kernels, called through the C ABI.

Default: N=1, both precision forms timed side by side; the headline line is
the FP32 form.  Under torchrun every rank casts its own replica batch into its
own tally (weak scaling, no collective in the timed region).

--impl reference times the FP64 CPU oracle on the host cores instead, on
bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import vrc_workloads as W  # noqa: E402

WORKLOAD = ("slab256: 256^3 mesh of 1 cm cells, 8 materials with 20,000-point tables "
            "(200 Lorentzian resonances each), 16 random axis-aligned slabs, 2^24 rays "
            "(uniform positions, isotropic directions, log-uniform energies, lognormal(0,0.5) "
            "weights), 16 log-uniform energy groups, seed 1")
GRADED = ("graded: 16x16-pin assembly (pitch 1.26 cm; fuel, void gap, cladding, moderator) on a "
          "rectilinear 420x420x5 mesh, 0.6 mm cells over the assembly growing 1.1x per cell to 2 cm "
          "through a 30 cm solution + graphite reflector, 6 materials (5 with 20,000-point tables), "
          "2^24 rays (70% in fuel discs), 1/E energies, one group, seed 5")
HISTORY = ("history: the slab256 rays grouped into histories of 1..15 consecutive rays "
           "(uniform, mean 8), cast per history in 16 calls of 2^20 rays each; per-history "
           "moments S1 += x_h, S2 += x_h^2 per (group, cell)")
DETECTORS = ("detectors: the slab256 rays as collision events, each scored at 8 detector "
             "points (a 2x2x2 lattice at 1/4 and 3/4 of the box) by the next-event estimator "
             "wt exp(-tau)/(4 pi R^2), tau by the grid walk from the event to the detector")
SURROGATE = ("surrogate32: 32^3 mesh of 1 cm cells, 16 materials (layout uniform-random) with "
             "20,000-point tables of 200 resonances, 2^24 rays, FP32 form; cross sections from the "
             "learned 64 -> 128 -> 128 -> 16 network (sinusoidal embedding of log10 E, SiLU, 1/v prior) "
             "where its validated error is within 1e-3, the table elsewhere, seed 4")
METRIC = "ray-cell segments/s at <=1e-4 tally rel. err vs FP64 oracle; % HBM roofline"
UNIT = "segments/s"
# Algorithmic bytes: per segment 8 B tally read + 8 B tally write + 1 B material
# id; per ray 32 B of ray data (x, y, z, u, v, w, E, wt as float32).
BYTES_PER_SEGMENT = 17
BYTES_PER_TALLY = 16
BYTES_PER_MATERIAL = 1
BYTES_PER_RAY = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["vrc", "reference"], default="vrc")
    ap.add_argument("--forms", default="plain,fp32", help="forms to time; the last is the headline")
    ap.add_argument("--sort", type=int, default=-1, help="ray sorting: -1 auto, 0 off, 1 on")
    ap.add_argument("--rays-per-warp", type=int, default=0,
                    help="cast ray assignment: 0 auto, -1 interleaved, R > 0 dynamic chunks of R rays")
    ap.add_argument("--n-rays", type=int, default=1 << 24)
    ap.add_argument("--mesh", type=int, default=256)
    ap.add_argument("--workload", choices=["slab256", "batched", "stream", "graded", "history",
                                           "detectors", "surrogate"],
                    default="slab256")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--problems", type=int, default=1024,
                    help="batched workload: the first N of its 1,024 problems (profiling a subset)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity-sample", action="store_true")
    ap.add_argument("--no-micro", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the pin-lattice, batched and surrogate workloads of the default line")
    ap.add_argument("--config-steps", type=int, default=5, help="timed steps of each extra workload")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU-baseline oracle sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    if args.workload == "graded":
        return W.graded_assembly(seed=5, n_rays=args.n_rays)
    return W.slab_room(seed=1, n=args.mesh, n_rays=args.n_rays)


def workload_text(args, prob):
    if args.workload == "graded":
        return GRADED, f"float64 [{prob.n_groups}][{prob.mesh.nz}][{prob.mesh.ny}][{prob.mesh.nx}]"
    return WORKLOAD, "float64 [16][256^3] (2 GiB)"


def headline_config(args, prob, world):
    """The headline line's config: what the workload is, the same for the
    GPU arm and the reference arm (measured figures go elsewhere)."""
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    return {"workload": workload_text(args, prob)[0], "rays_per_step": prob.n_rays,
            "form": forms[-1], "sort": args.sort, "tally": workload_text(args, prob)[1],
            "l2": ("inputs larger than L2 (512 MiB rays, 2 GiB tally, 16 MiB mesh); no flush"
                   if args.workload == "slab256" else
                   "inputs larger than L2 (512 MiB rays); tally 7 MB; no flush"),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


CAST_SOURCES = ("vrc_device.cuh", "vrc_math64.h", "vrc_cast.cu")
BATCHED_SOURCES = ("vrc_device.cuh", "vrc_math64.h", "vrc_batched.cu", "vrc_sort.cu")


def profiled_field(kernel_tag: str, workload_tag: str, field: str, sources=CAST_SOURCES):
    """A number from a committed ncu summary of this kernel on this workload
    (e.g. DRAM bytes per launch), if the summary was taken on the current
    kernel source (matched by the recorded hash of `sources`)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload_tag}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_1706_07476_gb300", "csrc", f), "rb").read())
    fields = dict(ln.split(":", 1) for ln in text.splitlines() if ln.startswith(("source_sha256:", field + ":")))
    if fields.get("source_sha256", "").strip() != h.hexdigest():
        return None
    try:
        return float(fields[field])
    except (KeyError, ValueError):
        return None


def profiled_traffic(kernel_tag: str, workload_tag: str):
    return profiled_field(kernel_tag, workload_tag, "traffic_bytes_per_launch")


def cpu_baseline(prob, target_s: float, oracle):
    """The FP64 oracle as it stands on all host cores, on the first rays of
    the same workload, sized to take about target_s seconds."""
    threads = oracle.hardware_threads()
    tally = np.zeros(prob.tally_size, np.float64)
    n = 1 << 14
    for _ in range(4):  # grow the sample until it takes about target_s
        tally[:] = 0.0
        sample = W.take_rays(prob, slice(0, n)).rays
        t0 = time.perf_counter()
        _, st = oracle.cast(prob, nthreads=threads, rays=sample, tally=tally)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or n >= prob.n_rays:
            break
        n = int(min(prob.n_rays, n * min(64.0, 0.9 * target_s / max(dt, 1e-3))))
    out = dict(value=st["segments"] / dt, unit=UNIT, cores=st["threads"], kind="oracle",
               sample=f"first {n} of the {prob.n_rays} rays of the {prob.name} workload "
                      f"({st['segments']} segments, {dt:.1f} s)")
    # the same oracle on one core, on a sample sized for about 3 s
    n1 = max(1024, min(n, int(n * 3.0 / max(dt * st["threads"], 1e-3))))
    t1 = np.zeros(prob.tally_size, np.float64)
    t0 = time.perf_counter()
    _, s1 = oracle.cast(prob, nthreads=1, rays=W.take_rays(prob, slice(0, n1)).rays, tally=t1)
    d1 = time.perf_counter() - t0
    out["value_one_core"] = s1["segments"] / d1
    out["sample_one_core"] = f"first {n1} rays ({s1['segments']} segments, {d1:.1f} s)"
    return out, tally, n


def roofline_figures(seg_per_step, live_per_step, rays_per_step, kernel_s, hbm):
    """Algorithmic HBM bytes per launch over the kernel time, two ways: every
    segment charged 17 B (tally read and write, material id), and only the
    segments that add a score charged the tally's 16 B (1 B material id for
    every walked segment); 32 B per ray in both."""
    alg = seg_per_step * BYTES_PER_SEGMENT + rays_per_step * BYTES_PER_RAY
    live = live_per_step * BYTES_PER_TALLY + seg_per_step * BYTES_PER_MATERIAL + rays_per_step * BYTES_PER_RAY
    return {"achieved_gbs": alg / kernel_s / 1e9, "frac": alg / kernel_s / 1e9 / hbm,
            "live_achieved_gbs": live / kernel_s / 1e9, "live_frac": live / kernel_s / 1e9 / hbm,
            "live_fraction_of_segments": live_per_step / max(seg_per_step, 1.0)}


def time_cast(vrc, torch, ctx, dev_rays, stream, steps, warmup):
    """Device-resident casts of one batch: CUDA events on the launching
    stream around `steps` casts after `warmup`, the library's own kernel
    timing, and the device counters of the timed casts."""
    for _ in range(warmup):
        vrc.vrc_cast_rays(ctx, dev_rays, stream=stream)
    rc, _ = vrc.vrc_sync(ctx, stream)
    assert rc == vrc.VRC_OK, rc
    vrc.vrc_reset_tally(ctx, stream)
    vrc.vrc_enable_timing(ctx, True)
    vrc.vrc_get_timing(ctx, stream, reset=True)
    torch.cuda.synchronize()
    l0 = vrc.vrc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        vrc.vrc_cast_rays(ctx, dev_rays, stream=stream)
    e1.record(stream)
    e1.synchronize()
    launches = vrc.vrc_launch_count() - l0
    rc, st = vrc.vrc_sync(ctx, stream)
    tm = vrc.vrc_get_timing(ctx, stream)
    vrc.vrc_enable_timing(ctx, False)
    assert rc == vrc.VRC_OK and st["overflow"] == 0, (rc, st)
    dt = e0.elapsed_time(e1) / 1e3
    return {"value": st["segments"] / dt, "ms_per_step": 1e3 * dt / steps,
            "kernel_ms": tm["cast_ms"] / max(tm["cast_launches"], 1),
            "sort_ms": tm["sort_ms"] / steps, "segments_per_step": st["segments"] / steps,
            "live_per_step": st["live"] / steps, "launches": launches, "steps": steps}


def parity_sample(vrc, ctx, prob, n_sample, stream, oracle):
    """The first n_sample rays of the workload cast into a fresh tally of the
    timed context, against the FP64 oracle on the same rays (Eq. 7 relative
    difference over cells with oracle tally >= 1e-30; segment counts)."""
    sub = W.take_rays(prob, slice(0, n_sample))
    want, st = oracle.cast(prob, rays=sub.rays)
    vrc.vrc_reset_tally(ctx, stream)
    vrc.vrc_cast_rays(ctx, sub.rays, stream=stream)
    rc, stats = vrc.vrc_sync(ctx, stream)
    got, _ = vrc.vrc_read_tally(ctx, stream=stream)
    sel = want >= 1e-30
    rel = np.abs(got[sel] - want[sel]) / want[sel]
    return {"rays": n_sample, "max_rel_err": float(rel.max()), "mean_rel_err": float(rel.mean()),
            "cells": int(sel.sum()), "segments_equal": bool(stats["segments"] == st["segments"]),
            "status": rc}


# --------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    prob = workload(args)
    threads = oracle.hardware_threads()
    per_step = max(1 << 12, min(prob.n_rays, 1 << 18))
    tally = np.zeros(prob.tally_size, np.float64)
    segs, times = [], []
    for s in range(args.warmup + args.steps):
        lo = (s * per_step) % prob.n_rays
        sample = W.take_rays(prob, slice(lo, lo + per_step)).rays
        t0 = time.perf_counter()
        _, st = oracle.cast(prob, nthreads=threads, rays=sample, tally=tally)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            segs.append(st["segments"])
            times.append(dt)
    value = sum(segs) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": headline_config(args, prob, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} consecutive rays of the {prob.name} workload per step "
                                   f"(each step a bounded sample of the step's 2^24 rays)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- batched form

PINLATTICE = ("pinlattice: 17x17 cylinders (pitch 1.26 cm, radius 0.45 cm) voxelised on a 544x544x64 "
              "mesh of 0.039375x0.039375x5 cm cells, 4 materials (core, void gap, cladding, moderator; "
              "20,000-point tables), 2^24 rays (70% starting in the cylinders), 1/E energies, seed 2")
BATCHED = ("batched1024: 1,024 independent problems, cubic meshes of 1 cm cells with side "
           "log-uniform in 16-128, 2-8 materials each from the 1,000-point table generator, "
           "uniform-random layout, ray counts log-uniform in 1e3-1e6 (1.4e8 rays), one group, "
           "seed 3; one persistent graph-captured launch per step")


def measure_batched(args, torch, vrc, local, steps, warmup, form, parity_problems=0):
    """The batched form: every step is one launch of the batch plan (all
    problems), timed with CUDA events; the plan's options come from the
    project's autotuner (sweep outside the timed region, cached per GPU).
    With parity_problems > 0, that many problems (evenly spaced) are checked
    cell by cell against the FP64 oracle after one more launch."""
    from paper_1706_07476_gb300 import autotune
    probs = W.batched_problems(seed=3, n_problems=args.problems)
    ctxs = [vrc.context_for(p, vrc.vrc_default_options(form=form, device=local)) for p in probs]
    rays = [{k: torch.from_numpy(p.rays[k]).cuda() for k in W.RAY_FIELDS} for p in probs]
    best, tuned_ms, table = autotune.tune_batched(torch, probs, ctxs, rays, form,
                                                  use_cache=not args.retune)
    batch = vrc.vrc_batch_create(ctxs, rays, vrc.vrc_default_batch_options(**best))
    stream = torch.cuda.Stream()
    for _ in range(warmup):
        vrc.vrc_batch_launch(batch, stream=stream)
    stream.synchronize()
    for c in ctxs:
        vrc.vrc_reset_tally(c)
        vrc.vrc_sync(c)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.__enter__()
    l0 = vrc.vrc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        vrc.vrc_batch_launch(batch, stream=stream)
    e1.record(stream)
    e1.synchronize()
    launches = vrc.vrc_launch_count() - l0
    sampler.__exit__(None, None, None)
    elapsed = e0.elapsed_time(e1) / 1e3
    seg = live = 0
    for c in ctxs:
        rc, st = vrc.vrc_sync(c)
        assert rc == vrc.VRC_OK and st["overflow"] == 0, (rc, st)
        seg += st["segments"]
        live += st["live"]
    n_rays = sum(p.n_rays for p in probs)
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    lf = roofline_figures(seg / steps, live / steps, n_rays, elapsed / steps, hbm)
    out = {
        "value": seg / elapsed, "ms_per_step": 1e3 * elapsed / steps, "steps": steps,
        "segments_per_step": seg / steps, "live_segments_per_step": live / steps,
        "rays_per_step": n_rays, "form": "fp32" if form else "plain",
        "autotuned_options": best, "tuned_ms": tuned_ms,
        "roofline": {"bound": "hbm", "achieved": lf["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                     "frac": lf["frac"], "live_frac": lf["live_frac"],
                     "traffic": profiled_field("k_cast_batched", "batched", "traffic_bytes_per_step",
                                               BATCHED_SOURCES),
                     "peak_source": f"{src} hbm_gbs", "kernel": "whole step (sort + k_cast_batched)"},
        "clocks": sampler.summary(), "gpu_launches": launches,
        "autotune_sweep": [{"options": o, "ms": ms} for o, ms in table],
    }
    if parity_problems:
        import oracle
        for c in ctxs:
            vrc.vrc_reset_tally(c)
        vrc.vrc_batch_launch(batch, stream=stream)
        stream.synchronize()
        worst, seg_ok = 0.0, True
        idx = np.linspace(0, len(probs) - 1, parity_problems).astype(int)
        for i in idx:
            want, st = oracle.cast(probs[i])
            got, rc = vrc.vrc_read_tally(ctxs[i])
            _, gst = vrc.vrc_sync(ctxs[i])
            sel = want >= 1e-30
            worst = max(worst, float((np.abs(got[sel] - want[sel]) / want[sel]).max()))
            seg_ok = seg_ok and gst["segments"] == st["segments"]
        out["parity_sample"] = {"problems": len(idx), "max_rel_err": worst, "segments_equal": seg_ok}
    batch.close()
    for c in ctxs:
        c.close()
    del rays
    torch.cuda.empty_cache()
    return out, probs


def run_batched(args, rank, world, local):
    """--workload batched: the batched form's own JSON line."""
    import torch
    from paper_1706_07476_gb300 import vrc
    torch.cuda.set_device(local)
    form = vrc.VRC_FORM_FP32 if args.forms.split(",")[-1].strip() == "fp32" else vrc.VRC_FORM_PLAIN
    m, probs = measure_batched(args, torch, vrc, local, args.steps, args.warmup, form)
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if form else "f64",
        "data": "synthetic",
        "config": {"workload": BATCHED, "rays_per_step": m["rays_per_step"],
                   "segments_per_step": m["segments_per_step"], "form": m["form"],
                   "autotuned_options": m["autotuned_options"], "tuned_ms": m["tuned_ms"],
                   "l2": "inputs larger than L2 (4.5 GB rays, 2.6 GB tallies); no flush"},
        "roofline": m["roofline"], "clocks": m["clocks"], "gpu_launches": m["gpu_launches"],
        "autotune_sweep": m["autotune_sweep"],
    }
    if not args.no_cpu_baseline:
        import oracle
        idx = np.linspace(0, len(probs) - 1, 64).astype(int)
        t0 = time.perf_counter()
        segs = sum(oracle.cast(probs[i])[1]["segments"] for i in idx)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": segs / dt, "unit": UNIT, "cores": oracle.hardware_threads(),
                                "kind": "oracle",
                                "sample": f"64 of the 1,024 problems, evenly spaced ({segs} segments, {dt:.1f} s)"}
    print(json.dumps(line), flush=True)
    return 0


def measure_pinlattice(args, torch, vrc, local, stream, steps, warmup, oracle=None):
    """The pin lattice (544 x 544 x 64 cells of 0.039 x 0.039 x 5 cm, 2^24
    rays, FP32 form, one group): device-resident casts timed like the
    headline, and a parity sample of 2^20 rays against the FP64 oracle."""
    prob = W.pin_lattice(seed=2)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, device=local))
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
    r = time_cast(vrc, torch, ctx, dev, stream, steps, warmup)
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    lf = roofline_figures(r["segments_per_step"], r["live_per_step"], prob.n_rays, r["kernel_ms"] / 1e3, hbm)
    out = {"workload": PINLATTICE, "form": "fp32", "rays_per_step": prob.n_rays, **r,
           "roofline": {"bound": "hbm", "achieved": lf["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                        "frac": lf["frac"], "live_frac": lf["live_frac"], "traffic": None,
                        "peak_source": f"{src} hbm_gbs", "kernel": "k_cast<fp32>"}}
    if oracle is not None:
        out["parity_sample"] = parity_sample(vrc, ctx, prob, 1 << 20, stream, oracle)
    ctx.close()
    del dev
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------------------- streaming

def run_stream(args, rank, world, local):
    """Producer overlap: CPU threads copy the slab256 rays into pinned
    buffers of 2^20 records (the stand-in for a random walk filling its ray
    buffer) while earlier buffers are uploaded and cast.  Reports the
    producer alone, the GPU alone (buffers filled beforehand) and the two
    overlapped, in rays/s and segments/s."""
    import concurrent.futures as cf
    import torch
    from paper_1706_07476_gb300 import vrc
    torch.cuda.set_device(local)
    prob = workload(args)
    records = np.ascontiguousarray(np.stack([prob.rays[k] for k in W.RAY_FIELDS], axis=1))
    cap = 1 << 20
    nbuf = (prob.n_rays + cap - 1) // cap
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, device=local))
    rs = vrc.RayStream(ctx, cap, 3)
    pool = cf.ThreadPoolExecutor(max_workers=8)

    def fill(buf, lo, n):
        parts = [(i * n // 8, (i + 1) * n // 8) for i in range(8)]
        list(pool.map(lambda ab: buf.__setitem__(slice(ab[0], ab[1]), records[lo + ab[0]:lo + ab[1]]), parts))

    def run(produce: bool, cast: bool):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in range(nbuf):
            lo = b * cap
            n = min(cap, prob.n_rays - lo)
            buf = rs.acquire()
            if produce:
                fill(buf, lo, n)
            if cast:
                rs.submit(n)
            else:
                rs.submit(0)
        rs.finish()
        return time.perf_counter() - t0

    for _ in range(max(1, args.warmup)):
        run(True, True)
    t_cpu = min(run(True, False) for _ in range(2))
    vrc.vrc_reset_tally(ctx)
    t_gpu = min(run(False, True) for _ in range(2))
    vrc.vrc_reset_tally(ctx)
    vrc.vrc_sync(ctx)
    t_both = [run(True, True) for _ in range(max(1, min(args.steps, 5)))]
    rc, st = vrc.vrc_sync(ctx)
    seg_per_pass = st["segments"] / len(t_both)
    tb = min(t_both)
    line = {
        "metric": "streamed ray buffers: rays/s and segments/s with producer overlap",
        "value": seg_per_pass / tb, "unit": UNIT, "n_gpus": world, "steps": len(t_both),
        "warmup": args.warmup, "ms_per_step": 1e3 * tb, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "buffer_rays": cap, "buffers": 3, "producer_threads": 8},
        "producer_only_rays_per_s": prob.n_rays / t_cpu,
        "gpu_only_rays_per_s": prob.n_rays / t_gpu,
        "overlapped_rays_per_s": prob.n_rays / tb,
        "overlap_efficiency": max(t_cpu, t_gpu) / tb,
        "gpu_time_over_cpu_time": t_gpu / t_cpu,
    }
    rs.close()
    ctx.close()
    pool.shutdown()
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- per-history moments

def measure_history(args, torch, vrc, local, prob, stream, steps, warmup):
    """Per-history moments: every step casts the slab256 rays in 16 calls of
    2^20 rays through vrc_cast_histories (sort of the rays with their
    history ids, cast into per-ray pair records with bucket counts, bucket
    scatter, fold into S1/S2), FP32 form, device inputs, timed with CUDA
    events on the calling stream; the plain tally cast of the same calls
    (sorted too) is timed beside it.  Returns the history figures, both
    modes and the launch count."""
    rng = np.random.default_rng(6)
    lengths = rng.integers(1, 16, size=prob.n_rays // 4)
    hist = np.repeat(np.arange(lengths.size, dtype=np.uint32), lengths)[:prob.n_rays]
    chunk = 1 << 20
    starts = list(range(0, prob.n_rays, chunk))
    # calls end on a history boundary: move each cut back to its history's first ray
    cuts = [0]
    for s0 in starts[1:]:
        c = s0
        while c > cuts[-1] and hist[c] == hist[c - 1]:
            c -= 1
        cuts.append(c)
    cuts.append(prob.n_rays)
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
    hdev = torch.from_numpy(hist.view(np.int32)).cuda()
    parts = [({k: v[a:b] for k, v in dev.items()}, hdev[a:b], int(hist[b - 1]) - int(hist[a]) + 1)
             for a, b in zip(cuts[:-1], cuts[1:])]
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, device=local))

    def step_hist():
        for r, h, nh in parts:
            vrc.vrc_cast_histories(ctx, r, h, nh, stream=stream)

    def step_tally():
        for r, _, _ in parts:
            vrc.vrc_cast_rays(ctx, r, stream=stream)

    out = {}
    for name, fn, mode in (("tally", step_tally, vrc.VRC_MOMENTS_OFF), ("history", step_hist, vrc.VRC_MOMENTS_HISTORY)):
        vrc.vrc_moments_enable(ctx, mode)
        for _ in range(warmup):
            fn()
        stream.synchronize()
        vrc.vrc_reset_tally(ctx, stream)
        vrc.vrc_moments_enable(ctx, mode)
        torch.cuda.synchronize()
        n = max(1, min(steps, 10))
        l0 = vrc.vrc_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - t0
        rc, st = vrc.vrc_sync(ctx, stream)
        assert rc == vrc.VRC_OK and st["overflow"] == 0, (rc, st)
        dt = e0.elapsed_time(e1) / 1e3
        out[name] = {"segments_per_s": st["segments"] / dt, "ms_per_step": 1e3 * dt / n,
                     "wall_ms_per_step": 1e3 * wall / n, "segments_per_step": st["segments"] / n,
                     "steps": n, "launches": vrc.vrc_launch_count() - l0}
    _, _, samples = vrc.vrc_moments_read(ctx)
    ctx.close()
    n_calls = len(parts)
    del dev, hdev, parts
    torch.cuda.empty_cache()
    H = out["history"]
    return {"workload": HISTORY, "form": "fp32", "value": H["segments_per_s"], "unit": UNIT,
            "ms_per_step": H["ms_per_step"], "segments_per_step": H["segments_per_step"],
            "rays_per_step": prob.n_rays, "calls_per_step": n_calls,
            "histories_per_step": int(hist[-1]) + 1, "steps": H["steps"],
            "history_over_tally_time": H["ms_per_step"] / out["tally"]["ms_per_step"],
            "modes": out, "histories_folded": samples, "gpu_launches": H["launches"],
            "parity": "tests/test_history_moments_gpu.py (the oracle's per-history moments are "
                      "per-history full casts, too slow at this size)"}


def run_history(args, rank, world, local):
    """The per-history workload on its own (measure_history), one JSON line."""
    import torch
    from paper_1706_07476_gb300 import vrc
    torch.cuda.set_device(local)
    prob = workload(args)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    m = measure_history(args, torch, vrc, local, prob, stream, args.steps, args.warmup)
    line = {
        "metric": "per-history moments: ray-cell segments/s", "value": m["value"],
        "unit": UNIT, "n_gpus": world, "steps": m["steps"], "warmup": args.warmup,
        "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": HISTORY, "rays_per_step": prob.n_rays, "calls_per_step": m["calls_per_step"],
                   "histories_per_step": m["histories_per_step"], "form": "fp32", "sort": "auto (each call)"},
        "history_over_tally_time": m["history_over_tally_time"],
        "modes": m["modes"], "histories_folded": m["histories_folded"], "gpu_launches": m["gpu_launches"],
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- next-event detectors

def run_detectors(args, rank, world, local):
    """Next-event estimator: every step scores all slab256 rays at 8 detector
    points through vrc_detector_flux (device rays, both forms), timed with
    CUDA events on the calling stream; the unit is (ray, detector) pairs."""
    import torch
    from paper_1706_07476_gb300 import vrc
    torch.cuda.set_device(local)
    prob = workload(args)
    hi = np.array(prob.mesh.hi)
    det = np.array([[fx, fy, fz] for fz in (0.25, 0.75) for fy in (0.25, 0.75) for fx in (0.25, 0.75)]) * hi
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {}
    launches = 0
    for form in [f.strip() for f in args.forms.split(",") if f.strip()]:
        fid = vrc.VRC_FORM_FP32 if form == "fp32" else vrc.VRC_FORM_PLAIN
        ctx = vrc.context_for(prob, vrc.vrc_default_options(form=fid, device=local))
        for _ in range(args.warmup):
            vrc.vrc_detector_flux(ctx, dev, det, stream=stream)
        steps = max(1, min(args.steps, 5))
        l0 = vrc.vrc_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            flux = vrc.vrc_detector_flux(ctx, dev, det, stream=stream)
        e1.record(stream)
        e1.synchronize()
        launches = vrc.vrc_launch_count() - l0
        dt = e0.elapsed_time(e1) / 1e3 / steps
        rc, _ = vrc.vrc_sync(ctx)
        assert rc == vrc.VRC_OK, rc
        out[form] = {"pairs_per_s": prob.n_rays * len(det) / dt, "ms_per_step": 1e3 * dt,
                     "flux_total": float(flux.sum())}
        ctx.close()
    head = out[list(out)[-1]]
    line = {
        "metric": "next-event detector estimates: (ray, detector) pairs/s", "value": head["pairs_per_s"],
        "unit": "pairs/s", "n_gpus": world, "steps": max(1, min(args.steps, 5)), "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if list(out)[-1] == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": DETECTORS, "rays_per_step": prob.n_rays, "detectors": len(det)},
        "forms": out, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- learned cross sections

def measure_surrogate(args, torch, vrc, local, stream, steps, warmup, oracle=None):
    """The surrogate workload: trains the network (vrc_train_surrogate, outside
    the timed regions), then times whole casts (sort, network, walk) with
    CUDA events: (a) table cross sections, (b) the surrogate where validation
    accepts it at 1e-3 (the table elsewhere), (c) the network on every ray;
    and (d) the network's forward pass alone on the 2^24 ray energies, whose
    two 128-wide layers run on tcgen05.  With the oracle, parity samples of
    (a) and (b) on 2^20 rays."""
    prob = W.surrogate_mesh(seed=4, n_rays=args.n_rays)
    ctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, device=local))
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
    t0 = time.perf_counter()
    rep = vrc.vrc_train_surrogate(ctx)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    out = {}
    for name, mode in (("table", vrc.VRC_XS_TABLE), ("surrogate_checked", vrc.VRC_XS_SURROGATE)):
        vrc.vrc_set_xs_mode(ctx, mode)
        out[name] = time_cast(vrc, torch, ctx, dev, stream, steps, warmup)
    every = vrc.vrc_train_surrogate(ctx, vrc.vrc_default_surrogate_options(steps=0, tol=1e30))
    out["network_everywhere"] = time_cast(vrc, torch, ctx, dev, stream, steps, warmup)
    out["network_everywhere"]["coverage"] = every["coverage"]
    vrc.vrc_train_surrogate(ctx, vrc.vrc_default_surrogate_options(steps=0))  # back to the 1e-3 bound
    params = torch.from_numpy(vrc.vrc_get_surrogate_params(ctx)).cuda()
    y = torch.empty((prob.n_rays, 16), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        vrc.vrc_mlp_forward(params, dev["E"], W.E_MIN_EV, W.E_MAX_EV, y, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        vrc.vrc_mlp_forward(params, dev["E"], W.E_MIN_EV, W.E_MAX_EV, y, stream=stream)
    e1.record(stream)
    e1.synchronize()
    dt_mlp = e0.elapsed_time(e1) / 1e3 / steps
    # the products issued on the tensor cores: two 128-wide layers with each
    # activation as a bfloat16 pair (hi, lo), and the 128 -> 16 output layer
    # as five products (activation hi, lo x weight hi, mid, lo)
    tensor_flop = 2.0 * prob.n_rays * (2 * 64 * 128 + 2 * 128 * 128 + 5 * 128 * 16)
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    res = {
        "workload": SURROGATE, "form": "fp32", "rays_per_step": prob.n_rays,
        "value": out["surrogate_checked"]["value"],
        "ms_per_step": out["surrogate_checked"]["ms_per_step"],
        "gain_vs_table": out["surrogate_checked"]["value"] / out["table"]["value"],
        "modes": out,
        "training": {"seconds": train_s, "coverage_at_1e-3": rep["coverage"],
                     "bins_accepted": rep["bins_accepted"], "bins": rep["bins"],
                     "max_rel_err_accepted": rep["max_rel_err_accepted"],
                     "median_rel_err": rep["median_rel_err"], "smooth_fraction": rep["smooth_fraction"],
                     "final_loss": rep["final_loss"]},
        "mlp_forward": {"ms": 1e3 * dt_mlp, "rays_per_s": prob.n_rays / dt_mlp,
                        "kernel": "k_mlp_apply_tc (tcgen05.mma kind::f16, M = 128, N = 128, 48 and 32)"},
        "roofline": {"bound": "tensor", "achieved": tensor_flop / dt_mlp / 1e12, "peak": peak,
                     "unit": "TFLOP/s", "frac": tensor_flop / dt_mlp / 1e12 / peak, "traffic": None,
                     "peak_source": f"{src} bf16_tflops (cuBLAS bf16 GEMM, burst)",
                     "algorithmic_flops": "2 x (2 x 64 x 128 + 2 x 128 x 128 + 5 x 128 x 16) per ray on the tensor cores",
                     "kernel": "k_mlp_apply_tc"},
    }
    if oracle is not None:
        par = {}
        for name, mode in (("table", vrc.VRC_XS_TABLE), ("surrogate_checked", vrc.VRC_XS_SURROGATE)):
            vrc.vrc_set_xs_mode(ctx, mode)
            par[name] = parity_sample(vrc, ctx, prob, 1 << 20, stream, oracle)
        res["parity_sample"] = par
    ctx.close()
    del dev, y
    torch.cuda.empty_cache()
    return res


def run_surrogate(args, rank, world, local):
    """--workload surrogate: the surrogate workload's own JSON line."""
    import torch
    from paper_1706_07476_gb300 import vrc
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    steps = max(1, min(args.steps, 10))
    m = measure_surrogate(args, torch, vrc, local, stream, steps, args.warmup)
    line = {
        "metric": "ray-cell segments/s with learned cross sections where validated (table elsewhere)",
        "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (network: bf16 tensor cores, f32 accumulate)",
        "data": "synthetic", "config": {"workload": SURROGATE, "rays_per_step": m["rays_per_step"]},
        **{k: m[k] for k in ("gain_vs_table", "modes", "training", "mlp_forward", "roofline")},
        "gpu_launches": m["modes"]["surrogate_checked"]["launches"],
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args, rank, world, local)
    if args.workload == "stream":
        return run_stream(args, rank, world, local)
    if args.workload == "history":
        return run_history(args, rank, world, local)
    if args.workload == "detectors":
        return run_detectors(args, rank, world, local)
    if args.workload == "surrogate":
        return run_surrogate(args, rank, world, local)

    import torch
    import torch.distributed as dist
    from paper_1706_07476_gb300 import micro, vrc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    prob = workload(args)
    dev_rays = {k: torch.from_numpy(v).cuda() for k, v in prob.rays.items()}
    # a dedicated stream: the legacy default stream has handle 0, which the C
    # ABI reads as "the context's own stream"
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    form_id = {"plain": vrc.VRC_FORM_PLAIN, "fp32": vrc.VRC_FORM_FP32}

    results = {}
    ctxs = {}
    clocks = None
    launches = 0
    for fi, form in enumerate(forms):
        headline = fi == len(forms) - 1
        ctx = vrc.context_for(prob, vrc.vrc_default_options(form=form_id[form], sort=args.sort,
                                                            rays_per_warp=args.rays_per_warp,
                                                            device=local))
        ctxs[form] = ctx
        for _ in range(args.warmup):
            vrc.vrc_cast_rays(ctx, dev_rays, stream=stream)
        rc, _ = vrc.vrc_sync(ctx, stream)
        assert rc == vrc.VRC_OK, rc
        vrc.vrc_reset_tally(ctx, stream)
        vrc.vrc_enable_timing(ctx, True)
        vrc.vrc_get_timing(ctx, stream, reset=True)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if headline else None
        if sampler:
            sampler.__enter__()
        l0 = vrc.vrc_launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            vrc.vrc_cast_rays(ctx, dev_rays, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        n_launch = vrc.vrc_launch_count() - l0
        if sampler:
            sampler.__exit__(None, None, None)
            clocks = sampler.summary()
            launches = n_launch
        barrier()
        elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
        rc, stats = vrc.vrc_sync(ctx, stream)
        timing = vrc.vrc_get_timing(ctx, stream)
        assert rc == vrc.VRC_OK and stats["overflow"] == 0 and stats["rejected"] == 0, (rc, stats)
        seg_per_step = stats["segments"] / args.steps
        total = sum_over_ranks(stats["segments"])
        kernel_s = timing["cast_ms"] / 1e3 / max(timing["cast_launches"], 1)
        alg_bytes = seg_per_step * BYTES_PER_SEGMENT + prob.n_rays * BYTES_PER_RAY
        results[form] = dict(value=total / elapsed, ms_per_step=1e3 * elapsed / args.steps,
                             segments_per_step=seg_per_step, kernel_ms=1e3 * kernel_s,
                             alg_gbs=alg_bytes / kernel_s / 1e9, launches=n_launch,
                             live_segments_per_step=stats["live"] / args.steps,
                             live_segments_per_s=sum_over_ranks(stats["live"]) / elapsed)

    head = forms[-1]
    R = results[head]

    # opt-in early exit (options.stop_at_zero): same tally, walks end once a
    # ray's transmitted fraction is exactly 0; reported beside the headline
    stop = None
    if head == "fp32" and rank == 0:
        sctx = vrc.context_for(prob, vrc.vrc_default_options(form=vrc.VRC_FORM_FP32, sort=args.sort,
                                                             stop_at_zero=1, device=local))
        for _ in range(args.warmup):
            vrc.vrc_cast_rays(sctx, dev_rays, stream=stream)
        vrc.vrc_reset_tally(sctx, stream)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            vrc.vrc_cast_rays(sctx, dev_rays, stream=stream)
        s1.record(stream)
        s1.synchronize()
        rc, sst = vrc.vrc_sync(sctx, stream)
        assert rc == vrc.VRC_OK, rc
        st_s = s0.elapsed_time(s1) / 1e3 / args.steps
        stop = {"rays_per_s": prob.n_rays / st_s, "ms_per_step": 1e3 * st_s,
                "walked_segments_per_step": sst["segments"] / args.steps,
                "speedup_vs_full_walk": R["ms_per_step"] / (1e3 * st_s),
                "note": "options.stop_at_zero=1: same tally; walks end once exp(-tau) is exactly 0 "
                        "in float32; not the headline, which walks every ray to the mesh exit"}
        sctx.close()

    # end to end: host rays from pinned memory through the C ABI, per-step
    # device->host read of the step's status and counters
    e2e = None
    ctx = ctxs[head]
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in prob.rays.items()}
    vrc.vrc_enable_timing(ctx, False)
    for _ in range(max(1, args.warmup)):
        vrc.vrc_cast_rays(ctx, pinned, stream=stream)
        vrc.vrc_sync(ctx, stream)
    vrc.vrc_reset_tally(ctx, stream)
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    seg = 0
    for _ in range(e2e_steps):
        vrc.vrc_cast_rays(ctx, pinned, stream=stream)
        rc, st = vrc.vrc_sync(ctx, stream)
    t1 = time.perf_counter()
    seg = st["segments"]
    barrier()
    e2e_t = max_over_ranks(t1 - t0)
    e2e = {"value": sum_over_ranks(seg) / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": BYTES_PER_RAY * prob.n_rays,
           "d2h_bytes_per_step": 4 * 8 + 4,
           "note": "vrc_cast_rays on pinned host rays (upload inside) + vrc_sync reading the "
                   "step's counters and status; the tally stays on the device"}

    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roof = {"bound": "hbm", "achieved": R["alg_gbs"], "peak": hbm, "unit": "GB/s",
            "frac": R["alg_gbs"] / hbm, "traffic": profiled_traffic(f"k_cast_{head}", args.workload),
            "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy)",
            "algorithmic_bytes": f"{BYTES_PER_SEGMENT} B/segment + {BYTES_PER_RAY} B/ray",
            "kernel": f"k_cast<{head}>", "kernel_ms": R["kernel_ms"]}
    # the same roofline with the tally's 16 B charged only to the segments
    # that add a score (a segment past the point where exp(-tau) is exactly 0
    # reads its material id and nothing else)
    lf = roofline_figures(R["segments_per_step"], R["live_segments_per_step"], prob.n_rays,
                          R["kernel_ms"] / 1e3, hbm)
    roof["live"] = {"achieved": lf["live_achieved_gbs"], "frac": lf["live_frac"],
                    "live_segments_per_step": R["live_segments_per_step"],
                    "live_fraction_of_segments": lf["live_fraction_of_segments"],
                    "algorithmic_bytes": "16 B per live segment + 1 B per segment + 32 B per ray"}
    # the kernel's binding limit is instruction issue: warp instructions per
    # segment from the committed profile, against 4 schedulers x SMs x clock
    wips = profiled_field(f"k_cast_{head}", args.workload, "warp_instructions_per_segment")
    if wips:
        props = torch.cuda.get_device_properties(local)
        sm_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        cap = props.multi_processor_count * 4 * sm_hz / wips
        kernel_rate = R["segments_per_step"] / (R["kernel_ms"] / 1e3)
        roof["issue_roof"] = {"warp_instructions_per_segment": wips, "cap_segments_per_s": cap,
                              "kernel_segments_per_s": kernel_rate, "frac": kernel_rate / cap,
                              "basis": "SMs x 4 schedulers x max SM clock / (warp instructions per "
                                       "segment from the committed ncu profile)"}

    extra = {}
    if not args.no_micro and rank == 0:
        try:
            red_hbm = micro.red_f64_rate(torch, 1 << 28, 1 << 28)
            red_l2 = micro.red_f64_rate(torch, 1 << 22, 1 << 28)
            extra["micro"] = {
                "red_f64_hbm_per_s": red_hbm, "red_f64_l2_per_s": red_l2,
                "fma_f64_flops": micro.arith_rate(torch, "fma_f64"),
                "fma_f32_flops": micro.arith_rate(torch, "fma_f32"),
                "expm1_f64_per_s": micro.arith_rate(torch, "expm1_f64", iters=500),
                "expm1_f32_per_s": micro.arith_rate(torch, "expm1_f32", iters=500),
            }
            roof["atomic_roof_segments_per_s"] = red_hbm
            roof["frac_of_atomic_roof"] = R["value"] / world / red_hbm
            roof["atomic_roof_basis"] = (
                "one segment per random float64 red on a 2 GiB array (no locality), measured in "
                "this run; the cast beats it because only segments whose transmitted fraction is "
                "not yet 0 issue a red, and the ray sort gives those reds L2 locality")
        except Exception as e:  # measurement aid only
            extra["micro"] = {"error": str(e)}

    line = {
        "metric": METRIC, "value": R["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": R["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if head == "fp32" else "f64", "data": "synthetic",
        "config": headline_config(args, prob, world),
        "segments_per_step": R["segments_per_step"],
        "forms": results,
        "stop_at_zero": stop,
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    line.update(extra)

    if rank == 0 and world == 1:
        import oracle
        if not args.no_cpu_baseline:
            cb, otally, n_sample = cpu_baseline(prob, args.cpu_seconds, oracle)
            line["cpu_baseline"] = cb
            if not args.no_parity_sample:
                # the timed configuration, on the sampled rays, against the oracle
                par = {}
                for form in forms:
                    c = ctxs[form]
                    vrc.vrc_reset_tally(c, stream)
                    sub = {k: v[:n_sample] for k, v in dev_rays.items()}
                    vrc.vrc_cast_rays(c, sub, stream=stream)
                    got, rc = vrc.vrc_read_tally(c, stream=stream)
                    sel = otally >= 1e-30
                    rel = np.abs(got[sel] - otally[sel]) / otally[sel]
                    par[form] = {"rays": n_sample, "max_rel_err": float(rel.max()),
                                 "mean_rel_err": float(rel.mean()), "cells": int(sel.sum())}
                line["parity_sample"] = par
    for c in ctxs.values():
        c.close()
    del dev_rays, pinned
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_configs and args.workload == "slab256":
        # the other workloads, a few steps each, each with its parity sample
        import oracle
        cs, cw = max(1, args.config_steps), max(3, min(args.warmup, 3))
        configs = {"pinlattice": measure_pinlattice(args, torch, vrc, local, stream, cs, cw, oracle)}
        m, _ = measure_batched(args, torch, vrc, local, cs, cw, vrc.VRC_FORM_FP32, parity_problems=16)
        m["workload"] = BATCHED
        configs["batched1024"] = m
        configs["surrogate32"] = measure_surrogate(args, torch, vrc, local, stream, cs, cw, oracle)
        configs["history"] = measure_history(args, torch, vrc, local, prob, stream, cs, cw)
        line["configs"] = configs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
