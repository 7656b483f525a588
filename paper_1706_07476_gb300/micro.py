"""Roofline microbenchmarks (include/vrc_micro.h) timed with CUDA events.

Measures, on the current device: scattered float64 atomic-add throughput on
an HBM-resident and an L2-resident array, and float64 / float32 FMA and
expm1 rates.  Used by bench.py to state the roofs the cast runs against.
"""
from __future__ import annotations

import ctypes as C

from paper_1706_07476_gb300 import vrc

_lib = vrc.library()
for _name, _args in {
    "vrc_micro_red_f64": [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p],
    "vrc_micro_fma_f64": [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p],
    "vrc_micro_fma_f32": [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p],
    "vrc_micro_expm1_f64": [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p],
    "vrc_micro_expm1_f32": [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p],
}.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = C.c_int


def _time(torch, fn, reps=3):
    s = torch.cuda.current_stream()
    best = float("inf")
    fn()  # warm-up
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        best = min(best, a.elapsed_time(b) / 1e3)
    return best


def red_f64_rate(torch, n_elems: int, updates: int) -> float:
    """Random float64 atomic adds per second on an array of n_elems doubles."""
    buf = torch.zeros(n_elems, dtype=torch.float64, device="cuda")
    s = int(torch.cuda.current_stream().cuda_stream)

    def run():
        rc = _lib.vrc_micro_red_f64(buf.data_ptr(), n_elems, updates, s)
        if rc:
            raise vrc.VrcError(rc, "micro red")

    t = _time(torch, run)
    total = float(buf.sum().item())
    assert abs(total - updates * 4) < 0.5, total  # one warm-up + three timed runs
    del buf
    return updates / t


def arith_rate(torch, kind: str, threads: int = 152 * 2048, iters: int = 2000) -> float:
    """Operations per second: FMA counted as 2 flops; expm1 as 1 evaluation."""
    dt = torch.float64 if kind.endswith("64") else torch.float32
    out = torch.empty(threads, dtype=dt, device="cuda")
    s = int(torch.cuda.current_stream().cuda_stream)
    fn = getattr(_lib, f"vrc_micro_{kind}")

    def run():
        rc = fn(out.data_ptr(), threads, iters, s)
        if rc:
            raise vrc.VrcError(rc, f"micro {kind}")

    t = _time(torch, run)
    work = (16 if kind.startswith("fma") else 4) * iters * threads
    return work / t
