"""FP64 CPU oracle for the VRC fluence estimator (Eqs. 1-4, Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never links, loads or calls it, and it never calls the CUDA
library; the two share only the seeded input generators (``vrc_workloads``).

The arithmetic lives in ``vrc_oracle.c`` (plain C, double precision, no fused
multiply-add contraction); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.  ``mlp.py`` holds the FP64 reference of
the learned cross-section surrogate.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-pthread", "-ffp-contract=off", "-fno-fast-math", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("material", C.c_void_p), ("xe", C.c_void_p), ("ye", C.c_void_p),
                ("ze", C.c_void_p)]


class _XS(C.Structure):
    _fields_ = [("n_materials", C.c_int32), ("E", C.c_void_p), ("S", C.c_void_p),
                ("offs", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, D, I64, I32, F = C.c_void_p, C.c_double, C.c_int64, C.c_int32, C.c_float
            lib.orc_sigma_t.argtypes = [P, P, I64, D]
            lib.orc_sigma_t.restype = D
            lib.orc_group.argtypes = [P, I32, D]
            lib.orc_group.restype = I32
            lib.orc_trace_dda.argtypes = [P, P, P, P, P, P, I64]
            lib.orc_trace_dda.restype = I64
            lib.orc_trace_brute.argtypes = [P, P, P, P, P, P, I64, P]
            lib.orc_trace_brute.restype = I64
            lib.orc_ray_segments.argtypes = [P, P, P, I32] + [F] * 8 + [P, P, P, P, P, I64]
            lib.orc_ray_segments.restype = I64
            lib.orc_cast.argtypes = [P, P, P, I32] + [P] * 8 + [I64, P, I32, P]
            lib.orc_cast.restype = I32
            lib.orc_point_detector.argtypes = [P, P, P, I32] + [P] * 5 + [I64, P, I32, P]
            lib.orc_point_detector.restype = I32
            lib.orc_hardware_threads.argtypes = []
            lib.orc_hardware_threads.restype = I32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Ctx:
    """Keeps the numpy buffers behind the ctypes structs alive."""

    def __init__(self, mesh, tables=None):
        self.mat = np.ascontiguousarray(mesh.material, dtype=np.uint8).reshape(-1)
        assert self.mat.size == mesh.nx * mesh.ny * mesh.nz
        # a rectilinear mesh carries its plane positions per axis
        self.edges = [None if getattr(mesh, a, None) is None
                      else np.ascontiguousarray(getattr(mesh, a), np.float64)
                      for a in ("xe", "ye", "ze")]
        for e, n in zip(self.edges, (mesh.nx, mesh.ny, mesh.nz)):
            assert e is None or (e.shape == (n + 1,) and np.all(np.diff(e) > 0))
        ep = [None if e is None else e.ctypes.data for e in self.edges]
        self.mesh = _Mesh(mesh.nx, mesh.ny, mesh.nz, mesh.x0, mesh.y0, mesh.z0,
                          mesh.dx, mesh.dy, mesh.dz, self.mat.ctypes.data, *ep)
        if tables is not None:
            Es, Ss, offs = [], [], [0]
            for t in tables:
                if t is None:
                    offs.append(offs[-1])
                else:
                    Es.append(np.asarray(t[0], np.float64))
                    Ss.append(np.asarray(t[1], np.float64))
                    offs.append(offs[-1] + len(t[0]))
            self.E = np.ascontiguousarray(np.concatenate(Es) if Es else np.zeros(1))
            self.S = np.ascontiguousarray(np.concatenate(Ss) if Ss else np.zeros(1))
            self.offs = np.asarray(offs, np.int64)
            self.xs = _XS(len(tables), self.E.ctypes.data, self.S.ctypes.data,
                          self.offs.ctypes.data)


def hardware_threads() -> int:
    return int(_load().orc_hardware_threads())


def sigma_t(E: np.ndarray, S: np.ndarray, e: float) -> float:
    """Lin-lin sigma_t(e) by binary search on one table (clamped outside)."""
    E = np.ascontiguousarray(E, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    return float(_load().orc_sigma_t(_ptr(E), _ptr(S), len(E), float(e)))


def group(edges, e: float) -> int:
    if edges is None:
        return int(_load().orc_group(None, 0, float(e)))
    edges = np.ascontiguousarray(edges, np.float64)
    return int(_load().orc_group(_ptr(edges), len(edges) - 1, float(e)))


def _cap(mesh):
    return mesh.nx + mesh.ny + mesh.nz + 3


def trace_dda(mesh, p, d):
    """Grid walk of the half-line p + t d (d unit).  Returns (cells, t_in, lens)."""
    ctx = _Ctx(mesh)
    cap = _cap(mesh)
    cells = np.zeros(cap, np.int64)
    tin = np.zeros(cap, np.float64)
    lens = np.zeros(cap, np.float64)
    p = np.asarray(p, np.float64)
    d = np.asarray(d, np.float64)
    n = _load().orc_trace_dda(C.byref(ctx.mesh), _ptr(p), _ptr(d), _ptr(cells), _ptr(tin),
                              _ptr(lens), cap)
    if n < 0:
        raise RuntimeError("grid walk exceeded its step bound")
    return cells[:n], tin[:n], lens[:n]


def trace_brute(mesh, p, d):
    """Plane-crossing traversal (positive-length segments only)."""
    ctx = _Ctx(mesh)
    cap = _cap(mesh) + 2
    cells = np.zeros(cap, np.int64)
    tin = np.zeros(cap, np.float64)
    lens = np.zeros(cap, np.float64)
    tbuf = np.zeros(cap + 8, np.float64)
    p = np.asarray(p, np.float64)
    d = np.asarray(d, np.float64)
    n = _load().orc_trace_brute(C.byref(ctx.mesh), _ptr(p), _ptr(d), _ptr(cells), _ptr(tin),
                                _ptr(lens), cap, _ptr(tbuf))
    if n < 0:
        raise RuntimeError("brute traversal buffer too small")
    return cells[:n], tin[:n], lens[:n]


def ray_segments(problem, i: int):
    """Per-step detail of ray i: dict of cells, t_in, lens, sigma, score."""
    ctx = _Ctx(problem.mesh, problem.tables)
    cap = _cap(problem.mesh)
    out = {k: np.zeros(cap, np.float64) for k in ("t_in", "lens", "sigma", "score")}
    cells = np.zeros(cap, np.int64)
    r = problem.rays
    edges = problem.group_edges
    keep = None if edges is None else np.ascontiguousarray(edges, np.float64)
    ep = None if keep is None else _ptr(keep)
    ng = 0 if keep is None else len(keep) - 1
    vals = [float(r[k][i]) for k in ("x", "y", "z", "u", "v", "w", "E", "wt")]
    n = _load().orc_ray_segments(C.byref(ctx.mesh), C.byref(ctx.xs), ep, ng, *vals, _ptr(cells),
                                 _ptr(out["t_in"]), _ptr(out["lens"]), _ptr(out["sigma"]),
                                 _ptr(out["score"]), cap)
    if n < 0:
        raise RuntimeError("grid walk exceeded its step bound")
    res = {k: v[:n] for k, v in out.items()}
    res["cells"] = cells[:n]
    return res


def cast(problem, nthreads: int = 0, rays: dict | None = None, tally: np.ndarray | None = None):
    """Eq. 4 tally of a ray batch, float64 [n_groups * ncells].

    Returns (tally, stats) with stats = dict(segments, rejected, overflow,
    threads).  ``tally`` may be passed to accumulate across batches.
    """
    ctx = _Ctx(problem.mesh, problem.tables)
    r = problem.rays if rays is None else rays
    arrs = [np.ascontiguousarray(r[k], np.float32)
            for k in ("x", "y", "z", "u", "v", "w", "E", "wt")]
    n = int(arrs[0].shape[0])
    if tally is None:
        tally = np.zeros(problem.tally_size, np.float64)
    assert tally.dtype == np.float64 and tally.flags.c_contiguous
    assert tally.size == problem.tally_size
    edges = problem.group_edges
    keep = None if edges is None else np.ascontiguousarray(edges, np.float64)
    ep = None if keep is None else _ptr(keep)
    ng = 0 if keep is None else len(keep) - 1
    stats = np.zeros(4, np.int64)
    rc = _load().orc_cast(C.byref(ctx.mesh), C.byref(ctx.xs), ep, ng, *[_ptr(a) for a in arrs],
                          n, _ptr(tally), int(nthreads), _ptr(stats))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return tally, dict(segments=int(stats[0]), rejected=int(stats[1]),
                       overflow=int(stats[2]), threads=int(stats[3]))


def batch_moments(batch_tallies):
    """Tally total and its standard deviation by the batch method: with B
    batch tallies t_b, total = sum_b t_b and sigma = sqrt(B/(B-1) *
    (sum_b t_b^2 - total^2/B)) (sigma = 0 for B < 2), float64 per cell."""
    T = np.asarray(batch_tallies, np.float64)
    B = T.shape[0]
    total = T.sum(axis=0)
    if B < 2:
        return total, np.zeros_like(total)
    var = (np.sum(T * T, axis=0) - total * total / B) * (B / (B - 1.0))
    return total, np.sqrt(np.maximum(var, 0.0))


def history_moments(problem, history, n_histories: int, rays: dict | None = None):
    """Per-history moments behind the sigma of Eqs. 5 and 8: x_h = the tally of
    the rays of history h (every ray with that id), total = sum_h x_h and
    sigma = sqrt(N/(N-1) (sum_h x_h^2 - total^2/N)) with N = n_histories;
    histories without rays count as zero scores.  Returns (total, sigma, S2),
    float64 per cell, S2 = sum_h x_h^2."""
    r = problem.rays if rays is None else rays
    hist = np.asarray(history).reshape(-1)
    ids = np.unique(hist)
    N = int(n_histories)
    if len(ids) > N:
        raise ValueError("more distinct history ids than n_histories")
    s1 = np.zeros(problem.tally_size, np.float64)
    s2 = np.zeros(problem.tally_size, np.float64)
    for h in ids:
        sel = np.flatnonzero(hist == h)
        x, _ = cast(problem, nthreads=1, rays={k: np.asarray(v)[sel] for k, v in r.items()})
        s1 += x
        s2 += x * x
    if N < 2:
        return s1, np.zeros_like(s1), s2
    var = (s2 - s1 * s1 / N) * (N / (N - 1.0))
    return s1, np.sqrt(np.maximum(var, 0.0)), s2


def point_detector(problem, detectors, rays: dict | None = None):
    """Next-event flux at each detector point from every ray event:
    sum over events of wt exp(-tau)/(4 pi R^2), float64 [n_det][n_groups]."""
    ctx = _Ctx(problem.mesh, problem.tables)
    r = problem.rays if rays is None else rays
    arrs = [np.ascontiguousarray(r[k], np.float32) for k in ("x", "y", "z", "E", "wt")]
    det = np.ascontiguousarray(detectors, np.float64).reshape(-1, 3)
    out = np.zeros((det.shape[0], problem.n_groups), np.float64)
    edges = problem.group_edges
    keep = None if edges is None else np.ascontiguousarray(edges, np.float64)
    ep = None if keep is None else _ptr(keep)
    ng = 0 if keep is None else len(keep) - 1
    rc = _load().orc_point_detector(C.byref(ctx.mesh), C.byref(ctx.xs), ep, ng,
                                    *[_ptr(a) for a in arrs], int(arrs[0].shape[0]), _ptr(det),
                                    det.shape[0], _ptr(out))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out
