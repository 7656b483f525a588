"""Python binding of libvrc (include/vrc.h): the same calls, argument marshalling only.

Every step of the cast runs in the library's CUDA kernels.  There is no
Python or CPU fallback: importing this module fails loudly when libvrc.so has
not been built, and every call raises :class:`VrcError` with the library's
message on failure.

Arrays may be numpy arrays (host), torch CPU tensors (host, pinned or not) or
torch CUDA tensors (device).  Streams may be ``None`` (the context's stream),
a ``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvrc.so")

VRC_OK = 0
VRC_ERR_ARG = -1
VRC_ERR_STATE = -2
VRC_ERR_CUDA = -3
VRC_ERR_OOM = -4
VRC_ERR_TRAVERSAL = -5
VRC_ERR_NONFINITE = -6
VRC_FORM_PLAIN = 0
VRC_FORM_FP32 = 1
VRC_PER_VOLUME = 1

RAY_FIELDS = ("x", "y", "z", "u", "v", "w", "E", "wt")


class VrcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libvrc error {code}: {msg}")
        self.code = code


class vrc_options(C.Structure):
    _fields_ = [("form", C.c_int32), ("sort", C.c_int32), ("sort_len_buckets", C.c_int32),
                ("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("device", C.c_int32),
                ("stop_at_zero", C.c_int32), ("rays_per_warp", C.c_int32)]


class vrc_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("material", C.c_void_p), ("n_materials", C.c_int32), ("n_groups", C.c_int32),
                ("group_edges", C.c_void_p)]


class vrc_rect_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x_edges", C.c_void_p), ("y_edges", C.c_void_p), ("z_edges", C.c_void_p),
                ("material", C.c_void_p), ("n_materials", C.c_int32), ("n_groups", C.c_int32),
                ("group_edges", C.c_void_p)]


class vrc_rays(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in RAY_FIELDS] + [("n", C.c_int64), ("on_device", C.c_int32)]


class vrc_stats(C.Structure):
    _fields_ = [("segments", C.c_int64), ("rays", C.c_int64), ("rejected", C.c_int64),
                ("overflow", C.c_int64), ("live", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "vrc_default_options": ([P], None),
        "vrc_create_mesh": ([P, P, P], C.c_int),
        "vrc_load_xs": ([P, I32, P, P, I64], C.c_int),
        "vrc_cast_rays": ([P, P, P], C.c_int),
        "vrc_sync": ([P, P, P], C.c_int),
        "vrc_read_tally": ([P, P, I64, I32, P], C.c_int),
        "vrc_tally_device_ptr": ([P], C.c_void_p),
        "vrc_context_stream": ([P], C.c_void_p),
        "vrc_create_rect_mesh": ([P, P, P], C.c_int),
        "vrc_reset_tally": ([P, P], C.c_int),
        "vrc_set_options": ([P, P], C.c_int),
        "vrc_destroy": ([P], None),
        "vrc_last_error": ([], C.c_char_p),
        "vrc_device_count": ([], C.c_int),
        "vrc_enable_timing": ([P, I32], C.c_int),
        "vrc_get_timing": ([P, P, P, P, P, I32], C.c_int),
        "vrc_launch_count": ([], C.c_int64),
        "vrc_debug_fail_alloc": ([I64], C.c_int),
        "vrc_sort_rays_static": ([P, P, P, P], C.c_int),
        "vrc_detector_flux": ([P, P, P, I32, P, P], C.c_int),
        "vrc_moments_enable": ([P, I32], C.c_int),
        "vrc_moments_fold": ([P, P], C.c_int),
        "vrc_moments_read": ([P, P, P, I64, P, P], C.c_int),
        "vrc_cast_histories": ([P, P, P, I64, P], C.c_int),
        "vrc_stream_create": ([P, I64, I32, P], C.c_int),
        "vrc_stream_acquire": ([P, P, P], C.c_int),
        "vrc_stream_submit": ([P, I64], C.c_int),
        "vrc_stream_finish": ([P], C.c_int),
        "vrc_stream_destroy": ([P], None),
        "vrc_default_surrogate_options": ([P], None),
        "vrc_mlp_forward": ([P, P, I64, C.c_double, C.c_double, P, P], C.c_int),
        "vrc_mlp_loss_grad": ([P, P, P, P, I64, I64, C.c_double, C.c_double, P, P, P], C.c_int),
        "vrc_train_surrogate": ([P, P, P], C.c_int),
        "vrc_set_xs_mode": ([P, I32], C.c_int),
        "vrc_get_surrogate_params": ([P, P], C.c_int),
        "vrc_default_batch_options": ([P], None),
        "vrc_batch_create": ([P, P, I32, P, P], C.c_int),
        "vrc_batch_launch": ([P, P], C.c_int),
        "vrc_batch_destroy": ([P], None),
        "vrc_cast_batched": ([P, P, I32, P], C.c_int),
        "vrc_version": ([], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def library():
    """The loaded ctypes library (for callers that need a symbol directly)."""
    return _lib


def vrc_last_error() -> str:
    return (_lib.vrc_last_error() or b"").decode()


def _check(rc: int, ok=(VRC_OK,)) -> int:
    if rc not in ok:
        raise VrcError(rc, vrc_last_error())
    return rc


def vrc_device_count() -> int:
    return int(_lib.vrc_device_count())


def vrc_version() -> int:
    return int(_lib.vrc_version())


def require_device():
    if vrc_device_count() < 1:
        raise RuntimeError("libvrc found no CUDA device")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None


def vrc_default_options(**kw) -> vrc_options:
    o = vrc_options()
    _lib.vrc_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


class Context:
    """Owns one vrc_ctx handle; destroyed explicitly or when collected."""

    def __init__(self, handle, ncells, n_groups, spacing):
        self.handle = handle
        self.ncells = ncells
        self.n_groups = n_groups
        self.spacing = spacing
        self._inflight = []

    @property
    def tally_size(self):
        return self.ncells * self.n_groups

    def close(self):
        if self.handle:
            _lib.vrc_destroy(self.handle)
            self.handle = None
        self._inflight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def vrc_create_mesh(mesh, n_materials: int, group_edges=None, options: vrc_options | None = None) -> Context:
    """mesh: object with nx, ny, nz, x0..z0, dx..dz and uint8 material [nz][ny][nx]."""
    mat = np.ascontiguousarray(mesh.material, dtype=np.uint8).reshape(-1)
    edges = None if group_edges is None else np.ascontiguousarray(group_edges, np.float64)
    d = vrc_mesh_desc(mesh.nx, mesh.ny, mesh.nz, mesh.x0, mesh.y0, mesh.z0, mesh.dx, mesh.dy,
                      mesh.dz, mat.ctypes.data, int(n_materials),
                      1 if edges is None else len(edges) - 1,
                      None if edges is None else edges.ctypes.data)
    h = C.c_void_p()
    _check(_lib.vrc_create_mesh(C.byref(d), None if options is None else C.byref(options),
                                C.byref(h)))
    return Context(h, mesh.nx * mesh.ny * mesh.nz, d.n_groups, (mesh.dx, mesh.dy, mesh.dz))


def vrc_create_rect_mesh(mesh, n_materials: int, group_edges=None,
                         options: vrc_options | None = None) -> Context:
    """mesh: object with float64 plane arrays xe, ye, ze and uint8 material [nz][ny][nx]."""
    mat = np.ascontiguousarray(mesh.material, dtype=np.uint8).reshape(-1)
    xe, ye, ze = (np.ascontiguousarray(e, np.float64) for e in (mesh.xe, mesh.ye, mesh.ze))
    edges = None if group_edges is None else np.ascontiguousarray(group_edges, np.float64)
    d = vrc_rect_mesh_desc(len(xe) - 1, len(ye) - 1, len(ze) - 1, xe.ctypes.data, ye.ctypes.data,
                           ze.ctypes.data, mat.ctypes.data, int(n_materials),
                           1 if edges is None else len(edges) - 1,
                           None if edges is None else edges.ctypes.data)
    h = C.c_void_p()
    _check(_lib.vrc_create_rect_mesh(C.byref(d), None if options is None else C.byref(options),
                                     C.byref(h)))
    return Context(h, (len(xe) - 1) * (len(ye) - 1) * (len(ze) - 1), d.n_groups, None)


def vrc_load_xs(ctx: Context, material: int, E, sigma):
    if E is None:
        _check(_lib.vrc_load_xs(ctx.handle, int(material), None, None, 0))
        return
    E = np.ascontiguousarray(E, np.float64)
    S = np.ascontiguousarray(sigma, np.float64)
    if E.shape != S.shape:
        raise ValueError("E and sigma must have the same length")
    _check(_lib.vrc_load_xs(ctx.handle, int(material), E.ctypes.data, S.ctypes.data, len(E)))


def vrc_context_stream(ctx: Context) -> int:
    return int(_lib.vrc_context_stream(ctx.handle) or 0)


def _order_device_inputs(ctx: Context, stream, tensors):
    """Makes the stream a library call runs on wait for torch's current stream
    (which produced the device tensors).  Returns the device tensors."""
    dev = [t for t in tensors if not isinstance(t, np.ndarray) and t.is_cuda]
    if dev:
        import torch
        handle = _stream_handle(stream) or vrc_context_stream(ctx)
        cur = torch.cuda.current_stream(dev[0].device)
        if handle != cur.cuda_stream:
            torch.cuda.ExternalStream(handle, device=dev[0].device).wait_stream(cur)
    return dev


def _hold_until_done(ctx: Context, stream, dev):
    """Keeps device inputs referenced until the stream has passed the call just
    enqueued, so the caching allocator cannot hand their memory to a later
    producer while the library still reads it.  Entries are dropped once their
    event completes, and all of them when the context is closed (vrc_destroy
    waits for the context's stream)."""
    ctx._inflight = [(e, t) for e, t in ctx._inflight if not e.query()]
    if dev:
        import torch
        handle = _stream_handle(stream) or vrc_context_stream(ctx)
        ev = torch.cuda.Event()
        ev.record(torch.cuda.ExternalStream(handle, device=dev[0].device))
        ctx._inflight.append((ev, dev))


def _ray_struct(rays: dict):
    arrs = [rays[k] for k in RAY_FIELDS]
    keep = []
    ptrs = []
    on_dev = None
    n = None
    for a in arrs:
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, np.float32)
            dev = False
            ptr, cnt = a.ctypes.data, a.shape[0]
        else:  # torch tensor
            if a.dtype != __import__("torch").float32 or not a.is_contiguous():
                raise TypeError("ray tensors must be contiguous float32")
            dev = a.is_cuda
            ptr, cnt = a.data_ptr(), a.shape[0]
        keep.append(a)
        if on_dev is None:
            on_dev, n = dev, cnt
        elif dev != on_dev or cnt != n:
            raise ValueError("ray arrays must all be on the same side and of the same length")
        ptrs.append(ptr)
    r = vrc_rays(*ptrs, int(n), int(bool(on_dev)))
    return r, keep


def vrc_cast_rays(ctx: Context, rays: dict, stream=None):
    r, keep = _ray_struct(rays)
    dev = _order_device_inputs(ctx, stream, keep)
    _check(_lib.vrc_cast_rays(ctx.handle, C.byref(r), _stream_handle(stream)))
    _hold_until_done(ctx, stream, dev)


def vrc_sort_rays_static(ctx: Context, rays: dict, out, stream=None):
    """No-allocation ray sort: device rays in; `out` is a caller-owned device
    float32 tensor of 8*n elements receiving x, y, z, u, v, w, E, wt blocks."""
    r, keep = _ray_struct(rays)
    dev = _order_device_inputs(ctx, stream, keep + ([] if out is None else [out]))
    ptr = None if out is None else out.data_ptr()
    _check(_lib.vrc_sort_rays_static(ctx.handle, C.byref(r), ptr, _stream_handle(stream)))
    _hold_until_done(ctx, stream, dev)


VRC_MLP_PARAMS = 26928
VRC_XS_TABLE = 0
VRC_XS_SURROGATE = 1


class vrc_surrogate_options(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("tol", C.c_float),
                ("seed", C.c_uint64), ("smooth", C.c_float)]


class vrc_surrogate_report(C.Structure):
    _fields_ = [("final_loss", C.c_float), ("bins", C.c_int32), ("bins_accepted", C.c_int32),
                ("coverage", C.c_float), ("max_rel_err_accepted", C.c_float),
                ("median_rel_err", C.c_float), ("train_points", C.c_int64),
                ("validation_points", C.c_int64), ("smooth_fraction", C.c_float)]


def vrc_default_surrogate_options(**kw) -> vrc_surrogate_options:
    o = vrc_surrogate_options()
    _lib.vrc_default_surrogate_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown surrogate option {k}")
        setattr(o, k, v)
    return o


def vrc_mlp_forward(params, E, e_lo: float, e_hi: float, out, stream=None):
    """Device tensors: params [VRC_MLP_PARAMS] f32, E [n] f32, out [n, 16] f32."""
    _check(_lib.vrc_mlp_forward(params.data_ptr(), E.data_ptr(), E.shape[0], float(e_lo),
                                float(e_hi), out.data_ptr(), _stream_handle(stream)))


def vrc_mlp_loss_grad(params, E, target, mask, count: int, e_lo: float, e_hi: float, grad, loss,
                      stream=None):
    """Device tensors; mask uint8 [n, 16] or None.  grad and loss are overwritten."""
    _check(_lib.vrc_mlp_loss_grad(params.data_ptr(), E.data_ptr(), target.data_ptr(),
                                  None if mask is None else mask.data_ptr(), E.shape[0],
                                  int(count), float(e_lo), float(e_hi), grad.data_ptr(),
                                  loss.data_ptr(), _stream_handle(stream)))


def vrc_train_surrogate(ctx: Context, options: vrc_surrogate_options | None = None) -> dict:
    rep = vrc_surrogate_report()
    _check(_lib.vrc_train_surrogate(ctx.handle, None if options is None else C.byref(options),
                                    C.byref(rep)))
    return {k: getattr(rep, k) for k, _ in rep._fields_}


def vrc_set_xs_mode(ctx: Context, mode: int):
    _check(_lib.vrc_set_xs_mode(ctx.handle, int(mode)))


def vrc_get_surrogate_params(ctx: Context) -> np.ndarray:
    out = np.empty(VRC_MLP_PARAMS, np.float32)
    _check(_lib.vrc_get_surrogate_params(ctx.handle, out.ctypes.data))
    return out


def vrc_detector_flux(ctx: Context, rays: dict, detectors, stream=None) -> np.ndarray:
    """Next-event flux at each detector, float64 [n_det][n_groups]."""
    r, keep = _ray_struct(rays)
    det = np.ascontiguousarray(detectors, np.float64).reshape(-1, 3)
    out = np.empty((det.shape[0], ctx.n_groups), np.float64)
    _order_device_inputs(ctx, stream, keep)
    _check(_lib.vrc_detector_flux(ctx.handle, C.byref(r), det.ctypes.data, det.shape[0],
                                  out.ctypes.data, _stream_handle(stream)))
    return out


VRC_MOMENTS_OFF = 0
VRC_MOMENTS_BATCH = 1
VRC_MOMENTS_HISTORY = 2


def vrc_moments_enable(ctx: Context, mode: int = VRC_MOMENTS_BATCH):
    _check(_lib.vrc_moments_enable(ctx.handle, int(mode)))


def vrc_cast_histories(ctx: Context, rays: dict, history, n_histories: int, stream=None):
    """Per-history cast: history is a uint32 array (numpy for host rays, a
    torch int32/uint32 tensor for device rays) with the history id of each ray."""
    r, keep = _ray_struct(rays)
    if isinstance(history, np.ndarray):
        if r.on_device:
            raise ValueError("history ids must be on the same side as the rays")
        h = np.ascontiguousarray(history, np.uint32)
        if h.shape[0] != r.n:
            raise ValueError("one history id per ray")
        hp = h.ctypes.data
        dev = []
    else:
        if not r.on_device or not history.is_cuda or history.element_size() != 4 or not history.is_contiguous():
            raise ValueError("device history ids: a contiguous 4-byte tensor beside device rays")
        if history.shape[0] != r.n:
            raise ValueError("one history id per ray")
        hp = history.data_ptr()
        dev = _order_device_inputs(ctx, stream, keep + [history])
    _check(_lib.vrc_cast_histories(ctx.handle, C.byref(r), hp, int(n_histories), _stream_handle(stream)))
    _hold_until_done(ctx, stream, dev)


def vrc_moments_fold(ctx: Context, stream=None):
    _check(_lib.vrc_moments_fold(ctx.handle, _stream_handle(stream)))


def vrc_moments_read(ctx: Context, stream=None):
    """Returns (total, sigma, samples): host float64 arrays and the batch or
    history count."""
    total = np.empty(ctx.tally_size, np.float64)
    sigma = np.empty(ctx.tally_size, np.float64)
    b = C.c_int64()
    _check(_lib.vrc_moments_read(ctx.handle, total.ctypes.data, sigma.ctypes.data, total.size,
                                 C.byref(b), _stream_handle(stream)))
    return total, sigma, b.value


class RayStream:
    """vrc_stream: pinned buffers of 32-byte ray records, filled by the caller
    while earlier buffers are uploaded and cast (double buffering)."""

    FIELDS = 8

    def __init__(self, ctx: Context, capacity: int, n_buffers: int = 2):
        h = C.c_void_p()
        _check(_lib.vrc_stream_create(ctx.handle, int(capacity), int(n_buffers), C.byref(h)))
        self.handle, self.ctx, self.capacity = h, ctx, int(capacity)

    def acquire(self) -> np.ndarray:
        """The next buffer as a (capacity, 8) float32 view: x y z u v w E wt."""
        ptr, cap = C.c_void_p(), C.c_int64()
        _check(_lib.vrc_stream_acquire(self.handle, C.byref(ptr), C.byref(cap)))
        buf = (C.c_float * (cap.value * self.FIELDS)).from_address(ptr.value)
        return np.ctypeslib.as_array(buf).reshape(cap.value, self.FIELDS)

    def submit(self, n: int):
        _check(_lib.vrc_stream_submit(self.handle, int(n)))

    def finish(self):
        _check(_lib.vrc_stream_finish(self.handle))

    def close(self):
        if self.handle:
            _lib.vrc_stream_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class vrc_batch_options(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk", C.c_int32),
                ("sort_len_buckets", C.c_int32), ("use_graph", C.c_int32), ("rays_per_warp", C.c_int32)]


def vrc_default_batch_options(**kw) -> vrc_batch_options:
    o = vrc_batch_options()
    _lib.vrc_default_batch_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown batch option {k}")
        setattr(o, k, int(v))
    return o


class Batch:
    """Owns one vrc_batch plan (and keeps its contexts and rays referenced)."""

    def __init__(self, handle, ctxs, keep):
        self.handle = handle
        self.ctxs = ctxs
        self._keep = keep

    def close(self):
        if self.handle:
            _lib.vrc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ctx_array(ctxs):
    arr = (C.c_void_p * len(ctxs))(*[c.handle.value if isinstance(c.handle, C.c_void_p) else c.handle
                                     for c in ctxs])
    return arr


def _rays_array(rays_list):
    structs, keep = [], []
    for rays in rays_list:
        r, k = _ray_struct(rays)
        structs.append(r)
        keep.append(k)
    arr = (vrc_rays * len(structs))(*structs)
    return arr, keep


def vrc_batch_create(ctxs, rays_list, options: vrc_batch_options | None = None) -> Batch:
    """ctxs: list of Context; rays_list: list of dicts of device tensors."""
    carr = _ctx_array(ctxs)
    rarr, keep = _rays_array(rays_list)
    h = C.c_void_p()
    _check(_lib.vrc_batch_create(carr, rarr, len(ctxs),
                                 None if options is None else C.byref(options), C.byref(h)))
    return Batch(h, list(ctxs), (carr, rarr, keep))


def vrc_batch_launch(batch: Batch, stream=None):
    # the Batch holds its rays and vrc_batch_destroy waits for its stream
    _order_device_inputs(batch.ctxs[0], stream, batch._keep[2][0] if batch._keep[2] else [])
    _check(_lib.vrc_batch_launch(batch.handle, _stream_handle(stream)))


def vrc_batch_destroy(batch: Batch):
    batch.close()


def vrc_cast_batched(ctxs, rays_list, stream=None):
    carr = _ctx_array(ctxs)
    rarr, keep = _rays_array(rays_list)
    _order_device_inputs(ctxs[0], stream, [t for k in keep for t in k])
    _check(_lib.vrc_cast_batched(carr, rarr, len(ctxs), _stream_handle(stream)))


def vrc_sync(ctx: Context, stream=None):
    """Waits; returns (status code, stats dict).  Raises only for ARG/CUDA errors."""
    st = vrc_stats()
    rc = _lib.vrc_sync(ctx.handle, _stream_handle(stream), C.byref(st))
    _check(rc, ok=(VRC_OK, VRC_ERR_NONFINITE, VRC_ERR_TRAVERSAL))
    return rc, dict(segments=st.segments, rays=st.rays, rejected=st.rejected, overflow=st.overflow,
                    live=st.live)


def vrc_read_tally(ctx: Context, out: np.ndarray | None = None, flags: int = 0, stream=None):
    """Copies the tally to host float64 [n_groups*ncells]; returns (array, status code)."""
    if out is None:
        out = np.empty(ctx.tally_size, np.float64)
    if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != ctx.tally_size:
        raise ValueError("out must be a contiguous float64 array of the tally size")
    rc = _lib.vrc_read_tally(ctx.handle, out.ctypes.data, out.size, int(flags), _stream_handle(stream))
    _check(rc, ok=(VRC_OK, VRC_ERR_NONFINITE, VRC_ERR_TRAVERSAL))
    return out, rc


def vrc_tally_device_ptr(ctx: Context) -> int:
    return int(_lib.vrc_tally_device_ptr(ctx.handle) or 0)


def vrc_reset_tally(ctx: Context, stream=None):
    _check(_lib.vrc_reset_tally(ctx.handle, _stream_handle(stream)))


def vrc_set_options(ctx: Context, options: vrc_options):
    _check(_lib.vrc_set_options(ctx.handle, C.byref(options)))


def vrc_enable_timing(ctx: Context, on: bool = True):
    _check(_lib.vrc_enable_timing(ctx.handle, int(bool(on))))


def vrc_get_timing(ctx: Context, stream=None, reset: bool = False):
    """Returns dict(cast_ms, sort_ms, cast_launches) summed since enable/reset."""
    cast_ms, sort_ms, n = C.c_double(), C.c_double(), C.c_int64()
    _check(_lib.vrc_get_timing(ctx.handle, _stream_handle(stream), C.byref(cast_ms),
                               C.byref(sort_ms), C.byref(n), int(bool(reset))))
    return dict(cast_ms=cast_ms.value, sort_ms=sort_ms.value, cast_launches=n.value)


def vrc_launch_count() -> int:
    return int(_lib.vrc_launch_count())


def vrc_debug_fail_alloc(n: int):
    """Test hook: the allocation after the next n fails as out of memory (n < 0 disarms)."""
    _check(_lib.vrc_debug_fail_alloc(int(n)))


def vrc_destroy(ctx: Context):
    ctx.close()


def context_for(problem, options: vrc_options | None = None) -> Context:
    """vrc_create_mesh (or vrc_create_rect_mesh for a mesh with plane arrays)
    + vrc_load_xs for a vrc_workloads.Problem."""
    if getattr(problem.mesh, "xe", None) is not None:
        ctx = vrc_create_rect_mesh(problem.mesh, problem.n_materials, problem.group_edges, options)
    else:
        ctx = vrc_create_mesh(problem.mesh, problem.n_materials, problem.group_edges, options)
    for m, t in enumerate(problem.tables):
        if t is None:
            vrc_load_xs(ctx, m, None, None)
        else:
            vrc_load_xs(ctx, m, t[0], t[1])
    return ctx
