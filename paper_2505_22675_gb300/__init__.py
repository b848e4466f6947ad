"""bathygrid: gridding scattered multibeam soundings on a GB300 GPU.

Thin Python binding of libbathygrid.so (include/bathygrid.h). Functions keep
the C names without the `bg_` prefix and only marshal arguments: every step
of the hot path (hash build, neighbour search, IDW, kriging) runs in the
library's CUDA kernels. PyTorch supplies device memory and streams.

    ctx = ctx_create(0)
    grid = grid_create(ctx, 0, 0, 200, 256, 256)
    s = soundings_upload(ctx, x_cm, y_cm, z_m)        # torch tensors or numpy arrays
    depth = torch.empty(256 * 256, device="cuda")
    interp_idw(s, grid, 8, 2.0, depth)
"""
from __future__ import annotations

import ctypes

from . import _capi
from ._capi import BGError, Request, Result, SoundingsInfo, Variogram, check

SPHERICAL = 0
EXPONENTIAL = 1
IDW = 0
OKRIGE = 1

__all__ = [
    "BGError", "Variogram", "SoundingsInfo", "SPHERICAL", "EXPONENTIAL", "IDW", "OKRIGE",
    "version", "launch_count", "alu_peak", "ALU_KINDS", "profile_enable", "profile_read", "ctx_create", "ctx_destroy",
    "ctx_device_bytes", "grid_create", "grid_destroy",
    "soundings_upload", "soundings_info", "soundings_destroy", "interp_idw", "interp_okrige",
    "interp_idw_okrige", "interp_idw_okrige_host", "interp_idw_points", "interp_okrige_points", "BILINEAR", "CATMULL_ROM", "resample_points",
    "resample_grid",
    "variogram", "interp_idw_noalloc", "submit", "poll", "wait", "cancel", "serve_stats",
    "serve_shutdown", "Request", "Result", "Batch", "batch_create", "batch_run", "batch_tune", "batch_set_shape", "batch_config",
    "batch_set_cell_target", "batch_status", "batch_destroy",
]


def _lib():
    return _capi.load()


def _ptr(t):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _is_cuda(t):
    return t is not None and getattr(t, "is_cuda", False)


def _stream(stream, *tensors):
    """cudaStream_t for the call: explicit, else torch's current stream when a
    tensor lives on the GPU, else NULL (legacy default stream)."""
    if stream is not None:
        return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    for t in tensors:
        if _is_cuda(t):
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


def version() -> str:
    return _lib().bg_version().decode()


def launch_count() -> int:
    """Kernels the library has launched since it was loaded."""
    out = ctypes.c_uint64()
    check(_lib().bg_launch_count(ctypes.byref(out)), "bg_launch_count")
    return out.value


ALU_KINDS = {"fp32_fma": 0, "int32_imad": 1, "int32_add_xor": 2, "fp64_fma": 3}


def alu_peak(kind: str, device: int = 0):
    """Measured ALU peak of `device` for one instruction kind (ALU_KINDS):
    (ops/s, SM MHz the measuring kernel ran at). FMAs count 2 flops."""
    ops = ctypes.c_double()
    mhz = ctypes.c_double()
    check(_lib().bg_alu_peak(device, ALU_KINDS[kind], ctypes.byref(ops), ctypes.byref(mhz)),
          "bg_alu_peak")
    return ops.value, mhz.value


PROFILE_STAGES = ("hash_build", "idw", "kriging_knn_ids", "kriging_solve")


def profile_enable(ctx, on: bool = True) -> None:
    """Record CUDA events around each interpolation kernel launch of ctx."""
    check(_lib().bg_profile_enable(ctx, int(bool(on))), "bg_profile_enable")


def profile_read(ctx) -> dict:
    """{stage: (total ms, launches, grid nodes)} since the last read; clears."""
    n = len(PROFILE_STAGES)
    ms = (ctypes.c_double * n)()
    la = (ctypes.c_int64 * n)()
    un = (ctypes.c_int64 * n)()
    check(_lib().bg_profile_read(ctx, ms, la, un, n), "bg_profile_read")
    return {name: (ms[i], la[i], un[i]) for i, name in enumerate(PROFILE_STAGES)}


def variogram(model: int = SPHERICAL, nugget_m2: float = 0.25, sill_m2: float = 100.0,
              range_m: float = 50.0) -> Variogram:
    """Variogram parameters; sill is the total sill (nugget + partial sill)."""
    return Variogram(model, nugget_m2, sill_m2, range_m)


def ctx_create(device: int = 0, hbm_budget_bytes: int = 0):
    out = ctypes.c_void_p()
    check(_lib().bg_ctx_create(device, hbm_budget_bytes, ctypes.byref(out)), "bg_ctx_create")
    return out


def ctx_destroy(ctx) -> None:
    check(_lib().bg_ctx_destroy(ctx), "bg_ctx_destroy")


def ctx_device_bytes(ctx) -> int:
    out = ctypes.c_int64()
    check(_lib().bg_ctx_device_bytes(ctx, ctypes.byref(out)), "bg_ctx_device_bytes")
    return out.value


def grid_create(ctx, x0_cm: int, y0_cm: int, cell_cm: int, nx: int, ny: int):
    out = ctypes.c_void_p()
    check(_lib().bg_grid_create(ctx, x0_cm, y0_cm, cell_cm, nx, ny, ctypes.byref(out)),
          "bg_grid_create")
    return out


def grid_destroy(grid) -> None:
    check(_lib().bg_grid_destroy(grid), "bg_grid_destroy")


def soundings_upload(ctx, x_cm, y_cm, z_m, cell_cm_hint: int = 0, stream=None):
    """Upload soundings (int32 cm, int32 cm, float32 m) and build the device hash.

    Device tensors are read in place; host tensors / numpy arrays are copied.
    """
    on_dev = [_is_cuda(t) for t in (x_cm, y_cm, z_m)]
    if any(on_dev) and not all(on_dev):
        raise ValueError("x, y and z must all be on the device or all on the host")
    n = int(x_cm.shape[0])
    if int(y_cm.shape[0]) != n or int(z_m.shape[0]) != n:
        raise ValueError("x, y and z must have the same length")
    _check_dtype(x_cm, "int32")
    _check_dtype(y_cm, "int32")
    _check_dtype(z_m, "float32")
    out = ctypes.c_void_p()
    check(_lib().bg_soundings_upload(ctx, _ptr(x_cm), _ptr(y_cm), _ptr(z_m), n, int(all(on_dev)),
                                     cell_cm_hint, _stream(stream, x_cm), ctypes.byref(out)),
          "bg_soundings_upload")
    return out


def soundings_info(s) -> SoundingsInfo:
    info = SoundingsInfo()
    check(_lib().bg_soundings_info_get(s, ctypes.byref(info)), "bg_soundings_info_get")
    return info


def soundings_destroy(s) -> None:
    check(_lib().bg_soundings_destroy(s), "bg_soundings_destroy")


def interp_idw(s, grid, k: int, power: float, depth_out, nbr_out=None, stream=None) -> None:
    """IDW over the k nearest valid soundings into depth_out (device, nx*ny float32)."""
    _check_dtype(depth_out, "float32")
    if nbr_out is not None:
        _check_dtype(nbr_out, "int32")
    check(_lib().bg_interp_idw(s, grid, k, power, _ptr(depth_out), _ptr(nbr_out),
                               _stream(stream, depth_out)), "bg_interp_idw")


def interp_okrige(s, grid, k: int, vgm: Variogram, depth_out, var_out=None, nbr_out=None,
                  stream=None) -> None:
    """Ordinary kriging over the k nearest valid soundings (depth and variance)."""
    _check_dtype(depth_out, "float32")
    if var_out is not None:
        _check_dtype(var_out, "float32")
    if nbr_out is not None:
        _check_dtype(nbr_out, "int32")
    check(_lib().bg_interp_okrige(s, grid, k, ctypes.byref(vgm), _ptr(depth_out), _ptr(var_out),
                                  _ptr(nbr_out), _stream(stream, depth_out)), "bg_interp_okrige")


def interp_idw_okrige(s, grid, k_idw: int, power: float, k_okrige: int, vgm: Variogram, idw_out,
                      depth_out, var_out=None, stream=None) -> None:
    """IDW (first k_idw neighbours) and ordinary kriging (k_okrige) in one pass;
    bitwise the results of interp_idw and interp_okrige called separately."""
    for t in (idw_out, depth_out):
        _check_dtype(t, "float32")
    if var_out is not None:
        _check_dtype(var_out, "float32")
    check(_lib().bg_interp_idw_okrige(s, grid, k_idw, power, k_okrige, ctypes.byref(vgm),
                                      _ptr(idw_out), _ptr(depth_out), _ptr(var_out),
                                      _stream(stream, depth_out)), "bg_interp_idw_okrige")


def interp_idw_okrige_host(s, grid, k_idw: int, power: float, k_okrige: int, vgm: Variogram,
                           idw_out, depth_out, var_out=None, idw_host=None, depth_host=None,
                           var_host=None, stream=None) -> None:
    """interp_idw_okrige that also copies each row chunk's grids to host arrays
    (CPU tensors, pinned for overlap) while the later chunks compute; the host
    arrays are complete once `stream` is synchronized."""
    for t in (idw_out, depth_out):
        _check_dtype(t, "float32")
    m = int(depth_out.shape[0])
    for t in (var_out, idw_host, depth_host, var_host):
        if t is not None:
            _check_dtype(t, "float32")
    for t in (idw_host, depth_host, var_host):
        if t is not None:
            if _is_cuda(t):
                raise ValueError("host destinations must be host tensors or arrays")
            if int(t.shape[0]) != m:
                raise ValueError("host destinations need nx*ny entries")
    check(_lib().bg_interp_idw_okrige_host(s, grid, k_idw, power, k_okrige, ctypes.byref(vgm),
                                           _ptr(idw_out), _ptr(depth_out), _ptr(var_out),
                                           _ptr(idw_host), _ptr(depth_host), _ptr(var_host),
                                           _stream(stream, depth_out)), "bg_interp_idw_okrige_host")


def _check_points(qx_cm, qy_cm, depth_out):
    for t, dt in ((qx_cm, "int32"), (qy_cm, "int32"), (depth_out, "float32")):
        _check_dtype(t, dt)
    m = int(qx_cm.shape[0])
    if int(qy_cm.shape[0]) != m or int(depth_out.shape[0]) < m:
        raise ValueError("qx, qy and depth_out must hold m entries")
    return m


def interp_idw_points(s, qx_cm, qy_cm, k: int, power: float, depth_out, nbr_out=None,
                      stream=None) -> None:
    """IDW at query points (device int32 cm arrays) into depth_out (device, m float32)."""
    m = _check_points(qx_cm, qy_cm, depth_out)
    if nbr_out is not None:
        _check_dtype(nbr_out, "int32")
    check(_lib().bg_interp_idw_points(s, _ptr(qx_cm), _ptr(qy_cm), m, k, power, _ptr(depth_out),
                                      _ptr(nbr_out), _stream(stream, depth_out)),
          "bg_interp_idw_points")


def interp_okrige_points(s, qx_cm, qy_cm, k: int, vgm: Variogram, depth_out, var_out=None,
                         nbr_out=None, stream=None) -> None:
    """Ordinary kriging at query points (device int32 cm arrays)."""
    m = _check_points(qx_cm, qy_cm, depth_out)
    if var_out is not None:
        _check_dtype(var_out, "float32")
    if nbr_out is not None:
        _check_dtype(nbr_out, "int32")
    check(_lib().bg_interp_okrige_points(s, _ptr(qx_cm), _ptr(qy_cm), m, k, ctypes.byref(vgm),
                                         _ptr(depth_out), _ptr(var_out), _ptr(nbr_out),
                                         _stream(stream, depth_out)), "bg_interp_okrige_points")


BILINEAR = 0
CATMULL_ROM = 1


def resample_points(src, grid_spec, method: int, qx_cm, qy_cm, out, how_out=None,
                    stream=None) -> None:
    """Bilinear / Catmull-Rom of a regular grid (device float32 [ny * nx], NaN =
    missing; grid_spec = (x0_cm, y0_cm, cell_cm, nx, ny)) at query points."""
    m = _check_points(qx_cm, qy_cm, out)
    _check_dtype(src, "float32")
    if how_out is not None:
        _check_dtype(how_out, "int8")
    x0, y0, cell, nx, ny = (int(v) for v in grid_spec)
    if int(src.shape[0]) != nx * ny:
        raise ValueError("src must hold nx * ny values")
    check(_lib().bg_resample_points(_ptr(src), x0, y0, cell, nx, ny, int(method), _ptr(qx_cm),
                                    _ptr(qy_cm), m, _ptr(out), _ptr(how_out),
                                    _stream(stream, out)), "bg_resample_points")


def resample_grid(src, grid_spec, method: int, out_spec, out, how_out=None, stream=None) -> None:
    """Bilinear / Catmull-Rom of a regular grid at every node of the output grid
    out_spec = (x0_cm, y0_cm, cell_cm, nx, ny), row-major into out."""
    _check_dtype(src, "float32")
    _check_dtype(out, "float32")
    if how_out is not None:
        _check_dtype(how_out, "int8")
    x0, y0, cell, nx, ny = (int(v) for v in grid_spec)
    ox0, oy0, ocell, onx, ony = (int(v) for v in out_spec)
    if int(src.shape[0]) != nx * ny or int(out.shape[0]) < onx * ony:
        raise ValueError("src must hold nx * ny values and out onx * ony")
    check(_lib().bg_resample_grid(_ptr(src), x0, y0, cell, nx, ny, int(method), ox0, oy0, ocell,
                                  onx, ony, _ptr(out), _ptr(how_out), _stream(stream, out)),
          "bg_resample_grid")


def interp_idw_noalloc(x_cm, y_cm, z_m, grid_spec, k: int, power: float, depth_out,
                      nbr_out=None, stream=None) -> None:
    """IDW without any device allocation (device inputs, at most 262,144 soundings).

    grid_spec = (x0_cm, y0_cm, cell_cm, nx, ny). For callers that cannot
    allocate device memory; the library's fixed 16 MiB device array serves as
    work space, so two overlapping calls must not run at once.
    """
    for t, dt in ((x_cm, "int32"), (y_cm, "int32"), (z_m, "float32"), (depth_out, "float32")):
        _check_dtype(t, dt)
    if nbr_out is not None:
        _check_dtype(nbr_out, "int32")
    x0, y0, cell, nx, ny = (int(v) for v in grid_spec)
    check(_lib().bg_interp_idw_noalloc(_ptr(x_cm), _ptr(y_cm), _ptr(z_m), int(x_cm.shape[0]),
                                       x0, y0, cell, nx, ny, k, power, _ptr(depth_out),
                                       _ptr(nbr_out), _stream(stream, depth_out)),
          "bg_interp_idw_noalloc")


# host arrays of submitted requests, kept alive until their ticket completes
_inflight = {}


def submit(ctx, x_cm, y_cm, z_m, grid_spec, method: int, k: int, depth_out, var_out=None,
           power: float = 2.0, vgm: Variogram | None = None) -> int:
    """Queue a gridding request on host arrays; returns its ticket.

    grid_spec = (x0_cm, y0_cm, cell_cm, nx, ny); method IDW (0) or OKRIGE (1).
    depth_out / var_out are host float32 arrays of nx*ny, written when the
    ticket completes; all arrays are kept alive here until then.
    """
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=d) for a, d in
            ((x_cm, np.int32), (y_cm, np.int32), (z_m, np.float32))]
    for a in (depth_out, var_out):
        if a is not None and (a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]):
            raise TypeError("outputs must be contiguous float32 numpy arrays")
    x0, y0, cell, nx, ny = (int(v) for v in grid_spec)
    r = Request()
    r.x_cm, r.y_cm, r.z_m = (a.ctypes.data for a in arrs)
    r.n = int(arrs[0].size)
    r.x0_cm, r.y0_cm, r.cell_cm, r.nx, r.ny = x0, y0, cell, nx, ny
    r.method, r.k, r.power = int(method), int(k), float(power)
    r.variogram = vgm if vgm is not None else variogram()
    r.depth_out = depth_out.ctypes.data
    r.var_out = var_out.ctypes.data if var_out is not None else None
    t = ctypes.c_uint64()
    check(_lib().bg_submit(ctx, ctypes.byref(r), ctypes.byref(t)), "bg_submit")
    _inflight[(ctx.value, t.value)] = (arrs, depth_out, var_out)
    return t.value


def poll(ctx, ticket: int):
    """Result of a finished ticket (then released), or None while it runs."""
    res = Result()
    st = check(_lib().bg_poll(ctx, ticket, ctypes.byref(res)), "bg_poll")
    if st == _capi.BG_PENDING:
        return None
    _inflight.pop((ctx.value, ticket), None)
    return res


def wait(ctx, ticket: int, timeout_ms: int = -1):
    """Block until the ticket finishes (BGError with BG_ERR_TIMEOUT on expiry)."""
    res = Result()
    check(_lib().bg_wait(ctx, ticket, int(timeout_ms), ctypes.byref(res)), "bg_wait")
    _inflight.pop((ctx.value, ticket), None)
    return res


def cancel(ctx, ticket: int) -> None:
    check(_lib().bg_cancel(ctx, ticket), "bg_cancel")


def serve_stats(ctx):
    """(queued, running, reserved device bytes) of the context's serving loop."""
    q, r, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(_lib().bg_serve_stats(ctx, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)),
          "bg_serve_stats")
    return q.value, r.value, b.value


def serve_shutdown(ctx) -> None:
    check(_lib().bg_serve_shutdown(ctx), "bg_serve_shutdown")


class Batch:
    """Handle of a batch of tiles (bg_batch_t) with references to its tensors."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep


def batch_create(ctx, tiles) -> Batch:
    """Lay out a batch. tiles: sequence of dicts with device tensors x_cm, y_cm
    (int32), z_m (float32), grid_spec (x0, y0, cell, nx, ny), method, k, and
    outputs depth_out (float32, nx*ny), var_out (kriging, or None); plus power
    (IDW) or vgm (kriging)."""
    arr = (_capi.Tile * max(1, len(tiles)))()
    keep = []
    for i, t in enumerate(tiles):
        for name, dt in (("x_cm", "int32"), ("y_cm", "int32"), ("z_m", "float32"),
                         ("depth_out", "float32")):
            _check_dtype(t[name], dt)
            if not _is_cuda(t[name]):
                raise ValueError(f"tile {i}: {name} must be a device tensor")
        r = arr[i]
        r.x_cm, r.y_cm, r.z_m = (t[n].data_ptr() for n in ("x_cm", "y_cm", "z_m"))
        r.n = int(t["x_cm"].shape[0])
        r.x0_cm, r.y0_cm, r.cell_cm, r.nx, r.ny = (int(v) for v in t["grid_spec"])
        r.method, r.k = int(t["method"]), int(t["k"])
        r.power = float(t.get("power", 2.0))
        r.variogram = t.get("vgm") or variogram()
        r.depth_out = t["depth_out"].data_ptr()
        vo = t.get("var_out")
        r.var_out = vo.data_ptr() if vo is not None else None
        keep.append(t)
    out = ctypes.c_void_p()
    check(_lib().bg_batch_create(ctx, arr, len(tiles), ctypes.byref(out)), "bg_batch_create")
    return Batch(out, keep)


def batch_run(b: Batch, stream=None) -> None:
    check(_lib().bg_batch_run(b.handle, _stream(stream, *(t["depth_out"] for t in b._keep[:1]))),
          "bg_batch_run")


def batch_set_cell_target(b: Batch, soundings_per_cell: float) -> None:
    check(_lib().bg_batch_set_cell_target(b.handle, float(soundings_per_cell)),
          "bg_batch_set_cell_target")


def batch_set_shape(b: Batch, knn_strip: int, solve_item: int) -> None:
    """k-NN nodes per thread along x (1, 2, 4) and solve block batches per
    claimed item (1, 2, 4, 8, 16) of the next runs; results do not change."""
    check(_lib().bg_batch_set_shape(b.handle, int(knn_strip), int(solve_item)),
          "bg_batch_set_shape")


def batch_config(b: Batch) -> dict:
    """{'soundings_per_cell', 'knn_strip', 'solve_item'} of the batch."""
    ppc, strip, item = ctypes.c_float(), ctypes.c_int(), ctypes.c_int()
    check(_lib().bg_batch_get_config(b.handle, ctypes.byref(ppc), ctypes.byref(strip),
                                     ctypes.byref(item)), "bg_batch_get_config")
    return {"soundings_per_cell": ppc.value, "knn_strip": strip.value, "solve_item": item.value}


def batch_tune(b: Batch, stream=None) -> float:
    """Tune the cell target, k-NN strip and solve item size (batch_config
    gives all three); returns the cell target."""
    best = ctypes.c_float()
    check(_lib().bg_batch_tune(b.handle, _stream(stream, *(t["depth_out"] for t in b._keep[:1])),
                               ctypes.byref(best)), "bg_batch_tune")
    return best.value


def batch_status(b: Batch) -> int:
    f = ctypes.c_int()
    check(_lib().bg_batch_status(b.handle, ctypes.byref(f)), "bg_batch_status")
    return f.value


def batch_destroy(b: Batch) -> None:
    check(_lib().bg_batch_destroy(b.handle), "bg_batch_destroy")
    b._keep = []


def _check_dtype(t, name):
    dt = str(t.dtype)
    if not dt.endswith(name):
        raise TypeError(f"expected {name}, got {dt}")
