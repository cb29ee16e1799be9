"""GB300 (sm_103a) ray-casting volume renderer for spectral data cubes.

Python binding of the C ABI in ``include/vr.h`` (``libvr.so``).  Functions named
``vr_*`` mirror the C entry points one to one and only marshal arguments; every
step of rendering runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if ``libvr.so`` is missing or
fails to load, every call raises.

The method is the ray-casting renderer of Hassan, Fluke & Barnes (Abstract,
Sec. 1: ray casting of HI spectral cubes larger than one machine's memory;
Sec. 3: renders of one orientation at a user-defined size, 5 x 5 wall of
1920 x 1080 panels).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvr.so")

VR_OK, VR_ERR_INVALID_ARG, VR_ERR_STATE, VR_ERR_OOM, VR_ERR_CUDA = 0, 1, 2, 3, 4
VR_ERR_TIMEOUT, VR_ERR_IO, VR_ERR_INTERNAL, VR_ERR_UNSUPPORTED = 5, 6, 7, 8
VR_F32, VR_F16, VR_BF16 = 0, 1, 2
VR_COMPOSITE, VR_MIP = 0, 1
DTYPES = {"f32": VR_F32, "f16": VR_F16, "bf16": VR_BF16}
MODES = {"composite": VR_COMPOSITE, "mip": VR_MIP}
VR_OPT_SINGLE_STORE = 1
VR_PATH_AUTO, VR_PATH_RAY, VR_PATH_BRICK, VR_PATH_SORTLAST, VR_PATH_LAYERED = 0, 1, 2, 3, 4
PATHS = {"auto": VR_PATH_AUTO, "ray": VR_PATH_RAY, "brick": VR_PATH_BRICK, "sortlast": VR_PATH_SORTLAST,
         "layered": VR_PATH_LAYERED}


class VrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


class vr_camera(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("eye", ctypes.c_double * 3), ("right", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fwd", ctypes.c_double * 3),
                ("win", ctypes.c_double * 4), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class vr_options(ctypes.Structure):
    _fields_ = [("brick", ctypes.c_int32), ("flags", ctypes.c_int32), ("step", ctypes.c_double),
                ("ert", ctypes.c_double)]


class vr_tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("block", ctypes.c_int32),
                ("group", ctypes.c_int32)]


class vr_stream_stats(ctypes.Structure):
    _fields_ = [("bricks_fetched", ctypes.c_uint64), ("bricks_culled", ctypes.c_uint64),
                ("bytes_h2d", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("generate_s", ctypes.c_double), ("wait_s", ctypes.c_double)]


REGION_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_void_p)


class vr_cube_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("nbx", ctypes.c_int32), ("nby", ctypes.c_int32), ("nbz", ctypes.c_int32),
                ("brick", ctypes.c_int32), ("pitch", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("brick_bytes", ctypes.c_int64), ("store_bytes", ctypes.c_int64)]


_P = ctypes.c_void_p
# name -> (restype, argtypes); every symbol include/vr.h declares.
SIGNATURES = {
    "vr_default_options": (None, [_P]),
    "vr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "vr_create": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "vr_destroy": (ctypes.c_int, [_P]),
    "vr_load_cube": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int, _P]),
    "vr_set_transfer_function": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float,
                                                ctypes.c_float]),
    "vr_set_camera": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "vr_render": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "vr_set_path": (ctypes.c_int, [_P, ctypes.c_int]),
    "vr_load_cube_streamed": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_uint64]),
    "vr_get_stream_stats": (ctypes.c_int, [_P, _P]),
    "vr_set_stream_timeout": (ctypes.c_int, [_P, ctypes.c_double]),
    "vr_get_tuning": (ctypes.c_int, [_P, _P]),
    "vr_set_tuning": (ctypes.c_int, [_P, _P]),
    "vr_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P]),
    "vr_set_graph": (ctypes.c_int, [_P, ctypes.c_int]),
    "vr_render_backward": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "vr_set_sample_counter": (ctypes.c_int, [_P, _P]),
    "vr_selftest_wait_timeout": (ctypes.c_int, [_P, _P]),
    "vr_set_kernel_events": (ctypes.c_int, [_P, _P, _P]),
    "vr_render_mip_noalloc": (ctypes.c_int, [_P, _P, _P, _P]),
    "vr_get_cube_info": (ctypes.c_int, [_P, _P]),
    "vr_pyramid_layout": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    "vr_image_pyramid": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "vr_overlay_boxes": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P]),
    "vr_sortlast_partials": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int32, _P, _P, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int64), _P]),
    "vr_sortlast_fold": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, _P, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "vr_last_error": (ctypes.c_char_p, [_P]),
}

# vr_footprint (include/vr.h) as a numpy record
FOOTPRINT = np.dtype([("brick", "<i4"), ("key", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("x1", "<i4"),
                      ("y1", "<i4"), ("offset", "<i8")])

_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libvr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(ctx, status: int, what: str):
    if status != VR_OK:
        lib = load_library()
        msg = lib.vr_last_error(ctx).decode() if ctx else ""
        name = lib.vr_status_string(status).decode()
        raise VrError(status, f"{what}: {name}: {msg}")


def _stream_handle(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def camera_struct(cam: dict) -> vr_camera:
    c = vr_camera()
    c.type = int(cam["type"])
    for k in ("eye", "right", "up", "fwd"):
        setattr(c, k, (ctypes.c_double * 3)(*[float(v) for v in cam[k]]))
    c.win = (ctypes.c_double * 4)(*[float(v) for v in cam["win"]])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


# ------------------------------------------------------------------ same-named entry points
def vr_create(device: int = 0, brick: int = 128, step: float = 0.5, ert: float = 0.99,
              single_store: bool = False):
    lib = load_library()
    o = vr_options()
    lib.vr_default_options(ctypes.byref(o))
    o.brick, o.step, o.ert = int(brick), float(step), float(ert)
    o.flags = VR_OPT_SINGLE_STORE if single_store else 0
    h = ctypes.c_void_p()
    st = lib.vr_create(ctypes.byref(h), int(device), ctypes.byref(o))
    if st != VR_OK:
        raise VrError(st, f"vr_create: {lib.vr_status_string(st).decode()}")
    return h


def vr_destroy(ctx):
    load_library().vr_destroy(ctx)


def vr_load_cube(ctx, src, storage: str = "f32", stream=None, device: int = 0):
    """src: float32 numpy array (host) or torch tensor (host or device), shape (nz, ny, nx)."""
    import torch
    lib = load_library()
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.float32)
        ptr, on_dev, shape = src.ctypes.data, 0, src.shape
    else:
        if src.dtype != torch.float32 or not src.is_contiguous():
            raise ValueError("vr_load_cube: need a contiguous float32 tensor")
        ptr, on_dev, shape = src.data_ptr(), int(src.is_cuda), tuple(src.shape)
    nz, ny, nx = shape
    st = lib.vr_load_cube(ctx, ctypes.c_void_p(ptr), on_dev, nx, ny, nz, DTYPES[storage],
                          _stream_handle(stream, device))
    _check(ctx, st, "vr_load_cube")


def vr_set_transfer_function(ctx, rgba, vmin: float, vmax: float):
    lib = load_library()
    t = np.ascontiguousarray(np.asarray(rgba, dtype=np.float32))
    st = lib.vr_set_transfer_function(ctx, t.ctypes.data_as(_P), int(t.shape[0]), float(vmin),
                                      float(vmax))
    _check(ctx, st, "vr_set_transfer_function")


def vr_set_camera(ctx, cams):
    lib = load_library()
    if isinstance(cams, dict):
        cams = [cams]
    arr = (vr_camera * len(cams))(*[camera_struct(c) for c in cams])
    st = lib.vr_set_camera(ctx, arr, len(cams))
    _check(ctx, st, "vr_set_camera")


def vr_render(ctx, mode: str, out_rgba, out_max=None, stream=None, device: int = 0):
    lib = load_library()
    st = lib.vr_render(ctx, MODES[mode], ctypes.c_void_p(out_rgba.data_ptr()),
                       None if out_max is None else ctypes.c_void_p(out_max.data_ptr()),
                       _stream_handle(stream, device))
    _check(ctx, st, "vr_render")


def vr_render_backward(ctx, mode: str, dL_dimg, dL_dtf, dL_dvol=None, stream=None, device: int = 0):
    """dL_dimg (ncams, H, W, 4), dL_dtf (n, 4), dL_dvol (nz, ny, nx) or None: device float32."""
    lib = load_library()
    st = lib.vr_render_backward(ctx, MODES[mode], ctypes.c_void_p(dL_dimg.data_ptr()),
                                ctypes.c_void_p(dL_dtf.data_ptr()),
                                None if dL_dvol is None else ctypes.c_void_p(dL_dvol.data_ptr()),
                                _stream_handle(stream, device))
    _check(ctx, st, "vr_render_backward")


VR_NOALLOC_MAX_PIXELS = 1 << 21


def vr_render_mip_noalloc(ctx, out_rgba, out_max=None, stream=None, device: int = 0):
    """MIP into caller-provided device tensors with no device allocation by the library
    (scratch is a fixed array inside libvr.so; see include/vr.h)."""
    lib = load_library()
    st = lib.vr_render_mip_noalloc(ctx, ctypes.c_void_p(out_rgba.data_ptr()),
                                   None if out_max is None else ctypes.c_void_p(out_max.data_ptr()),
                                   _stream_handle(stream, device))
    _check(ctx, st, "vr_render_mip_noalloc")


def vr_sortlast_partials(ctx, mode: str, bricks, partial=None, stream=None, device: int = 0):
    """Footprints (numpy FOOTPRINT array, in the order of `bricks`) and the float4 count of
    the partial images of the listed bricks for camera 0; with `partial` (a float32 device
    tensor of at least 4 x that many values) also renders the images into it."""
    ids = np.ascontiguousarray(bricks, dtype=np.int32)
    foot = np.zeros(ids.size, FOOTPRINT)
    need = ctypes.c_int64(0)
    cap = 0 if partial is None else partial.numel() // 4
    st = load_library().vr_sortlast_partials(
        ctx, MODES[mode], ids.ctypes.data_as(ctypes.c_void_p) if ids.size else None, int(ids.size),
        foot.ctypes.data_as(ctypes.c_void_p) if ids.size else None,
        None if partial is None else ctypes.c_void_p(partial.data_ptr()), cap, ctypes.byref(need),
        _stream_handle(stream, device))
    _check(ctx, st, "vr_sortlast_partials")
    return foot, need.value


def vr_sortlast_fold(ctx, mode: str, partial, foot, y0: int, y1: int, out, stream=None, device: int = 0):
    """Fold the partial images (float32 device tensor, footprints `foot`, FOOTPRINT array)
    over rows [y0, y1) of camera 0 into out (device tensor, (y1 - y0) x width x 4)."""
    f = np.ascontiguousarray(foot, dtype=FOOTPRINT)
    cap = 0 if partial is None else partial.numel() // 4
    st = load_library().vr_sortlast_fold(
        ctx, MODES[mode], None if partial is None or cap == 0 else ctypes.c_void_p(partial.data_ptr()), cap,
        f.ctypes.data_as(ctypes.c_void_p), int(f.size), int(y0), int(y1), ctypes.c_void_p(out.data_ptr()),
        _stream_handle(stream, device))
    _check(ctx, st, "vr_sortlast_fold")


def vr_pyramid_layout(width: int, height: int, tile: int = 0):
    """(levels counting level 0, floats the packed levels 1.. take)."""
    lv, nf = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(None, load_library().vr_pyramid_layout(width, height, tile, ctypes.byref(lv), ctypes.byref(nf)),
           "vr_pyramid_layout")
    return lv.value, nf.value


def vr_image_pyramid(ctx, rgba, out, tile: int = 0, stream=None, device: int = 0):
    """Levels 1.. of the premultiplied RGBA image rgba (device tensor, height x width x 4
    float32) into out (device tensor of vr_pyramid_layout floats); see include/vr.h."""
    h, w = int(rgba.shape[-3]), int(rgba.shape[-2])
    lib = load_library()
    st = lib.vr_image_pyramid(ctx, ctypes.c_void_p(rgba.data_ptr()), w, h, tile,
                              ctypes.c_void_p(out.data_ptr()), _stream_handle(stream, device))
    _check(ctx, st, "vr_image_pyramid")


def vr_overlay_boxes(ctx, cams, boxes, colours, rgba, stream=None, device: int = 0):
    """Wireframe bounding cubes (boxes: nbox x 6 x0 y0 z0 x1 y1 z1, colours: nbox x 4 straight
    RGBA; host arrays) drawn over the premultiplied images rgba (device tensor, ncams x H x W
    x 4) of the cameras cams; see include/vr.h."""
    import numpy as np
    if isinstance(cams, dict):
        cams = [cams]
    arr = (vr_camera * len(cams))(*[camera_struct(c) for c in cams])
    b = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
    c = np.ascontiguousarray(colours, dtype=np.float32).reshape(-1, 4)
    if len(b) != len(c):
        raise ValueError("one colour per box")
    lib = load_library()
    st = lib.vr_overlay_boxes(ctx, arr, len(cams), b.ctypes.data_as(ctypes.c_void_p), len(b),
                              c.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(rgba.data_ptr()),
                              _stream_handle(stream, device))
    _check(ctx, st, "vr_overlay_boxes")


def vr_get_tuning(ctx) -> dict:
    t = vr_tuning()
    _check(ctx, load_library().vr_get_tuning(ctx, ctypes.byref(t)), "vr_get_tuning")
    return {k: getattr(t, k) for k, _ in vr_tuning._fields_}


def vr_set_tuning(ctx, tuning: dict):
    t = vr_tuning(**{k: int(tuning[k]) for k, _ in vr_tuning._fields_})
    _check(ctx, load_library().vr_set_tuning(ctx, ctypes.byref(t)), "vr_set_tuning")


def vr_autotune(ctx, mode: str, scratch_rgba, reps: int = 5, stream=None, device: int = 0):
    """Time every candidate launch shape for `mode`; keeps and returns the fastest
    (dict with the tuning and its ms per render)."""
    t = vr_tuning()
    ms = ctypes.c_double()
    st = load_library().vr_autotune(ctx, MODES[mode], ctypes.c_void_p(scratch_rgba.data_ptr()), int(reps),
                                    ctypes.byref(t), ctypes.byref(ms), _stream_handle(stream, device))
    _check(ctx, st, "vr_autotune")
    d = {k: getattr(t, k) for k, _ in vr_tuning._fields_}
    d["ms"] = ms.value
    return d


def vr_set_graph(ctx, enable: bool = True):
    _check(ctx, load_library().vr_set_graph(ctx, int(bool(enable))), "vr_set_graph")


def vr_load_cube_streamed(ctx, fn, user, dims, storage: str = "f16", cache_bytes: int = 1 << 30):
    """Out-of-core cube of dims (nx, ny, nz) pulled on demand from the region callback
    `fn` (a C function pointer as ctypes.c_void_p, or a REGION_FN) with `user` (a
    ctypes object or address kept alive by the caller)."""
    lib = load_library()
    uptr = ctypes.c_void_p(ctypes.addressof(user)) if isinstance(user, ctypes.Structure) else user
    fptr = ctypes.cast(fn, ctypes.c_void_p)
    nx, ny, nz = dims
    st = lib.vr_load_cube_streamed(ctx, fptr, uptr, int(nx), int(ny), int(nz), DTYPES[storage],
                                   int(cache_bytes))
    _check(ctx, st, "vr_load_cube_streamed")


def vr_get_stream_stats(ctx) -> dict:
    s = vr_stream_stats()
    _check(ctx, load_library().vr_get_stream_stats(ctx, ctypes.byref(s)), "vr_get_stream_stats")
    return {k: getattr(s, k) for k, _ in vr_stream_stats._fields_}


def vr_set_stream_timeout(ctx, seconds: float):
    _check(ctx, load_library().vr_set_stream_timeout(ctx, float(seconds)), "vr_set_stream_timeout")


def vr_set_path(ctx, path: str = "auto"):
    st = load_library().vr_set_path(ctx, PATHS[path])
    _check(ctx, st, "vr_set_path")


def vr_selftest_wait_timeout(ctx, stream=None, device: int = 0):
    """Make one bounded device wait expire on purpose (no copy in flight) and leave its
    status for the next render to report."""
    st = load_library().vr_selftest_wait_timeout(ctx, _stream_handle(stream, device))
    _check(ctx, st, "vr_selftest_wait_timeout")


def vr_set_sample_counter(ctx, counter=None):
    lib = load_library()
    st = lib.vr_set_sample_counter(ctx, None if counter is None else
                                   ctypes.c_void_p(counter.data_ptr()))
    _check(ctx, st, "vr_set_sample_counter")


def vr_set_kernel_events(ctx, start=None, stop=None):
    """start/stop: torch.cuda.Event(enable_timing=True) (or None, None to turn off)."""
    lib = load_library()
    h = (lambda e: None if e is None else ctypes.c_void_p(e.cuda_event))
    if start is not None:
        start.record()  # make sure the underlying CUDA events exist
        stop.record()
    st = lib.vr_set_kernel_events(ctx, h(start), h(stop))
    _check(ctx, st, "vr_set_kernel_events")


def vr_get_cube_info(ctx) -> dict:
    lib = load_library()
    info = vr_cube_info()
    _check(ctx, lib.vr_get_cube_info(ctx, ctypes.byref(info)), "vr_get_cube_info")
    return {k: getattr(info, k) for k, _ in vr_cube_info._fields_}


# ------------------------------------------------------------------ convenience object
class Renderer:
    """A context plus its output buffers.  All rendering happens in libvr.so."""

    def __init__(self, device: int = 0, brick: int = 128, step: float = 0.5, ert: float = 0.99,
                 single_store: bool = False):
        import torch
        self.device = int(device)
        self.torch_device = torch.device("cuda", self.device)
        self.ctx = vr_create(self.device, brick, step, ert, single_store)
        self.cams = []

    def close(self):
        if self.ctx is not None:
            vr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_cube(self, vol, storage="f32", stream=None):
        vr_load_cube(self.ctx, vol, storage, stream, self.device)

    def set_transfer_function(self, rgba, vmin, vmax):
        vr_set_transfer_function(self.ctx, rgba, vmin, vmax)

    def set_camera(self, cams):
        if isinstance(cams, dict):
            cams = [cams]
        vr_set_camera(self.ctx, cams)
        self.cams = list(cams)

    def set_path(self, path="auto"):
        vr_set_path(self.ctx, path)

    def overlay(self, rgba, boxes, colours, cams=None, stream=None):
        """Draw a catalogue's bounding cubes over images rendered with this renderer's
        cameras (or cams), in place."""
        vr_overlay_boxes(self.ctx, self.cams if cams is None else cams, boxes, colours, rgba, stream,
                         self.device)
        return rgba

    def pyramid(self, rgba, tile: int = 0, out=None, stream=None):
        """Packed levels 1.. of an image (height x width x 4) of this renderer's device."""
        import torch
        rgba = rgba.contiguous()
        _, nf = vr_pyramid_layout(int(rgba.shape[-2]), int(rgba.shape[-3]), tile)
        if out is None:
            out = torch.empty(max(nf, 4), dtype=torch.float32, device=self.torch_device)
        vr_image_pyramid(self.ctx, rgba, out, tile, stream, self.device)
        return out[:nf]

    def cube_info(self):
        return vr_get_cube_info(self.ctx)

    def render(self, mode="composite", out=None, out_max=None, with_max=False, stream=None):
        import torch
        n, h, w = len(self.cams), self.cams[0]["height"], self.cams[0]["width"]
        if out is None:
            out = torch.empty((n, h, w, 4), dtype=torch.float32, device=self.torch_device)
        if with_max and out_max is None:
            out_max = torch.empty((n, h, w), dtype=torch.float32, device=self.torch_device)
        vr_render(self.ctx, mode, out, out_max, stream, self.device)
        return (out, out_max) if with_max else out


# ------------------------------------------------------------------ autograd
def _autograd_function():
    import torch

    class VolumeRenderFunction(torch.autograd.Function):
        """image = render(tf, volume); backward calls vr_render_backward.

        The renderer must hold the cube `volume` (VolumeRenderer.render loads it when the
        tensor changes) and the table `tf`; both are copied into the library."""

        @staticmethod
        def forward(ctx, tf, volume, renderer, mode):
            out = renderer.render(mode)
            ctx.renderer = renderer
            ctx.mode = mode
            ctx.tf_shape = tuple(tf.shape)
            ctx.vol_shape = tuple(volume.shape) if volume is not None else None
            ctx.need_vol = volume is not None and volume.requires_grad
            return out

        @staticmethod
        def backward(ctx, grad):
            r = ctx.renderer
            dtf = torch.empty(ctx.tf_shape, dtype=torch.float32, device=r.torch_device)
            dvol = (torch.empty(ctx.vol_shape, dtype=torch.float32, device=r.torch_device)
                    if ctx.need_vol else None)
            vr_render_backward(r.ctx, ctx.mode, grad.contiguous().float(), dtf, dvol,
                               device=r.device)
            return dtf, dvol, None, None

    return VolumeRenderFunction


_VRF = None


class VolumeRenderer(Renderer):
    """Renderer whose render(tf, volume) takes part in torch autograd: gradients flow to
    the transfer-function table and (if it requires grad) the float32 volume."""

    def __init__(self, device=0, brick=128, step=0.5, ert=0.99, vmin=-1.0, vmax=20.0,
                 storage="f32"):
        super().__init__(device, brick, step, ert)
        self.vmin, self.vmax, self.storage = float(vmin), float(vmax), storage
        self._vol_key = None

    def render(self, mode="composite", out=None, out_max=None, with_max=False, stream=None,
               tf=None, volume=None):
        if tf is None:
            return super().render(mode, out, out_max, with_max, stream)
        global _VRF
        if _VRF is None:
            _VRF = _autograd_function()
        key = (id(volume), volume._version, volume.data_ptr()) if volume is not None else None
        if volume is not None and key != self._vol_key:
            self.load_cube(volume.detach().contiguous(), self.storage, stream)
            self._vol_key = key
        self.set_transfer_function(tf.detach().float().cpu().numpy(), self.vmin, self.vmax)
        return _VRF.apply(tf, volume, _Plain(self), mode)


class _Plain:
    """The non-autograd face of a VolumeRenderer (what the autograd function calls)."""

    def __init__(self, r):
        self._r = r
        self.ctx, self.device, self.torch_device = r.ctx, r.device, r.torch_device

    def render(self, mode):
        return Renderer.render(self._r, mode)


# ------------------------------------------------------------------ autotuning cache
def autotune(renderer: Renderer, mode: str, reps: int = 5, cache: str | None = None) -> dict:
    """Pick the launch shape for `mode` on the renderer's current cube and cameras with
    vr_autotune, remembering the result in a JSON file keyed by GPU, cube, storage type,
    image size, camera count and mode (so a later run on the same workload reuses it)."""
    import json

    import torch
    info = renderer.cube_info()
    n, h, w = len(renderer.cams), renderer.cams[0]["height"], renderer.cams[0]["width"]
    key = "|".join(str(x) for x in (torch.cuda.get_device_name(renderer.device), info["nx"], info["ny"],
                                    info["nz"], info["dtype"], info["brick"], w, h, n, mode))
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        vr_set_tuning(renderer.ctx, table[key])
        return dict(table[key], cached=True)
    scratch = torch.empty((n, h, w, 4), dtype=torch.float32, device=renderer.torch_device)
    best = vr_autotune(renderer.ctx, mode, scratch, reps, device=renderer.device)
    if cache:
        table[key] = best
        tmp = cache + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return dict(best, cached=False)
