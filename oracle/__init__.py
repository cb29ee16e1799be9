"""FP64 CPU oracle for the ray-casting volume renderer (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  It shares no code
with the CUDA renderer; both consume the same inputs from ``synth``.

What it computes (steps in order; the paper -- Hassan, Fluke & Barnes, Abstract
and Secs. 1 and 3 -- names ray casting of spectral cubes, larger-than-memory
decomposition and high-resolution renders of one orientation, but prints no
formulas, so each step is the standard definition):

1. camera ray per pixel centre (rows top-down; orthographic rays start on the
   image plane, perspective rays at the eye);
2. slab intersection with [0,nx]x[0,ny]x[0,nz], t >= 0;
3. samples t_k = k*step, k in [ceil(t_near/step), ceil(t_far/step));
4. trilinear interpolation, cell-centred voxels, clamp to edge;
5. node-centred linear transfer-function lookup over [vmin, vmax], clamped;
6. front-to-back "over" with termination after the sample at which
   1 - T >= ert; MIP outputs TF(max v) straight;
7. the adjoint of 6 (reverse sweep with suffix colour / transmittance);
8. the image pyramid of a render (2 x 2 box filter of premultiplied RGBA per level);
9. the catalogue overlay: wireframe bounding cubes projected and drawn over a render.

Parity pins: see tests/test_oracle_pins.py (closed forms for constant cubes,
single-peak MIP, brute force along the spectral axis, sort-last invariance,
finite differences for the adjoint).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
# A prebuilt oracle library to load instead (the mutation test points this at
# deliberately broken copies to show that the pins catch them).
_LIB_OVERRIDE = os.environ.get("VR_ORACLE_LIB")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_oracle.so (gcc -O2, strict IEEE: no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=gnu11",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcCamera(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("eye", ctypes.c_double * 3), ("right", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fwd", ctypes.c_double * 3),
                ("win", ctypes.c_double * 4), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class OrcScene(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("vol", ctypes.c_void_p), ("tf", ctypes.c_void_p), ("ntf", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double),
                ("step", ctypes.c_double), ("ert", ctypes.c_double), ("dk0", ctypes.c_int32),
                ("dk1", ctypes.c_int32), ("pos_err", ctypes.c_double), ("dstop", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


_P = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if _LIB_OVERRIDE:
                lib = ctypes.CDLL(_LIB_OVERRIDE)
            else:
                build()
                lib = ctypes.CDLL(_LIB)
            lib.orc_render.restype = ctypes.c_int
            lib.orc_render.argtypes = [_P, _P, _P, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int]
            lib.orc_render_sortlast.restype = ctypes.c_int
            lib.orc_render_sortlast.argtypes = [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P,
                                                _P, ctypes.c_int]
            lib.orc_backward.restype = ctypes.c_int
            lib.orc_backward.argtypes = [_P, _P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int]
            lib.orc_touch.restype = ctypes.c_int
            lib.orc_touch.argtypes = [_P, _P, _P, ctypes.c_int64, _P, ctypes.c_int]
            lib.orc_brick_partial.restype = ctypes.c_int
            lib.orc_brick_partial.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int64, _P,
                                              ctypes.c_int64, _P, _P, _P, _P]
            lib.orc_round_bf16.restype = None
            lib.orc_round_bf16.argtypes = [_P, _P, ctypes.c_int64]
            lib.orc_overlay.restype = ctypes.c_int
            lib.orc_overlay.argtypes = [_P, _P, ctypes.c_int64, _P, _P, _P]
            lib.orc_pyramid.restype = ctypes.c_int
            lib.orc_pyramid.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P,
                                        ctypes.POINTER(ctypes.c_int64)]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def camera_struct(cam: dict) -> OrcCamera:
    c = OrcCamera()
    c.type = int(cam["type"])
    for k in ("eye", "right", "up", "fwd"):
        setattr(c, k, (ctypes.c_double * 3)(*[float(v) for v in cam[k]]))
    c.win = (ctypes.c_double * 4)(*[float(v) for v in cam["win"]])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


U32 = 2.0 ** -24  # unit roundoff of FP32


def pos_err_bricked(brick: int, far: float = 0.0) -> float:
    """Sample-position error bound (voxels, per axis) of a renderer that steps samples in
    brick-local FP32 coordinates: |g| <= brick + 2 rounded three times (anchor, offset,
    step FMA), plus the drift of the FP32-rounded step vector over one brick, at most
    u (brick + 1), plus the float-float anchor's own error for a sample `far` voxels
    from the origin (2^-40 far)."""
    return U32 * (4 * brick + 7) + 2.0 ** -40 * far


def pos_err_marcher(step: float, far: float = 0.0, span: int = 12) -> float:
    """Sample-position error bound (voxels, per axis) of a renderer that re-anchors each ray
    in float-float every `span` samples and steps in FP32 relative to the anchor's voxel:
    the remainder at the anchor (in [0, 1], one rounding), the stepped coordinate
    q = q0 + j e (|q| <= 1 + (span - 1) step, one rounding) and the drift of the
    FP32-rounded step vector over the span (at most u (span - 1) step), plus the
    float-float anchor's own error for a sample `far` voxels from the origin."""
    return U32 * (2.0 + 2.0 * (span - 1) * float(step)) + 2.0 ** -40 * far


class Scene:
    """A cube (float32 values as stored), a transfer function and march settings.

    pos_err is the error model behind the ambiguity windows (see oracle.c): a bound on the
    renderer's sample-position error in voxels per axis.  The default is the bricked
    stepping bound for 128^3 bricks, the largest brick edge the renderer uses."""

    def __init__(self, vol: np.ndarray, tf: np.ndarray, vmin: float, vmax: float,
                 step: float = 0.5, ert: float = 0.99, pos_err: float | None = None):
        vol = np.ascontiguousarray(vol, dtype=np.float32)
        tf = np.ascontiguousarray(tf, dtype=np.float32)
        assert vol.ndim == 3 and tf.ndim == 2 and tf.shape[1] == 4 and tf.shape[0] >= 2
        self.vol, self.tf = vol, tf
        self.nz, self.ny, self.nx = vol.shape
        self.vmin, self.vmax, self.step, self.ert = float(vmin), float(vmax), float(step), float(ert)
        self.pos_err = pos_err_bricked(128) if pos_err is None else float(pos_err)

    def _struct(self, mode: int, ert=None, dk0=0, dk1=0, dstop=0) -> OrcScene:
        s = OrcScene()
        s.nx, s.ny, s.nz = self.nx, self.ny, self.nz
        s.vol, s.tf = self.vol.ctypes.data, self.tf.ctypes.data
        s.ntf, s.mode = self.tf.shape[0], int(mode)
        s.vmin, s.vmax, s.step = self.vmin, self.vmax, self.step
        s.ert = self.ert if ert is None else float(ert)
        s.dk0, s.dk1 = int(dk0), int(dk1)
        s.pos_err, s.dstop = self.pos_err, int(dstop)
        return s


def _nthreads(n):
    return int(n) if n else (os.cpu_count() or 1)


def render(scene: Scene, cam: dict, mode: str = "composite", pixels=None, *, ert=None, dk0=0,
           dk1=0, dstop=0, nthreads=None) -> dict:
    """Render pixels (flat py*W+px; None = whole image) -> dict(rgba, max, nsamples, flags).
    dk0, dk1, dstop select an alternative outcome of an ambiguous ray (see variants)."""
    lib = _load()
    m = {"composite": 0, "mip": 1}[mode]
    s = scene._struct(m, ert, dk0, dk1, dstop)
    c = camera_struct(cam)
    if pixels is None:
        npix = cam["width"] * cam["height"]
        pix = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix.size
    rgba = np.zeros((npix, 4), np.float64)
    vmax = np.zeros(npix, np.float64)
    ns = np.zeros(npix, np.int64)
    fl = np.zeros(npix, np.int32)
    rc = lib.orc_render(ctypes.byref(s), ctypes.byref(c), None if pix is None else _ptr(pix),
                        npix, _ptr(rgba), _ptr(vmax), _ptr(ns), _ptr(fl), _nthreads(nthreads))
    if rc:
        raise ValueError("orc_render: bad arguments")
    return dict(rgba=rgba, max=vmax, nsamples=ns, flags=fl)


def render_sortlast(scene: Scene, cam: dict, brick: int, mode: str = "composite", pixels=None,
                    *, ert=None, nthreads=None) -> dict:
    lib = _load()
    m = {"composite": 0, "mip": 1}[mode]
    s = scene._struct(m, ert)
    c = camera_struct(cam)
    if pixels is None:
        npix, pix = cam["width"] * cam["height"], None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix.size
    rgba = np.zeros((npix, 4), np.float64)
    vmax = np.zeros(npix, np.float64)
    rc = lib.orc_render_sortlast(ctypes.byref(s), ctypes.byref(c), int(brick),
                                 None if pix is None else _ptr(pix), npix, _ptr(rgba), _ptr(vmax),
                                 _nthreads(nthreads))
    if rc:
        raise ValueError("orc_render_sortlast: bad arguments")
    return dict(rgba=rgba, max=vmax)


def brick_partial(scene: Scene, cam: dict, brick: int, brick_id: int, pixels=None) -> dict:
    """Partial image of one brick of the brick^3 decomposition: per pixel (flat py*W+px;
    None = whole image) the brick's samples composited front to back from T = 1 with no
    termination, as ct = (C0, C1, C2, T), plus their maximum and count, and the brick's
    visibility key (ascending = front to back)."""
    lib = _load()
    s = scene._struct(0, 2.0)
    c = camera_struct(cam)
    if pixels is None:
        pixels = np.arange(cam["width"] * cam["height"], dtype=np.int64)
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    ct = np.zeros((pix.size, 4), np.float64)
    mx = np.zeros(pix.size, np.float64)
    ns = np.zeros(pix.size, np.int64)
    key = ctypes.c_int64(0)
    rc = lib.orc_brick_partial(ctypes.byref(s), ctypes.byref(c), int(brick), int(brick_id), _ptr(pix),
                               pix.size, _ptr(ct), _ptr(mx), _ptr(ns), ctypes.byref(key))
    if rc:
        raise ValueError("orc_brick_partial: bad arguments")
    return dict(ct=ct, max=mx, nsamples=ns, key=int(key.value))


def backward(scene: Scene, cams: list, dimg: np.ndarray, mode: str = "composite", *,
             with_volume=True, ert=None, nthreads=None, ambiguity=False):
    """dL/dTF (ntf x 4) and dL/dvol (nz, ny, nx) for dL/dI = dimg (ncams, H, W, 4).
    With ambiguity=True also returns a third array (nz, ny, nx): per voxel, a bound on how
    far a renderer's voxel gradient may legitimately be from dL/dvol (samples within
    rounding of a table node or of the MIP maximum, rays whose end sample or termination
    is within rounding of its threshold)."""
    lib = _load()
    m = {"composite": 0, "mip": 1}[mode]
    s = scene._struct(m, ert)
    arr = (OrcCamera * len(cams))(*[camera_struct(c) for c in cams])
    g = np.ascontiguousarray(dimg, dtype=np.float64)
    assert g.shape == (len(cams), cams[0]["height"], cams[0]["width"], 4)
    dtf = np.zeros((scene.tf.shape[0], 4), np.float64)
    with_volume = with_volume or ambiguity
    dvol = np.zeros(scene.vol.shape, np.float64) if with_volume else None
    amb = np.zeros(scene.vol.shape, np.float64) if ambiguity else None
    nt = _nthreads(nthreads)
    if with_volume:  # one voxel accumulator (two with the ambiguity bound) per thread
        per = dvol.nbytes * (2 if ambiguity else 1)
        nt = max(1, min(nt, int(4e9 // max(1, per))))
    rc = lib.orc_backward(ctypes.byref(s), arr, len(cams), _ptr(g), _ptr(dtf),
                          None if dvol is None else _ptr(dvol), None if amb is None else _ptr(amb),
                          nt)
    if rc:
        raise ValueError("orc_backward: bad arguments")
    return (dtf, dvol, amb) if ambiguity else (dtf, dvol)


def touched(scene: Scene, cam: dict, mode: str = "mip", pixels=None, nthreads=None) -> np.ndarray:
    """Byte mask (nz, ny, nx) of the voxels read by the executed samples."""
    lib = _load()
    m = {"composite": 0, "mip": 1}[mode]
    s = scene._struct(m)
    c = camera_struct(cam)
    mask = np.zeros(scene.vol.shape, np.uint8)
    if pixels is None:
        npix, pix = cam["width"] * cam["height"], None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pix.size
    rc = lib.orc_touch(ctypes.byref(s), ctypes.byref(c), None if pix is None else _ptr(pix), npix,
                       _ptr(mask), _nthreads(nthreads))
    if rc:
        raise ValueError("orc_touch: bad arguments")
    return mask


def round_storage(vol: np.ndarray, storage: str) -> np.ndarray:
    """The float32 cube as the renderer stores it: 'f32' unchanged, 'f16' IEEE binary16,
    'bf16' bfloat16, both round-to-nearest-even, returned widened to float32."""
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    if storage == "f32":
        return vol
    if storage == "f16":
        return vol.astype(np.float16).astype(np.float32)
    if storage == "bf16":
        out = np.empty_like(vol)
        _load().orc_round_bf16(_ptr(vol), _ptr(out), vol.size)
        return out
    raise ValueError(storage)


def pyramid(img: np.ndarray, tile: int = 0):
    """Levels 1.. of a premultiplied RGBA image (H, W, 4): each level halves the size
    (rounding up) and averages the pixels of each 2 x 2 block that lie inside the level.
    Returns (number of levels counting the input, packed levels as float64, row-major or
    in tile x tile tiles -- the layout of vr_image_pyramid)."""
    a = np.ascontiguousarray(img, dtype=np.float32)
    assert a.ndim == 3 and a.shape[2] == 4
    h, w = a.shape[:2]
    lib = _load()
    n = ctypes.c_int64(0)
    levels = lib.orc_pyramid(_ptr(a), w, h, int(tile), None, ctypes.byref(n))
    if levels < 0:
        raise ValueError("orc_pyramid: bad arguments")
    out = np.zeros(n.value, np.float64)
    lib.orc_pyramid(_ptr(a), w, h, int(tile), _ptr(out), ctypes.byref(n))
    return levels, out


def overlay(img: np.ndarray, cam: dict, boxes: np.ndarray, colours: np.ndarray):
    """Wireframe bounding cubes (nbox, 6: x0 y0 z0 x1 y1 z1) drawn over the premultiplied
    image (H, W, 4) of camera cam, box i in straight colour colours[i]; a pixel covered by
    several boxes takes the highest index.  Returns (image float64, key int32 (H, W):
    index + 1 of the box drawn at each pixel, 0 = none)."""
    out = np.ascontiguousarray(img, dtype=np.float64).copy()
    h, w = out.shape[:2]
    assert (h, w) == (cam["height"], cam["width"])
    bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
    col = np.ascontiguousarray(colours, dtype=np.float32).reshape(-1, 4)
    assert len(col) == len(bx)
    key = np.zeros((h, w), np.int32)
    c = camera_struct(cam)
    if _load().orc_overlay(ctypes.byref(c), _ptr(bx), len(bx), _ptr(col), _ptr(out), _ptr(key)):
        raise ValueError("orc_overlay: bad arguments")
    return out, key


def pyramid_sizes(w: int, h: int):
    """(width, height) of levels 1.. (down to 1 x 1)."""
    out = []
    while w > 1 or h > 1:
        w, h = (w + 1) // 2, (h + 1) // 2
        out.append((w, h))
    return out


def l2_loss(img: np.ndarray, target: np.ndarray):
    """L = mean((I - I*)^2) over every value, and dL/dI."""
    d = np.asarray(img, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def variants(flags: int):
    """(dstop, dk0, dk1) combinations that a flagged ray may legitimately take: its first
    sample one earlier or later (bit 0), its end one earlier or later (bit 1), its
    termination one sample earlier or later (bit 2)."""
    k0s = (0, -1, 1) if flags & 1 else (0,)
    k1s = (0, -1, 1) if flags & 2 else (0,)
    ds = (0, -1, 1) if flags & 4 else (0,)
    return [(e, a, b) for e in ds for a in k0s for b in k1s]
