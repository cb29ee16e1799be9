"""Seeded synthetic inputs shared by the oracle, the CUDA renderer, tests and bench.

Nothing in this package implements the rendering method: it only produces
input data -- HI-like spectral cubes (``generate``), cameras
(``ortho_view``, ``orbit_view``, ``wall_views``, ``random_views``) and
transfer-function tables (``viridis_ramp_tf``, ``hidden_tf``) -- plus the
workload definitions (``CONFIGS``) that name them.

Workload definitions follow the paper's data: HI spectral-line cubes stored
as 32-bit floats (the HIPASS cube of Sec. 3 is 1721 x 1721 x 1025 voxels in
12 GB, i.e. 4 bytes a voxel), with a long spectral axis, and rendered to the
5 x 5 wall of 1920 x 1080 panels of Sec. 3.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into synth/_synth.so (plain C, gcc, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class SynParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("sigma", ctypes.c_double),
                ("nsrc", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("amp_lo", ctypes.c_double), ("amp_hi", ctypes.c_double),
                ("fwhm_s_lo", ctypes.c_double), ("fwhm_s_hi", ctypes.c_double),
                ("fwhm_z_lo", ctypes.c_double), ("fwhm_z_hi", ctypes.c_double),
                ("ripple_amp", ctypes.c_double), ("ripple_period", ctypes.c_double),
                ("trunc", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.syn_region.restype = ctypes.c_int
            lib.syn_region.argtypes = [ctypes.POINTER(SynParams)] + [ctypes.c_int64] * 6 + [
                ctypes.c_void_p, ctypes.c_int]
            lib.syn_sources.restype = ctypes.c_int
            lib.syn_sources.argtypes = [ctypes.POINTER(SynParams), ctypes.c_void_p]
            lib.syn_ripple_phase.restype = ctypes.c_double
            lib.syn_ripple_phase.argtypes = [ctypes.POINTER(SynParams)]
            _lib = lib
    return _lib


class SynCbUser(ctypes.Structure):
    _fields_ = [("p", SynParams), ("nthreads", ctypes.c_int32), ("pad_", ctypes.c_int32)]


def region_callback(p: dict, nthreads: int | None = None):
    """(C function pointer, user struct) of the generator's region callback, for
    renderers that pull cube regions on demand (the struct must be kept alive)."""
    lib = _load()
    u = SynCbUser()
    u.p = _params(p)
    u.nthreads = int(nthreads or os.cpu_count() or 1)
    fn = ctypes.cast(lib.syn_region_cb, ctypes.c_void_p)
    return fn, u


def lib_handle():
    """The loaded generator library (for callers that want its C entry points)."""
    return _load()


# --------------------------------------------------------------------------------------------
# Workload definitions.  Sizes, source counts and ranges are the five workloads of the
# method's evaluation plan; seeds are 1234 + workload index.
# --------------------------------------------------------------------------------------------

def cube_params(nx, ny, nz, *, seed, nsrc, ripple=False, sigma=1.0, amp=(5.0, 20.0),
                fwhm_s=(2.0, 6.0), fwhm_z=(4.0, 20.0), ripple_amp=0.5, ripple_period=256.0,
                trunc=4.0) -> dict:
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), seed=int(seed), sigma=float(sigma),
                nsrc=int(nsrc), amp_lo=amp[0], amp_hi=amp[1], fwhm_s_lo=fwhm_s[0],
                fwhm_s_hi=fwhm_s[1], fwhm_z_lo=fwhm_z[0], fwhm_z_hi=fwhm_z[1],
                ripple_amp=float(ripple_amp) if ripple else 0.0,
                ripple_period=float(ripple_period), trunc=float(trunc))


CONFIGS = {
    # 128^3 noise + 20 sources, orthographic view rotated 30 deg about y and 20 deg about x,
    # 512 x 512, composite with termination at alpha 0.99, plus MIP of the same view.
    "small": dict(cube=cube_params(128, 128, 128, seed=1235, nsrc=20),
                  image=(512, 512), step=0.5, ert=0.99, storage=("f32",)),
    # 1024 x 1024 x 2048 (RA x Dec x channel), 2000 sources + continuum ripple, perspective
    # 1920 x 1080, 36-frame orbit in 10 degree steps, 128^3 bricks with a 1-voxel ghost.
    "survey": dict(cube=cube_params(1024, 1024, 2048, seed=1236, nsrc=2000, ripple=True),
                   image=(1920, 1080), step=0.5, ert=0.99, frames=36,
                   storage=("f32", "f16", "bf16")),
    # 2048 x 2048 x 1024 FP16, same source model (same source density: 4000 sources),
    # 5 x 5 wall of 1920 x 1080 panels as 25 off-axis frusta of one camera.
    "wall": dict(cube=cube_params(2048, 2048, 1024, seed=1237, nsrc=4000, ripple=True),
                 image=(1920, 1080), panels=(5, 5), step=0.5, ert=0.99, storage=("f16",)),
    # 256^3 FP32, noise + 50 sources, 64 seeded views at 512 x 512, hidden TF.
    "diff": dict(cube=cube_params(256, 256, 256, seed=1238, nsrc=50),
                 image=(512, 512), views=64, view_seed=7, tf_seed=99, step=0.5, ert=0.99,
                 storage=("f32",)),
    # The paper's HIPASS cube shape (Sec. 3: 1721 x 1721 x 1025, 32-bit floats, 12 GB), same
    # source density as the survey (2830 sources); one perspective orientation rendered as a
    # high-resolution static image at 3000 x 3000 and 8000 x 8000.
    "hipass": dict(cube=cube_params(1721, 1721, 1025, seed=1240, nsrc=2830, ripple=True),
                   images=((3000, 3000), (8000, 8000)), az=30.0, step=0.5, ert=0.99,
                   storage=("f32",)),
    # 4096 x 4096 x 8192 FP16, same source model (density-scaled: 128000 sources),
    # streamed out of core; 1920 x 1080 perspective, 10-frame orbit.
    "ooc": dict(cube=cube_params(4096, 4096, 8192, seed=1239, nsrc=128000, ripple=True),
                image=(1920, 1080), step=0.5, ert=0.99, frames=10, storage=("f16",)),
}


def _params(p: dict) -> SynParams:
    s = SynParams()
    for k, v in p.items():
        setattr(s, k, v)
    return s


def generate(p: dict, region=None, nthreads: int | None = None, out: np.ndarray | None = None
             ) -> np.ndarray:
    """Cube values as float32, shape (sz, sy, sx) (x fastest).

    ``region`` = (x0, y0, z0, sx, sy, sz); default the whole cube.  Any region is
    bit-identical to the same voxels of the whole cube.
    """
    lib = _load()
    if region is None:
        region = (0, 0, 0, p["nx"], p["ny"], p["nz"])
    x0, y0, z0, sx, sy, sz = (int(v) for v in region)
    if out is None:
        out = np.empty((sz, sy, sx), dtype=np.float32)
    else:
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == sx * sy * sz
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    sp = _params(p)
    rc = lib.syn_region(ctypes.byref(sp), x0, y0, z0, sx, sy, sz,
                        out.ctypes.data_as(ctypes.c_void_p), int(nthreads))
    if rc != 0:
        raise ValueError(f"syn_region failed for region {region} of {p['nx']}x{p['ny']}x{p['nz']}")
    return out


def sources(p: dict) -> np.ndarray:
    """Source table (nsrc, 6): amp, cx, cy, cz, sigma_spatial, sigma_spectral."""
    lib = _load()
    out = np.zeros((max(p["nsrc"], 1), 6), dtype=np.float64)
    sp = _params(p)
    lib.syn_sources(ctypes.byref(sp), out.ctypes.data_as(ctypes.c_void_p))
    return out[: p["nsrc"]]


def catalogue(p: dict, k: float = 2.0) -> np.ndarray:
    """Source-finder style catalogue of the cube's sources: one bounding cube per source,
    (nsrc, 6) as x0, y0, z0, x1, y1, z1 = centre -+ k sigma (spatial sigma on x, y,
    spectral on z), clipped to the cube [0, n]."""
    s = sources(p)
    c = s[:, 1:4]
    r = np.stack([s[:, 4], s[:, 4], s[:, 5]], axis=1) * k
    n = np.array([p["nx"], p["ny"], p["nz"]], np.float64)
    lo = np.clip(c - r, 0.0, n)
    hi = np.clip(c + r, 0.0, n)
    return np.ascontiguousarray(np.concatenate([lo, hi], axis=1))


def ripple_phase(p: dict) -> float:
    lib = _load()
    sp = _params(p)
    return float(lib.syn_ripple_phase(ctypes.byref(sp)))


# --------------------------------------------------------------------------------------------
# Cameras.  A camera is a dict {type: 0 ortho | 1 perspective, eye, right, up, fwd, win=(l,r,b,t),
# width, height}.  Pixel (px, py), py = 0 the top row, maps to window coordinates
# u = l + (px + 1/2)(r - l)/width, v = t - (py + 1/2)(t - b)/height.
# --------------------------------------------------------------------------------------------

def _rx(deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _ry(deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _cam(t, eye, right, up, fwd, win, w, h) -> dict:
    return dict(type=int(t), eye=[float(v) for v in eye], right=[float(v) for v in right],
                up=[float(v) for v in up], fwd=[float(v) for v in fwd],
                win=[float(v) for v in win], width=int(w), height=int(h))


def _centre_radius(dims):
    nx, ny, nz = dims
    c = np.array([nx / 2.0, ny / 2.0, nz / 2.0])
    return c, 0.5 * math.sqrt(nx * nx + ny * ny + nz * nz)


def ortho_view(dims, width=512, height=512, rx_deg=20.0, ry_deg=30.0) -> dict:
    """Orthographic view: canonical basis (right +x, up +y, forward +z) rotated by
    Rx(rx) Ry(ry); square window = bounding-sphere diameter; image plane 2R before
    the cube centre (R = half-diagonal)."""
    c, r = _centre_radius(dims)
    m = _rx(rx_deg) @ _ry(ry_deg)
    right, up, fwd = m[:, 0], m[:, 1], m[:, 2]
    eye = c - 2.0 * r * fwd
    aspect = width / height
    return _cam(0, eye, right, up, fwd, (-r * aspect, r * aspect, -r, r), width, height)


def look_at(dims, fwd, width, height, fov_deg=60.0, dist_factor=2.0, up_hint=(0.0, 1.0, 0.0)):
    c, r = _centre_radius(dims)
    f = np.asarray(fwd, dtype=np.float64)
    f = f / np.linalg.norm(f)
    u0 = np.asarray(up_hint, dtype=np.float64)
    if abs(float(np.dot(u0, f))) > 0.99:
        u0 = np.array([1.0, 0.0, 0.0])
    right = np.cross(u0, f)
    right /= np.linalg.norm(right)
    up = np.cross(f, right)
    eye = c - dist_factor * r * f
    t = math.tan(math.radians(fov_deg) / 2.0)
    a = width / height
    return _cam(1, eye, right, up, f, (-t * a, t * a, -t, t), width, height)


def orbit_view(dims, az_deg, width=1920, height=1080, fov_deg=60.0) -> dict:
    """Perspective orbit about the Dec (y) axis: eye at 2R from the centre, vertical
    field of view 60 deg, azimuth 0 looking along +z (the spectral axis)."""
    a = math.radians(az_deg)
    return look_at(dims, (math.sin(a), 0.0, math.cos(a)), width, height, fov_deg)


def orbit(dims, frames, step_deg=10.0, width=1920, height=1080):
    return [orbit_view(dims, i * step_deg, width, height) for i in range(frames)]


def wall_views(cam: dict, cols=5, rows=5) -> list[dict]:
    """Split one camera into cols x rows off-axis sub-frusta.  Panel (c, r) (r = 0 the top
    row) covers global pixels [c W, (c+1) W) x [r H, (r+1) H) of the full camera, where
    W, H are the panel sizes; bezels are ignored."""
    l, r_, b, t = cam["win"]
    W, H = cam["width"] // cols, cam["height"] // rows
    assert W * cols == cam["width"] and H * rows == cam["height"]
    out = []
    for rr in range(rows):
        for cc in range(cols):
            win = (l + (r_ - l) * cc / cols, l + (r_ - l) * (cc + 1) / cols,
                   t - (t - b) * (rr + 1) / rows, t - (t - b) * rr / rows)
            out.append(_cam(cam["type"], cam["eye"], cam["right"], cam["up"], cam["fwd"], win, W, H))
    return out


def random_views(dims, n, seed, width=512, height=512):
    """n perspective views from seeded directions uniform on the sphere (2R, 60 deg)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        out.append(look_at(dims, v, width, height))
    return out


def axis_view(dims, width, height, plane_offset=0.0) -> dict:
    """Orthographic view straight down +z with pixel centres on voxel centres
    (pixel (px, py) looks down column x = px + 1/2, y = ny - 1/2 - py); the image
    plane is at z = plane_offset."""
    nx, ny, nz = dims
    return _cam(0, (0.0, 0.0, plane_offset), (1, 0, 0), (0, 1, 0), (0, 0, 1),
                (0.0, float(width), float(ny - height), float(ny)), width, height)


# --------------------------------------------------------------------------------------------
# Transfer functions: n x 4 float32 straight (non-premultiplied) RGBA tables.
# --------------------------------------------------------------------------------------------

_VIRIDIS_ANCHORS = np.array([[0.267, 0.005, 0.329], [0.229, 0.322, 0.546], [0.128, 0.567, 0.551],
                             [0.369, 0.789, 0.383], [0.993, 0.906, 0.144]])


def viridis_ramp_tf(n=256) -> np.ndarray:
    """Linear alpha ramp alpha_i = i/(n-1) with viridis-like colours (dark purple ->
    teal -> yellow), piecewise linear between five anchors."""
    x = np.linspace(0.0, 1.0, n)
    xa = np.linspace(0.0, 1.0, len(_VIRIDIS_ANCHORS))
    rgb = np.stack([np.interp(x, xa, _VIRIDIS_ANCHORS[:, c]) for c in range(3)], axis=1)
    return np.concatenate([rgb, x[:, None]], axis=1).astype(np.float32)


def hidden_tf(seed, n=256) -> np.ndarray:
    """Seeded smooth RGBA table (used as the unknown target table of the gradient workload)."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, n)
    knots = np.linspace(0.0, 1.0, 9)
    rgb = np.stack([np.interp(x, knots, rng.uniform(0.05, 0.95, size=9)) for _ in range(3)], 1)
    gamma = rng.uniform(0.7, 1.6)
    alpha = 0.9 * x ** gamma
    return np.concatenate([rgb, alpha[:, None]], axis=1).astype(np.float32)
