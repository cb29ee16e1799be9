"""The C ABI library loads and exports every symbol include/*.h declares; host-side
argument checks answer without a GPU (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(vr_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1012_2909_gb300 import _build
    _build.build()
    import paper_1012_2909_gb300 as vr
    return vr.load_library()


def test_every_declared_symbol_is_exported(lib):
    import paper_1012_2909_gb300 as vr
    names = _declared()
    assert names, "no declarations found"
    for n in sorted(names):
        assert hasattr(lib, n), f"libvr.so does not export {n}"
    # and the Python binding marshals every one of them under the same name
    assert names == set(vr.SIGNATURES), names ^ set(vr.SIGNATURES)


def test_host_side_checks(lib):
    import paper_1012_2909_gb300 as vr
    assert lib.vr_status_string(vr.VR_ERR_STATE) == b"VR_ERR_STATE"
    o = vr.vr_options()
    lib.vr_default_options(ctypes.byref(o))
    assert (o.brick, o.step, o.ert) == (128, 0.5, 0.99)
    h = ctypes.c_void_p()
    assert lib.vr_create(None, 0, None) == vr.VR_ERR_INVALID_ARG
    bad = vr.vr_options(brick=100, step=0.5, ert=0.99)
    assert lib.vr_create(ctypes.byref(h), 0, ctypes.byref(bad)) == vr.VR_ERR_INVALID_ARG
    assert lib.vr_set_camera(None, None, 1) == vr.VR_ERR_INVALID_ARG
    assert lib.vr_render(None, 0, None, None, None) == vr.VR_ERR_INVALID_ARG
    assert lib.vr_destroy(None) == vr.VR_OK
    assert lib.vr_last_error(None) == b"no context"


def test_abi_struct_layouts():
    """The ctypes mirrors match the C declarations' sizes (all fields 8-byte aligned)."""
    import paper_1012_2909_gb300 as vr
    assert ctypes.sizeof(vr.vr_camera) == 8 + 12 * 8 + 4 * 8 + 8
    assert ctypes.sizeof(vr.vr_options) == 24
    assert ctypes.sizeof(vr.vr_cube_info) == 3 * 8 + 6 * 4 + 2 * 8
    assert vr.FOOTPRINT.itemsize == 6 * 4 + 8  # vr_footprint


def test_pyramid_layout_matches_the_oracle():
    """vr_pyramid_layout is host arithmetic: level count and buffer size for every layout."""
    import numpy as np
    import oracle
    import paper_1012_2909_gb300 as vr
    for w, h in ((1, 1), (7, 1), (1, 5), (5, 3), (64, 64), (100, 37), (1000, 999)):
        for tile in (0, 8, 64):
            levels, packed = oracle.pyramid(np.zeros((h, w, 4), np.float32), tile)
            assert vr.vr_pyramid_layout(w, h, tile) == (levels, packed.size)
    assert vr.vr_pyramid_layout(1 << 20, 3, 0)[0] == 21  # the largest side accepted
    for bad in ((0, 5, 0), (5, 0, 0), (4, 4, 12), (4, 4, 4), (4, 4, 8192), ((1 << 20) + 1, 4, 0)):
        with pytest.raises(vr.VrError):
            vr.vr_pyramid_layout(*bad)


def _code(path):
    """Source text without comments."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def test_device_code_keeps_fp64_to_the_table_gradient_reduction():
    """The render and adjoint kernels compute in FP32 and float-float pairs: `double`
    appears in no device source except the body of the final table-gradient reduction
    (k_tfgrad_reduce) and the catalogue overlay, which is off the render path and follows
    the oracle's double-precision projection.  vr_api.cu and the host structs of
    vr_internal.cuh are host code."""
    csrc = os.path.join(ROOT, "paper_1012_2909_gb300", "csrc")
    host_or_exempt = {"vr_api.cu", "vr_overlay.cu", "vr_internal.cuh"}
    for path in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        name = os.path.basename(path)
        if name in host_or_exempt:
            continue
        code = _code(path)
        if name == "vr_adjoint.cu":
            start = code.index("k_tfgrad_reduce(")
            body_end = code.index("\n}", start)
            assert re.search(r"\bdouble\b", code[start:body_end])
            code = code[:start] + code[body_end:]
        assert not re.search(r"\bdouble\b", code), name
