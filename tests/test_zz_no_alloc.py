"""vr_render_mip_noalloc: the MIP render for callers that cannot allocate device memory
while they render (real-time loops that must not meet cudaMalloc's implicit
synchronisation, programs whose device memory belongs to another allocator).
It must give the same images as vr_render's brick path, call after call, although every
call reuses one fixed scratch array inside the library.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4  # the FP32-voxel RGBA tolerance the parity tests use


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_vr_render_on_consecutive_calls():
    import paper_1012_2909_gb300 as vr

    lib = vr.load_library()
    dims = (150, 130, 260)
    vol = synth.generate(synth.cube_params(*dims, seed=404, nsrc=12, ripple=True,
                                           ripple_period=64.0))
    r = vr.Renderer(0, brick=64)
    r.load_cube(vol, "f16")
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    r.set_path("brick")
    stream = torch.cuda.current_stream()
    # two calls in a row with different views and sizes; the second one with and
    # without out_max (then the running maxima live in the library's array)
    views = [synth.orbit_view(dims, 25.0, 320, 200), synth.orbit_view(dims, 160.0, 256, 256)]
    for cam in views:
        r.set_camera(cam)
        ref, ref_max = r.render("mip", with_max=True)
        torch.cuda.synchronize()
        for with_max in (True, False):
            out = torch.full_like(ref, float("nan"))
            mx = torch.full_like(ref_max, float("nan")) if with_max else None
            st = lib.vr_render_mip_noalloc(r.ctx, _ptr(out), _ptr(mx),
                                           ctypes.c_void_p(stream.cuda_stream))
            assert st == vr.VR_OK, lib.vr_last_error(r.ctx)
            torch.cuda.synchronize()
            err = (out - ref).abs().max().item()
            assert err <= TOL, err
            if with_max:
                hit = torch.isfinite(ref_max)
                assert torch.equal(torch.isfinite(mx), hit)
                assert (mx[hit] - ref_max[hit]).abs().max().item() <= TOL * 10
        # and the last call's image against the FP64 oracle on the same stored (FP16) values
        from parity import compare
        import oracle
        sc = oracle.Scene(oracle.round_storage(vol, "f16"), synth.viridis_ramp_tf(), -1.0, 20.0, 0.5, 0.99)
        compare(out[0].cpu().numpy().reshape(-1, 4), sc, cam, "mip", tol=TOL, path="brick")
    r.close()


def test_noalloc_rejects_images_above_its_limit():
    import paper_1012_2909_gb300 as vr

    lib = vr.load_library()
    dims = (64, 64, 64)
    r = vr.Renderer(0, brick=32)
    r.load_cube(np.zeros(dims, np.float32), "f32")
    r.set_transfer_function(synth.viridis_ramp_tf(), 0.0, 1.0)
    w, h = 2049, 1025  # 2,100,225 pixels > VR_NOALLOC_MAX_PIXELS = 2,097,152
    assert w * h > vr.VR_NOALLOC_MAX_PIXELS
    r.set_camera(synth.orbit_view(dims, 0.0, w, h))
    out = torch.empty((1, h, w, 4), device="cuda")
    st = lib.vr_render_mip_noalloc(r.ctx, _ptr(out), None,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == vr.VR_ERR_INVALID_ARG
    assert b"VR_NOALLOC_MAX_PIXELS" in lib.vr_last_error(r.ctx)
    r.close()
