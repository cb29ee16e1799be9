"""Out-of-core rendering: bricks pulled from a region callback through a small HBM cache.

Parity: the streamed images equal the FP64 oracle (composite with termination, MIP) and
the in-core renders of the same cube.  Failure handling is exercised on the host: a
callback that fails gives VR_ERR_IO, one that overruns the deadline VR_ERR_TIMEOUT, and
the context keeps working afterwards."""
import ctypes
import time

import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = (150, 130, 170)  # 5 x 5 x 6 bricks of 32


@pytest.fixture(scope="module")
def cube():
    p = synth.cube_params(*DIMS, seed=909, nsrc=14, ripple=True, ripple_period=40.0)
    return p, synth.generate(p)


def _streamed(vr, p, storage, cache_bricks, brick=32):
    r = vr.Renderer(0, brick=brick)
    fn, user = synth.region_callback(p, nthreads=4)
    slot = (brick + 2) * (brick + 2) * ((brick + 2 + 7) // 8 * 8) * (4 if storage == "f32" else 2)
    vr.vr_load_cube_streamed(r.ctx, fn, user, DIMS, storage, cache_bytes=cache_bricks * (slot + 256))
    r._keep = (fn, user)
    return r


@pytest.mark.parametrize("storage", ["f16", "bf16", "f32"])
def test_streamed_equals_oracle_and_in_core(cube, storage):
    import paper_1012_2909_gb300 as vr
    p, vol = cube
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view(DIMS, az, 61, 45) for az in (15.0, 200.0)]
    sc = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 0.99)
    rs = _streamed(vr, p, storage, cache_bricks=9)
    rs.set_transfer_function(tf, -1.0, 20.0)
    rs.set_camera(cams)
    ri = vr.Renderer(0, brick=32)
    ri.load_cube(vol, storage)
    ri.set_transfer_function(tf, -1.0, 20.0)
    ri.set_camera(cams)
    for mode, path in (("composite", "layered"), ("mip", "brick")):
        out, mx = rs.render(mode, with_max=True)
        ri.set_path(path)
        ref, rmx = ri.render(mode, with_max=True)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        for i, c in enumerate(cams):
            compare(out[i].cpu().numpy().reshape(-1, 4), sc, c, mode, tol=1e-4,
                    gpu_max=mx[i].cpu().numpy() if mode == "mip" else None, max_tol=2e-3, path=path)
    st = vr.vr_get_stream_stats(rs.ctx)
    print(st)
    assert st["bricks_fetched"] > 9 and st["batches"] > 1 and st["bytes_h2d"] > 0
    assert st["bricks_culled"] > 0  # the composite never fetched bricks behind terminated rays
    rs.close()
    ri.close()


def test_callback_failure_and_deadline(cube):
    import paper_1012_2909_gb300 as vr
    p, vol = cube
    state = {"fail": False, "sleep": 0.0}

    def region(user, x0, y0, z0, sx, sy, sz, dst):
        if state["fail"]:
            return 7
        if state["sleep"]:
            time.sleep(state["sleep"])
        out = np.ctypeslib.as_array(ctypes.cast(dst, ctypes.POINTER(ctypes.c_float)), shape=(sz * sy * sx,))
        out[:] = synth.generate(p, region=(x0, y0, z0, sx, sy, sz), nthreads=2).reshape(-1)
        return 0

    cb = vr.REGION_FN(region)
    r = vr.Renderer(0, brick=32)
    vr.vr_load_cube_streamed(r.ctx, cb, None, DIMS, "f16", cache_bytes=12 * (34 * 34 * 40 * 2 + 256))
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    r.set_camera(synth.orbit_view(DIMS, 40.0, 40, 30))
    good = r.render("mip").clone()
    torch.cuda.synchronize()
    r.set_camera(synth.orbit_view(DIMS, 130.0, 40, 30))  # needs bricks not yet cached
    state["fail"] = True
    with pytest.raises(vr.VrError) as e:
        r.render("mip")
    assert e.value.status == vr.VR_ERR_IO
    state["fail"] = False
    state["sleep"] = 0.3
    vr.vr_set_stream_timeout(r.ctx, 0.1)
    with pytest.raises(vr.VrError) as e:
        r.render("composite")
    assert e.value.status == vr.VR_ERR_TIMEOUT
    # recovery: normal deadline, same images as a fresh context
    state["sleep"] = 0.0
    vr.vr_set_stream_timeout(r.ctx, 60.0)
    r.set_camera(synth.orbit_view(DIMS, 40.0, 40, 30))
    again = r.render("mip")
    torch.cuda.synchronize()
    assert torch.equal(again, good)
    r.close()


def test_cache_smaller_than_a_brick_is_rejected(cube):
    import paper_1012_2909_gb300 as vr
    p, _ = cube
    r = vr.Renderer(0, brick=32)
    fn, user = synth.region_callback(p)
    with pytest.raises(vr.VrError) as e:
        vr.vr_load_cube_streamed(r.ctx, fn, user, DIMS, "f16", cache_bytes=1000)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    r.close()


def test_cache_beyond_device_memory_is_out_of_memory(cube):
    """A brick cache that cannot be allocated (a 32768^3 cube with a 1 PB budget) answers
    VR_ERR_OOM without calling the region callback, and the same context then loads and
    renders a cube correctly."""
    import paper_1012_2909_gb300 as vr
    p, vol = cube
    r = vr.Renderer(0, brick=32)
    calls = []

    @vr.REGION_FN
    def never(user, x0, y0, z0, sx, sy, sz, out):
        calls.append(1)
        return 1

    with pytest.raises(vr.VrError) as e:
        vr.vr_load_cube_streamed(r.ctx, never, None, (1 << 15, 1 << 15, 1 << 15), "f16", cache_bytes=1 << 50)
    assert e.value.status == vr.VR_ERR_OOM
    assert not calls
    tf = synth.viridis_ramp_tf()
    cam = synth.orbit_view(DIMS, 75.0, 48, 36)
    r.load_cube(vol, "f16")
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cam)
    img = r.render("composite")
    torch.cuda.synchronize()
    sc = oracle.Scene(oracle.round_storage(vol, "f16"), tf, -1.0, 20.0, 0.5, 0.99)
    compare(img[0].cpu().numpy().reshape(-1, 4), sc, cam, "composite", tol=1e-4)
    r.close()
