"""Failure detection on the GPU without a fault.  A bounded device wait is made to expire
on purpose (vr_selftest_wait_timeout: a barrier phase that no copy completes, with no copy
in flight, waited on with the brick pass's own bounded wait).  The next render must report
VR_ERR_INTERNAL once, and the context must go on rendering correctly."""
import time

import pytest

import oracle
import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_expired_wait_is_reported_once_and_the_context_recovers():
    import paper_1012_2909_gb300 as vr

    dims = (40, 36, 48)
    vol = synth.generate(synth.cube_params(*dims, seed=12, nsrc=5))
    tf = synth.viridis_ramp_tf()
    cam = synth.orbit_view(dims, 50.0, 40, 30)
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    r = vr.Renderer(0, brick=32)
    r.load_cube(vol, "f32")
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cam)
    r.set_path("brick")
    for render in (lambda: r.render("mip"),
                   lambda: vr.vr_render_mip_noalloc(r.ctx, torch.empty((1, 30, 40, 4), device="cuda"))):
        t0 = time.perf_counter()
        vr.vr_selftest_wait_timeout(r.ctx)
        assert time.perf_counter() - t0 < 60.0  # the wait is bounded
        with pytest.raises(vr.VrError) as e:
            render()
        assert e.value.status == vr.VR_ERR_INTERNAL
        # reported once: the same context renders again, and correctly
        img = r.render("mip")
        torch.cuda.synchronize()
        compare(img[0].cpu().numpy().reshape(-1, 4), sc, cam, "mip", tol=1e-4)
    r.close()
