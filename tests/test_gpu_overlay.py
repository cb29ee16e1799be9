"""Catalogue overlay (wireframe bounding cubes over a render) against the oracle, through
the C ABI.  The drawn pixels come from double-precision arithmetic with one rounding per
operation in the same order on both sides, and every box has its own random colour, so
a pixel decided differently shows as a colour error far above the tolerance; the
tolerance (2e-6) only covers the FP32 blend against the FP64 one."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vr():
    import paper_1012_2909_gb300 as vr
    return vr


def _cam(type_, eye, fwd, right=(1, 0, 0), up=(0, 1, 0), win=(-0.5, 0.5, -0.5, 0.5), w=1, h=1):
    return dict(type=type_, eye=list(eye), right=list(right), up=list(up), fwd=list(fwd), win=list(win),
                width=w, height=h)


def _compare(vr, r, img, cams, boxes, colours):
    """GPU overlay of img (ncams, H, W, 4) against the oracle, camera by camera."""
    gpu = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    r.overlay(gpu, boxes, colours, cams=cams)
    got = gpu.cpu().numpy().astype(np.float64)
    drawn = 0
    for i, c in enumerate(cams):
        want, key = oracle.overlay(img[i].astype(np.float32).astype(np.float64), c, boxes, colours)
        err = float(np.abs(got[i] - want).max())
        assert err <= 2e-6, (i, err)
        drawn += int(np.count_nonzero(key))
    return drawn


def test_closed_form_scenes(vr):
    r = vr.Renderer(0)
    rng = np.random.default_rng(11)
    ortho = _cam(0, (0, 0, -10), (0, 0, 1), win=(0, 64, 0, 32), w=64, h=32)
    boxes = np.array([[10.5, 5.5, 1.0, 20.5, 9.5, 3.0], [2.5, 2.5, 0, 12.5, 12.5, 1],
                      [8.5, 4.5, 0, 30.5, 10.5, 1], [50.5, 20.5, 0, 80.5, 40.5, 1]])
    cols = rng.random((4, 4)).astype(np.float32)
    img = rng.random((1, 32, 64, 4))
    assert _compare(vr, r, img, [ortho], boxes, cols) > 0
    persp = _cam(1, (0, 0, -40), (0, 0, 1), win=(-1, 1, -1, 1), w=96, h=96)
    assert _compare(vr, r, rng.random((1, 96, 96, 4)), [persp], np.array([[3.0, -5.0, 2.0, 11.0, 4.0, 9.0]]),
                    cols[:1]) > 0
    # a box straddling the eye plane (near clipping) and one behind the eye
    inside = _cam(1, (0, 0, 0), (0, 0, 1), win=(-1, 1, -1, 1), w=48, h=48)
    _compare(vr, r, rng.random((1, 48, 48, 4)), [inside],
             np.array([[-2.0, -1.0, -5.0, 3.0, 2.0, 6.0], [-2, -2, -9, 2, 2, -3]]), cols[:2])
    # no boxes: the image is unchanged
    _compare(vr, r, img, [ortho], np.zeros((0, 6)), np.zeros((0, 4), np.float32))
    r.close()


def test_survey_render_with_its_catalogue(vr):
    cfg = synth.CONFIGS["survey"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    r = vr.Renderer(0)
    r.load_cube(synth.generate(p), "f16")
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    boxes = synth.catalogue(p)
    cols = np.random.default_rng(2000).random((len(boxes), 4)).astype(np.float32)
    for az in (0.0, 130.0):
        cam = synth.orbit_view(dims, az)
        r.set_camera(cam)
        img = r.render("composite").cpu().numpy()
        assert _compare(vr, r, img, [cam], boxes, cols) > 10_000
    r.close()


def test_orthographic_and_wall_panels(vr):
    cfg = synth.CONFIGS["small"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    r = vr.Renderer(0)
    r.load_cube(synth.generate(p), "f32")
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    boxes = synth.catalogue(p)
    cols = np.random.default_rng(20).random((len(boxes), 4)).astype(np.float32)
    ortho = synth.ortho_view(dims, 512, 512)
    r.set_camera(ortho)
    assert _compare(vr, r, r.render("mip").cpu().numpy(), [ortho], boxes, cols) > 500
    panels = synth.wall_views(synth.orbit_view(dims, 30.0, 5 * 96, 5 * 54), 5, 5)
    r.set_camera(panels)
    assert _compare(vr, r, r.render("composite").cpu().numpy(), panels, boxes, cols) > 500
    r.close()


def test_bad_arguments(vr):
    r = vr.Renderer(0)
    c = _cam(0, (0, 0, -10), (0, 0, 1), win=(0, 8, 0, 8), w=8, h=8)
    flat = torch.zeros(8 * 8 * 4 + 1, device="cuda")
    box, col = np.array([[1, 1, 1, 5, 5, 5.0]]), np.ones((1, 4), np.float32)
    with pytest.raises(vr.VrError) as e:  # 4-byte offset: not 16-byte aligned
        r.overlay(flat[1:].view(1, 8, 8, 4), box, col, cams=[c])
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    c2 = dict(c, width=16)
    with pytest.raises(vr.VrError) as e:
        r.overlay(torch.zeros((2, 8, 8, 4), device="cuda"), box, col, cams=[c, c2])
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    img = torch.zeros((1, 8, 8, 4), device="cuda")
    with pytest.raises(vr.VrError) as e:  # a non-finite box is refused, the image is untouched
        r.overlay(img, np.array([[1, 1, 1, np.nan, 5, 5.0]]), col, cams=[c])
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    with pytest.raises(vr.VrError) as e:
        r.overlay(img, box, col, cams=[dict(c, eye=[0.0, np.inf, -10.0])])
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert not img.any()
    r.close()
