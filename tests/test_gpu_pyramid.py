"""Image pyramid of a render against the oracle, through the C ABI.

Tolerance: a level averages at most four FP32 values of the level before it (three
roundings of a sum of values in [0, 1], then an exact scaling), so every level adds at
most 3 * 2^-24 * 4 / 4 < 2.5e-7 of absolute error; the test allows 2.5e-7 per level."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def r():
    import paper_1012_2909_gb300 as vr
    rr = vr.Renderer(0)
    yield rr
    rr.close()


def _check(r, img, tile):
    levels, want = oracle.pyramid(img, tile)
    got = r.pyramid(torch.from_numpy(img).cuda(), tile).cpu().numpy().astype(np.float64)
    assert got.size == want.size
    if want.size:
        err = float(np.abs(got - want).max())
        assert err <= 2.5e-7 * levels, (img.shape, tile, err)
    return levels


@pytest.mark.parametrize("tile", [0, 8, 64])
def test_random_images_odd_and_degenerate_sizes(r, tile):
    rng = np.random.default_rng(tile + 1)
    for w, h in ((1, 1), (7, 1), (1, 5), (5, 3), (33, 32), (64, 64), (100, 37), (257, 129), (1000, 999)):
        _check(r, rng.random((h, w, 4)).astype(np.float32), tile)


def test_pyramid_of_a_render(r):
    cfg = synth.CONFIGS["small"]
    p = cfg["cube"]
    vol = synth.generate(p)
    import paper_1012_2909_gb300 as vr
    rr = vr.Renderer(0)
    rr.load_cube(vol, "f32")
    rr.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    rr.set_camera(synth.ortho_view((p["nx"], p["ny"], p["nz"]), 512, 512))
    img = rr.render("composite")[0]
    for tile in (0, 256):
        levels, want = oracle.pyramid(img.cpu().numpy(), tile)
        got = rr.pyramid(img, tile).cpu().numpy()
        assert levels == 10 and float(np.abs(got - want).max()) <= 2.5e-7 * levels
    rr.close()


def test_full_size_8000_squared(r):
    """The size of the paper-scale static render: 8000 x 8000, row-major and 256-tiled."""
    g = torch.Generator(device="cuda").manual_seed(8000)
    img = torch.rand((8000, 8000, 4), device="cuda", generator=g)
    host = img.cpu().numpy()
    for tile in (0, 256):
        levels, want = oracle.pyramid(host, tile)
        got = r.pyramid(img, tile).cpu().numpy()
        assert levels == 14 and got.size == want.size
        assert float(np.abs(got.astype(np.float64) - want).max()) <= 2.5e-7 * levels


def test_bad_arguments(r):
    import paper_1012_2909_gb300 as vr
    img = torch.zeros((8, 8, 4), device="cuda")
    out = torch.zeros(1024, device="cuda")
    with pytest.raises(vr.VrError) as e:
        vr.vr_image_pyramid(r.ctx, img, out, tile=12)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    flat = torch.zeros(8 * 8 * 4 + 1, device="cuda")
    with pytest.raises(vr.VrError) as e:  # 4-byte offset: not 16-byte aligned
        vr.vr_image_pyramid(r.ctx, flat[1:].view(8, 8, 4), out)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
