"""Object-space sort-last through the C ABI on one GPU, its ranks played by brick
partitions of one context (the exchange runs in memory with dist.Loopback): each
partition renders its partials with vr_sortlast_partials, the rows go to the band
owners, and each owner folds its band with vr_sortlast_fold.  The stitched bands equal
the single-device sort-last render bit for bit (same partial values, same per-pixel
order) and the oracle within the FP32 tolerance; MIP folds by maximum."""
import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _virtual_ranks(vr, r, mode, world, H, W):
    from paper_1012_2909_gb300 import dist
    info = vr.vr_get_cube_info(r.ctx)
    parts = dist.partition_bricks((info["nbx"], info["nby"], info["nbz"]), world)
    outgoing = []
    for rank in range(world):
        foot, need = vr.vr_sortlast_partials(r.ctx, mode, parts[rank])
        partial = torch.empty((max(need, 1), 4), device="cuda")
        foot, _ = vr.vr_sortlast_partials(r.ctx, mode, parts[rank], partial)
        torch.cuda.synchronize()
        outgoing.append([dist.pack(foot, partial, *dist.band_rows(H, world, d)) for d in range(world)])
    incoming = dist.Loopback(world).alltoall_all(outgoing)
    img = torch.empty((H, W, 4), device="cuda")
    for d in range(world):
        y0, y1 = dist.band_rows(H, world, d)
        rfoot, rpay = dist.unpack(incoming[d])
        band = torch.empty((y1 - y0, W, 4), device="cuda")
        vr.vr_sortlast_fold(r.ctx, mode, rpay.cuda(), rfoot, y0, y1, band)
        img[y0:y1] = band
    torch.cuda.synchronize()
    return img


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_virtual_ranks_equal_sortlast_and_oracle(storage):
    import paper_1012_2909_gb300 as vr
    dims, brick = (96, 80, 72), 32
    vol = synth.generate(synth.cube_params(*dims, seed=44, nsrc=8, ripple=True, ripple_period=32.0))
    tf = synth.viridis_ramp_tf()
    r = vr.Renderer(0, brick=brick)
    r.load_cube(vol, storage)
    r.set_transfer_function(tf, -1.0, 20.0)
    sc = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 2.0)
    for cam in (synth.orbit_view(dims, 33.0, 57, 43), synth.ortho_view(dims, 57, 43, rx_deg=-25.0, ry_deg=70.0),
                synth.look_at(dims, (0.1, -0.4, 1.0), 57, 43, dist_factor=0.3)):
        r.set_camera(cam)
        r.set_path("sortlast")
        ref = r.render("composite").clone()
        for world in (1, 2, 3, 5):
            img = _virtual_ranks(vr, r, "composite", world, cam["height"], cam["width"])
            assert torch.equal(img, ref[0]), world
        compare(img.cpu().numpy().reshape(-1, 4), sc, cam, "composite", tol=1e-4, path="sortlast")
        img = _virtual_ranks(vr, r, "mip", 3, cam["height"], cam["width"])
        compare(img.cpu().numpy().reshape(-1, 4), sc, cam, "mip", tol=1e-4, path="sortlast")
    r.close()


def test_partials_argument_checks():
    import paper_1012_2909_gb300 as vr
    dims = (40, 36, 48)
    vol = synth.generate(synth.cube_params(*dims, seed=3, nsrc=3))
    r = vr.Renderer(0, brick=16)
    r.load_cube(vol, "f32")
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    with pytest.raises(vr.VrError) as e:  # no camera yet
        vr.vr_sortlast_partials(r.ctx, "composite", [0])
    assert e.value.status == vr.VR_ERR_STATE
    r.set_camera(synth.orbit_view(dims, 10.0, 32, 24))
    for bad in ([-1], [0, 0], [10 ** 6]):
        with pytest.raises(vr.VrError) as e:
            vr.vr_sortlast_partials(r.ctx, "composite", bad)
        assert e.value.status == vr.VR_ERR_INVALID_ARG
    foot, need = vr.vr_sortlast_partials(r.ctx, "composite", [0, 1, 2])
    assert need > 0 and list(foot["brick"]) == [0, 1, 2]
    small = torch.empty((max(need - 1, 1), 4), device="cuda")
    with pytest.raises(vr.VrError) as e:
        vr.vr_sortlast_partials(r.ctx, "composite", [0, 1, 2], small)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    out = torch.empty((24, 32, 4), device="cuda")
    with pytest.raises(vr.VrError) as e:  # a footprint beyond the buffer
        vr.vr_sortlast_fold(r.ctx, "composite", small, foot, 0, 24, out)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    with pytest.raises(vr.VrError) as e:  # bad rows
        vr.vr_sortlast_fold(r.ctx, "composite", small, foot[:0], 5, 5, out)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    vr.vr_sortlast_fold(r.ctx, "composite", None, foot[:0], 0, 24, out)  # nothing to fold
    torch.cuda.synchronize()
    assert torch.count_nonzero(out) == 0
    r.close()
