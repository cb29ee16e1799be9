"""CUDA-graph mode and launch-shape tuning change how the work is launched, never the
result: images must be bitwise identical to the direct, default-shape renders."""
import json

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def scene():
    import paper_1012_2909_gb300 as vr
    dims = (96, 80, 112)
    vol = synth.generate(synth.cube_params(*dims, seed=12, nsrc=10, ripple=True, ripple_period=40.0))
    r = vr.Renderer(0, brick=32)
    r.load_cube(vol, "f16")
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    yield vr, r, dims
    r.close()


def _render(r, mode):
    out = r.render(mode)
    torch.cuda.synchronize()
    return out.clone()


@pytest.mark.parametrize("mode,path", [("composite", "ray"), ("mip", "ray"), ("mip", "brick")])
def test_graph_mode_is_bitwise_identical(scene, mode, path):
    vr, r, dims = scene
    r.set_path(path)
    for step, az in enumerate((10.0, 55.0, 120.0)):  # camera changes go through graph updates
        cams = synth.wall_views(synth.orbit_view(dims, az, 5 * 16, 5 * 12), 5, 5) if step == 2 else \
            [synth.orbit_view(dims, az, 64, 48), synth.orbit_view(dims, az + 5.0, 64, 48)]
        r.set_camera(cams)
        vr.vr_set_graph(r.ctx, False)
        ref = _render(r, mode)
        vr.vr_set_graph(r.ctx, True)
        got = _render(r, mode)
        got2 = _render(r, mode)  # replay of the same graph
        vr.vr_set_graph(r.ctx, False)
        assert torch.equal(got, ref) and torch.equal(got2, ref)
    r.set_path("auto")


def test_every_tuning_gives_the_same_image(scene):
    vr, r, dims = scene
    r.set_camera([synth.orbit_view(dims, 33.0, 70, 50), synth.orbit_view(dims, 200.0, 70, 50)])
    default = vr.vr_get_tuning(r.ctx)
    for mode, path in (("composite", "ray"), ("mip", "ray"), ("mip", "brick")):
        r.set_path(path)
        ref = _render(r, mode)
        for tw, th in ((8, 4), (4, 8), (16, 2), (2, 16), (32, 1)):
            for block in (64, 128, 256):
                for group in (4, 8, 16):
                    if path == "ray" and group != 8:
                        continue
                    if path == "brick" and (tw, th, block) != (8, 4, 128):
                        continue
                    vr.vr_set_tuning(r.ctx, dict(tile_w=tw, tile_h=th, block=block, group=group))
                    assert torch.equal(_render(r, mode), ref), (mode, path, tw, th, block, group)
    vr.vr_set_tuning(r.ctx, default)
    with pytest.raises(vr.VrError) as e:
        vr.vr_set_tuning(r.ctx, dict(tile_w=8, tile_h=8, block=128, group=8))
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    r.set_path("auto")


def test_autotune_and_cache(scene, tmp_path):
    vr, r, dims = scene
    r.set_camera(synth.wall_views(synth.orbit_view(dims, 70.0, 5 * 32, 5 * 18), 5, 5))
    cache = str(tmp_path / "tune.json")
    for mode in ("composite", "mip"):
        ref = _render(r, mode)
        t = vr.autotune(r, mode, reps=2, cache=cache)
        assert not t["cached"] and t["ms"] > 0
        assert torch.equal(_render(r, mode), ref)
        t2 = vr.autotune(r, mode, reps=2, cache=cache)
        assert t2["cached"]
    assert len(json.load(open(cache))) == 2
