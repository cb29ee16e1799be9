"""GPU renderer vs the FP64 oracle, element by element, through the C ABI.

Tolerances (max abs RGBA error per pixel): 1e-4 for FP32 voxels; for FP16 / BF16
storage the kernel is held to the same 1e-4 against the oracle run on the rounded
cube, and to 2e-3 against the oracle on the FP32 source where the storage error
allows it (FP16).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vr():
    import paper_1012_2909_gb300 as vr
    return vr


def _render(vr, vol, tf, cams, mode, storage="f32", brick=128, step=0.5, ert=0.99, vmin=-1.0,
            vmax=20.0, path="auto"):
    r = vr.Renderer(0, brick=brick, step=step, ert=ert)
    r.set_path(path)
    r.load_cube(vol, storage)
    r.set_transfer_function(tf, vmin, vmax)
    r.set_camera(cams)
    out, mx = r.render(mode, with_max=True)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), mx.cpu().numpy()
    r.close()
    return res


def test_small_workload_full_image(vr):
    """128^3 float32 noise + 20 sources, ortho 512^2 rotated 30/20 deg, step 0.5, ERT 0.99."""
    cfg = synth.CONFIGS["small"]
    vol = synth.generate(cfg["cube"])
    tf = synth.viridis_ramp_tf()
    cam = synth.ortho_view((128, 128, 128), 512, 512)
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    for mode in ("composite", "mip"):
        img, mx = _render(vr, vol, tf, [cam], mode)
        st = compare(img[0].reshape(-1, 4), sc, cam, mode, tol=1e-4,
                     gpu_max=mx[0] if mode == "mip" else None, max_tol=2e-3)
        print(mode, st)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_precision_storage(vr, storage):
    p = synth.cube_params(96, 80, 72, seed=77, nsrc=12, ripple=True, ripple_period=32.0)
    vol = synth.generate(p)
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view((96, 80, 72), az, 64, 48) for az in (0.0, 35.0)]
    rounded = oracle.round_storage(vol, storage)
    sc_r = oracle.Scene(rounded, tf, -1.0, 20.0, 0.5, 0.99)
    sc_f = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    for mode in ("composite", "mip"):
        img, mx = _render(vr, vol, tf, cams, mode, storage=storage, brick=32)
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc_r, c, mode, tol=1e-4,
                    gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3)
            if storage == "f16":
                compare(img[i].reshape(-1, 4), sc_f, c, mode, tol=2e-3)


@pytest.mark.parametrize("brick", [8, 16])
def test_ragged_cube_bricks_and_tiles(vr, brick):
    dims = (45, 37, 29)  # not multiples of the brick; image not a multiple of 8 x 4
    p = synth.cube_params(*dims, seed=3, nsrc=6)
    vol = synth.generate(p)
    tf = synth.viridis_ramp_tf(64)
    cams = [synth.orbit_view(dims, 17.0, 37, 23),
            synth.random_views(dims, 1, seed=9, width=37, height=23)[0],
            synth.look_at(dims, (0.3, -0.2, 1.0), 37, 23, dist_factor=0.3),  # eye inside
            synth.look_at(dims, (1.0, 0.0, 0.0), 37, 23, fov_deg=5.0,
                          up_hint=(0.0, 0.0, 1.0)) | {"eye": [500.0, 500.0, 500.0]}]  # miss
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    for mode in ("composite", "mip"):
        img, mx = _render(vr, vol, tf, cams, mode, brick=brick)
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc, c, mode, tol=1e-4,
                    gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3)
        assert np.all(img[3] == 0)


@pytest.mark.parametrize("step", [0.37, 0.731, 1.3])
def test_odd_step_sizes(vr, step):
    """Steps whose division is inexact (the sample range comes from an FP32 slab test
    screened by a rounding bound, with a float-float fallback): ray-path composite and MIP and
    the brick-path MIP, perspective, orthographic and inside-the-cube views."""
    dims = (45, 37, 71)  # ragged against 32^3 bricks
    p = synth.cube_params(*dims, seed=4, nsrc=8)
    vol = synth.generate(p)
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view(dims, 23.0, 41, 29),
            synth.ortho_view(dims, 41, 29),
            synth.look_at(dims, (0.3, -0.2, 1.0), 41, 29, dist_factor=0.3)]  # eye inside
    sc = oracle.Scene(vol, tf, -1.0, 20.0, step, 0.99)
    for mode, path in (("composite", "ray"), ("mip", "ray"), ("mip", "brick")):
        img, mx = _render(vr, vol, tf, cams, mode, brick=32, step=step, path=path)
        for i, c in enumerate(cams):
            st = compare(img[i].reshape(-1, 4), sc, c, mode, tol=1e-4,
                         gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3, path=path)
            assert st["nsamples"] > 0


@pytest.mark.parametrize("ntf,ert,vrange", [(2, 0.05, (-1.0, 20.0)), (1024, 2.0, (-1.0, 20.0)),
                                             (1024, 0.5, (2.0, 3.0))])
def test_transfer_function_and_termination_extremes(vr, ntf, ert, vrange):
    """The smallest (2 entries) and largest (1024) tables, termination after the first
    few samples (ert 0.05), termination disabled (ert > 1), and a narrow value range that
    clamps most samples at both ends: every path against the oracle."""
    dims = (45, 37, 71)
    vol = synth.generate(synth.cube_params(*dims, seed=9, nsrc=8))
    tf = synth.hidden_tf(17, ntf)
    cams = [synth.orbit_view(dims, 41.0, 41, 29), synth.ortho_view(dims, 41, 29)]
    sc = oracle.Scene(vol, tf, vrange[0], vrange[1], 0.5, ert)
    for mode, path in (("composite", "ray"), ("mip", "ray"), ("mip", "brick")):
        img, mx = _render(vr, vol, tf, cams, mode, brick=32, ert=ert, vmin=vrange[0], vmax=vrange[1],
                          path=path)
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc, c, mode, tol=1e-4,
                    gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3, path=path)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_transparent_bricks_are_skipped_exactly(vr, storage):
    """A table that is transparent below 6 sigma: the composite marcher skips every brick
    whose stored maximum maps below the transparent nodes (noise-only bricks), executes
    fewer samples than the rays hold, and still equals the oracle."""
    dims = (80, 72, 96)
    vol = synth.generate(synth.cube_params(*dims, seed=13, nsrc=6))
    tf = synth.viridis_ramp_tf()
    node_v = -1.0 + 21.0 * np.arange(256) / 255.0
    tf[node_v < 6.0, 3] = 0.0
    cams = [synth.orbit_view(dims, 35.0, 48, 40), synth.ortho_view(dims, 48, 40)]
    r = vr.Renderer(0, brick=16)
    r.load_cube(vol, storage)
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cams)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    vr.vr_set_sample_counter(r.ctx, counter)
    img = r.render("composite").cpu().numpy()
    vr.vr_set_sample_counter(r.ctx, None)
    r.close()
    sc = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 0.99)
    total = 0
    for i, c in enumerate(cams):
        st = compare(img[i].reshape(-1, 4), sc, c, "composite", tol=1e-4)
        total += st["nsamples"]
    assert int(counter.item()) < 0.8 * total, (int(counter.item()), total)


def test_fine_step(vr):
    """A step of 0.05 voxel (20 samples per voxel, thousands per ray), every path."""
    dims = (24, 20, 36)
    vol = synth.generate(synth.cube_params(*dims, seed=10, nsrc=4))
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view(dims, 77.0, 24, 18), synth.ortho_view(dims, 24, 18)]
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.05, 0.99)
    for mode, path in (("composite", "ray"), ("mip", "ray"), ("mip", "brick")):
        img, mx = _render(vr, vol, tf, cams, mode, brick=8 if path == "ray" else 32, step=0.05, path=path)
        for i, c in enumerate(cams):
            st = compare(img[i].reshape(-1, 4), sc, c, mode, tol=1e-4,
                         gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3, path=path)
            assert st["nsamples"] > 0


def test_distant_narrow_view(vr):
    """An eye ~1e5 voxels away with a 0.02 degree field of view: the FP32 screen of the
    sample range fails for most rays, so the float-float slab test decides them, and the
    anchors o + k e are far from the origin."""
    dims = (45, 37, 71)
    vol = synth.generate(synth.cube_params(*dims, seed=6, nsrc=8))
    tf = synth.viridis_ramp_tf()
    cam = synth.look_at(dims, (0.3, 0.2, 1.0), 41, 29, fov_deg=0.02, dist_factor=2000.0)
    assert np.linalg.norm(np.asarray(cam["eye"])) > 5e4
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    for mode, path in (("composite", "ray"), ("mip", "ray"), ("mip", "brick")):
        img, mx = _render(vr, vol, tf, [cam], mode, brick=32, path=path)
        st = compare(img[0].reshape(-1, 4), sc, cam, mode, tol=1e-4,
                     gpu_max=mx[0] if mode == "mip" else None, max_tol=2e-3, path=path)
        assert st["nsamples"] > 0


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_shifted_copy_reads_bit_identical(vr, storage):
    """The marcher's paired loads (x-neighbours from the store or from its copy shifted by
    one element, 16-bit stores) give the single-store images bit for bit: the same
    operations on the same values.  Ragged cube, perspective and orthographic views, both
    modes."""
    dims = (45, 37, 71)
    vol = synth.generate(synth.cube_params(*dims, seed=8, nsrc=8))
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view(dims, 23.0, 41, 29), synth.ortho_view(dims, 41, 29)]
    imgs, store = {}, {}
    for single in (False, True):
        r = vr.Renderer(0, brick=32, single_store=single)
        r.set_path("ray")
        r.load_cube(vol, storage)
        store[single] = r.cube_info()["store_bytes"]
        r.set_transfer_function(tf, -1.0, 20.0)
        r.set_camera(cams)
        imgs[single] = [r.render(m, with_max=True) for m in ("composite", "mip")]
        torch.cuda.synchronize()
        imgs[single] = [(o.cpu().numpy(), mx.cpu().numpy()) for o, mx in imgs[single]]
        r.close()
    # the shifted copy is kept for a small 16-bit cube, never for FP32
    assert store[False] == (1 if storage == "f32" else 2) * store[True]
    for (a, am), (b, bm) in zip(imgs[False], imgs[True]):
        assert np.array_equal(a, b)
        assert np.array_equal(am, bm)
    sc = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 0.99)
    compare(imgs[True][0][0][0].reshape(-1, 4), sc, cams[0], "composite", tol=1e-4)


def test_axis_aligned_and_face_grazing_rays(vr):
    dims = (16, 12, 20)
    vol = synth.generate(synth.cube_params(*dims, seed=4, nsrc=3))
    tf = synth.viridis_ramp_tf()
    cams = [synth.axis_view(dims, 16, 12, plane_offset=-2.25),
            # pixel centres exactly on the x = 0 and x = 16 faces (and every integer between)
            dict(type=0, eye=[0.0, 0.0, -1.1], right=[1, 0, 0], up=[0, 1, 0], fwd=[0, 0, 1],
                 win=[-0.5, 16.5, 0.0, 12.0], width=17, height=12)]
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 1.0, 0.99)
    for mode in ("composite", "mip"):
        for c in cams:
            img, mx = _render(vr, vol, tf, [c], mode, brick=8, step=1.0)
            compare(img[0].reshape(-1, 4), sc, c, mode, tol=1e-4,
                    gpu_max=mx[0] if mode == "mip" else None, max_tol=2e-3)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (9, 1, 4)])
def test_degenerate_cubes(vr, dims):
    rng = np.random.default_rng(1)
    vol = (rng.normal(size=dims[::-1]) * 5 + 4).astype(np.float32)
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view(dims, 20.0, 19, 13), synth.ortho_view(dims, 19, 13)]
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    for mode in ("composite", "mip"):
        img, mx = _render(vr, vol, tf, cams, mode, brick=8)
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc, c, mode, tol=1e-4,
                    gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3)
    # staged cells (bricks of 32: one brick holding one ragged cell): brick-pass MIP and
    # the sort-last partial passes
    img, mx = _render(vr, vol, tf, cams, "mip", brick=32, path="brick")
    for i, c in enumerate(cams):
        compare(img[i].reshape(-1, 4), sc, c, "mip", tol=1e-4, gpu_max=mx[i], max_tol=2e-3, path="brick")
    sc_off = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 2.0)
    img, _ = _render(vr, vol, tf, cams, "composite", brick=32, path="sortlast")
    for i, c in enumerate(cams):
        compare(img[i].reshape(-1, 4), sc_off, c, "composite", tol=1e-4, path="sortlast")


def test_many_cameras_and_sample_count(vr):
    dims = (40, 36, 52)
    vol = synth.generate(synth.cube_params(*dims, seed=8, nsrc=10))
    tf = synth.viridis_ramp_tf()
    cams = synth.random_views(dims, 40, seed=2, width=16, height=12)  # > one launch of 32
    sc = oracle.Scene(vol, tf, -1.0, 20.0, 0.5, 0.99)
    r = vr.Renderer(0, brick=16)
    r.load_cube(vol)
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cams)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    vr.vr_set_sample_counter(r.ctx, counter)
    for mode in ("composite", "mip"):
        counter.zero_()
        out = r.render(mode)
        torch.cuda.synchronize()
        img = out.cpu().numpy()
        total, flagged = 0, 0
        for i, c in enumerate(cams):
            st = compare(img[i].reshape(-1, 4), sc, c, mode, tol=1e-4)
            total += st["nsamples"]
            flagged += st["n_flagged"]
        got = int(counter.item())
        if flagged == 0:
            assert got == total
        else:
            assert abs(got - total) <= 2 * flagged
    r.close()


def test_render_into_torch_stream_and_reuse(vr):
    dims = (32, 32, 32)
    vol = torch.from_numpy(synth.generate(synth.cube_params(*dims, seed=5, nsrc=4))).cuda()
    tf = synth.viridis_ramp_tf()
    cam = synth.orbit_view(dims, 45.0, 40, 30)
    r = vr.Renderer(0, brick=16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r.load_cube(vol, "f16")  # device source
        r.set_transfer_function(tf, -1.0, 20.0)
        r.set_camera(cam)
        a = r.render("mip")
        b = r.render("mip")
    s.synchronize()
    assert torch.equal(a, b)  # deterministic
    sc = oracle.Scene(oracle.round_storage(vol.cpu().numpy(), "f16"), tf, -1.0, 20.0)
    compare(a[0].cpu().numpy().reshape(-1, 4), sc, cam, "mip", tol=1e-4)
    r.close()


def test_status_codes(vr):
    r = vr.Renderer(0)
    out = torch.empty((1, 4, 4, 4), device="cuda")
    with pytest.raises(vr.VrError) as e:
        r.set_camera(synth.orbit_view((8, 8, 8), 0.0, 4, 4))
        r.render("mip", out=out)
    assert e.value.status == vr.VR_ERR_STATE
    with pytest.raises(vr.VrError) as e:
        r.set_transfer_function(np.zeros((1, 4), np.float32), 0.0, 1.0)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    with pytest.raises(vr.VrError) as e:
        r.set_transfer_function(np.zeros((4, 4), np.float32), 1.0, 1.0)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    r.load_cube(np.zeros((8, 8, 8), np.float32))
    r.set_transfer_function(synth.viridis_ramp_tf(), 0.0, 1.0)
    big = torch.empty(4 * 4 * 4 + 1, device="cuda")
    with pytest.raises(vr.VrError) as e:  # misaligned output is rejected, not written
        vr.vr_render(r.ctx, "mip", big[1:])
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    bad = dict(synth.orbit_view((8, 8, 8), 0.0, 4, 4))
    bad["type"] = 7
    with pytest.raises(vr.VrError) as e:
        r.set_camera(bad)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    far = dict(synth.orbit_view((8, 8, 8), 0.0, 4, 4), eye=[0.0, 0.0, -2e9])
    with pytest.raises(vr.VrError) as e:  # beyond the float-float set-up's range
        r.set_camera(far)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    flat = dict(synth.orbit_view((8, 8, 8), 0.0, 4, 4), fwd=[0.0, 0.0, 0.0])  # no forward axis
    with pytest.raises(vr.VrError) as e:
        r.set_camera(flat)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    huge = synth.orbit_view((8, 8, 8), 0.0, 32768, 32769)  # more than 2^30 pixels in one image
    with pytest.raises(vr.VrError) as e:
        r.set_camera(huge)
    assert e.value.status == vr.VR_ERR_INVALID_ARG
    r.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("brick", [32, 64])
def test_brick_path_mip(vr, storage, brick):
    """Object-order MIP (TMA-staged cells) on ragged cubes, several views, both camera types."""
    for dims in ((96, 80, 72), (45, 37, 29), (33, 70, 130)):
        p = synth.cube_params(*dims, seed=sum(dims), nsrc=8, ripple=True, ripple_period=32.0)
        vol = synth.generate(p)
        tf = synth.viridis_ramp_tf()
        cams = [synth.orbit_view(dims, az, 61, 47) for az in (0.0, 33.0, 90.0, 200.0)]
        cams += [synth.ortho_view(dims, 61, 47, rx_deg=15.0, ry_deg=-40.0),
                 synth.axis_view(dims, 61, 47, plane_offset=-3.3) | {"width": 61, "height": 47},
                 synth.look_at(dims, (0.2, 0.5, 1.0), 61, 47, dist_factor=0.35)]  # eye inside
        sc = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 0.99)
        img, mx = _render(vr, vol, tf, cams, "mip", storage=storage, brick=brick, path="brick")
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc, c, "mip", tol=1e-4, gpu_max=mx[i], max_tol=2e-3)


def test_brick_path_rejects_composite_and_small_bricks(vr):
    vol = np.zeros((40, 40, 40), np.float32)
    r = vr.Renderer(0, brick=16)
    r.load_cube(vol)
    r.set_transfer_function(synth.viridis_ramp_tf(), 0.0, 1.0)
    r.set_camera(synth.orbit_view((40, 40, 40), 0.0, 8, 8))
    r.set_path("brick")
    for mode in ("mip", "composite"):
        with pytest.raises(vr.VrError) as e:
            r.render(mode)
        assert e.value.status == vr.VR_ERR_UNSUPPORTED
    r.set_path("auto")
    r.render("mip")  # falls back to the ray path
    torch.cuda.synchronize()
    r.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_survey_workload_sampled_pixels(vr, storage):
    """Full-size 1024 x 1024 x 2048 cube (2000 sources + ripple), perspective 1920 x 1080,
    two orbit frames; 4096 seeded pixels checked against the oracle, for the image-order
    composite and MIP, the brick-pass MIP and the sort-last composite (per-brick partial
    images from staged cells, folded in visibility order; no termination)."""
    cfg = synth.CONFIGS["survey"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    vol = synth.generate(p)
    tf = synth.viridis_ramp_tf()
    cams = [synth.orbit_view(dims, az) for az in (0.0, 130.0)]
    r = vr.Renderer(0, brick=128)
    r.load_cube(vol, storage)
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cams)
    ref_vol = oracle.round_storage(vol, storage)
    del vol
    sc = oracle.Scene(ref_vol, tf, -1.0, 20.0, 0.5, 0.99)
    rng = np.random.default_rng(2024)
    pix = rng.choice(1920 * 1080, 4096, replace=False)
    for mode, path in (("composite", "ray"), ("mip", "ray"), ("mip", "brick")):
        r.set_path(path)
        out, mx = r.render(mode, with_max=True)
        torch.cuda.synchronize()
        img = out.cpu().numpy().reshape(2, -1, 4)
        mxs = mx.cpu().numpy().reshape(2, -1)
        for i, c in enumerate(cams):
            st = compare(img[i][pix], sc, c, mode, pixels=pix, tol=1e-4,
                         gpu_max=mxs[i][pix] if mode == "mip" else None, max_tol=2e-3, path=path)
            print(storage, mode, path, i, st)
    sc_off = oracle.Scene(ref_vol, tf, -1.0, 20.0, 0.5, 2.0)
    r.set_path("sortlast")
    out = r.render("composite")
    torch.cuda.synchronize()
    img = out.cpu().numpy().reshape(2, -1, 4)
    for i, c in enumerate(cams):
        st = compare(img[i][pix], sc_off, c, "composite", pixels=pix, tol=1e-4, path="sortlast")
        print(storage, "composite", "sortlast", i, st)
    r.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_wall_25_frusta_one_launch(vr, storage):
    """5 x 5 wall: 25 off-axis frusta of one camera rendered together (one persistent
    launch per mode); each panel equals the oracle, and the mosaic equals the oracle's
    render of the single big camera (the panels are exact sub-windows)."""
    dims = (160, 144, 96)
    vol = synth.generate(synth.cube_params(*dims, seed=71, nsrc=30, ripple=True, ripple_period=48.0))
    tf = synth.viridis_ramp_tf()
    big = synth.orbit_view(dims, 35.0, 5 * 24, 5 * 14)
    panels = synth.wall_views(big, 5, 5)
    sc = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 0.99)
    for mode in ("composite", "mip"):
        img, mx = _render(vr, vol, tf, panels, mode, storage=storage, brick=32)
        mosaic = np.zeros((5 * 14, 5 * 24, 4), np.float32)
        for i in range(25):
            rr, cc = divmod(i, 5)
            mosaic[14 * rr:14 * rr + 14, 24 * cc:24 * cc + 24] = img[i]
        compare(mosaic.reshape(-1, 4), sc, big, mode, tol=1e-4)
        for i in (0, 7, 24):
            compare(img[i].reshape(-1, 4), sc, panels[i], mode, tol=1e-4,
                    gpu_max=mx[i] if mode == "mip" else None, max_tol=2e-3)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_sortlast_and_layered_composite(vr, storage):
    """Object-order composite: per-brick partial images folded in visibility order equal
    the oracle's composite without termination; the layered form (running state carried
    from layer to layer) equals the oracle's composite with termination."""
    for dims, brick in (((96, 80, 72), 32), ((45, 37, 29), 16), ((130, 70, 200), 64)):
        p = synth.cube_params(*dims, seed=sum(dims) + 1, nsrc=8, ripple=True, ripple_period=32.0)
        vol = synth.generate(p)
        tf = synth.viridis_ramp_tf()
        cams = [synth.orbit_view(dims, az, 53, 41) for az in (0.0, 47.0, 160.0, 290.0)]
        cams += [synth.ortho_view(dims, 53, 41, rx_deg=-25.0, ry_deg=70.0),
                 synth.look_at(dims, (0.1, -0.4, 1.0), 53, 41, dist_factor=0.3)]  # eye inside
        rounded = oracle.round_storage(vol, storage)
        sc_off = oracle.Scene(rounded, tf, -1.0, 20.0, 0.5, 2.0)
        sc_on = oracle.Scene(rounded, tf, -1.0, 20.0, 0.5, 0.99)
        img, _ = _render(vr, vol, tf, cams, "composite", storage=storage, brick=brick, path="sortlast")
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc_off, c, "composite", tol=1e-4, path="sortlast")
        img, _ = _render(vr, vol, tf, cams, "composite", storage=storage, brick=brick, path="layered")
        for i, c in enumerate(cams):
            compare(img[i].reshape(-1, 4), sc_on, c, "composite", tol=1e-4, path="layered")
    # visibility passes of the staged cells at their edge cases: an orthographic view
    # straight along z (two axes give equal keys), perspective eyes exactly on cell
    # boundary planes (inside the cube and outside it), and a view that misses the cube
    dims, brick = (130, 70, 200), 64
    vol = synth.generate(synth.cube_params(*dims, seed=331, nsrc=8, ripple=True, ripple_period=32.0))
    tf = synth.viridis_ramp_tf()

    def aim(eye, target, w=53, h=41, fov=60.0):
        f = np.asarray(target, np.float64) - np.asarray(eye, np.float64)
        f /= np.linalg.norm(f)
        right = np.cross((0.0, 1.0, 0.0), f)
        right /= np.linalg.norm(right)
        up = np.cross(f, right)
        t = np.tan(np.radians(fov) / 2.0)
        return dict(type=1, eye=[float(v) for v in eye], right=[float(v) for v in right],
                    up=[float(v) for v in up], fwd=[float(v) for v in f],
                    win=[-t * w / h, t * w / h, -t, t], width=w, height=h)

    cams = [synth.ortho_view(dims, 53, 41, rx_deg=0.0, ry_deg=0.0),
            aim((64.0, 32.0, 96.0), (10.0, 60.0, 190.0)),     # inside, on x, y and z cell planes
            aim((64.0, 32.0, -160.0), (70.0, 40.0, 100.0)),   # outside, on x and y cell planes
            aim((65.0, 35.0, 500.0), (65.0, 35.0, 900.0))]    # looks away: every ray misses
    img, _ = _render(vr, vol, tf, cams, "composite", storage=storage, brick=brick, path="sortlast")
    sc_off = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 2.0)
    for i, c in enumerate(cams):
        compare(img[i].reshape(-1, 4), sc_off, c, "composite", tol=1e-4, path="sortlast")
    assert not img[3].any()
    # the lane groups of other sizes join their runs in another rounding order
    r = vr.Renderer(0, brick=brick)
    r.set_path("sortlast")
    r.load_cube(vol, storage)
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cams[1])
    for group in (4, 16):
        t = vr.vr_get_tuning(r.ctx)
        t["group"] = group
        vr.vr_set_tuning(r.ctx, t)
        out = r.render("composite")
        torch.cuda.synchronize()
        compare(out[0].cpu().numpy().reshape(-1, 4), sc_off, cams[1], "composite", tol=1e-4, path="sortlast")
    r.close()
    # a 1024-entry table: the partial images come from whole-brick marches instead of
    # staged cells (whose shared copy of the table holds at most 256 entries)
    dims, brick = (96, 80, 72), 32
    vol = synth.generate(synth.cube_params(*dims, seed=249, nsrc=8, ripple=True, ripple_period=32.0))
    tf = synth.viridis_ramp_tf(1024)
    cams = [synth.orbit_view(dims, az, 53, 41) for az in (20.0, 200.0)]
    img, _ = _render(vr, vol, tf, cams, "composite", storage=storage, brick=brick, path="sortlast")
    sc_off = oracle.Scene(oracle.round_storage(vol, storage), tf, -1.0, 20.0, 0.5, 2.0)
    for i, c in enumerate(cams):
        compare(img[i].reshape(-1, 4), sc_off, c, "composite", tol=1e-4, path="sortlast")
