"""Object-space sort-last through the C ABI on one GPU.  Ranks played by brick
partitions of one context (the exchange runs in memory with dist.Loopback): each
partition renders its partials with vr_sortlast_partials, the rows go to the band
owners, and each owner folds its band with vr_sortlast_fold.  The stitched bands equal
the single-device sort-last render bit for bit (same partial values, same per-pixel
order) and the oracle within the FP32 tolerance; MIP folds by maximum.  And two ranks
as two processes on the same GPU, exchanging over gloo."""
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


def _two_proc_scene():
    dims = (96, 80, 72)
    vol = synth.generate(synth.cube_params(*dims, seed=45, nsrc=8, ripple=True, ripple_period=32.0))
    return vol, synth.viridis_ramp_tf(), synth.orbit_view(dims, 35.0, 64, 48)


def _band_worker(rank, world, port, q):
    """One rank in its own process on the same GPU: its slab of bricks rendered by the
    library, the partials exchanged over gloo (staged through host memory), its band
    folded.  No kernel of one rank waits on another: the exchange is on the host."""
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as tdist

    import paper_1012_2909_gb300 as vr
    from paper_1012_2909_gb300 import dist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    try:
        vol, tf, cam = _two_proc_scene()
        r = vr.Renderer(0, brick=32)
        r.load_cube(vol, "f16")
        r.set_transfer_function(tf, -1.0, 20.0)
        r.set_camera(cam)
        tr = dist.TorchTransport()
        for mode in ("composite", "mip"):
            y0, y1, band = dist.render_band(r, mode, tr)
            torch.cuda.synchronize()
            out.append((mode, y0, y1, band.cpu().numpy()))
        tdist.barrier()
        r.close()
    finally:
        tdist.destroy_process_group()
    q.put((rank, out))


def test_two_processes_over_gloo():
    """Two ranks as two processes sharing the GPU, the partial images exchanged by
    dist.TorchTransport over gloo: the bands stitch to the single-process sort-last
    image bit for bit (composite), and to the oracle (MIP)."""
    import socket

    import torch.multiprocessing as mp

    import paper_1012_2909_gb300 as vr
    world = 2
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_band_worker, args=(rk, world, port, q)) for rk in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    vol, tf, cam = _two_proc_scene()
    W, H = cam["width"], cam["height"]
    r = vr.Renderer(0, brick=32)
    r.load_cube(vol, "f16")
    r.set_transfer_function(tf, -1.0, 20.0)
    r.set_camera(cam)
    r.set_path("sortlast")
    ref = r.render("composite")[0].cpu().numpy()
    r.close()
    sc = oracle.Scene(oracle.round_storage(vol, "f16"), tf, -1.0, 20.0, 0.5, 2.0)
    rows = []
    for rk in range(world):
        for mode, y0, y1, band in res[rk]:
            rows.append((mode, y0, y1))
            if mode == "composite":
                np.testing.assert_array_equal(band, ref[y0:y1])
            else:
                compare(band.reshape(-1, 4), sc, cam, "mip", pixels=np.arange(y0 * W, y1 * W), tol=1e-4,
                        path="sortlast")
    for mode in ("composite", "mip"):  # the bands tile the image
        spans = sorted((y0, y1) for m, y0, y1 in rows if m == mode)
        assert spans[0][0] == 0 and spans[-1][1] == H
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))


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
