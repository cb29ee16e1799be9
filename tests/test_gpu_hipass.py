"""High-resolution static render of one orientation (Sec. 3) on a cube of the paper's
HIPASS shape: 1721 x 1721 x 1025 FP32 (12 GB), ragged against the 128^3 bricks on every
axis (the last brick layer along the spectral axis is one voxel thick), rendered at
3000 x 3000 and 8000 x 8000 (at 3000 x 3000 also the sort-last composite, whose partial
images come from staged cells).  Seeded pixels of every image are checked against the
FP64 oracle (max abs RGBA error 1e-4, MIP maximum 2e-3)."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_hipass_static_render_sampled_pixels():
    import paper_1012_2909_gb300 as vr
    cfg = synth.CONFIGS["hipass"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    vol = synth.generate(p)
    tf = synth.viridis_ramp_tf()
    r = vr.Renderer(0, brick=128, step=cfg["step"], ert=cfg["ert"])
    r.load_cube(vol, "f32")
    r.set_transfer_function(tf, -1.0, 20.0)
    sc = oracle.Scene(vol, tf, -1.0, 20.0, cfg["step"], cfg["ert"])
    sc_off = oracle.Scene(vol, tf, -1.0, 20.0, cfg["step"], 2.0)  # sort-last: no termination
    rng = np.random.default_rng(1721)
    for W, H in cfg["images"]:
        cam = synth.orbit_view(dims, cfg["az"], W, H)
        r.set_camera(cam)
        pix = rng.choice(W * H, 4096, replace=False)
        runs = [("composite", "ray"), ("mip", "brick")]
        if W * H <= 9_000_000:
            runs += [("mip", "ray"), ("composite", "sortlast")]
        for mode, path in runs:
            r.set_path(path)
            out, mx = r.render(mode, with_max=True)
            torch.cuda.synchronize()
            img = out.reshape(-1, 4)[torch.from_numpy(pix).cuda()].cpu().numpy()
            mxs = mx.reshape(-1)[torch.from_numpy(pix).cuda()].cpu().numpy()
            st = compare(img, sc_off if path == "sortlast" else sc, cam, mode, pixels=pix, tol=1e-4,
                         gpu_max=mxs if mode == "mip" else None, max_tol=2e-3, path=path)
            print(W, H, mode, path, st)
            assert st["nsamples"] > (1_000_000 if mode == "mip" else 50_000), st  # the view sees the cube
            del out, mx
    r.close()
