"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one part of the method by a closed form, a library routine, brute
force written differently from the oracle, or an invariant of the mathematics:

* constant cube: accumulated alpha 1-(1-a)^n and colour rgb*(1-(1-a)^n), with n from
  hand-derived ray/box chords; with termination n_ERT = ceil(ln 0.01 / ln(1-a));
* transfer function: numpy.interp over the node grid, clamped;
* single-peak MIP: the peak value, and the trilinear hat off-centre;
* axis-aligned views: numpy brute force along the spectral axis, composited by the
  closed-form product sum_j a_j c_j prod_{i<j}(1 - a_i) and cumulative products;
* sort-last: partial images per brick folded in visibility order equal the direct
  render (associativity of "over"; max is exact);
* 5 x 5 style mosaic: sub-frusta equal the crops of the one big render;
* adjoint: central finite differences of the FP64 loss;
* bfloat16 rounding: torch's conversion and hand-made ties.
"""
import math

import numpy as np
import pytest

import oracle
import synth

TOL = 1e-12


def cam(type_, eye, fwd, right=(1, 0, 0), up=(0, 1, 0), win=(-0.5, 0.5, -0.5, 0.5), w=1, h=1):
    return dict(type=type_, eye=list(eye), right=list(right), up=list(up), fwd=list(fwd),
                win=list(win), width=w, height=h)


# ------------------------------------------------------------------------- constant cube
@pytest.mark.parametrize("a", [0.02, 0.1, 0.37, 0.8])
def test_constant_cube_closed_form(a):
    vol = np.full((10, 6, 8), 3.0, np.float32)  # nz, ny, nx
    a32 = float(np.float32(a))
    rgb = np.array([0.2, 0.5, 0.9], np.float32).astype(np.float64)
    tf = np.tile(np.array([0.2, 0.5, 0.9, a], np.float32), (5, 1))
    s = 1 / math.sqrt(2)
    rays = [
        # orthographic along +z from z = -1.3: t in [1.3, 11.3) -> k = 3..22 (20 samples)
        (cam(0, (4.1, 2.2, -1.3), (0, 0, 1)), 20),
        # orthographic along (1,0,1)/sqrt2 from (-2, 3.3, -1): enters x=0 at t=2 sqrt2,
        # leaves x=8 at t=10 sqrt2 -> k = ceil(5.657)=6 .. ceil(28.28)-1=28 (23 samples)
        (cam(0, (-2, 3.3, -1), (s, 0, s), right=(s, 0, -s)), 23),
        # perspective along +z from z = -5.2: t in [5.2, 15.2) -> k = 11..30 (20 samples)
        (cam(1, (4, 3, -5.2), (0, 0, 1)), 20),
        # perspective through an off-centre pixel, direction (-0.35, 0, 1), sec = sqrt(1.1225):
        # enters z=0 at t = 5.2 sec = 5.509, leaves x=0 at depth 4/0.35, t = 12.108
        # -> k = 12..24 (13 samples); an unnormalised direction would give 12
        (cam(1, (4, 3, -5.2), (0, 0, 1), win=(-0.7, 0.0, -0.5, 0.5)), 13),
        # perspective from inside the cube at z = 2.3 along +z: t in [0, 7.7) -> k = 0..15
        (cam(1, (4, 3, 2.3), (0, 0, 1)), 16),
    ]
    for c, n in rays:
        sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=2.0)
        r = oracle.render(sc, c, "composite")
        assert r["nsamples"][0] == n
        A = 1 - (1 - a32) ** n
        np.testing.assert_allclose(r["rgba"][0, 3], A, atol=TOL)
        np.testing.assert_allclose(r["rgba"][0, :3], rgb * A, atol=TOL)
        # early termination at accumulated alpha 0.99
        sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=0.99)
        r = oracle.render(sc, c, "composite")
        n_ert = min(n, math.ceil(math.log(0.01) / math.log(1 - a32)))
        assert r["nsamples"][0] == n_ert
        np.testing.assert_allclose(r["rgba"][0, 3], 1 - (1 - a32) ** n_ert, atol=TOL)


def test_empty_ray_and_miss():
    vol = np.ones((4, 4, 4), np.float32)
    tf = synth.viridis_ramp_tf(8)
    sc = oracle.Scene(vol, tf, 0.0, 2.0)
    miss = cam(1, (10, 10, -5), (0, 0, 1))
    for mode in ("composite", "mip"):
        r = oracle.render(sc, miss, mode)
        assert r["nsamples"][0] == 0 and np.all(r["rgba"] == 0)
    assert oracle.render(sc, miss, "mip")["max"][0] == -np.inf


# --------------------------------------------------------------------- transfer function
def test_tf_lookup_matches_numpy_interp():
    tf = synth.hidden_tf(3, n=17)
    vmin, vmax = -1.0, 20.0
    nodes = np.linspace(vmin, vmax, tf.shape[0])
    for val in [-5.0, -1.0, -0.3, 0.0, 2.7, 7.77, 19.99, 20.0, 33.0]:
        vol = np.full((3, 3, 3), val, np.float32)
        sc = oracle.Scene(vol, tf, vmin, vmax)
        r = oracle.render(sc, cam(0, (1.5, 1.5, -0.7), (0, 0, 1)), "mip")
        v32 = float(np.float32(val))
        want = [np.interp(v32, nodes, tf[:, c].astype(np.float64)) for c in range(4)]
        np.testing.assert_allclose(r["rgba"][0], want, atol=1e-12)
        assert r["max"][0] == v32


# ---------------------------------------------------------------------- single-peak MIP
@pytest.mark.parametrize("dx,dy", [(0.0, 0.0), (0.3, 0.0), (-0.2, 0.45)])
def test_single_peak_mip(dx, dy):
    vol = np.zeros((9, 9, 9), np.float32)
    V = 7.0
    vol[4, 4, 4] = V  # centre (4.5, 4.5, 4.5)
    tf = synth.viridis_ramp_tf()
    sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5)
    # image plane z = -1: samples at z = -1 + k/2, one of them exactly at z = 4.5
    r = oracle.render(sc, cam(0, (4.5 + dx, 4.5 + dy, -1.0), (0, 0, 1)), "mip")
    np.testing.assert_allclose(r["max"][0], V * (1 - abs(dx)) * (1 - abs(dy)), atol=1e-12)
    # plane z = -0.75: nearest samples at 4.25 / 4.75 -> hat value 0.75 along z
    r = oracle.render(sc, cam(0, (4.5 + dx, 4.5 + dy, -0.75), (0, 0, 1)), "mip")
    np.testing.assert_allclose(r["max"][0], V * (1 - abs(dx)) * (1 - abs(dy)) * 0.75, atol=1e-12)


# ------------------------------------------------------- axis-aligned brute force (numpy)
def _column_view(nx, ny, xoff, z0):
    # orthographic down +z; pixel (px, py) at x = px + 0.5 + xoff, y = ny - 0.5 - py
    return dict(type=0, eye=[0.0, 0.0, z0], right=[1, 0, 0], up=[0, 1, 0], fwd=[0, 0, 1],
                win=[xoff, xoff + (nx - 1), 0.0, float(ny)], width=nx - 1, height=ny)


def _brute(vol, tf, vmin, vmax, xoff, z0, step, ert):
    nz, ny, nx = vol.shape
    W, H = nx - 1, ny
    nodes = np.linspace(vmin, vmax, tf.shape[0])
    t_near, t_far = -z0, nz - z0
    ks = np.arange(math.ceil(t_near / step), math.ceil(t_far / step))
    zs = z0 + ks * step
    img = np.zeros((H, W, 4))
    mip = np.zeros((H, W))
    for py in range(H):
        y = ny - 1 - py
        for px in range(W):
            fx = xoff
            col = (1 - fx) * vol[:, y, px].astype(np.float64) + fx * vol[:, y, px + 1]
            vals = np.interp(zs - 0.5, np.arange(nz), col)  # clamps at both ends
            mip[py, px] = vals.max()
            rgba = np.stack([np.interp(vals, nodes, tf[:, c].astype(np.float64))
                             for c in range(4)], 1)
            a = rgba[:, 3]
            trans = np.cumprod(1 - a)                      # T after each sample
            n = len(a)
            if ert <= 1:
                hit = np.nonzero(1 - trans >= ert)[0]
                if len(hit):
                    n = hit[0] + 1
            before = np.concatenate([[1.0], trans[:-1]])   # prod_{i<j} (1 - a_i)
            img[py, px, :3] = (a[:n, None] * rgba[:n, :3] * before[:n, None]).sum(0)
            img[py, px, 3] = 1 - trans[n - 1]
    return img, mip


@pytest.mark.parametrize("step,z0,xoff", [(1.0, -2.25, 0.0), (0.5, -2.3, 0.3), (0.25, -0.6, 0.7)])
@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_axis_aligned_bruteforce(step, z0, xoff, ert):
    rng = np.random.default_rng(11)
    nz, ny, nx = 14, 5, 7
    vol = rng.normal(size=(nz, ny, nx)).astype(np.float32) * 4 + 3
    tf = synth.viridis_ramp_tf()
    sc = oracle.Scene(vol, tf, -1.0, 20.0, step=step, ert=ert)
    c = _column_view(nx, ny, xoff, z0)
    want, wmip = _brute(vol, tf, -1.0, 20.0, xoff, z0, step, ert)
    r = oracle.render(sc, c, "composite")
    assert not np.any(r["flags"] & 3)
    np.testing.assert_allclose(r["rgba"].reshape(ny, nx - 1, 4), want, atol=1e-12)
    r = oracle.render(sc, c, "mip")
    np.testing.assert_allclose(r["max"].reshape(ny, nx - 1), wmip, atol=1e-12)


# ------------------------------------------------------------------ sort-last invariance
def _small_scene(ert=2.0, seed=5, dims=(20, 17, 23)):
    p = synth.cube_params(*dims, seed=seed, nsrc=4, ripple=True, ripple_period=16.0)
    vol = synth.generate(p)
    return oracle.Scene(vol, synth.viridis_ramp_tf(), -1.0, 20.0, step=0.5, ert=ert)


@pytest.mark.parametrize("brick", [4, 8, 16])
def test_sortlast_equals_direct(brick):
    sc = _small_scene()
    dims = (sc.nx, sc.ny, sc.nz)
    views = [synth.ortho_view(dims, 24, 20), synth.orbit_view(dims, 40.0, 24, 20),
             synth.random_views(dims, 1, seed=3, width=24, height=20)[0]]
    for v in views:
        d = oracle.render(sc, v, "composite")
        s = oracle.render_sortlast(sc, v, brick, "composite")
        np.testing.assert_allclose(s["rgba"], d["rgba"], atol=1e-12)
        d = oracle.render(sc, v, "mip")
        s = oracle.render_sortlast(sc, v, brick, "mip")
        assert np.array_equal(s["max"], d["max"])
        assert np.array_equal(s["rgba"], d["rgba"])


def test_termination_changes_at_most_one_percent():
    sc = _small_scene(ert=0.99)
    dims = (sc.nx, sc.ny, sc.nz)
    v = synth.orbit_view(dims, 20.0, 32, 24)
    on = oracle.render(sc, v, "composite")["rgba"]
    off = oracle.render(sc, v, "composite", ert=2.0)["rgba"]
    assert np.max(np.abs(on - off)) <= 0.01 + 1e-12


# ------------------------------------------------------------------------------ mosaic
def test_mosaic_equals_big_render():
    sc = _small_scene(ert=0.99)
    dims = (sc.nx, sc.ny, sc.nz)
    big = synth.orbit_view(dims, 25.0, 5 * 8, 5 * 6)
    full = oracle.render(sc, big, "composite")["rgba"].reshape(30, 40, 4)
    for i, p in enumerate(synth.wall_views(big, 5, 5)):
        rr, cc = divmod(i, 5)
        part = oracle.render(sc, p, "composite")["rgba"].reshape(6, 8, 4)
        np.testing.assert_allclose(part, full[6 * rr:6 * rr + 6, 8 * cc:8 * cc + 8], atol=1e-9)


# ------------------------------------------------------------------------------ adjoint
def _loss(sc, views, target, mode):
    imgs = np.stack([oracle.render(sc, v, mode)["rgba"].reshape(v["height"], v["width"], 4)
                     for v in views])
    return oracle.l2_loss(imgs, target)


def _nsamp(sc, views, mode):
    return np.concatenate([oracle.render(sc, v, mode)["nsamples"] for v in views])


@pytest.mark.parametrize("mode", ["composite", "mip"])
def test_adjoint_matches_finite_differences(mode):
    p = synth.cube_params(12, 10, 9, seed=21, nsrc=3)
    vol = synth.generate(p)
    tf = synth.viridis_ramp_tf(32)
    sc = oracle.Scene(vol, tf, -1.0, 20.0, step=0.5, ert=0.99)
    views = synth.random_views((12, 10, 9), 2, seed=4, width=12, height=10)
    tsc = oracle.Scene(vol, synth.hidden_tf(99, 32), -1.0, 20.0, step=0.5, ert=0.99)
    target = np.stack([oracle.render(tsc, v, mode)["rgba"].reshape(10, 12, 4) for v in views])
    L0, dimg = _loss(sc, views, target, mode)
    dtf, dvol = oracle.backward(sc, views, dimg.reshape(2, 10, 12, 4), mode)
    base_ns = _nsamp(sc, views, mode)
    rng = np.random.default_rng(1)

    def fd(perturb):
        lp, ln_ = [], []
        for sgn, acc in ((1, lp), (-1, ln_)):
            s2, h = perturb(sgn)
            if not np.array_equal(_nsamp(s2, views, mode), base_ns):
                return None
            acc.append((_loss(s2, views, target, mode)[0], h))
        (l1, h1), (l2, h2) = lp[0], ln_[0]
        return (l1 - l2) / (h1 - h2)

    checked = 0
    cand = [tuple(x) for x in np.argwhere(np.abs(dtf) > 1e-6 * np.abs(dtf).max())]
    rng.shuffle(cand)
    gmax = np.abs(dtf).max()
    for (i, c) in cand[:12]:
        def pert(sgn, i=i, c=c):
            t2 = tf.copy()
            t2[i, c] = np.float32(tf[i, c] + sgn * 1e-3)
            return oracle.Scene(vol, t2, -1.0, 20.0, 0.5, 0.99), float(t2[i, c]) - float(tf[i, c])
        g = fd(pert)
        if g is None:
            continue
        rel = abs(g - dtf[i, c]) / max(abs(g), 1e-2 * gmax)
        assert rel <= 1e-3, (i, c, g, dtf[i, c])
        checked += 1
    assert checked >= 6
    vmaxg = np.abs(dvol).max()
    cand = [tuple(x) for x in np.argwhere(np.abs(dvol) > 1e-3 * vmaxg)]
    rng.shuffle(cand)
    checked = 0
    for idx in cand[:12]:
        def pertv(sgn, idx=idx):
            v2 = vol.copy()
            v2[idx] = np.float32(vol[idx] + sgn * 1e-3)
            return oracle.Scene(v2, tf, -1.0, 20.0, 0.5, 0.99), float(v2[idx]) - float(vol[idx])
        g = fd(pertv)
        if g is None:
            continue
        rel = abs(g - dvol[idx]) / max(abs(g), 1e-2 * vmaxg)
        assert rel <= 1e-3, (idx, g, dvol[idx])
        checked += 1
    assert checked >= 6


# ---------------------------------------------------------------------- touched voxels
def test_touch_census_axis_ray():
    vol = np.zeros((6, 5, 4), np.float32)
    sc = oracle.Scene(vol, synth.viridis_ramp_tf(), 0.0, 1.0)
    # one ray down +z through voxel centre (1.5, 2.5): corners x in {1,2}, y in {2,3}
    m = oracle.touched(sc, cam(0, (1.5, 2.5, -0.7), (0, 0, 1)), "mip")
    want = np.zeros_like(m)
    want[:, 2:4, 1:3] = 1
    assert np.array_equal(m, want)
    # one ray along +x through (y, z) = (2.5, 1.5): corners y in {2,3}, z in {1,2}, every x
    m = oracle.touched(sc, cam(0, (-0.7, 2.5, 1.5), (1, 0, 0), right=(0, 0, -1)), "mip")
    want = np.zeros_like(m)
    want[1:3, 2:4, :] = 1
    assert np.array_equal(m, want)


# ---------------------------------------------------------------------- storage rounding
def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    x = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 1e-30, 3.0e38, 0.1, 19.37],
                 np.float32)
    got = oracle.round_storage(x, "bf16")
    assert got[0] == 1.0 and got[1] == 1 + 2 ** -6  # ties to even
    rng = np.random.default_rng(0)
    y = (rng.normal(size=10000) * 10).astype(np.float32)
    want = torch.from_numpy(y).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.round_storage(y, "bf16"), want)
    assert np.array_equal(oracle.round_storage(y, "f16"),
                          torch.from_numpy(y).to(torch.float16).to(torch.float32).numpy())


# ---------------------------------------------------------------------- image pyramid
def test_pyramid_hand_example_3x3():
    rng = np.random.default_rng(3)
    a32 = rng.random((3, 3, 4)).astype(np.float32)
    a = a32.astype(np.float64)
    levels, out = oracle.pyramid(a32)
    assert levels == 3 and out.size == 4 * (4 + 1)
    want1 = np.array([[(a[0, 0] + a[0, 1] + a[1, 0] + a[1, 1]) / 4, (a[0, 2] + a[1, 2]) / 2],
                      [(a[2, 0] + a[2, 1]) / 2, a[2, 2]]])
    np.testing.assert_allclose(out[:16].reshape(2, 2, 4), want1, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[16:], want1.reshape(4, 4).mean(axis=0), rtol=0, atol=1e-15)


def test_pyramid_constant_image_and_level_count():
    c = np.array([0.1, 0.2, 0.3, 0.7], np.float32)
    for h, w in ((13, 7), (1, 9), (6, 1), (1, 1)):
        levels, out = oracle.pyramid(np.tile(c, (h, w, 1)))
        # levels: ceil(log2(max(w, h))) + 1
        assert levels == int(np.ceil(np.log2(max(w, h)))) + 1
        assert np.array_equal(out.reshape(-1, 4), np.tile(c.astype(np.float64), (out.size // 4, 1)))


def test_pyramid_power_of_two_block_means():
    rng = np.random.default_rng(4)
    a = rng.random((32, 16, 4)).astype(np.float32)  # H = 32, W = 16
    levels, out = oracle.pyramid(a)
    assert levels == 6
    lev = a.astype(np.float64)
    off = 0
    for w, h in oracle.pyramid_sizes(16, 32):
        lh, lw = lev.shape[:2]
        # 2 x 2 block means where both sides are even; a side of 1 averages the pairs of the other
        nxt = lev.reshape(lh // 2 if lh > 1 else 1, 2 if lh > 1 else 1,
                          lw // 2 if lw > 1 else 1, 2 if lw > 1 else 1, 4).mean(axis=(1, 3))
        got = out[off:off + 4 * w * h].reshape(h, w, 4)
        np.testing.assert_allclose(got, nxt, rtol=0, atol=1e-15)
        np.testing.assert_allclose(got.mean(axis=(0, 1)), a.astype(np.float64).mean(axis=(0, 1)),
                                   rtol=0, atol=1e-12)  # the mean is preserved
        off += 4 * w * h
        lev = nxt
    assert off == out.size


def test_pyramid_tiled_layout():
    rng = np.random.default_rng(5)
    a = rng.random((6, 10, 4)).astype(np.float32)  # H = 6, W = 10
    _, flat = oracle.pyramid(a, tile=0)
    _, tiled = oracle.pyramid(a, tile=4)
    off_f = off_t = 0
    for w, h in oracle.pyramid_sizes(10, 6):
        lev = flat[off_f:off_f + 4 * w * h].reshape(h, w, 4)
        tx, ty = -(-w // 4), -(-h // 4)
        blk = tiled[off_t:off_t + 4 * tx * ty * 16].reshape(ty * tx, 4, 4, 4)
        for y in range(4 * ty):
            for x in range(4 * tx):
                v = blk[(y // 4) * tx + x // 4, y % 4, x % 4]
                if x < w and y < h:
                    assert np.array_equal(v, lev[y, x])
                else:
                    assert not v.any()  # padding of edge tiles
        off_f += 4 * w * h
        off_t += 4 * tx * ty * 16
    assert off_f == flat.size and off_t == tiled.size


# ---------------------------------------------------------------------- catalogue overlay
def _ortho_xy(w=64, h=32):
    # looks along +z; window = the pixel grid: pixel (px, py) centre at u = px + 1/2, v = h - py - 1/2
    return cam(0, (0, 0, -10), (0, 0, 1), win=(0, w, 0, h), w=w, h=h)


def _outline(x0, x1, y0, y1, w, h):
    m = np.zeros((h, w), bool)
    for x in range(x0, x1 + 1):
        for y in (y0, y1):
            if 0 <= x < w and 0 <= y < h:
                m[y, x] = True
    for y in range(y0, y1 + 1):
        for x in (x0, x1):
            if 0 <= x < w and 0 <= y < h:
                m[y, x] = True
    return m


def test_overlay_axis_aligned_outline_and_blend():
    c = _ortho_xy()
    bg = np.tile(np.array([0.2, 0.1, 0.0, 0.5]), (32, 64, 1))
    col = np.array([[1.0, 0.5, 0.25, 0.75]], np.float32)
    # u = 10.5 -> pixel column 10, u = 20.5 -> 20; v = 5.5 -> row 26, v = 9.5 -> row 22
    out, key = oracle.overlay(bg, c, np.array([[10.5, 5.5, 1.0, 20.5, 9.5, 3.0]]), col)
    want = _outline(10, 20, 22, 26, 64, 32)
    assert np.array_equal(key > 0, want)
    a = 0.75
    blend = np.array([a * 1.0 + (1 - a) * 0.2, a * 0.5 + (1 - a) * 0.1, a * 0.25, a + (1 - a) * 0.5])
    np.testing.assert_allclose(out[want], np.tile(blend, (want.sum(), 1)), rtol=0, atol=1e-15)
    assert np.array_equal(out[~want], bg[~want])


def test_overlay_priority_and_clipping():
    c = _ortho_xy()
    boxes = np.array([[2.5, 2.5, 0, 12.5, 12.5, 1],      # box 0
                      [8.5, 4.5, 0, 30.5, 10.5, 1],      # box 1 overlaps box 0
                      [50.5, 20.5, 0, 80.5, 40.5, 1]])   # box 2 leaves the image
    out, key = oracle.overlay(np.zeros((32, 64, 4)), c, boxes, np.ones((3, 4), np.float32))
    m0 = _outline(2, 12, 19, 29, 64, 32)
    m1 = _outline(8, 30, 21, 27, 64, 32)
    m2 = _outline(50, 80, -9, 11, 64, 32)
    want = np.zeros((32, 64), np.int32)
    want[m0] = 1
    want[m1] = 2   # a pixel of several boxes keeps the highest index
    want[m2] = 3
    assert np.array_equal(key, want)


def test_overlay_perspective_against_a_pinhole_projection():
    d, W = 40.0, 96
    c = cam(1, (0, 0, -d), (0, 0, 1), win=(-1, 1, -1, 1), w=W, h=W)
    box = np.array([3.0, -5.0, 2.0, 11.0, 4.0, 9.0])
    _, key = oracle.overlay(np.zeros((W, W, 4)), c, box[None], np.ones((1, 4), np.float32))

    def pix(p):  # pinhole: u = x / (z + d), v = y / (z + d); pixel centres at integers
        u, v = p[0] / (p[2] + d), p[1] / (p[2] + d)
        return np.array([(u + 1) / 2 * W - 0.5, (1 - v) / 2 * W - 0.5])

    corners = [np.array([box[0 + 3 * i], box[1 + 3 * j], box[2 + 3 * k]])
               for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    for p in corners:  # every corner pixel is drawn
        x, y = np.floor(pix(p) + 0.5).astype(int)
        assert key[y, x] == 1
    segs = [(pix(corners[a]), pix(corners[b])) for a in range(8) for b in range(a + 1, 8)
            if bin(a ^ b).count("1") == 1]
    assert len(segs) == 12
    ys, xs = np.nonzero(key)
    for x, y in zip(xs, ys):  # every drawn pixel is within rounding of a projected edge
        best = min(np.linalg.norm(np.array([x, y]) - (p + np.clip(np.dot([x, y] - p, q - p) /
                   max(np.dot(q - p, q - p), 1e-12), 0, 1) * (q - p))) for p, q in segs)
        assert best <= 0.71
    for p, q in segs:  # and every edge is drawn without gaps (8-connected walk)
        n = int(np.ceil(np.abs(q - p).max())) * 4 + 1
        for f in np.linspace(0, 1, n):
            x, y = np.floor(p + f * (q - p) + 0.5).astype(int)
            assert key[max(y - 1, 0):y + 2, max(x - 1, 0):x + 2].any()


def test_overlay_box_behind_the_camera_draws_nothing():
    c = cam(1, (0, 0, 0), (0, 0, 1), win=(-1, 1, -1, 1), w=32, h=32)
    _, key = oracle.overlay(np.zeros((32, 32, 4)), c, np.array([[-2, -2, -9, 2, 2, -3]]),
                            np.ones((1, 4), np.float32))
    assert not key.any()


# ------------------------------------------------------- ambiguity windows (reading R11)
# The windows are derived from the renderer's FP32 arithmetic (oracle.c header).  For a
# constant cube and a constant table the value has no position error and the alpha only
# lerp rounding, so the termination window is a few 1e-7: a ray whose 1 - (1-a)^n lands
# 1e-9 from the threshold must be flagged, one landing 3e-6 away must not.
def _const_ray(a, nz=60):
    vol = np.full((nz, 3, 3), 2.0, np.float32)
    tf = np.tile(np.array([0.3, 0.6, 0.2, a], np.float32), (4, 1))
    c = cam(0, (1.5, 1.5, -1.3), (0, 0, 1))  # t in [1.3, 61.3): k = 3 .. 122 at step 0.5
    return vol, tf, c


@pytest.mark.parametrize("delta,flagged", [(1e-9, True), (3e-6, False)])
def test_termination_window_constant_cube(delta, flagged):
    a = float(np.float32(0.1))
    vol, tf, c = _const_ray(a)
    n = 44  # 1 - 0.9^44 = 0.9903
    A = 1 - (1 - a) ** n
    sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=A - delta, pos_err=oracle.pos_err_marcher(0.5))
    r = oracle.render(sc, c, "composite")
    assert r["nsamples"][0] == n
    assert bool(r["flags"][0] & 4) == flagged
    assert not r["flags"][0] & 3


def test_termination_variants_stop_one_sample_apart():
    a = float(np.float32(0.1))
    vol, tf, c = _const_ray(a)
    n = 44
    sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=1 - (1 - a) ** n - 1e-12)
    for ds in (-1, 0, 1):
        r = oracle.render(sc, c, "composite", dstop=ds)
        assert r["nsamples"][0] == n + ds
        np.testing.assert_allclose(r["rgba"][0, 3], 1 - (1 - a) ** (n + ds), atol=TOL)
    assert sorted(oracle.variants(4)) == [(-1, 0, 0), (0, 0, 0), (1, 0, 0)]


def test_termination_window_scales_with_position_error():
    """A cube that ramps along the ray (1 per voxel) under a linear alpha table: the value
    error is pos_err per voxel of displacement, so a ray 1e-6 from the threshold is flagged
    with a 1e-4 voxel position error and not without one; 1e-4 away it is never flagged."""
    nz = 80
    vol = np.broadcast_to(np.arange(nz, dtype=np.float32)[:, None, None] * 0.25, (nz, 3, 3)).copy()
    tf = synth.viridis_ramp_tf()
    c = cam(0, (1.5, 1.5, -0.7), (0, 0, 1))
    base = oracle.Scene(vol, tf, -1.0, 20.0, step=0.5, ert=2.0)
    r = oracle.render(base, c, "composite")
    # accumulated alpha after each sample from the exact render with no termination
    alphas = [oracle.render(base, c, "composite", ert=2.0, dk1=-(int(r["nsamples"][0]) - j))["rgba"][0, 3]
              for j in range(1, int(r["nsamples"][0]) + 1)]
    n = next(j for j, A in enumerate(alphas, 1) if A > 0.9)
    A = alphas[n - 1]
    for pe, delta, flagged in ((1e-4, 1e-6, True), (0.0, 1e-6, False), (1e-4, 1e-4, False)):
        sc = oracle.Scene(vol, tf, -1.0, 20.0, step=0.5, ert=A - delta, pos_err=pe)
        out = oracle.render(sc, c, "composite")
        assert out["nsamples"][0] == n
        assert bool(out["flags"][0] & 4) == flagged, (pe, delta)


@pytest.mark.parametrize("end,delta,flagged", [(0, 1e-12, True), (0, 1e-8, False),
                                               (1, 1e-12, True), (1, 1e-8, False)])
def test_end_sample_window(end, delta, flagged):
    """t_near/step (end 0) or t_far/step (end 1) within 1e-12 of an integer is flagged; 1e-8
    away is beyond the float-float set-up bound (2^-43 (|o| + n + t) / (|d| step), about
    5e-12 here, windowed at 2^7 times that) and is not."""
    vol = np.full((10, 3, 3), 2.0, np.float32)
    tf = synth.viridis_ramp_tf(8)
    # orthographic along +z from z0: t_near = -z0, t_far = 10 - z0; step 0.3 (the two ends'
    # fractions then differ by 1/3)
    z0 = -0.3 * (5 + delta) if end == 0 else 10 - 0.3 * (40 + delta)
    sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.3, ert=2.0)
    r = oracle.render(sc, cam(0, (1.5, 1.5, z0), (0, 0, 1)), "mip")
    bit = 1 << end
    assert bool(r["flags"][0] & bit) == flagged
    assert not r["flags"][0] & (3 ^ bit)


# ----------------------------------------- adjoint: bound on legitimate deviations (R14)
def test_adjoint_node_alternative_bound():
    """Every sample of a constant cube sits exactly on a table node: the voxel gradient may
    take either one-sided slope.  The ambiguity bound must cover the gradient computed with
    the other side's slope (a table whose segment right of the node continues the left
    slope), and is zero for a value between nodes."""
    vol = np.full((12, 4, 4), 7.0, np.float32)   # node 7 of 11 over [0, 10]
    tf = synth.hidden_tf(5, n=11)
    c = [cam(1, (2.0, 2.0, -6.0), (0, 0, 1), win=(-0.2, 0.2, -0.2, 0.2), w=3, h=2)]
    g = np.random.default_rng(2).normal(size=(1, 2, 3, 4))
    sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=2.0)
    _, dvol, amb = oracle.backward(sc, c, g, "composite", ambiguity=True)
    tf2 = tf.copy()
    tf2[8] = 2 * tf[7] - tf[6]     # the left segment's slope continued past node 7
    _, dvol2 = oracle.backward(oracle.Scene(vol, tf2, 0.0, 10.0, step=0.5, ert=2.0), c, g, "composite")
    d = np.abs(dvol2 - dvol)
    assert d.max() > 0 and np.all(d <= amb + 1e-12)
    vol3 = np.full((12, 4, 4), 7.4, np.float32)  # between nodes 7 and 8
    _, _, amb3 = oracle.backward(oracle.Scene(vol3, tf, 0.0, 10.0, step=0.5, ert=2.0), c, g, "composite",
                                 ambiguity=True)
    assert np.all(amb3 == 0)


def test_adjoint_termination_alternative_bound():
    """A ray whose termination is within rounding of the threshold may stop one sample
    earlier: the bound must cover the gradient of that outcome (termination moved one
    sample earlier by a threshold just below the earlier sample's accumulated alpha)."""
    a = float(np.float32(0.1))
    vol = np.broadcast_to(np.linspace(1.0, 2.0, 60, dtype=np.float32)[:, None, None], (60, 3, 3)).copy()
    tf = np.array([[0.3, 0.6, 0.2, a], [0.9, 0.1, 0.5, a]], np.float32)
    c = [cam(0, (1.5, 1.5, -1.3), (0, 0, 1))]
    g = np.array([0.3, -0.2, 0.5, 0.7]).reshape(1, 1, 1, 4)
    n = 44
    ert = 1 - (1 - a) ** n - 1e-12
    sc = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=ert)
    assert oracle.render(sc, c[0], "composite")["flags"][0] & 4
    _, dvol, amb = oracle.backward(sc, c, g, "composite", ambiguity=True)
    _, dvol_early = oracle.backward(sc, c, g, "composite", ert=1 - (1 - a) ** (n - 1) - 1e-12)
    d = np.abs(dvol_early - dvol)
    assert d.max() > 0 and np.all(d <= amb + 1e-12)
    # far from the threshold: no flag, and no ambiguity away from table nodes
    sc2 = oracle.Scene(vol, tf, 0.0, 10.0, step=0.5, ert=0.995)
    assert not oracle.render(sc2, c[0], "composite")["flags"][0]
    assert np.all(oracle.backward(sc2, c, g, "composite", ambiguity=True)[2] == 0)


# -------------------------------------------------- per-brick partial images (sort-last)
@pytest.mark.parametrize("brick", [8, 16])
def test_brick_partials_fold_to_the_direct_render(brick):
    """The bricks' partial images folded per pixel in ascending (key, brick id) with
    C += T C_b, T *= T_b equal the direct render without termination (associativity of
    "over"), their maxima give the MIP maximum, and their sample counts add up."""
    sc = _small_scene()
    dims = (sc.nx, sc.ny, sc.nz)
    nb = [-(-d // brick) for d in dims]
    for v in (synth.orbit_view(dims, 40.0, 20, 16), synth.ortho_view(dims, 20, 16)):
        direct = oracle.render(sc, v, "composite", ert=2.0)
        mip = oracle.render(sc, v, "mip")
        parts = [oracle.brick_partial(sc, v, brick, b) for b in range(nb[0] * nb[1] * nb[2])]
        order = sorted(range(len(parts)), key=lambda b: (parts[b]["key"], b))
        C = np.zeros((direct["rgba"].shape[0], 3))
        T = np.ones(direct["rgba"].shape[0])
        for b in order:
            C += T[:, None] * parts[b]["ct"][:, :3]
            T *= parts[b]["ct"][:, 3]
        np.testing.assert_allclose(C, direct["rgba"][:, :3], atol=1e-12)
        np.testing.assert_allclose(1 - T, direct["rgba"][:, 3], atol=1e-12)
        m = np.max([p_["max"] for p_ in parts], axis=0)
        assert np.array_equal(m, mip["max"])
        assert np.array_equal(np.sum([p_["nsamples"] for p_ in parts], axis=0), direct["nsamples"])
