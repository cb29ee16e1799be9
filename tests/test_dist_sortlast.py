"""Object-space sort-last across ranks on CPU (two and three gloo ranks): the brick
partition, the band ownership, the packing of partial images, the exchange itself and the
fold order, checked against the oracle's sort-last render (the paper's decomposition of a
cube over nodes whose partial images are combined, Abstract and Sec. 1).

The partial images come from the oracle (what the library's vr_sortlast_partials computes
on a GPU) and the fold arithmetic is written out here in numpy in the order that
dist.fold_order gives (what vr_sortlast_fold does on a GPU): what is under test is the host
side of the exchange, which runs unchanged over NCCL between GPUs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

DIMS = (40, 36, 44)
BRICK = 16


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    import oracle
    import synth
    vol = synth.generate(synth.cube_params(*DIMS, seed=21, nsrc=5, ripple=True, ripple_period=16.0))
    return oracle.Scene(vol, synth.viridis_ramp_tf(), -1.0, 20.0, 0.5, 2.0)


def _views():
    import synth
    return [synth.orbit_view(DIMS, 35.0, 26, 21), synth.ortho_view(DIMS, 26, 21, rx_deg=-20.0, ry_deg=110.0)]


def _local_partials(sc, cam, bricks, mode):
    """This rank's partial images, from the oracle: footprint = bounding box of the
    pixels with samples in the brick; images packed row-major from offset 0."""
    import oracle
    from paper_1012_2909_gb300 import FOOTPRINT
    W, H = cam["width"], cam["height"]
    feet, parts, off = [], [], 0
    for b in bricks:
        pb = oracle.brick_partial(sc, cam, BRICK, int(b))
        has = (pb["nsamples"] > 0).reshape(H, W)
        if not has.any():
            feet.append((b, pb["key"], 0, 0, -1, -1, off))
            continue
        ys, xs = np.nonzero(has)
        x0, x1, y0, y1 = xs.min(), xs.max(), ys.min(), ys.max()
        img = pb["ct"].reshape(H, W, 4) if mode == "composite" else np.stack(
            [pb["max"], np.zeros_like(pb["max"]), np.zeros_like(pb["max"]), np.zeros_like(pb["max"])], 1
        ).reshape(H, W, 4)
        parts.append(img[y0:y1 + 1, x0:x1 + 1].reshape(-1, 4))
        feet.append((b, pb["key"], x0, y0, x1, y1, off))
        off += parts[-1].shape[0]
    foot = np.array(feet, dtype=FOOTPRINT)
    partial = torch.from_numpy(np.concatenate(parts).astype(np.float32)) if parts else torch.zeros((0, 4))
    return foot, partial


def _fold(foot, payload, order, W, y0, y1, mode):
    pay = payload.numpy().astype(np.float64)
    C = np.zeros((y1 - y0, W, 3))
    T = np.ones((y1 - y0, W))
    M = np.full((y1 - y0, W), -np.inf)
    for i in order:
        f = foot[i]
        w = f["x1"] - f["x0"] + 1
        img = pay[f["offset"]:f["offset"] + (f["y1"] - f["y0"] + 1) * w].reshape(-1, w, 4)
        ys = slice(f["y0"] - y0, f["y1"] - y0 + 1)
        xs = slice(f["x0"], f["x1"] + 1)
        if mode == "composite":
            C[ys, xs] += T[ys, xs, None] * img[..., :3]
            T[ys, xs] *= img[..., 3]
        else:
            M[ys, xs] = np.maximum(M[ys, xs], img[..., 0])
    return C, T, M


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_1012_2909_gb300 import dist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scene()
        nb = [-(-d // BRICK) for d in DIMS]
        mine = dist.partition_bricks(nb, world)[rank]
        tr = dist.TorchTransport()
        out = []
        for vi, cam in enumerate(_views()):
            W, H = cam["width"], cam["height"]
            y0, y1 = dist.band_rows(H, world, rank)
            for mode in ("composite", "mip"):
                foot, partial = _local_partials(sc, cam, mine, mode)
                rfoot, rpay = dist.exchange_partials(foot, partial, H, tr)
                order = dist.fold_order(rfoot)
                C, T, M = _fold(rfoot, rpay, order, W, y0, y1, mode)
                out.append((vi, mode, y0, y1, sorted(int(b) for b in rfoot["brick"]),
                            [(int(f["y0"]), int(f["y1"])) for f in rfoot], C, T, M))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()
    q.put((rank, out))


@pytest.mark.parametrize("world", [2, 3, 4])  # 4 ranks over 3 brick layers: one rank holds no brick
def test_exchange_and_fold_equal_the_oracle_sortlast(world):
    import oracle
    from paper_1012_2909_gb300 import dist
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = _scene()
    nb = [-(-d // BRICK) for d in DIMS]
    # the partition covers every brick exactly once
    parts = dist.partition_bricks(nb, world)
    allb = np.concatenate(parts)
    assert np.array_equal(np.sort(allb), np.arange(nb[0] * nb[1] * nb[2]))
    for vi, cam in enumerate(_views()):
        W, H = cam["width"], cam["height"]
        bands = [dist.band_rows(H, world, r) for r in range(world)]
        assert bands[0][0] == 0 and bands[-1][1] == H
        assert all(bands[r][1] == bands[r + 1][0] for r in range(world - 1))
        # which bricks meet which band: every brick with samples in a band reaches its owner
        meets = {}
        for b in range(nb[0] * nb[1] * nb[2]):
            pb = oracle.brick_partial(sc, cam, BRICK, b)
            rows = np.nonzero((pb["nsamples"] > 0).reshape(H, W).any(axis=1))[0]
            meets[b] = rows
        for mode in ("composite", "mip"):
            ref = oracle.render_sortlast(sc, cam, BRICK, mode, ert=2.0)
            for r in range(world):
                (vi_, mode_, y0, y1, recv, rows, C, T, M) = next(
                    o for o in res[r] if o[0] == vi and o[1] == mode)
                assert (y0, y1) == bands[r]
                want = sorted(b for b, rs in meets.items() if len(rs) and rs.min() < y1 and rs.max() >= y0)
                assert recv == want, (r, mode)
                assert all(y0 <= a <= b < y1 for a, b in rows)  # clipped to the owner's band
                pix = np.arange(y0 * W, y1 * W)
                if mode == "composite":
                    got = np.concatenate([C.reshape(-1, 3), (1 - T).reshape(-1, 1)], 1)
                    np.testing.assert_allclose(got, ref["rgba"][pix], atol=1e-6)
                else:
                    np.testing.assert_allclose(M.reshape(-1), ref["max"][pix], atol=1e-6)
