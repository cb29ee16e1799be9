"""Object-space sort-last across ranks: the paper's distributed decomposition.

The paper renders a cube larger than one node's memory by giving each node a part
of it and combining the nodes' images (Abstract, Sec. 1).  Here each rank holds a
slab of bricks (partition_bricks), renders the partial image of every brick it holds
(vr_sortlast_partials: per footprint pixel (C, T) for "over", or the maximum for MIP),
and sends each partial's rows to the owner of the image band they fall in
(band_rows: rank r owns a contiguous band of rows).  The owner folds everything it
received in global visibility order -- ascending (key, brick), the same order every
rank computes for the same camera -- with vr_sortlast_fold.  A band holds the partials
of every brick whose footprint meets it, whoever rendered them, so the bands put
together equal the single-device sort-last image.

The exchange is one all-to-all step: the per-destination counts go first (all_gather
of a small integer tensor), then every pair of ranks swaps its payloads with
point-to-point sends and receives (supported by gloo and NCCL alike).  An in-process
transport (Loopback) runs the same packing and unpacking for ranks that share one
device.  Nothing here computes pixels: that is the library's kernels.
"""
from __future__ import annotations

import numpy as np

HEADER = 8  # int64 words per footprint on the wire: brick, key, x0, y0, x1, y1, offset, -


def partition_bricks(nb, world: int):
    """Linear brick ids (x fastest) of each rank: contiguous slabs of brick z-layers, the
    layers spread as evenly as possible (rank r gets layers [r n / world, (r+1) n / world))."""
    nbx, nby, nbz = (int(v) for v in nb)
    out = []
    for r in range(world):
        z0, z1 = r * nbz // world, (r + 1) * nbz // world
        out.append(np.arange(z0 * nbx * nby, z1 * nbx * nby, dtype=np.int32))
    return out


def band_rows(height: int, world: int, rank: int):
    """Image rows [y0, y1) owned by `rank`: contiguous bands, as even as possible."""
    return rank * height // world, (rank + 1) * height // world


def pack(foot, partial, y0: int, y1: int):
    """The rows [y0, y1) of every partial image that meets them: (headers int64 (k, HEADER),
    payload float32 (npix, 4), same device as `partial`).  A header's rectangle is the
    clipped one and its offset counts pixels from the start of the payload."""
    import torch

    heads, parts, off = [], [], 0
    for f in foot:
        if f["x1"] < f["x0"] or f["y1"] < y0 or f["y0"] >= y1:
            continue
        a, b = max(int(f["y0"]), y0), min(int(f["y1"]), y1 - 1)
        w = int(f["x1"]) - int(f["x0"]) + 1
        first = int(f["offset"]) + (a - int(f["y0"])) * w
        n = (b - a + 1) * w
        heads.append([int(f["brick"]), int(f["key"]), int(f["x0"]), a, int(f["x1"]), b, off, 0])
        parts.append(partial.view(-1, 4)[first:first + n])
        off += n
    h = np.asarray(heads, np.int64).reshape(-1, HEADER)
    if parts:
        payload = torch.cat(parts).contiguous()
    else:
        payload = torch.zeros((0, 4), dtype=torch.float32, device=partial.device)
    return h, payload


def unpack(messages):
    """Received (headers, payload) pairs, one per source rank -> (FOOTPRINT array with
    offsets into the concatenated payload, concatenated payload)."""
    import torch

    from . import FOOTPRINT

    feet, pays, base = [], [], 0
    for h, pay in messages:
        for row in np.asarray(h, np.int64).reshape(-1, HEADER):
            feet.append((row[0], row[1], row[2], row[3], row[4], row[5], base + row[6]))
        pays.append(pay.reshape(-1, 4))
        base += int(pay.reshape(-1, 4).shape[0])
    foot = np.array(feet, dtype=FOOTPRINT) if feet else np.zeros(0, FOOTPRINT)
    if pays:
        payload = torch.cat(pays).contiguous()
    else:
        payload = torch.zeros((0, 4), dtype=torch.float32)
    return foot, payload


def fold_order(foot):
    """Indices of `foot` in the global visibility order: ascending key, ties by brick id."""
    return np.lexsort((foot["brick"], foot["key"])) if len(foot) else np.zeros(0, np.int64)


class TorchTransport:
    """The exchange over a torch.distributed process group: NCCL moves device tensors
    directly; gloo moves host tensors, so device payloads are staged through host memory
    (host_staging None: staged exactly when the group's backend is gloo) and handed back
    on their device."""

    def __init__(self, group=None, host_staging=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        if host_staging is None:
            host_staging = str(dist.get_backend(group)) == "gloo"
        self.host_staging = bool(host_staging)

    def alltoall(self, outgoing):
        """outgoing[d] = (headers, payload) for rank d -> incoming[s] from rank s."""
        import torch

        dist, world, me = self.dist, self.world, self.rank
        dev = outgoing[me][1].device  # where the payloads live and are handed back
        comm = torch.device("cpu") if self.host_staging else dev  # where they travel
        counts = torch.tensor([[h.shape[0], p.shape[0]] for h, p in outgoing], dtype=torch.int64)
        counts = counts.to(comm)
        table = [torch.zeros_like(counts) for _ in range(world)]
        dist.all_gather(table, counts, group=self.group)
        table = [t.cpu().numpy() for t in table]  # table[s][d] = what s sends to d
        reqs, incoming = [], [None] * world
        recv_h, recv_p = {}, {}
        # every rank knows every count, so empty messages are simply not sent
        for s in range(world):
            if s == me:
                continue
            nh, npx = (int(v) for v in table[s][me])
            recv_h[s] = torch.zeros((nh, HEADER), dtype=torch.int64, device=comm)
            recv_p[s] = torch.zeros((npx, 4), dtype=torch.float32, device=comm)
            if nh:
                reqs.append(dist.irecv(recv_h[s], src=s, group=self.group))
            if npx:
                reqs.append(dist.irecv(recv_p[s], src=s, group=self.group))
        sends = []
        for d in range(world):
            if d == me:
                continue
            h, p = outgoing[d]
            th = torch.as_tensor(h, dtype=torch.int64).reshape(-1, HEADER).to(comm).contiguous()
            tp = p.to(comm).contiguous()
            sends += [th, tp]
            if th.shape[0]:
                reqs.append(dist.isend(th, dst=d, group=self.group))
            if tp.shape[0]:
                reqs.append(dist.isend(tp, dst=d, group=self.group))
        for q in reqs:
            q.wait()
        for s in range(world):
            if s == me:
                incoming[s] = outgoing[me]
            else:
                incoming[s] = (recv_h[s].cpu().numpy(), recv_p[s].to(dev))
        return incoming


class Loopback:
    """All ranks in one process (for example several bricks groups on one device): the
    messages of one exchange round are handed over in memory."""

    def __init__(self, world: int):
        self.world = world

    def alltoall_all(self, outgoing_by_rank):
        """outgoing_by_rank[s][d] -> incoming_by_rank[d][s]."""
        return [[outgoing_by_rank[s][d] for s in range(self.world)] for d in range(self.world)]


def exchange_partials(foot, partial, height: int, transport):
    """One rank's side of the exchange: send the rows of its partials to each band owner
    and return what it received for its own band, as (FOOTPRINT array, payload)."""
    world, me = transport.world, transport.rank
    outgoing = [pack(foot, partial, *band_rows(height, world, d)) for d in range(world)]
    return unpack(transport.alltoall(outgoing))


def render_band(renderer, mode: str, transport, out=None):
    """Distributed sort-last render of camera 0 (exactly one camera set): this rank's
    bricks are its partition_bricks slab; returns (y0, y1, band image (y1 - y0, W, 4))."""
    import torch

    from . import vr_get_cube_info, vr_sortlast_fold, vr_sortlast_partials

    info = vr_get_cube_info(renderer.ctx)
    cam = renderer.cams[0]
    W, H = int(cam["width"]), int(cam["height"])
    world, me = transport.world, transport.rank
    mine = partition_bricks((info["nbx"], info["nby"], info["nbz"]), world)[me]
    dev = renderer.device
    foot, need = vr_sortlast_partials(renderer.ctx, mode, mine, device=dev)
    partial = torch.empty((max(need, 1), 4), dtype=torch.float32, device=f"cuda:{dev}")
    foot, _ = vr_sortlast_partials(renderer.ctx, mode, mine, partial, device=dev)
    torch.cuda.synchronize(dev)
    rfoot, rpay = exchange_partials(foot, partial, H, transport)
    y0, y1 = band_rows(H, world, me)
    if out is None:
        out = torch.empty((y1 - y0, W, 4), dtype=torch.float32, device=f"cuda:{dev}")
    rpay = rpay.to(f"cuda:{dev}")
    vr_sortlast_fold(renderer.ctx, mode, rpay, rfoot, y0, y1, out, device=dev)
    return y0, y1, out
