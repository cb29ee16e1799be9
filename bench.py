#!/usr/bin/env python
"""Benchmark of the ray-casting renderer on the survey workload.

Workload (one step = one frame of the orbit, rendered in both modes):
  1024 x 1024 x 2048 (RA x Dec x channel) synthetic HI-like cube -- noise sigma = 1,
  2000 seeded Gaussian sources, continuum ripple along the channel axis -- stored as
  FP16 bricks (128^3 + 1-voxel ghost), perspective 1920 x 1080, 36-frame orbit in 10 deg
  steps about the Dec axis, step 0.5 voxel; composite with early termination at alpha
  0.99 (image-order marcher) and MIP (object-order TMA-staged brick pass).
  The same frames are also timed on the plain FP32 store for comparison.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same workload
(bounded pixel samples per step) as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "samples/s & ms/frame vs plain FP32 path at stated RGBA error; % HBM roofline"
WORKLOAD = "survey"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=36)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", default="f16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile", choices=["mip", "composite", "both", "pyramid", "sortlast", "layered", "adjoint"],
                    default=None,
                    help="only render --warmup + --steps orbit frames (for ncu); no timing legs")
    ap.add_argument("--cube", default=None,
                    help="NX,NY,NZ: override the cube size (same source density) for small captures")
    ap.add_argument("--frame", type=int, default=None, help="with --profile: render this frame only")
    ap.add_argument("--ooc-full-mip", type=int, default=0,
                    help="render this many full-view MIP frames of the out-of-core cube (minutes each) and exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the wall / gradient / out-of-core measurements")
    return ap.parse_args()


def workload_config(storage, world):
    """The `config` of both arms' JSON lines.  The brick-store size follows the layout of
    vr_load_cube: 128^3 bricks with a 1-voxel ghost, rows padded to 16 bytes, 256-byte slots."""
    bpv = 2 if storage in ("f16", "bf16") else 4
    rows = 130
    pitch = -(-rows // (16 // bpv)) * (16 // bpv)
    slot = -(-(rows * rows * pitch * bpv) // 256) * 256
    store = slot * (1024 // 128) * (1024 // 128) * (2048 // 128)
    return {"workload": "survey 1024x1024x2048 HI-like cube (2000 sources + ripple), "
                        f"{storage} bricks 128^3+ghost, 1920x1080 perspective, "
                        "36-frame orbit, step 0.5, composite (ERT 0.99) + MIP per step",
            "storage": storage, "compute": "f32", "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 ({store / 1e9:.2f} GB store)"}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(times_ms, samples, world, device="cpu"):
    """Whole-job figures over the ranks: the maximum of each time (the slowest rank
    sets the job time) and the sum of the work.  world == 1 returns them unchanged."""
    if world <= 1:
        return list(times_ms), float(samples)
    import torch
    import torch.distributed as tdist
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    s = torch.tensor([float(samples)], dtype=torch.float64, device=device)
    tdist.all_reduce(s, op=tdist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], float(s.item())


def kernel_source_hash():
    """sha256 prefix of the brick pass's sources with comments and blank space removed, so
    that an edit of a comment does not orphan the committed counters."""
    import hashlib
    h = hashlib.sha256()
    for f in ("vr_brick.cu", "vr_device.cuh", "vr_ff.cuh", "vr_tma.cuh"):
        with open(os.path.join(ROOT, "paper_1012_2909_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_hash):
    """DRAM bytes per launch of the brick pass from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "k_brick_mip_survey_f16.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"kernel source hash:\s*([0-9a-f]+)", text)
    mt = re.search(r"dram bytes per launch \(full frame\):\s*([0-9.eE+]+)", text)
    if not mh or not mt or mh.group(1) != kernel_hash:
        return None
    return float(mt.group(1))


def load_touch_table():
    path = os.path.join(ROOT, "tests", "golden", "survey_touched_voxels.json")
    with open(path) as f:
        return json.load(f)


def oracle_sample(vol_rounded, tf, cam, pixels, cfg):
    """Time the FP64 oracle on the listed pixels, both modes; returns (samples, seconds, results)."""
    import oracle
    # the ambiguity windows of the composite follow the image-order marcher's error model
    far = max(abs(x) for x in cam["eye"]) + max(abs(x) for x in cam["win"]) + max(vol_rounded.shape)
    sc = oracle.Scene(vol_rounded, tf, -1.0, 20.0, cfg["step"], cfg["ert"],
                      pos_err=oracle.pos_err_marcher(cfg["step"], far))
    t0 = time.perf_counter()
    rc = oracle.render(sc, cam, "composite", pixels)
    rm = oracle.render(sc, cam, "mip", pixels)
    dt = time.perf_counter() - t0
    return int(rc["nsamples"].sum() + rm["nsamples"].sum()), dt, (rc, rm)


def summarise_extras(ex):
    """The few figures of the extra measurements that the headline is read with."""
    out = {}

    def pick(name, keys):
        d = ex.get(name) or {}
        v = {k: (round(d[k], 4) if isinstance(d.get(k), float) else d.get(k)) for k in keys if k in d}
        if "error" in d:
            v["error"] = str(d["error"])[:120]
        if v:
            out[name] = v

    pick("paths", ["composite_ray_ms", "composite_layered_ms", "composite_sortlast_ms", "mip_brick_ms",
                   "mip_ray_ms"])
    pick("wall", ["mip_batched_ms", "mip_25_single_ms", "mip_batching_speedup", "composite_batched_ms",
                  "composite_batching_speedup", "mip_speedup_vs_fp32_single", "composite_speedup_vs_fp32_single"])
    pick("diff", ["forward_ms", "backward_ms"])
    h = (ex.get("hipass") or {}).get("8000x8000") or {}
    if h:
        out["hipass_8000"] = {k: round(h[k], 3) for k in ("mip_ms", "composite_ms", "pyramid_tile0_ms")
                              if k in h}
    o = ex.get("ooc") or {}
    if o:
        out["ooc"] = {k: (round(o[k], 4) if isinstance(o[k], float) else o[k]) for k in o
                      if k in ("cold_frame_s", "warm_frame_s", "composite_orbit_s", "composite_orbit_generate_s",
                               "composite_orbit_floor_s", "mip_frame_s", "mip_bricks", "h2d_link_gbs",
                               "generate_gbs")}
    return out


def sample_pixels(W, H, n, seed):
    """n distinct seeded pixels (flat py*W+px) drawn uniformly over the image."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(W * H, size=min(n, W * H), replace=False))



def _events_ms(fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def path_times(r, cams, out):
    """ms per frame of every render path on the same frames: composite through the
    image-order marcher (ERT), sort-last partial images folded in visibility order and the
    layered carried state (both without termination); MIP through the brick pass and the
    marcher."""
    res = {"frames": len(cams)}
    for mode, paths in (("composite", ("ray", "sortlast", "layered")), ("mip", ("brick", "ray"))):
        for path in paths:
            r.set_path(path)
            tot = 0.0
            for cam in cams:
                r.set_camera(cam)
                r.render(mode, out=out)  # first render of a view: plans and scratch
                tot += _events_ms(lambda: r.render(mode, out=out), 2)
            res[f"{mode}_{path}_ms"] = tot / len(cams)
    r.set_path("auto")
    return res


def extra_wall(dev):
    """5 x 5 wall of 1920 x 1080 panels (25 off-axis frusta of one camera) on the
    2048 x 2048 x 1024 FP16 cube: batched (one graph launch per mode, autotuned)
    versus the 25 panels rendered one by one, on the FP16 store and on the plain
    FP32 store with default launch shapes."""
    import torch

    import paper_1012_2909_gb300 as vr
    import synth
    cfg = synth.CONFIGS["wall"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    W, H = cfg["image"]
    vol = synth.generate(p)
    r = vr.Renderer(dev, brick=128, step=cfg["step"], ert=cfg["ert"])
    r.load_cube(vol, "f16")
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    big = synth.orbit_view(dims, 30.0, 5 * W, 5 * H)
    panels = synth.wall_views(big, 5, 5)
    out = {}
    counter = torch.zeros(1, dtype=torch.int64, device=f"cuda:{dev}")
    r.set_camera(panels)
    r.set_path("ray")
    vr.vr_set_sample_counter(r.ctx, counter)
    for mode in ("composite", "mip"):
        counter.zero_()
        r.render(mode)
        torch.cuda.synchronize()
        out[f"{mode}_samples"] = int(counter.item())
    vr.vr_set_sample_counter(r.ctx, None)
    r.set_path("auto")
    tune = {m: vr.autotune(r, m, reps=2) for m in ("composite", "mip")}
    img = torch.empty((25, H, W, 4), device=f"cuda:{dev}")
    vr.vr_set_graph(r.ctx, True)
    for mode in ("composite", "mip"):
        out[f"{mode}_batched_ms"] = _events_ms(lambda: r.render(mode, out=img), 3)
    vr.vr_set_graph(r.ctx, False)
    one = torch.empty((1, H, W, 4), device=f"cuda:{dev}")
    for mode in ("composite", "mip"):
        def singles():
            for c in panels:
                r.set_camera(c)
                r.render(mode, out=one)
        out[f"{mode}_25_single_ms"] = _events_ms(singles, 1)
        r.set_camera(panels)
    for mode in ("composite", "mip"):
        out[f"{mode}_samples_per_s"] = out[f"{mode}_samples"] / (out[f"{mode}_batched_ms"] / 1e3)
        out[f"{mode}_batching_speedup"] = out[f"{mode}_25_single_ms"] / out[f"{mode}_batched_ms"]
    out["tuning"] = {m: {k: v for k, v in t.items() if k != "cached"} for m, t in tune.items()}
    r.close()
    # the plain FP32 single-view path on the same panels
    r = vr.Renderer(dev, brick=128, step=cfg["step"], ert=cfg["ert"])
    r.load_cube(vol, "f32")
    del vol
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    for mode in ("composite", "mip"):
        def singles32():
            for c in panels:
                r.set_camera(c)
                r.render(mode, out=one)
        singles32()  # first use allocates the per-pixel scratch
        out[f"{mode}_fp32_25_single_ms"] = _events_ms(singles32, 1)
        out[f"{mode}_speedup_vs_fp32_single"] = out[f"{mode}_fp32_25_single_ms"] / out[f"{mode}_batched_ms"]
    r.close()
    out["workload"] = ("2048x2048x1024 FP16, 25 x 1920x1080 off-axis frusta (9600x5400), graph mode; "
                       "baseline: FP32 store, one panel per render, default launch shapes")
    return out


def _measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("hbm_gbs", 6800.0))
    except OSError:
        return 6800.0


def extra_hipass(dev):
    """High-resolution static render (one orientation) of the paper's HIPASS-shaped cube,
    1721 x 1721 x 1025 FP32, at 3000 x 3000 and 8000 x 8000: MIP (brick pass) and
    composite (image order, termination 0.99)."""
    import torch

    import paper_1012_2909_gb300 as vr
    import synth
    cfg = synth.CONFIGS["hipass"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    vol = synth.generate(p)
    r = vr.Renderer(dev, brick=128, step=cfg["step"], ert=cfg["ert"])
    r.load_cube(vol, "f32")
    del vol
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    counter = torch.zeros(1, dtype=torch.int64, device=f"cuda:{dev}")
    out = {"workload": "1721x1721x1025 FP32 (HIPASS shape, 2830 sources + ripple), perspective, "
                       "one orientation, step 0.5"}
    for W, H in cfg["images"]:
        r.set_camera(synth.orbit_view(dims, cfg["az"], W, H))
        img = torch.empty((1, H, W, 4), device=f"cuda:{dev}")
        res = {}
        for mode in ("composite", "mip"):
            r.set_path("ray")
            vr.vr_set_sample_counter(r.ctx, counter)
            counter.zero_()
            r.render(mode, out=img)
            torch.cuda.synchronize()
            n = int(counter.item())
            vr.vr_set_sample_counter(r.ctx, None)
            r.set_path("auto")
            r.render(mode, out=img)
            ms = _events_ms(lambda: r.render(mode, out=img), 3)
            res[f"{mode}_ms"] = ms
            res[f"{mode}_samples"] = n
            res[f"{mode}_samples_per_s"] = n / (ms / 1e3)
        if W * H >= 64_000_000:
            # pyramid of the composite render: HBM-bound; algorithmic bytes = level 0 read once
            # plus every level written once (edge-tile padding not counted)
            r.render("composite", out=img)
            lw, lh, written = W, H, 0
            while lw > 1 or lh > 1:
                lw, lh = (lw + 1) // 2, (lh + 1) // 2
                written += lw * lh
            alg = 16 * (W * H + written)
            peak = _measured_peak()
            for tile in (0, 256):
                pyr = r.pyramid(img[0], tile)
                ms = _events_ms(lambda: r.pyramid(img[0], tile, out=pyr), 5)
                res[f"pyramid_tile{tile}_ms"] = ms
                res[f"pyramid_tile{tile}_gbs"] = alg / (ms / 1e3) / 1e9
                res[f"pyramid_tile{tile}_frac_of_measured_hbm"] = alg / (ms / 1e3) / 1e9 / peak
                del pyr
            res["pyramid_algorithmic_bytes"] = alg
            # catalogue overlay: the sources' bounding cubes as wireframes over the render
            import numpy as np
            boxes = synth.catalogue(p)
            cols = np.random.default_rng(2830).random((len(boxes), 4)).astype(np.float32)
            r.overlay(img, boxes, cols)  # first use allocates the scratch
            res["overlay_ms"] = _events_ms(lambda: r.overlay(img, boxes, cols), 5)
            res["overlay_boxes"] = len(boxes)
        out[f"{W}x{H}"] = res
        del img
    r.close()
    return out


def extra_diff(dev):
    """Gradient workload: 256^3 FP32 (noise + 50 sources), 64 seeded views at 512^2,
    L2 loss against images of a hidden table; forward + adjoint per step."""
    import torch

    import paper_1012_2909_gb300 as vr
    import synth
    cfg = synth.CONFIGS["diff"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    vol = synth.generate(p)
    views = synth.random_views(dims, cfg["views"], seed=cfg["view_seed"], width=512, height=512)
    r = vr.Renderer(dev, brick=128, step=cfg["step"], ert=cfg["ert"])
    r.load_cube(vol, "f32")
    r.set_camera(views)
    r.set_transfer_function(synth.hidden_tf(cfg["tf_seed"]), -1.0, 20.0)
    target = r.render("composite").clone()
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    dtf = torch.empty((256, 4), device=f"cuda:{dev}")
    dvol = torch.empty(vol.shape, device=f"cuda:{dev}")
    img = torch.empty_like(target)

    def step():
        r.render("composite", out=img)
        dimg = 2.0 * (img - target) / img.numel()
        vr.vr_render_backward(r.ctx, "composite", dimg, dtf, dvol)

    step()
    fwd = _events_ms(lambda: r.render("composite", out=img), 3)
    both = _events_ms(step, 3)
    r.close()
    return {"workload": "256^3 FP32, 64 views 512x512, L2 loss, forward + adjoint (table + voxels)",
            "forward_ms": fwd, "step_ms": both, "backward_ms": both - fwd}


def extra_ooc(dev, cache_gib=32, frames=10):
    """Out-of-core: 4096 x 4096 x 8192 FP16 cube (256 GiB) produced brick by brick from the
    generator into page-locked memory and streamed to a 32 GiB HBM cache.

    * composite: the 10-frame orbit (10 deg steps) at 1920 x 1080; a frame fetches only
      the bricks in front of terminated rays that are not cached yet;
    * MIP: every brick a ray crosses is needed (about 275 GB a frame at full view), so the
      MIP frames cover a bounded share of the cube, labelled: the central panel of a
      20 x 20 split of the same view (1/400 of the image, all depths), at 1920 x 1080, for
      the first 2 orbit positions.

    Per frame the stages are reported apart: host generation (time inside the region
    callback), the host-to-device link (the bytes copied and their floor at the measured
    pinned copy rate), the host's waits on the device, and the rest; the frame's floor is
    its largest stage."""
    import synth
    r, frame, dims, W, H, h2d_gbs = _ooc_session(dev, cache_gib)
    cams = synth.orbit(dims, frames, 10.0, W, H)
    comp = [frame(c, "composite") for c in cams]
    warm = frame(cams[-1], "composite")  # the last view again: everything cached
    mip = []
    for c in cams[:2]:
        big = dict(c, width=W * 20, height=H * 20)
        mip.append(frame(synth.wall_views(big, 20, 20)[210], "mip"))  # panel (10, 10) of 20 x 20
    r.close()
    tot = lambda xs, k: sum(x[k] for x in xs)  # noqa: E731
    return {"workload": "4096x4096x8192 FP16 (256 GiB) streamed from the generator, 32 GiB cache, 1920x1080; "
                        f"composite: {frames}-frame orbit (10 deg steps); MIP: central 1/400 panel of the "
                        "view (bounded share of the cube), 2 orbit positions",
            "h2d_link_gbs": h2d_gbs,
            "composite_frames": comp, "composite_warm_repeat": warm, "mip_frames": mip,
            "composite_orbit_s": tot(comp, "wall_s"), "composite_orbit_generate_s": tot(comp, "generate_s"),
            "composite_orbit_floor_s": tot(comp, "floor_s"),
            "mip_frame_s": [m["wall_s"] for m in mip], "mip_bricks": [m["bricks_fetched"] for m in mip],
            "cold_frame_s": comp[0]["wall_s"], "warm_frame_s": warm["wall_s"],
            "generate_gbs": tot(comp, "h2d_gb") / max(tot(comp, "generate_s"), 1e-9)}


def run_ooc_full_mip(a):
    """Full-view MIP frames of the out-of-core cube (every brick a ray crosses, about
    275 GB of FP16 a frame, produced by the generator): minutes a frame, so a separate
    run, not a bench extra.  Prints one JSON line with the stages of every frame."""
    import synth
    r, frame, dims, W, H, h2d_gbs = _ooc_session(0, 32)
    cams = synth.orbit(dims, max(a.ooc_full_mip, 1), 10.0, W, H)
    out = [frame(c, "mip") for c in cams]
    r.close()
    print(json.dumps({"ooc_full_mip": {"workload": "4096x4096x8192 FP16 (256 GiB) streamed from the generator, "
                                                   "32 GiB cache, 1920x1080 full view, orbit positions 10 deg apart",
                                       "h2d_link_gbs": h2d_gbs, "frames": out}}), flush=True)


def _ooc_session(dev, cache_gib):
    """The out-of-core cube loaded through the generator's region callback, with the
    measured pinned host-to-device rate and a frame timer that separates the stages."""
    import torch

    import paper_1012_2909_gb300 as vr
    import synth
    cfg = synth.CONFIGS["ooc"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    # the host-to-device link: one pinned 1 GiB buffer copied a few times
    host = torch.empty(1 << 28, dtype=torch.float32, pin_memory=True)
    devb = torch.empty(1 << 28, dtype=torch.float32, device=f"cuda:{dev}")
    h2d_ms = _events_ms(lambda: devb.copy_(host, non_blocking=True), 4)
    h2d_gbs = host.numel() * 4 / (h2d_ms / 1e3) / 1e9
    del host, devb
    torch.cuda.empty_cache()
    r = vr.Renderer(dev, brick=128, step=cfg["step"], ert=cfg["ert"])
    fn, user = synth.region_callback(p)
    r.region_user = user  # the callback reads it at every render: keep it alive with the renderer
    vr.vr_load_cube_streamed(r.ctx, fn, user, dims, "f16", cache_bytes=cache_gib << 30)
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    W, H = cfg["image"]

    def frame(cam, mode):
        r.set_camera(cam)
        st0 = vr.vr_get_stream_stats(r.ctx)
        t0 = time.time()
        r.render(mode)
        torch.cuda.synchronize()
        wall = time.time() - t0
        st = vr.vr_get_stream_stats(r.ctx)
        d = {k: st[k] - st0[k] for k in ("bricks_fetched", "bricks_culled", "bytes_h2d", "batches",
                                         "generate_s", "wait_s")}
        link = d["bytes_h2d"] / 1e9 / h2d_gbs
        stages = {"generate_s": d["generate_s"], "link_floor_s": link, "device_wait_s": d["wait_s"],
                  "other_s": max(0.0, wall - d["generate_s"] - d["wait_s"])}
        return {"wall_s": wall, "bricks_fetched": d["bricks_fetched"], "bricks_culled": d["bricks_culled"],
                "batches": d["batches"], "h2d_gb": d["bytes_h2d"] / 1e9, **stages,
                "floor_s": max(stages["generate_s"], link), "wall_over_floor": wall / max(1e-9, max(
                    stages["generate_s"], link))}

    return r, frame, dims, W, H, h2d_gbs


# ------------------------------------------------------------------------------ our arm
def run_ours(a):
    import numpy as np
    import torch

    import paper_1012_2909_gb300 as vr
    import synth

    rank, local, world = dist_env()
    dev = local
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    cfg = synth.CONFIGS[WORKLOAD]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    W, H = cfg["image"]
    tf = synth.viridis_ramp_tf()
    cams = synth.orbit(dims, cfg["frames"])
    t0 = time.time()
    vol = synth.generate(p)
    gen_s = time.time() - t0

    def make(storage):
        r = vr.Renderer(dev, brick=128, step=cfg["step"], ert=cfg["ert"])
        r.load_cube(vol, storage)
        r.set_transfer_function(tf, -1.0, 20.0)
        return r

    rq = make(a.storage)
    r32 = make("f32")
    info = rq.cube_info()
    torch.cuda.synchronize()

    # executed samples per frame and mode (deterministic; counted once, untimed)
    counter = torch.zeros(1, dtype=torch.int64, device=f"cuda:{dev}")
    nsamp = {"composite": [], "mip": []}
    rq.set_path("ray")
    vr.vr_set_sample_counter(rq.ctx, counter)
    for c in cams:
        rq.set_camera(c)
        for mode in ("composite", "mip"):
            counter.zero_()
            rq.render(mode)
            torch.cuda.synchronize()
            nsamp[mode].append(int(counter.item()))
    vr.vr_set_sample_counter(rq.ctx, None)
    rq.set_path("auto")

    out_c = torch.empty((1, H, W, 4), device=f"cuda:{dev}")
    out_m = torch.empty((1, H, W, 4), device=f"cuda:{dev}")
    max_m = torch.empty((1, H, W), device=f"cuda:{dev}")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(a.steps)]

    def step(r, i, kernel_events=None, bufs=None):
        f = i % len(cams)
        oc, om, mm = bufs if bufs is not None else (out_c, out_m, max_m)
        r.set_camera(cams[f])
        r.render("composite", out=oc)
        if kernel_events is not None:
            vr.vr_set_kernel_events(r.ctx, *kernel_events)
        r.render("mip", out=om, out_max=mm, with_max=True)
        if kernel_events is not None:
            vr.vr_set_kernel_events(r.ctx, None, None)
        return nsamp["composite"][f] + nsamp["mip"][f]

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    def timed(r, kernel=False):
        for i in range(a.warmup):
            step(r, i)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        samples = 0
        ev[0].record()
        for i in range(a.steps):
            samples += step(r, i, kev[i] if kernel else None)
        ev[1].record()
        torch.cuda.synchronize()
        barrier()
        ms = ev[0].elapsed_time(ev[1])
        return ms, samples

    with ClockSampler(dev) as clk:
        ms, samples = timed(rq, kernel=True)
    clocks = clk.summary()
    kernel_ms = [kev[i][0].elapsed_time(kev[i][1]) for i in range(a.steps)]
    ms32, samples32 = timed(r32)

    # max over ranks of the times, sum of the samples
    (ms, ms32), total_samples = aggregate([ms, ms32], samples, world, f"cuda:{dev}")

    # end to end through the public API: camera from the host in, both images out to
    # pinned host memory, every step.  Double-buffered as an application would run it:
    # step i renders into buffer set i % 2 while a copy stream reads step i - 1 back.
    bufs = [(torch.empty_like(out_c), torch.empty_like(out_m), torch.empty_like(max_m)) for _ in range(2)]
    hosts = [(torch.empty((1, H, W, 4), pin_memory=True), torch.empty((1, H, W, 4), pin_memory=True))
             for _ in range(2)]
    cstream = torch.cuda.Stream()
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    main = torch.cuda.current_stream()

    def e2e_step(i):
        b = i % 2
        if i >= 2:
            main.wait_event(copied[b])  # the read-back of step i - 2 has left buffer set b
        n = step(rq, i, bufs=bufs[b])
        rendered[b].record(main)
        with torch.cuda.stream(cstream):
            cstream.wait_event(rendered[b])
            hosts[b][0].copy_(bufs[b][0], non_blocking=True)
            hosts[b][1].copy_(bufs[b][1], non_blocking=True)
            copied[b].record(cstream)
        return n

    for i in range(a.warmup):
        e2e_step(i)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    esamples = 0
    for i in range(a.steps):
        esamples += e2e_step(i)
    for b in range(2):
        main.wait_event(copied[b])  # every read-back is inside the timed region
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    (e2e_ms,), _ = aggregate([e2e_ms], 0, world, f"cuda:{dev}")

    # roofline of the dominant kernel (the MIP brick pass)
    touch = load_touch_table()
    bpv = 2 if a.storage in ("f16", "bf16") else 4
    frames = [i % len(cams) for i in range(a.steps)]
    alg_bytes = [touch["mip"][f] * bpv for f in frames]
    avg_kernel_s = statistics.mean(kernel_ms) / 1e3
    achieved = statistics.mean(alg_bytes) / avg_kernel_s / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    khash = kernel_source_hash()
    traffic = profiled_traffic(khash)

    mip_ms = statistics.mean(kernel_ms)
    res = {
        "metric": METRIC,
        "value": total_samples / (ms / 1e3),
        "unit": "samples/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{a.storage} storage, f32 arithmetic",
        "storage_dtype": a.storage,
        "data": "synthetic",
        "config": workload_config(a.storage, world),
        "ms_per_frame": {"composite": None, "mip_brick_kernel": mip_ms},
        "rays_per_s": W * H * 2 * a.steps / (ms / 1e3) * world,
        "fp32_path": {"ms_per_step": ms32 / a.steps,
                      "samples_per_s": samples32 / (ms32 / 1e3),
                      "speedup_of_storage_path": ms32 / ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_brick_mip", "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                     "algorithmic_bytes_per_launch": statistics.mean(alg_bytes),
                     "kernel_source_hash": khash},
        "e2e": {"value": total_samples / (e2e_ms / 1e3) if world == 1 else
                float(esamples) * world / (e2e_ms / 1e3),
                "unit": "samples/s", "h2d_bytes_per_step": 144,
                "d2h_bytes_per_step": 2 * H * W * 4 * 4},
        # per step: k_march (composite); k_pixel_setup, k_cell_list, k_brick_mip,
        # k_mip_finalize (MIP)
        "gpu_launches": 5 * a.steps,
        "clocks": clocks,
        "generation_s": gen_s,
    }

    # CPU baseline: the oracle on a bounded pixel sample of frame 0, rank 0 at N = 1
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        vol_r = oracle.round_storage(vol, a.storage)
        del vol
        cam = cams[0]
        pix = sample_pixels(W, H, 1024, seed=5)
        s0, t0_, _ = oracle_sample(vol_r, tf, cam, pix, cfg)
        npx = int(min(W * H, max(1024, 1024 * a.cpu_seconds / max(t0_, 1e-3))))
        pix = sample_pixels(W, H, npx, seed=6)
        s1, t1, (rc, rm) = oracle_sample(vol_r, tf, cam, pix, cfg)
        # parity of the timed frame on the same pixels
        rq.set_camera(cam)
        oc = rq.render("composite")
        om = rq.render("mip")
        torch.cuda.synchronize()
        gc = oc[0].cpu().numpy().reshape(-1, 4)[pix]
        gm = om[0].cpu().numpy().reshape(-1, 4)[pix]
        ec = np.abs(gc - rc["rgba"]).max(axis=1)
        em = np.abs(gm - rm["rgba"]).max(axis=1)
        flagged = rc["flags"] != 0
        res["cpu_baseline"] = {"value": s1 / t1, "unit": "samples/s", "cores": os.cpu_count(),
                               "kind": "oracle",
                               "sample": f"{len(pix)} seeded pixels of orbit frame 0, "
                                         f"composite + MIP, FP64, {t1:.1f} s"}
        res["rgba_max_abs_err"] = {"composite_unflagged": float(ec[~flagged].max()),
                                   "composite_flagged_rays": int(flagged.sum()),
                                   "mip": float(em.max()), "pixels": int(len(pix)),
                                   "reference": "FP64 oracle on the rounded cube",
                                   "tolerance": 2e-3 if a.storage != "f32" else 1e-4}
    # per-mode frame time (composite) from one extra timed pass over every orbit frame
    # (its cost varies about 3.5x around the orbit with the cube's projected area)
    tot = 0.0
    for cam in cams:
        rq.set_camera(cam)
        rq.render("composite", out=out_c)
        e0.record()
        rq.render("composite", out=out_c)
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    res["ms_per_frame"]["composite"] = tot / len(cams)
    if rank == 0 and not a.no_extras:
        res["extras"] = {}
        t0 = time.time()
        res["extras"]["paths"] = path_times(rq, cams[::6], out_c)
        res["extras"]["paths"]["wall_s"] = time.time() - t0
        del rq, r32
        torch.cuda.empty_cache()
        for name, fn in (("wall", extra_wall), ("hipass", extra_hipass), ("diff", extra_diff),
                         ("ooc", extra_ooc)):
            t0 = time.time()
            try:
                res["extras"][name] = fn(dev)
            except Exception as exc:  # report, do not lose the main line
                res["extras"][name] = {"error": f"{type(exc).__name__}: {exc}"}
            res["extras"][name]["wall_s"] = time.time() - t0
            torch.cuda.empty_cache()
    if rank == 0:
        # the detailed extras go on a line of their own (no "metric" key) before the
        # result line, and the result line carries a short summary of them, so that the
        # result line stays short enough to be kept whole
        extras = res.pop("extras", None)
        if extras is not None:
            print(json.dumps({"extras": extras}), flush=True)
            res["extras_summary"] = summarise_extras(extras)
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


# ------------------------------------------------------------------------ reference arm
def run_reference(a):
    import numpy as np

    import oracle
    import synth

    rank, _, world = dist_env()
    if rank != 0:
        return
    cfg = synth.CONFIGS[WORKLOAD]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    tf = synth.viridis_ramp_tf()
    cams = synth.orbit(dims, cfg["frames"])
    vol = oracle.round_storage(synth.generate(p), a.storage)
    sc = oracle.Scene(vol, tf, -1.0, 20.0, cfg["step"], cfg["ert"])
    rng = np.random.default_rng(3)
    W, H = cfg["image"]
    npix = 16384  # per step: large enough that thread start-up does not dominate the oracle's time

    def one(i):
        cam = cams[i % len(cams)]
        # seeded pixels in the central band of the image, where the cube projects
        xs = rng.integers(W // 4, 3 * W // 4, npix)
        ys = rng.integers(H // 8, 7 * H // 8, npix)
        pix = np.unique(ys * W + xs)
        rc = oracle.render(sc, cam, "composite", pix)
        rm = oracle.render(sc, cam, "mip", pix)
        return int(rc["nsamples"].sum() + rm["nsamples"].sum())

    for i in range(a.warmup):
        one(i)
    t0 = time.perf_counter()
    samples = sum(one(i) for i in range(a.steps))
    dt = time.perf_counter() - t0
    v = samples / dt
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s",
           "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": dt * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(a.storage, world),
           "cpu_baseline": {"value": v, "unit": "samples/s", "cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": f"{npix} seeded pixels per step (central band), "
                                      "composite + MIP, FP64"},
           "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_profile(a):
    """Render frames of the workload and nothing else, so that a profiler sees only the
    renderer's kernels (used by the commands in profiles/)."""
    import torch

    import paper_1012_2909_gb300 as vr
    import synth

    if a.profile == "pyramid":
        # pyramid of a seeded 8000 x 8000 premultiplied image (the size of the paper-scale
        # static render), row-major levels, warm-up passes then timed passes
        g = torch.Generator(device="cuda").manual_seed(8000)
        img = torch.rand((8000, 8000, 4), device="cuda", generator=g)
        r = vr.Renderer(0)
        out = r.pyramid(img)
        for _ in range(a.warmup):
            r.pyramid(img, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.steps):
            r.pyramid(img, out=out)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile": "pyramid", "image": [8000, 8000],
                          "ms_per_pyramid": e0.elapsed_time(e1) / max(a.steps, 1)}))
        r.close()
        return

    if a.profile == "adjoint":
        # forward + adjoint of the gradient workload (256^3 FP32, L2 loss against a hidden
        # table's images), 8 of its 64 views at 512 x 512 per step
        dcfg = synth.CONFIGS["diff"]
        pd = dcfg["cube"]
        ddims = (pd["nx"], pd["ny"], pd["nz"])
        vol = synth.generate(pd)
        views = synth.random_views(ddims, 8, seed=dcfg["view_seed"], width=512, height=512)
        r = vr.Renderer(0, brick=128, step=dcfg["step"], ert=dcfg["ert"])
        r.load_cube(vol, "f32")
        r.set_camera(views)
        r.set_transfer_function(synth.hidden_tf(dcfg["tf_seed"]), -1.0, 20.0)
        target = r.render("composite").clone()
        r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
        dtf = torch.empty((256, 4), device="cuda")
        dvol = torch.empty(vol.shape, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(a.warmup + a.steps):
            if i == a.warmup:
                torch.cuda.synchronize()
                e0.record()
            img = r.render("composite")
            dimg = (2.0 * (img - target) / img.numel()).contiguous()
            vr.vr_render_backward(r.ctx, "composite", dimg, dtf, dvol)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile": "adjoint", "cube": ddims, "views": len(views),
                          "ms_per_step": e0.elapsed_time(e1) / max(a.steps, 1)}))
        r.close()
        return

    cfg = synth.CONFIGS[WORKLOAD]
    p = dict(cfg["cube"])
    if a.cube:
        nx, ny, nz = (int(v) for v in a.cube.split(","))
        scale = nx * ny * nz / (p["nx"] * p["ny"] * p["nz"])
        p.update(nx=nx, ny=ny, nz=nz, nsrc=max(1, int(round(p["nsrc"] * scale))))
    dims = (p["nx"], p["ny"], p["nz"])
    vol = synth.generate(p)
    r = vr.Renderer(0, brick=128, step=cfg["step"], ert=cfg["ert"])
    r.load_cube(vol, a.storage)
    del vol
    r.set_transfer_function(synth.viridis_ramp_tf(), -1.0, 20.0)
    cams = synth.orbit(dims, cfg["frames"])
    modes = ["composite", "mip"] if a.profile == "both" else [a.profile]
    if a.profile in ("sortlast", "layered"):  # the object-order composite paths
        r.set_path(a.profile)
        modes = ["composite"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = a.warmup + a.steps
    for i in range(n):
        if i == a.warmup:
            torch.cuda.synchronize()
            e0.record()
        r.set_camera(cams[a.frame if a.frame is not None else i % len(cams)])
        for m in modes:
            r.render(m)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile": a.profile, "cube": dims, "storage": a.storage, "frames": a.steps,
                      "ms_per_frame": e0.elapsed_time(e1) / max(a.steps, 1)}))
    r.close()


def main():
    a = parse()
    if a.ooc_full_mip:
        run_ooc_full_mip(a)
        return
    if a.profile:
        run_profile(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
