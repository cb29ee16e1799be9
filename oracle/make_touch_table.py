"""Write tests/golden/survey_touched_voxels.json with the oracle's touched-voxel census.

For every frame of the survey workload's 36-frame orbit (1024 x 1024 x 2048 cube,
1920 x 1080 perspective, step 0.5) it counts the voxels that the executed samples
read (the 8 clamped trilinear corners of each sample):

* MIP: every sample of every ray is executed, so the count depends on geometry only;
* composite: samples stop at termination (alpha 0.99), so the count depends on the
  cube values; they are taken on the seeded cube as float16-rounded storage.

These counts times the bytes per stored voxel are the algorithmic bytes of one
frame.  Run:  python oracle/make_touch_table.py [--frames N]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "survey_touched_voxels.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=36)
    ap.add_argument("--composite", action="store_true", help="also count composite frames")
    a = ap.parse_args()
    cfg = synth.CONFIGS["survey"]
    p = cfg["cube"]
    dims = (p["nx"], p["ny"], p["nz"])
    tf = synth.viridis_ramp_tf()
    cams = synth.orbit(dims, a.frames)
    res = {"workload": "survey 1024x1024x2048, 1920x1080 perspective orbit, 10 deg steps, step 0.5",
           "source": "oracle.touched (8 clamped trilinear corners of every executed sample)",
           "mip": [], "composite": []}
    zeros = np.zeros((p["nz"], p["ny"], p["nx"]), np.float32)
    sc = oracle.Scene(zeros, tf, -1.0, 20.0, cfg["step"], cfg["ert"])
    for i, c in enumerate(cams):
        t = time.time()
        m = oracle.touched(sc, c, "mip")
        res["mip"].append(int(np.count_nonzero(m)))
        del m
        print(f"frame {i} mip {res['mip'][-1]} ({time.time() - t:.1f}s)", flush=True)
    if a.composite:
        vol = oracle.round_storage(synth.generate(p), "f16")
        sc = oracle.Scene(vol, tf, -1.0, 20.0, cfg["step"], cfg["ert"])
        for i, c in enumerate(cams):
            m = oracle.touched(sc, c, "composite")
            res["composite"].append(int(np.count_nonzero(m)))
            del m
            print(f"frame {i} composite {res['composite'][-1]}", flush=True)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
