"""Helpers that compare renderer output with the FP64 oracle, pixel by pixel.

A pixel passes if its max-abs RGBA error is within the tolerance against the
oracle's primary result, or -- for a ray the oracle flags as ambiguous (a first
or last sample, or the termination sample, within rounding of its threshold) --
against one of the oracle's alternative outcomes for that ray.
"""
import copy

import numpy as np

import oracle


def far_extent(scene, cam):
    """Largest coordinate magnitude (voxels) a sample of this view can have: the eye (or
    the orthographic image plane) and the cube."""
    return (max(abs(float(x)) for x in cam["eye"]) + max(abs(float(x)) for x in cam["win"]) +
            max(scene.nx, scene.ny, scene.nz))


def model_scene(scene, cam, mode, path):
    """The scene with the error model of the render path under test (the oracle's
    ambiguity windows follow from it): the image-order marcher ("auto" and "ray"
    composite) re-anchors every 12 samples; the other paths step in brick-local FP32
    (bound for 128^3 bricks, the largest edge used)."""
    sc = copy.copy(scene)
    far = far_extent(scene, cam)
    if mode == "composite" and path in ("auto", "ray"):
        sc.pos_err = oracle.pos_err_marcher(scene.step, far)
    else:
        sc.pos_err = oracle.pos_err_bricked(128, far)
    return sc


def compare(gpu_rgba, scene, cam, mode, pixels=None, tol=1e-4, gpu_max=None, max_tol=None,
            path="auto"):
    """gpu_rgba: (npix, 4) for the listed pixels (flat py*W+px; None = all), rendered by
    render path `path`.  Returns dict(max_err, n_flagged, n_variant, max_err_max)."""
    scene = model_scene(scene, cam, mode, path)
    ref = oracle.render(scene, cam, mode, pixels)
    g = np.asarray(gpu_rgba, dtype=np.float64).reshape(-1, 4)
    err = np.abs(g - ref["rgba"]).max(axis=1)
    bad = np.nonzero(err > tol)[0]
    n_variant = 0
    pix_all = np.arange(cam["width"] * cam["height"]) if pixels is None else np.asarray(pixels)
    for i in bad:
        fl = int(ref["flags"][i])
        best = err[i]
        if fl:
            for ds, dk0, dk1 in oracle.variants(fl):
                if (ds, dk0, dk1) == (0, 0, 0):
                    continue
                alt = oracle.render(scene, cam, mode, pix_all[i:i + 1], dstop=ds,
                                    dk0=dk0, dk1=dk1)
                best = min(best, float(np.abs(g[i] - alt["rgba"][0]).max()))
        if best > tol:
            raise AssertionError(
                f"pixel {int(pix_all[i])}: max abs error {best:.3e} > {tol:.1e} "
                f"(flags {fl}); gpu {g[i]}, oracle {ref['rgba'][i]}")
        err[i] = best
        n_variant += 1
    out = dict(max_err=float(err.max()) if err.size else 0.0,
               n_flagged=int(np.count_nonzero(ref["flags"])), n_variant=n_variant,
               nsamples=int(ref["nsamples"].sum()))
    if gpu_max is not None:
        gm = np.asarray(gpu_max, dtype=np.float64).reshape(-1)
        hit = ref["nsamples"] > 0
        assert np.all(np.isneginf(gm[~hit])), "MIP max must be -inf for rays without samples"
        d = np.abs(gm[hit] - ref["max"][hit])
        out["max_err_max"] = float(d.max()) if d.size else 0.0
        if max_tol is not None:
            assert out["max_err_max"] <= max_tol, out
    return out
