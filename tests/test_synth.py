"""The input generator's contract (CPU): any region equals the same voxels of the whole
cube, whatever its offsets (the noise of voxels 2m and 2m + 1 comes from one
Box-Muller pair, so a region may start or end inside a pair), and the noise is unit
Gaussian with the two members of a pair uncorrelated."""
import numpy as np
import pytest

import synth


def test_regions_equal_slices_of_the_whole_cube():
    # odd nx: rows start alternately on the first and the second voxel of a pair
    p = synth.cube_params(37, 20, 9, seed=77, nsrc=6, ripple=True, ripple_period=8.0)
    whole = synth.generate(p)
    one = synth.generate(p, nthreads=1)
    assert np.array_equal(whole, one)
    for x0 in (0, 1, 2, 5, 35, 36):
        for sx in (1, 2, 3, 37 - x0):
            if x0 + sx > 37:
                continue
            for (y0, sy, z0, sz) in ((0, 20, 0, 9), (3, 5, 4, 2), (19, 1, 8, 1)):
                reg = synth.generate(p, region=(x0, y0, z0, sx, sy, sz))
                assert np.array_equal(reg, whole[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx]), (x0, sx, y0, z0)


def test_noise_is_unit_gaussian_and_pairs_are_uncorrelated():
    p = synth.cube_params(64, 64, 64, seed=5, nsrc=0)
    v = synth.generate(p).astype(np.float64).reshape(-1)
    n = v.size
    assert abs(v.mean()) < 5.0 / np.sqrt(n)
    assert abs(v.std() - 1.0) < 5.0 / np.sqrt(2 * n)
    # fourth moment of a unit normal is 3
    assert abs(np.mean(v ** 4) - 3.0) < 0.05
    even, odd = v[0::2], v[1::2]
    r = np.corrcoef(even, odd)[0, 1]
    assert abs(r) < 5.0 / np.sqrt(n // 2)
    # tail mass beyond 3 sigma: 0.27 % for a unit normal
    tail = np.mean(np.abs(v) > 3.0)
    assert tail == pytest.approx(0.0027, rel=0.15)
