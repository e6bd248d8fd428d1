"""Host helpers of bench.py (no GPU): the 1 % uncertainty statistic and the
bremsstrahlung-tail statistic of the variance-reduction line."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_rel_uncertainty_selects_high_dose_voxels():
    d = np.array([1.0, 0.6, 0.4, 0.0])
    v = np.array([0.01, 0.0036, 1.0, 0.0]) * 1e-2
    # voxels >= 50 % of max: the first two, relative sigma 0.01 and 0.01
    assert abs(bench.rel_uncertainty(d, v, 0.5) - 0.01) < 1e-12


def test_tail_uncertainty_takes_the_slabs_beyond_the_peak():
    nz, nxy = 10, 4
    prof = np.array([0.5, 1.0, 0.8, 0.3, 0.005, 0.0008, 0.0007, 0.0006, 0.0005, 0.0])
    d = np.repeat(prof[:, None] / nxy, nxy, axis=1).ravel()
    rel = np.where(np.repeat(prof[:, None], nxy, axis=1).ravel() < 1e-3, 0.2, 0.01)
    v = (rel * d) ** 2
    U, n = bench.tail_uncertainty(d, v, nz)
    # tail from slab 5 (the first below 0.1 % of the peak) on; slab 9 has no
    # dose, the others are >= 10 % of the tail maximum
    assert n == 4 * nxy
    assert abs(U - 0.2) < 1e-12
