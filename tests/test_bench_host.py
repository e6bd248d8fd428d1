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


def test_algorithmic_budget_and_pipe_roofline():
    """The roofline arithmetic on made-up counts: the per-kernel split of the
    method's operations adds up to the whole, and the binding pipe is the one
    whose time at its peak is longest."""
    st = {"n_tent": 1000, "n_real": 400, "n_e_steps": 2000, "n_cross": 3000, "n_hard": 500,
          "n_particles": 300, "n_hist": 100}
    ost = {"n_compton": 70, "n_pe": 10, "n_rayleigh": 15, "n_pair": 5, "n_hard_el": 200,
           "n_hard_inel": 100, "n_hard_br": 20, "n_delta": 180}
    mix = bench.event_mix(ost)
    assert abs(sum(mix[k] for k in ("compton", "pe", "rayleigh", "pair")) - 1) < 1e-12
    assert abs(sum(mix[k] for k in ("hard_el", "hard_inel", "hard_br", "delta")) - 1) < 1e-12
    parts = [bench.algorithmic_ops(st, mix, k) for k in ("photon", "charged", "knock")]
    whole = bench.algorithmic_ops(st, mix, "all")
    extra = [st["n_particles"] * x for x in bench.ALGO_BUDGET["particle"]]
    for i in range(3):
        assert abs(sum(p[i] for p in parts) + extra[i] - whole[i]) < 1e-6 * whole[i]
    # a class II step draws two Philox blocks: 40 multiplies of the half-rate pipe
    assert bench.ALGO_BUDGET["e_step"][1] == 2 * bench.PHILOX[1]
    peaks = {"ffma": 4e13, "imad": 2e13, "lg2": 5e12}
    r = bench.pipe_roofline((4e13, 1e12, 1e11), 2.0, peaks)
    assert r["pipe"] == "issue" and abs(r["frac"] - (4e13 + 1e12 + 1e11) / 4e13 / 2.0) < 1e-12
    r = bench.pipe_roofline((1e12, 1e12, 1e13), 4.0, peaks)
    assert r["pipe"] == "sfu" and abs(r["frac"] - 0.5) < 1e-12
