"""Pins of the oracle's variance reduction (interaction forcing of hard
inelastic collisions and hard bremsstrahlung, bremsstrahlung photon
splitting), each against the analog simulation it must reproduce:

* splitting alone with photons absorbed where they are made: the n copies of
  weight 1/n deposit exactly what the one analog photon deposits, so the dose
  equals the analog dose to rounding, and every history closes its ledger;
* a forcing window that excludes every particle changes nothing (bit for bit);
* forcing + splitting on a 1 MeV electron beam with photons tracked: the dose
  agrees with the analog dose (permutation gate on batch doses), and the
  energy ledger closes in expectation. Dropping the 1/F weight of a forced
  secondary, or letting the particle always take the forced loss, moves the
  dose by many sigma (the forced events outnumber the analog ones F to 1).
"""
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from parity import permutation_gate

NTH = max(1, min(16, os.cpu_count() or 1))


def beam(eabs_g):
    ph = S.water_cube(16, 0.05)
    src = S.Source(S.ELECTRON, 0, 0.425, 0.425, 0, 0, 1.0)
    return ph, src, S.Transport(eabs_g=eabs_g, eabs_e=0.02, wcc=0.005, wcr=0.005)


def test_splitting_alone_equals_analog_when_photons_are_absorbed():
    ph, src, tp = beam(eabs_g=1e3)
    a = O.run(ph, src, tp, 400, seed=4, n_batches=4)
    b = O.run(ph, src, tp, 400, seed=4, n_batches=4, vr=S.VR(n_split_brems=4))
    assert a.stats["n_hard_br"] > 20
    np.testing.assert_allclose(b.sum_q, a.sum_q, rtol=1e-12, atol=1e-15)
    assert b.stats["max_ledger_rel"] < 1e-9
    assert b.stats["n_e_steps"] == a.stats["n_e_steps"]


def test_forcing_outside_its_window_changes_nothing():
    ph, src, tp = beam(eabs_g=1e-3)
    a = O.run(ph, src, tp, 300, seed=6, n_batches=4)
    b = O.run(ph, src, tp, 300, seed=6, n_batches=4,
              vr=S.VR(f_inel=7.0, f_brems=50.0, w_lo=1.5, w_hi=2.0))
    np.testing.assert_array_equal(b.sum_q, a.sum_q)
    assert b.stats["n_hard_inel"] == a.stats["n_hard_inel"]


def _forced_case(args):
    vr, seed, k0, K, n = args
    ph, src, tp = beam(eabs_g=1e-3)
    out = []
    for k in range(k0, k0 + K):
        r = O.run(ph, src, tp, n, seed=seed, first_hist=k * n, n_batches=1, vr=vr)
        st = r.stats
        out.append((r.dose, (st["e_src"] - st["e_dep"] - st["e_esc"]) / st["e_src"],
                    st["n_hard_inel"], st["n_hard_br"]))
    return out


def test_forcing_and_splitting_reproduce_the_analog_dose():
    import multiprocessing as mp
    vr = S.VR(f_inel=5.0, f_brems=20.0, n_split_brems=2)
    K, n = 24, 1500
    jobs = []
    for v, seed in ((None, 11), (vr, 12)):
        jobs += [(v, seed, k, 1, n) for k in range(K)]
    with mp.get_context("spawn").Pool(NTH) as pool:
        res = pool.map(_forced_case, jobs)
    ana = [r[0] for r in res[:K]]
    frc = [r[0] for r in res[K:]]
    Ba = np.array([x[0] for x in ana])
    Bf = np.array([x[0] for x in frc])
    g = permutation_gate(Bf, Ba, thr=0.01, n_perm=1000)
    print("forced vs analog", g)
    assert g["pass"], g
    # the forced run did force: many more hard events per history
    assert sum(x[2] for x in frc) > 3 * sum(x[2] for x in ana)
    assert sum(x[3] for x in frc) > 10 * sum(x[3] for x in ana)
    # the analog ledger closes per batch to rounding; the forced one in
    # expectation (batch residuals centred on zero)
    assert max(abs(x[1]) for x in ana) < 1e-9
    rf = np.array([x[1] for x in frc])
    assert np.std(rf) > 0
    assert abs(rf.mean()) < 4.0 * rf.std(ddof=1) / np.sqrt(K)


def test_invalid_vr_rejected():
    ph, src, tp = beam(eabs_g=1e-3)
    for bad in (S.VR(f_inel=0.5), S.VR(n_split_brems=0), S.VR(w_lo=2.0, w_hi=1.0)):
        with pytest.raises(ValueError):
            O.run(ph, src, tp, 10, vr=bad)
    with pytest.raises(RuntimeError):    # the adjoint is written for analog histories
        O.adjoint(ph, src, tp, None, 10, vr=S.VR(f_brems=2.0))
