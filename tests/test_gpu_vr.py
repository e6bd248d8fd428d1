"""Variance reduction on the GPU (interaction forcing, bremsstrahlung
splitting; gbmc_set_vr), against the oracle and against the GPU's own analog
runs:

* parity with the oracle running the same variance reduction (permutation
  gate on batch doses), plain and wavefront kernels;
* splitting alone with photons absorbed where they are made reproduces the
  analog run (same electron histories, copies' deposits sum to the photon's);
* a forcing window that excludes every particle reproduces the analog run;
* the wavefront kernels replay the plain kernel's weighted histories;
* the adjoint refuses weighted histories, bad parameters are refused.
"""
import multiprocessing as mp

import numpy as np
import pytest

import paper_2003_00796_gb300 as G
import synthetic as S
from test_gpu_parity import NTHREADS
from parity import permutation_gate

pytestmark = pytest.mark.gpu

VR = S.VR(f_inel=5.0, f_brems=20.0, n_split_brems=2)


def beam_workload(eabs_g=1e-3, vr=None):
    ph = S.water_cube(16, 0.05)
    src = S.Source(S.ELECTRON, 0, 0.425, 0.425, 0, 0, 1.0)
    tp = S.Transport(eabs_g=eabs_g, eabs_e=0.02, wcc=0.005, wcr=0.005)
    return S.Workload("beam1MeV_water16", ph, src, tp, 0, 1, vr)


def gpu_run(w, n, seed, kernel=G.KERNEL_PLAIN, first=0, n_batches=8):
    e = G.Engine(0, kernel=kernel, n_batches=n_batches).setup(w)
    e.run(n, seed=seed, first_hist=first)
    d, v = e.dose()
    st = e.stats()
    e.close()
    return d, v, st


def _oracle_batch(args):
    nk, seed, k = args
    import oracle as O2
    w = beam_workload(vr=VR)
    return O2.run(w.phantom, w.source, w.transport, nk, seed=seed, first_hist=k * nk,
                  n_batches=1, vr=VR).dose


@pytest.mark.parametrize("kernel", [G.KERNEL_PLAIN, G.KERNEL_WAVEFRONT])
def test_vr_parity_with_oracle(kernel):
    w = beam_workload(vr=VR)
    K, nk = 24, 4000
    Bg = np.array([gpu_run(w, nk, 21, kernel, first=k * nk, n_batches=2)[0] for k in range(K)])
    with mp.get_context("spawn").Pool(NTHREADS) as pool:
        Bo = np.array(pool.map(_oracle_batch, [(nk, 22, k) for k in range(K)]))
    res = permutation_gate(Bg, Bo, thr=0.01, n_perm=1000)
    print("vr parity", kernel, res)
    assert res["pass"], res
    assert res["n_vox"] >= 50


def test_splitting_alone_reproduces_analog_when_photons_are_absorbed():
    a = gpu_run(beam_workload(eabs_g=1e3), 20_000, 5)
    b = gpu_run(beam_workload(eabs_g=1e3, vr=S.VR(n_split_brems=4)), 20_000, 5)
    for k in ("n_hist", "n_e_steps", "n_hard", "n_cross"):
        assert a[2][k] == b[2][k], k
    big = a[0] > 1e-3 * a[0].max()
    rel = np.abs(b[0][big] - a[0][big]) / a[0][big]
    assert np.median(rel) < 1e-5 and rel.max() < 1e-3


def test_forcing_outside_its_window_reproduces_analog():
    a = gpu_run(beam_workload(), 20_000, 6)
    b = gpu_run(beam_workload(vr=S.VR(f_inel=7.0, f_brems=50.0, w_lo=1.5, w_hi=2.0)), 20_000, 6)
    for k in ("n_hist", "n_e_steps", "n_hard", "n_cross", "n_tent", "n_real"):
        assert a[2][k] == b[2][k], k
    big = a[0] > 1e-2 * a[0].max()
    rel = np.abs(b[0][big] - a[0][big]) / a[0][big]
    assert np.median(rel) < 1e-5


def test_wavefront_replays_plain_with_vr():
    w = beam_workload(vr=VR)
    a = gpu_run(w, 20_000, 7, G.KERNEL_PLAIN)
    b = gpu_run(w, 20_000, 7, G.KERNEL_WAVEFRONT)
    for k in ("n_hist", "n_e_steps", "n_hard", "n_tent"):
        assert abs(a[2][k] - b[2][k]) <= 1e-3 * a[2][k], k
    big = a[0] > 1e-2 * a[0].max()
    rel = np.abs(b[0][big] - a[0][big]) / a[0][big]
    assert np.median(rel) < 1e-5
    assert a[2]["error_flags"] == 0 and b[2]["error_flags"] == 0


def test_vr_refusals():
    w = beam_workload(vr=VR)
    e = G.Engine(0).setup(w)
    with pytest.raises(G.GbmcError) as ex:
        e.adjoint(np.ones(w.phantom.n_vox), 100)
    assert ex.value.status == 4
    for bad in (S.VR(f_inel=0.5), S.VR(n_split_brems=0), S.VR(n_split_brems=65),
                S.VR(w_lo=2.0, w_hi=1.0)):
        with pytest.raises(G.GbmcError):
            e.set_vr(bad)
    e.set_vr(None)
    e.set_majorant([1.2])
    m, _ = e.adjoint(np.ones(w.phantom.n_vox), 1000)
    assert np.all(np.isfinite(m))
    e.close()
