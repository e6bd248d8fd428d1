"""The library's event counters against the oracle's: per history, the
numbers of tentative photon collisions (Woodcock flights, escapes included),
real photon interactions, class II steps, voxel crossings of charged
particles, and hard events of class II steps (delta events included) are
random variables with the same distribution in both engines, so their means
over independent runs agree within their standard errors. These are the
method's work counts (Sec. 4.1: JUMP, STEP and KNOCK calls); a kernel that
skipped or repeated steps, or mis-sampled a flight or a hard-event rate, would
move them even where the dose still agreed."""
import os

import numpy as np
import pytest

import oracle as O
import paper_2003_00796_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))
GPU_KEYS = ("n_tent", "n_real", "n_e_steps", "n_cross", "n_hard")


def _oracle_counts(st):
    return {"n_tent": st["n_tent"], "n_real": st["n_real"], "n_e_steps": st["n_e_steps"],
            "n_cross": st["n_cross"],
            "n_hard": st["n_hard_el"] + st["n_hard_inel"] + st["n_hard_br"] + st["n_delta"]}


def _grf32():
    ph = S.grf_three_material(32, 0.4, seed=2)
    edges, wts = S.kramers_spectrum(6.0, 0.1, 64)
    return S.Workload("grf32", ph, S.Source(S.PHOTON, 1, 6.4, 6.4, 4.0, 4.0, 6.0, edges, wts),
                      S.Transport(), 0, 1)


def _ct48():
    ph = S.ct_phantom(48, 0.2, seed=3)
    return S.Workload("ct48", ph, S.Source(S.ELECTRON, 1, 4.8, 4.8, 0.5, 0.5, 20.0),
                      S.Transport(), 0, 1)


def _vr_beam():
    """1 MeV electron pencil in water with interaction forcing (x5 inelastic,
    x20 bremsstrahlung) and bremsstrahlung splitting in two: the forced
    event rates and the split photons' flights."""
    ph = S.water_cube(16, 0.05)
    src = S.Source(S.ELECTRON, 0, 0.425, 0.425, 0, 0, 1.0)
    tp = S.Transport(eabs_g=1e-3, eabs_e=0.02, wcc=0.005, wcr=0.005)
    return S.Workload("beam1MeV_water16_vr", ph, src, tp, 0, 1,
                      S.VR(f_inel=5.0, f_brems=20.0, n_split_brems=2))


# case: (workload, histories per run, independent runs K per engine); z is
# t-distributed with about 2K - 2 degrees of freedom
CASES = {"grf32_photon_field": (_grf32, 8_000, 10), "ct48_electron_20MeV": (_ct48, 400, 10),
         "vr_beam_1MeV": (_vr_beam, 1_000, 6)}
Z_MAX = 5.0     # P(|t| > 5) <= 5e-4 per comparison at 10 degrees of freedom
_ORACLE = {}


def _oracle_runs(case, w, n, K):
    """K oracle runs of n histories (shared by both kernels' tests)."""
    if case not in _ORACLE:
        o = np.zeros((K, len(GPU_KEYS)))
        for k in range(K):
            r = O.run(w.phantom, w.source, w.transport, n, seed=202, first_hist=k * n, n_batches=4,
                      n_threads=NTHREADS, vr=getattr(w, "vr", None))
            oc = _oracle_counts(r.stats)
            o[k] = [float(oc[c]) for c in GPU_KEYS]
        _ORACLE[case] = o
    return _ORACLE[case]


@pytest.mark.parametrize("kernel", [G.KERNEL_PLAIN, G.KERNEL_WAVEFRONT])
@pytest.mark.parametrize("case", sorted(CASES))
def test_event_counts_match_oracle(case, kernel):
    make, n, K = CASES[case]
    w = make()
    e = G.Engine(0, kernel=kernel, n_batches=4, queue_cap=1 << 16).setup(w)
    g = np.zeros((K, len(GPU_KEYS)))
    prev = np.zeros(len(GPU_KEYS))
    for k in range(K):
        e.run(n, seed=101, first_hist=k * n)
        st = e.stats()
        cur = np.array([float(st[c]) for c in GPU_KEYS])
        g[k] = cur - prev
        prev = cur
    assert e.stats()["error_flags"] == 0
    e.close()
    o = _oracle_runs(case, w, n, K)
    for j, key in enumerate(GPU_KEYS):
        mg, mo = g[:, j].mean() / n, o[:, j].mean() / n
        se = np.sqrt(g[:, j].var(ddof=1) / K + o[:, j].var(ddof=1) / K) / n
        if mo == 0.0 and mg == 0.0:
            continue
        z = (mg - mo) / se if se > 0 else np.inf
        print(f"{case} kernel {kernel} {key}: gpu {mg:.5g} oracle {mo:.5g} per history, z {z:+.2f}")
        assert abs(z) < Z_MAX, (key, mg, mo, z)
