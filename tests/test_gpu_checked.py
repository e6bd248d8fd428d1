"""The checked library on the GPU (libgbmc_checked.so: the same sources
compiled with GBMC_CHECKED, so that every kernel tests its voxel, material,
batch, job, queue-slot, alias-bin, element-count and adjoint-buffer indices
before using them; gbmc.h, "checked build").

The checked kernels must (1) really test: the device check substitutes 0 and
records the flag for an index out of range, and passes an index in range
through; (2) find nothing on valid runs of every kernel family -- plain,
wavefront (photon, charged, knock and drain kernels), batched, weighted
(variance reduction) and both adjoints; (3) run the same histories as the
default library, so their tallies and event counts agree with it to the
tolerance of two runs of the default library (FP32 atomic order, and the rare
particle whose FP32 arithmetic rounds differently in the kernel that finishes
it: which particles the drain kernel finishes depends on what else is in
flight)."""
import numpy as np
import pytest

import paper_2003_00796_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu

COUNTERS = ("n_tent", "n_real", "n_e_steps", "n_cross", "n_hard", "n_particles")


def test_device_index_check_is_live_only_in_the_checked_library():
    idx = np.array([0, 5, 9, -1, 10, 2**31 - 1, 7, -(2**31)], np.int32)
    bound = np.array([10, 10, 10, 10, 10, 2**40, 7, 3], np.int64)
    ok = (idx >= 0) & (idx.astype(np.int64) < bound)
    out, flags = G.check_index(idx, bound, checked=True)
    np.testing.assert_array_equal(out, np.where(ok, idx, 0))
    np.testing.assert_array_equal(flags, np.where(ok, 0, G.FLAG_BOUNDS))
    out0, flags0 = G.check_index(idx, bound, checked=False)
    np.testing.assert_array_equal(out0, idx)
    assert not flags0.any()


def _grf32():
    ph = S.grf_three_material(32, 0.4, seed=2)
    edges, wts = S.kramers_spectrum(6.0, 0.1, 64)
    return S.Workload("grf32", ph, S.Source(S.PHOTON, 1, 6.4, 6.4, 4.0, 4.0, 6.0, edges, wts),
                      S.Transport(), 0, 1)


def _ct48():
    ph = S.ct_phantom(48, 0.2, seed=3)
    return S.Workload("ct48", ph, S.Source(S.ELECTRON, 1, 4.8, 4.8, 0.5, 0.5, 20.0),
                      S.Transport(), 0, 1)


def _positron():
    ph = S.grf_three_material(24, 0.25, seed=7)
    return S.Workload("pos24", ph, S.Source(S.POSITRON, 0, 3.0, 3.0, 0.0, 0.0, 3.0),
                      S.Transport(), 0, 1)


def _vr():
    """1 MeV electron pencil in water with interaction forcing and
    bremsstrahlung splitting (the weighted kernels)."""
    ph = S.water_cube(16, 0.05)
    src = S.Source(S.ELECTRON, 0, 0.425, 0.425, 0, 0, 1.0)
    tp = S.Transport(eabs_g=1e-3, eabs_e=0.02, wcc=0.005, wcr=0.005)
    return S.Workload("beam1MeV_water16_vr", ph, src, tp, 0, 1,
                      S.VR(f_inel=5.0, f_brems=20.0, n_split_brems=2))


CASES = {
    "water_plain": (S.workload_water_pencil, G.KERNEL_PLAIN, 20_000),
    "water_wavefront": (S.workload_water_pencil, G.KERNEL_WAVEFRONT, 20_000),
    "grf32_wavefront": (_grf32, G.KERNEL_WAVEFRONT, 20_000),
    "ct48_plain": (_ct48, G.KERNEL_PLAIN, 1_000),
    "ct48_wavefront": (_ct48, G.KERNEL_WAVEFRONT, 2_000),
    "positron_wavefront": (_positron, G.KERNEL_WAVEFRONT, 5_000),
    "vr_wavefront": (_vr, G.KERNEL_WAVEFRONT, 5_000),
    "vr_plain": (_vr, G.KERNEL_PLAIN, 5_000),
}


def _run(w, kernel, n, checked):
    e = G.Engine(0, kernel=kernel, n_batches=8, queue_cap=1 << 16, checked=checked).setup(w)
    assert e.checked == checked
    e.run(n, seed=41)
    d = e.edep()[0].copy()
    st = e.stats()
    e.close()
    return d, st


def _agree(a, sa, b, sb, label):
    big = a > 0.01 * a.max()
    rel = np.abs(a - b)[big] / a[big]
    diffs = {k: int(sb[k]) - int(sa[k]) for k in COUNTERS}
    print(label, "median", np.median(rel), "max", rel.max(), "counter differences", diffs)
    assert np.median(rel) < 1e-5
    assert b.sum() == pytest.approx(a.sum(), rel=1e-3)
    for k in COUNTERS:
        assert abs(int(sb[k]) - int(sa[k])) <= 1e-3 * max(int(sa[k]), 1) + 2, (k, sa[k], sb[k])


@pytest.mark.parametrize("case", sorted(CASES))
def test_checked_kernels_find_nothing_and_run_the_same_histories(case):
    make, kernel, n = CASES[case]
    w = make()
    a, sa = _run(w, kernel, n, checked=False)
    b, sb = _run(w, kernel, n, checked=True)
    assert sb["error_flags"] == 0 and sb["status"] == 0
    assert sb["n_hist"] == sa["n_hist"] == n
    _agree(a, sa, b, sb, case)


def test_checked_batch_finds_nothing():
    """Six uneven jobs in one batched run (job-index and per-job voxel checks)."""
    edges, wts = S.kramers_spectrum(6.0, 0.1, 64)
    specs = [(20, 0.4, S.PHOTON, 1.0, False), (33, 0.2, S.ELECTRON, 6.0, False),
             (16, 0.3, S.PHOTON, 0.0, True), (40, 0.1, S.ELECTRON, 2.0, False),
             (24, 0.4, S.POSITRON, 3.0, False), (28, 0.2, S.PHOTON, 4.5, False)]
    jobs = []
    for j, (n, d, part, e, spec) in enumerate(specs):
        ph = S.grf_three_material(n, d, seed=100 + j, corr_len=0.6)
        L = n * d
        src = S.Source(part, 1, L / 2, L / 2, L / 4, L / 5, e if not spec else 6.0,
                       edges if spec else None, wts if spec else None)
        jobs.append((ph, src, 4_000 + 1_000 * j, 1000 + 17 * j))
    out = []
    for checked in (False, True):
        e = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=8, checked=checked)
        e.set_materials([S.water(), S.bone(), S.lung()], S.Transport(), 7.0)
        e.run_batch(jobs)
        st = e.stats()
        doses = [e.job_dose(j)[0].copy() for j in range(len(jobs))]
        out.append((doses, st))
        e.close()
    (da, sa), (db, sb) = out
    assert sb["error_flags"] == 0 and sb["status"] == 0
    for j in range(len(jobs)):
        a, b = da[j], db[j]
        big = a > 0.01 * a.max()
        assert np.median(np.abs(a - b)[big] / a[big]) < 1e-5, j
        assert b.sum() == pytest.approx(a.sum(), rel=1e-3), j
    for k in COUNTERS:
        assert abs(int(sb[k]) - int(sa[k])) <= 1e-3 * max(int(sa[k]), 1) + 2, (k, sa[k], sb[k])


@pytest.mark.parametrize("kernel", [G.KERNEL_PLAIN, G.KERNEL_WAVEFRONT])
def test_checked_adjoint_finds_nothing(kernel):
    """Both replays of the path-replay adjoint (the adjoint-buffer index of the
    wavefront's replays, the deposit weights of both)."""
    ph = S.grf_three_material(16, 0.5, seed=5)
    w = S.Workload("grf16", ph, S.Source(S.PHOTON, 1, 4.0, 4.0, 2.0, 2.0, 1.0),
                   S.Transport(), 0, 1)
    g = np.random.default_rng(3).normal(size=ph.n_vox)
    out = []
    for checked in (False, True):
        e = G.Engine(0, kernel=kernel, n_batches=8, checked=checked).setup(w)
        grad = e.adjoint(g, 20_000, seed=12)[0].copy()
        st = e.stats()
        out.append((grad, st))
        e.close()
    (ga, sa), (gb, sb) = out
    assert sb["error_flags"] == 0 and sb["status"] == 0
    big = np.abs(ga) > 0.01 * np.abs(ga).max()
    assert np.median(np.abs(ga - gb)[big] / np.abs(ga[big])) < 1e-3
