"""Batched runs (gbmc_run_batch): jobs with their own phantoms, sources and
seeds in one wavefront pass loop. Each job's histories are those of a single
run with the same phantom, source and key (seed, job id), so the batch must
reproduce single runs job by job: doses equal up to the order of FP32 atomics,
event counts equal up to the rare particle whose FP32 arithmetic rounds
differently in the kernel that finishes it (a run's last particles are run to
the end by the drain kernel, and which particles those are depends on what
else is in flight)."""
import numpy as np
import pytest

import paper_2003_00796_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu

E_MAX = 7.0


def small_jobs():
    """Six uneven jobs: photons and electrons, mono and binned sources."""
    edges, wts = S.kramers_spectrum(6.0, 0.1, 64)
    specs = [  # (side, voxel cm, particle, energy, spectrum)
        (20, 0.4, S.PHOTON, 1.0, False),
        (33, 0.2, S.ELECTRON, 6.0, False),
        (16, 0.3, S.PHOTON, 0.0, True),
        (40, 0.1, S.ELECTRON, 2.0, False),
        (24, 0.4, S.POSITRON, 3.0, False),
        (28, 0.2, S.PHOTON, 4.5, False),
    ]
    jobs = []
    for j, (n, d, part, e, spec) in enumerate(specs):
        ph = S.grf_three_material(n, d, seed=100 + j, corr_len=0.6)
        L = n * d
        src = S.Source(part, 1, L / 2, L / 2, L / 4, L / 5, e if not spec else 6.0,
                       edges if spec else None, wts if spec else None)
        jobs.append((ph, src, 20_000 + 7_000 * j, 1000 + 17 * j))
    return jobs


def engine(kernel=G.KERNEL_WAVEFRONT):
    e = G.Engine(0, kernel=kernel, n_batches=8)
    e.set_materials([S.water(), S.bone(), S.lung()], S.Transport(), E_MAX)
    return e


def test_batch_reproduces_single_runs():
    jobs = small_jobs()
    eb = engine()
    eb.run_batch(jobs)
    sb = eb.stats()
    totals = {k: 0 for k in ("n_hist", "n_tent", "n_real", "n_e_steps", "n_cross", "n_hard", "n_particles")}
    for j, (ph, src, n, seed) in enumerate(jobs):
        db, vb = eb.job_dose(j)
        es = engine()
        es.load_phantom(ph)
        es.set_source(src)
        # the job's key is (lo32(seed), hi32(seed) ^ j); a single run uses job id 0
        es.run(n, seed=seed ^ (j << 32))
        ds, vs = es.dose()
        st = es.stats()
        es.close()
        for k in totals:
            totals[k] += st[k]
        big = ds > 0.05 * ds.max()
        assert big.sum() > 10, j
        rel = np.abs(db[big] - ds[big]) / ds[big]
        assert np.median(rel) < 1e-5, (j, np.median(rel))
        assert rel.max() < 1e-2, (j, rel.max())
        np.testing.assert_allclose(vb[big], vs[big], rtol=1e-2)
    assert sb["n_hist"] == totals["n_hist"]
    for k, v in totals.items():
        assert abs(sb[k] - v) <= 1e-5 * v + 2, (k, sb[k], v)
    eb.close()


def test_batch_matches_plain_single_runs_statistically():
    """A batched job against the plain (one history per thread) kernel on the
    same histories: same physics, independent code path for the queues."""
    jobs = small_jobs()[:2]
    eb = engine()
    eb.run_batch(jobs)
    for j, (ph, src, n, seed) in enumerate(jobs):
        db, _ = eb.job_dose(j)
        es = engine(G.KERNEL_PLAIN)
        es.load_phantom(ph)
        es.set_source(src)
        es.run(n, seed=seed ^ (j << 32))
        ds, _ = es.dose()
        es.close()
        big = ds > 0.05 * ds.max()
        rel = np.abs(db[big] - ds[big]) / ds[big]
        assert np.median(rel) < 1e-5, (j, np.median(rel))
    eb.close()


def test_batch_rejects_bad_jobs():
    jobs = small_jobs()[:2]
    e = engine()
    with pytest.raises(G.GbmcError):
        e.run_batch([])
    bad = S.grf_three_material(8, 0.5, seed=1)
    bad.rho[0, 0, 0] = -1.0
    with pytest.raises(G.GbmcError):
        e.run_batch([jobs[0], (bad, jobs[1][1], 100, 1)])
    hot = S.Source(S.PHOTON, 0, 1.0, 1.0, 0, 0, 50.0)    # above the tables' energy range
    with pytest.raises(G.GbmcError):
        e.run_batch([(jobs[0][0], hot, 100, 1)])
    # the context stays usable
    e.run_batch(jobs[:1])
    d, v = e.job_dose(0)
    assert d.max() > 0 and np.all(np.isfinite(v))
    e.close()


def test_autotune_single_and_batch():
    e = engine()
    w = S.workload_grf_spectrum(32, 0)
    e.load_phantom(w.phantom)
    e.set_source(w.source)
    cap = 1 << 24
    got = e.autotune(400_000, seed=3)
    assert got["charged_budget"] in (8, 16, 32)
    assert got["photon_budget"] in (4, 8, 16)
    assert got["pass_target"] in (cap // 8, cap // 4, cap // 2)
    assert e.stats()["n_hist"] == 0          # trials leave no trace in the tally
    e.run(100_000, seed=5)
    d, v = e.dose()
    assert d.max() > 0
    jobs = small_jobs()[:3]
    got_b = e.autotune(60_000, seed=3, jobs=jobs)
    assert got_b["pass_target"] in (cap // 8, cap // 4, cap // 2)
    e.run_batch(jobs)
    for j in range(3):
        d, v = e.job_dose(j)
        assert d.max() > 0
    e.close()


def test_repeated_batches_reuse_their_buffers_and_reject_bad_phantoms():
    """A second run of the same jobs keeps the job buffers (same voxel and
    batch counts) and gives the same doses up to FP32 atomic order; a batch
    with another shape allocates anew; a phantom with a material id beyond
    the context's materials is found by the device-side validation and
    reported with its job index, and the context stays usable."""
    jobs = small_jobs()[:3]
    e = engine()
    e.run_batch(jobs)
    first = [e.job_dose(j)[0] for j in range(3)]
    e.run_batch(jobs)
    for j in range(3):
        d = e.job_dose(j)[0]
        big = first[j] > 0.05 * first[j].max()
        assert np.median(np.abs(d[big] - first[j][big]) / first[j][big]) < 1e-5, j
    other = small_jobs()[3:5]
    e.run_batch(other)
    assert e.job_dose(1)[0].size == other[1][0].mat.size
    bad_ph = S.grf_three_material(16, 0.3, seed=7)
    bad_ph.mat = bad_ph.mat.copy()
    bad_ph.mat[3, 4, 5] = 7
    with pytest.raises(G.GbmcError) as ex:
        e.run_batch([jobs[0], (bad_ph, jobs[1][1], 1000, 3)])
    assert ex.value.status == 1 and "job 1" in str(ex.value)
    e.run_batch(jobs)
    d = e.job_dose(0)[0]
    big = first[0] > 0.05 * first[0].max()
    assert np.median(np.abs(d[big] - first[0][big]) / first[0][big]) < 1e-5
    e.close()
