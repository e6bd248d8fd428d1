"""Device-memory limit of a context (gbmc_set_mem_limit): the failure path of
every kind of allocation, exercised without exhausting the GPU. An allocation
beyond the limit fails as a failed cudaMalloc would (GBMC_ERR_OOM, nothing
allocated); the state being built stays unset and is refused by the runs
(GBMC_ERR_STATE); with the limit raised the same calls succeed and the runs
make the same histories as an unlimited context."""
import numpy as np
import pytest

import paper_2003_00796_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu

OOM, STATE = 3, 4


def _status(fn, *a, **k):
    with pytest.raises(G.GbmcError) as x:
        fn(*a, **k)
    return x.value.status


def _same(a, b):
    big = a > 0.01 * a.max()
    assert np.median(np.abs(a - b)[big] / a[big]) < 1e-5
    assert b.sum() == pytest.approx(a.sum(), rel=1e-3)


def _jobs():
    specs = [(20, 0.4, S.PHOTON, 1.0), (33, 0.2, S.ELECTRON, 6.0), (16, 0.3, S.PHOTON, 3.0)]
    out = []
    for j, (n, d, part, e) in enumerate(specs):
        ph = S.grf_three_material(n, d, seed=100 + j, corr_len=0.6)
        L = n * d
        out.append((ph, S.Source(part, 1, L / 2, L / 2, L / 4, L / 5, e), 3_000, 1000 + 17 * j))
    return out


def test_memory_limit_fails_like_oom_and_the_context_recovers():
    w = S.workload_grf_spectrum(24, 0)
    n = 20_000
    opts = dict(kernel=G.KERNEL_WAVEFRONT, n_batches=8, queue_cap=1 << 16)
    ref = G.Engine(0, **opts).setup(w)
    ref.run(n, seed=3)
    d_ref = ref.edep()[0].copy()
    full, lim = ref.mem_info()
    assert lim == 0 and full > 0
    mats = [S.water(), S.bone(), S.lung()]
    ref.set_materials(mats, S.Transport(), 7.0)
    ref.run_batch(_jobs())
    b_ref = [ref.job_dose(j)[0].copy() for j in range(3)]
    ref.close()

    e = G.Engine(0, **opts)
    # tables: refused below their size; nothing held
    e.set_mem_limit(1024)
    assert _status(e.set_materials, w.phantom.materials, w.transport, 7.0) == OOM
    assert e.mem_info() == (0, 1024)
    e.set_mem_limit(0)
    e.setup(w)
    held = e.mem_info()[0]
    # wavefront queues: the run is refused before any launch and the tally is untouched
    e.set_mem_limit(held + 4096)
    assert _status(e.run, n, seed=3) == OOM
    assert e.mem_info()[0] == held
    assert e.moments()[2] == 0
    e.set_mem_limit(0)
    e.run(n, seed=3)
    _same(d_ref, e.edep()[0])
    assert e.mem_info()[0] == full
    # a phantom that does not fit: the context has none until one is loaded
    big = S.grf_three_material(48, 0.2, seed=4)
    e.set_mem_limit(full)
    assert _status(e.load_phantom, big) == OOM
    assert _status(e.run, 1_000, seed=1) == STATE
    e.set_mem_limit(0)
    e.load_phantom(big)
    e.run(1_000, seed=1)
    assert e.stats()["error_flags"] == 0
    # a batched run that fails part-way: its doses cannot be read; the next one runs
    e.set_materials(mats, S.Transport(), 7.0)
    held = e.mem_info()[0]
    n0 = 20 ** 3
    e.set_mem_limit(held + 5 * n0 + 1000)     # the first job's phantom fits, the second's not
    assert _status(e.run_batch, _jobs()) == OOM
    assert _status(e.job_dose, 0) == STATE
    e.set_mem_limit(0)
    e.run_batch(_jobs())
    for j in range(3):
        _same(b_ref[j], e.job_dose(j)[0])
    e.close()
