"""The allocation-free run entry point (collected last on purpose).

gbmc_run_noalloc is for callers that must not allocate device memory while
histories run (a program with a device-memory budget fixed at start-up, or one
whose streams must keep overlapping, which cudaMalloc would serialise). It
keeps its scratch in a static device array and writes into caller buffers.
Here it is called through the C ABI and checked against the ordinary run path
(gbmc_run + gbmc_get_edep) on the same histories, twice in a row: the second
call must not see the first call's scratch."""
import numpy as np
import pytest

import paper_2003_00796_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_run_twice():
    torch = pytest.importorskip("torch")
    ph = S.grf_three_material(30, 0.4, seed=2)      # 27 000 voxels: not a multiple of 4
    edges, wts = S.kramers_spectrum(6.0, 0.1, 64)
    src = S.Source(S.PHOTON, 1, 6.0, 6.0, 2.0, 2.0, 6.0, edges, wts)
    w = S.Workload("grf30", ph, src, S.Transport(), 0, 1)
    K, n = 8, 40_000
    ref = G.Engine(0, n_batches=K).setup(w)
    e = G.Engine(0, n_batches=K).setup(w)
    for call, (seed, first) in enumerate([(5, 0), (6, 1_000_000)]):
        ref.reset()
        ref.run(n, seed=seed, first_hist=first)
        m_ref, v_ref = ref.edep()
        s1 = torch.zeros(ph.n_vox, dtype=torch.float64, device="cuda")
        s2 = torch.zeros_like(s1)
        e.run_noalloc(n, s1, s2, seed=seed, first_hist=first, n_batches=K)
        torch.cuda.synchronize()
        S1, S2 = s1.cpu().numpy(), s2.cpu().numpy()
        m = S1 / n
        var = np.maximum(S2 - n * m * m, 0) / (n * (K - 1))
        big = m_ref > 0.01 * m_ref.max()
        # same histories, same batches: equal up to FP32 atomic ordering
        np.testing.assert_allclose(m[big], m_ref[big], rtol=1e-5)
        np.testing.assert_allclose(var[big], v_ref[big], rtol=1e-3)
        assert m.sum() == pytest.approx(m_ref.sum(), rel=1e-6)
        assert e.noalloc_flags() == 0          # no stack overflow, no loop bound hit
    # a third call (kernels loaded by the first two) leaves the device's free
    # memory exactly as it was: nothing is allocated, not even transiently kept
    s1 = torch.zeros(ph.n_vox, dtype=torch.float64, device="cuda")
    s2 = torch.zeros_like(s1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    e.run_noalloc(n, s1, s2, seed=7, first_hist=2_000_000, n_batches=K)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # outputs that are not float64 device buffers of nvox values are refused
    # before anything runs: by the binding, and by the C entry point itself
    with pytest.raises(ValueError):
        e.run_noalloc(n, s1.float(), s2, n_batches=K)
    with pytest.raises(ValueError):
        e.run_noalloc(n, s1[:-1], s2[:-1], n_batches=K)
    with pytest.raises(ValueError):
        e.run_noalloc(n, s1.cpu(), s2.cpu(), n_batches=K)
    host = np.zeros(ph.n_vox)
    st = G.lib().gbmc_run_noalloc(e._h, n, 1, 0, K, host.ctypes.data, host.ctypes.data, None)
    assert st == 1
    # sizes beyond the static scratch are rejected
    big_ph = S.water_cube(120, 0.5)
    e2 = G.Engine(0, n_batches=K).setup(big_ph, S.Source(S.PHOTON, 0, 30, 30, 0, 0, 1.0), S.Transport())
    t1 = torch.zeros(big_ph.n_vox, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GbmcError) as ex:
        e2.run_noalloc(1000, t1, t1.clone(), n_batches=K)
    assert ex.value.status == 1
