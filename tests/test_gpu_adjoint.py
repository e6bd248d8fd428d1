"""GPU path-replay adjoint (gbmc_adjoint and the torch.autograd wrapper):

* parity with the oracle's likelihood-ratio gradient (same estimator, FP64,
  CPU) on a 16^3 crop of the three-material phantom, in kerma mode and with
  coupled electron transport, by the batch permutation gate;
* agreement with central finite differences of the GPU forward dose with
  common random numbers and a fixed majorant, on 32 sampled voxels of the
  high-fluence region (kerma mode, where the estimator is exact);
* the autograd wrapper returns the adjoint's gradient for L = sum (D - T)^2.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
import paper_2003_00796_gb300 as G
import synthetic as S
from parity import batch_stats, permutation_gate

pytestmark = pytest.mark.gpu

KERMA = S.Transport(eabs_e=1e3)
NPROC = max(1, min(16, os.cpu_count() or 1))


def crop_case(n=16, transport=KERMA):
    ph = S.crop(S.grf_three_material(128, 0.2, seed=2), n)
    edges, wts = S.kramers_spectrum(6.0, 0.1, 64)
    L = n * 0.2
    src = S.Source(S.PHOTON, 1, L / 2, L / 2, 0.4 * L, 0.4 * L, 6.0, edges, wts)
    # dL/dD = 1 everywhere (L = total dose): the gradient the estimator
    # resolves best per history; any fixed g tests the same estimator
    g = np.ones(ph.n_vox)
    rho_maj = [1.05 * float(ph.rho[ph.mat == m].max()) if np.any(ph.mat == m) else 1.0
               for m in range(len(ph.materials))]
    return S.Workload(f"crop{n}", ph, src, transport, 0, 1), g, rho_maj


def gpu_grad_batches(w, g, rho_maj, n, seed, K):
    e = G.Engine(0, kernel=G.KERNEL_PLAIN, n_batches=8).setup(w)
    e.set_majorant(rho_maj)
    nk = n // K
    B = [e.adjoint(g, nk, seed=seed, first_hist=k * nk)[0].copy() for k in range(K)]
    e.close()
    return np.array(B)


def _oracle_grad(args):
    w, g, rho_maj, nk, seed, k = args
    import oracle as O2
    m, _, _ = O2.adjoint(w.phantom, w.source, w.transport, g, nk, seed=seed, first_hist=k * nk,
                         n_batches=2, rho_maj=rho_maj)
    return m


def oracle_grad_batches(w, g, rho_maj, n, seed, K):
    nk = n // K
    with mp.get_context("spawn").Pool(NPROC) as pool:
        return np.array(pool.map(_oracle_grad, [(w, g, rho_maj, nk, seed, k) for k in range(K)]))


def grad_parity(w, g, rho_maj, n, K=20):
    Bo = oracle_grad_batches(w, g, rho_maj, n, seed=21, K=K)
    Bg = gpu_grad_batches(w, g, rho_maj, n, seed=22, K=K)
    mo, vo = batch_stats(Bo)
    mg, vg = batch_stats(Bg)
    # voxels whose gradient both engines resolve (|mean| above 4 sigma)
    sel = (np.abs(mo) > 4 * np.sqrt(vo)) & (np.abs(mg) > 4 * np.sqrt(vg))
    res = permutation_gate(Bg, Bo, n_perm=1000, sel=sel)
    print("gradient parity", w.transport.eabs_e, res)
    return res


def test_gradient_parity_kerma_mode():
    w, g, rho_maj = crop_case()
    res = grad_parity(w, g, rho_maj, 3_200_000, K=32)
    assert res["n_vox"] >= 30
    assert res["pass"], res


def test_gradient_parity_coupled_transport():
    w, g, rho_maj = crop_case(transport=S.Transport())
    res = grad_parity(w, g, rho_maj, 1_600_000, K=16)
    assert res["n_vox"] >= 10
    assert res["pass"], res


def _fd_setup(n=32):
    w, rho_t = S.workload_differentiable(n, 0)
    w.transport = KERMA
    ph = w.phantom
    rho_maj = [1.1 * float(ph.rho[ph.mat == m].max()) for m in range(len(ph.materials))]
    return w, rho_t, rho_maj


def test_adjoint_matches_central_differences_crn():
    """dJ/drho_v of J = sum_u g_u D_u, g = 2 (D - T) (the gradient of the
    config's loss at the current dose), on 32 voxels of the high-fluence
    region: adjoint vs central differences (h = 1e-3 relative) of the GPU
    forward with common random numbers and a fixed majorant."""
    w, rho_t, rho_maj = _fd_setup()
    ph = w.phantom
    e = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=8).setup(w)
    e.set_majorant(rho_maj)
    N = 4_000_000
    e.run(N, seed=31)
    D, _ = e.dose()
    wt = S.Workload("target", S.Phantom(ph.mat, rho_t, ph.dx, ph.dy, ph.dz, ph.materials),
                    w.source, w.transport, 0, 1)
    et = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=8).setup(wt)
    et.run(N, seed=32)
    T, _ = et.dose()
    et.close()
    g = 2.0 * (D - T)
    # adjoint: K batches of independent histories
    K, na = 16, 16_000_000
    Ba = np.array([e.adjoint(g, na // K, seed=33, first_hist=k * (na // K))[0].copy()
                   for k in range(K)])
    ma, va = batch_stats(Ba)
    # 32 voxels among the highest-dose ones, seeded choice
    top = np.argsort(D)[-400:]
    vox = np.random.default_rng(4).choice(top, 32, replace=False)
    h, nf, KF = 1e-3, 4_000_000, 8
    rho0 = ph.rho.reshape(-1).astype(np.float32)
    fd = np.zeros((KF, len(vox)))
    for i, v in enumerate(vox):
        J = []
        for sgn in (1.0, -1.0):
            r = rho0.copy()
            r[v] = np.float32(rho0[v] * (1.0 + sgn * h))
            e.load_phantom(ph, rho=r.reshape(ph.rho.shape))
            Jk = []
            for k in range(KF):
                e.reset()
                e.run(nf // KF, seed=34, first_hist=k * (nf // KF))
                Jk.append(g @ e.dose()[0])
            J.append((np.array(Jk), float(r[v])))
        fd[:, i] = (J[0][0] - J[1][0]) / (J[0][1] - J[1][1])
    e.close()
    mf, vf = batch_stats(fd)
    z = (ma[vox] - mf) / np.sqrt(va[vox] + vf)
    print("adjoint vs FD: z", np.round(z, 2), "adj", ma[vox][:6], "fd", mf[:6])
    assert np.mean(np.abs(z) < 3.0) >= 0.9, z
    assert np.mean(z * z) < 2.0, z
    assert abs(z.mean()) < 4.0 / np.sqrt(len(z)), z
    # the comparison has power: the gradients are resolved, not all noise
    assert np.mean(np.abs(ma[vox]) > 3.0 * np.sqrt(va[vox])) > 0.5


def test_autograd_wrapper_returns_the_adjoint():
    import torch
    from paper_2003_00796_gb300.autograd import dose
    w, rho_t, rho_maj = _fd_setup(16)
    ph = w.phantom
    e = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=8).setup(w)
    e.set_majorant(rho_maj)
    mat = torch.from_numpy(ph.mat).cuda()
    rho = torch.from_numpy(ph.rho.copy()).cuda().requires_grad_(True)
    T = torch.from_numpy(ph.rho.copy() * 0.0 + 1.0).double().cuda() * 1e-3
    D = dose(rho, e, ph, mat, 200_000, seed=41, adj_hist=300_000, adj_seed=42)
    L = ((D - T) ** 2).sum()
    L.backward()
    gr = rho.grad.double().cpu().numpy().reshape(-1)
    # the same adjoint by hand: g = dL/dD = 2 (D - T), same replay histories
    g = (2.0 * (D.detach() - T)).reshape(-1).contiguous()
    e.load_phantom(ph, mat=mat, rho=rho.detach())
    ref, _ = e.adjoint(g, 300_000, seed=42)
    e.close()
    big = np.abs(ref) > 0.05 * np.abs(ref).max()
    assert big.sum() > 20
    np.testing.assert_allclose(gr[big], ref[big], rtol=2e-3)
    assert np.all(np.isfinite(gr))


def test_majorant_below_phantom_maximum_is_rejected():
    w, _, _ = crop_case()
    e = G.Engine(0).setup(w)
    with pytest.raises(G.GbmcError):
        e.set_majorant([0.5] * len(w.phantom.materials))
    e.close()
