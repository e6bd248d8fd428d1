"""GPU path-replay adjoint (gbmc_adjoint and the torch.autograd wrapper):

* parity with the oracle's likelihood-ratio gradient (same estimator, FP64,
  CPU) on a 16^3 crop of the three-material phantom, in kerma mode and with
  coupled electron transport, by the batch permutation gate;
* agreement with central finite differences of the GPU forward dose with
  common random numbers and a fixed majorant, along 32 block directions of the
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
    # voxels whose gradient the pooled 2K batches resolve (|mean| above 4 sigma);
    # the selection treats the two engines alike, so the permutation null holds
    mp_, vp_ = batch_stats(np.concatenate([Bg, Bo], 0))
    sel = np.abs(mp_) > 4 * np.sqrt(vp_)
    res = permutation_gate(Bg, Bo, n_perm=1000, sel=sel)
    res["resolved_gpu"] = int(np.sum(np.abs(mg) > 4 * np.sqrt(vg)))
    res["resolved_oracle"] = int(np.sum(np.abs(mo) > 4 * np.sqrt(vo)))
    res["corr"] = float(np.corrcoef(mg[sel], mo[sel])[0, 1]) if sel.sum() > 2 else float("nan")
    print("gradient parity", w.transport.eabs_e, res)
    return res


def test_gradient_parity_kerma_mode():
    w, g, rho_maj = crop_case()
    res = grad_parity(w, g, rho_maj, 3_200_000, K=32)
    assert res["n_vox"] >= 20
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
    """Directional derivatives of J = sum_u g_u D_u along 32 directions that
    scale the densities of a 4^3-voxel block by (1 + h): the adjoint's
    sum_{v in block} rho_v dJ/drho_v against central differences
    [J(1 + h) - J(1 - h)] / (2 h) of the GPU forward with common random
    numbers and a fixed majorant (kerma mode, where the estimator is exact).
    g is the indicator of the downstream quarter of the phantom (J = its summed
    dose) and the blocks lie upstream in the field, so each derivative is
    resolved (the block's attenuation shadows the region). A single 2 mm voxel
    holds too few interactions for a per-voxel difference at any affordable
    history count (with common random numbers it rests on a handful of
    acceptance flips, far from normal errors), and the gradient of the loss
    sum (D - T)^2 is mostly noise at this scale; the loss's own gradient is
    exercised by the autograd test."""
    w, rho_t, rho_maj = _fd_setup()
    rho_maj = [1.15 / 1.1 * r for r in rho_maj]
    ph = w.phantom
    e = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=8).setup(w)
    e.set_majorant(rho_maj)
    e.run(8_000_000, seed=31)
    D, _ = e.dose()
    nz, ny, nx = ph.rho.shape
    zi = np.repeat(np.arange(nz), ny * nx)
    g = (zi >= 3 * nz // 4).astype(np.float64)
    rho0 = ph.rho.reshape(-1).astype(np.float32)
    blk = (np.arange(nz)[:, None, None] // 4 * (ny // 4) * (nx // 4)
           + np.arange(ny)[None, :, None] // 4 * (nx // 4) + np.arange(nx)[None, None, :] // 4)
    blk = blk.reshape(-1)
    nb = blk.max() + 1
    bdose = np.bincount(blk, weights=D, minlength=nb)
    bz = np.bincount(blk, weights=zi, minlength=nb) / np.bincount(blk, minlength=nb)
    bdose[bz >= nz // 2] = 0.0          # upstream half only
    blocks = np.random.default_rng(4).choice(np.argsort(bdose)[-48:], 32, replace=False)
    # adjoint: K batches of independent histories, projected on the directions
    K, na = 16, 256_000_000
    Ba = np.array([e.adjoint(g, na // K, seed=33, first_hist=k * (na // K))[0].copy()
                   for k in range(K)])
    Pa = np.array([[np.sum(Ba[k][blk == b] * rho0[blk == b]) for b in blocks] for k in range(K)])
    ma, va = batch_stats(Pa)
    # central differences, KF batches per side
    h, nf, KF = 0.05, 64_000_000, 8
    fd = np.zeros((KF, len(blocks)))
    for i, b in enumerate(blocks):
        J = []
        for sgn in (1.0, -1.0):
            r = rho0.copy()
            r[blk == b] = (rho0[blk == b] * (1.0 + sgn * h)).astype(np.float32)
            e.load_phantom(ph, rho=r.reshape(ph.rho.shape))
            Jk = []
            for k in range(KF):
                e.reset()
                e.run(nf // KF, seed=34, first_hist=k * (nf // KF))
                Jk.append(g @ e.dose()[0])
            J.append(np.array(Jk))
        fd[:, i] = (J[0] - J[1]) / (2.0 * h)
    e.close()
    mf, vf = batch_stats(fd)
    z = (ma - mf) / np.sqrt(va + vf)
    print("adjoint vs FD (block directions): z", np.round(z, 2))
    print("  adj", ma[:6], "+-", np.sqrt(va[:6]), "\n  fd ", mf[:6], "+-", np.sqrt(vf[:6]))
    assert np.mean(np.abs(z) < 3.0) >= 0.9, z
    assert np.mean(z * z) < 2.0, z
    assert abs(z.mean()) < 4.0 / np.sqrt(len(z)), z
    # the comparison has power: most directional derivatives are resolved by
    # both methods
    assert np.mean(np.abs(ma) > 3.0 * np.sqrt(va)) > 0.5
    assert np.mean(np.abs(mf) > 3.0 * np.sqrt(vf)) > 0.5


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


@pytest.mark.parametrize("coupled", [False, True])
def test_wavefront_adjoint_replays_plain(coupled):
    """The wavefront adjoint (G_h in a per-history buffer, particles of a
    history in different lanes and passes) runs the same histories as the
    plain one (G_h in a register): equal up to the order of FP32 sums."""
    w, g, rho_maj = crop_case(transport=S.Transport() if coupled else KERMA)
    out = []
    for kern in (G.KERNEL_PLAIN, G.KERNEL_WAVEFRONT):
        e = G.Engine(0, kernel=kern, n_batches=8).setup(w)
        e.set_majorant(rho_maj)
        m, v = e.adjoint(g, 200_000, seed=51)
        out.append((m.copy(), v.copy()))
        e.close()
    (mp_, vp_), (mw, vw) = out
    big = np.abs(mp_) > 0.05 * np.abs(mp_).max()
    assert big.sum() > 50
    rel = np.abs(mw[big] - mp_[big]) / np.abs(mp_[big])
    assert np.median(rel) < 1e-4, np.median(rel)
    assert np.percentile(rel, 99) < 1e-2
    np.testing.assert_allclose(mw.sum(), mp_.sum(), rtol=1e-3)
