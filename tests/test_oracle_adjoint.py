"""Pins of the oracle's likelihood-ratio dose gradient (the path-replay adjoint's
reference), each against something other than the estimator itself:

* the derivatives of the uncollided fraction exp(-kappa sum rho dz) of a pencil
  beam and of the probability that its first real interaction is in a given
  voxel, closed forms (pin the virtual and the real score terms, their signs,
  kappa and the fixed majorant);
* the score alone has mean zero in every voxel (pins the balance of the real
  term 1/rho against the virtual term);
* central finite differences of the oracle's own forward dose with common
  random numbers and a fixed majorant (pins the whole estimator: G_h, the
  score, the explicit -g D / rho term).
All in "kerma mode" (electrons absorbed where they are made), where the
estimator is exact: only the photon Woodcock acceptance depends on density."""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O
import synthetic as S

KERMA = S.Transport(eabs_e=1e3)


def column_phantom(seed=1, nz=10):
    rng = np.random.default_rng(seed)
    mat = np.zeros((nz, 3, 3), np.uint8)
    rho = rng.uniform(0.5, 1.5, (nz, 3, 3)).astype(np.float32)
    return S.Phantom(mat, rho, 1.0, 1.0, 1.0, [S.water()])


def small_phantom():
    rng = np.random.default_rng(2)
    n = 4
    mat = np.zeros((n, n, n), np.uint8)
    mat[2:] = 1
    rho = (np.where(mat == 0, 1.0, 1.6) * rng.uniform(0.8, 1.2, (n, n, n))).astype(np.float32)
    ph = S.Phantom(mat, rho, 1.0, 1.0, 1.0, [S.water(), S.bone()])
    src = S.Source(S.PHOTON, 1, 2.0, 2.0, 1.0, 1.0, 1.0)
    g = rng.uniform(-1.0, 1.0, n ** 3)
    return ph, src, g


RHO_MAJ = [2.0, 2.5]


@pytest.mark.parametrize("j0", [-1, 3])
def test_primary_event_derivative_closed_form(j0):
    """dP/drho along a pencil beam for P = uncollided fraction (j0 = -1) and
    P = probability that the first real interaction is in column voxel j0."""
    ph = column_phantom()
    src = S.Source(S.PHOTON, 0, 1.5, 1.5, 0.0, 0.0, 1.0)   # centre of the middle column
    target = -1 if j0 < 0 else j0 * 9 + 4
    m, var = O.lr_primary(ph, src, KERMA, 100_000, target=target, seed=3, rho_maj=[2.0])
    kappa = O.lib().or_mu_total(O.material(S.water()), 1.0)
    col = ph.rho[:, 1, 1].astype(np.float64)     # chords of 1 cm
    nz = len(col)
    if j0 < 0:
        exact = np.full(nz, -kappa * np.exp(-kappa * col.sum()))
    else:
        before = np.exp(-kappa * col[:j0].sum())
        P = before * (1.0 - np.exp(-kappa * col[j0]))
        exact = np.zeros(nz)
        exact[:j0] = -kappa * P
        exact[j0] = before * kappa * np.exp(-kappa * col[j0])
    on = m.reshape(ph.mat.shape)[:, 1, 1]
    sd = np.sqrt(var.reshape(ph.mat.shape)[:, 1, 1])
    live = exact != 0.0
    z = (on[live] - exact[live]) / sd[live]
    assert np.all(np.abs(z) < 4.5), z
    np.testing.assert_allclose(on[live], exact[live], rtol=0.1)
    assert np.all(on[~live] == 0.0)
    off = m.reshape(ph.mat.shape).copy()
    off[:, 1, 1] = 0.0
    assert np.all(off == 0.0)     # the primary never leaves its column before the event


def test_score_has_mean_zero():
    ph, src, _ = small_phantom()
    m, var, _ = O.adjoint(ph, src, KERMA, None, 30_000, seed=9, n_batches=20, rho_maj=RHO_MAJ)
    hit = var > 0
    z = m[hit] / np.sqrt(var[hit])
    assert hit.sum() > 40
    assert np.max(np.abs(z)) < 5.0
    # chi-square of 64 (weakly correlated) voxels: generous bound
    assert np.mean(z * z) < 2.0


def _fd_batch(args):
    k, v, n_per, h = args
    import oracle as O2
    import synthetic as S2
    ph, src, g = small_phantom()
    out = []
    for sgn in (1.0, -1.0):
        r = ph.rho.astype(np.float64).reshape(-1).copy()
        r[v] *= 1.0 + sgn * h
        r32 = r.astype(np.float32)
        p2 = S2.Phantom(ph.mat, r32.reshape(ph.mat.shape), 1.0, 1.0, 1.0, ph.materials)
        res = O2.run(p2, src, KERMA, n_per, seed=7, first_hist=k * n_per, n_batches=1,
                     rho_maj=RHO_MAJ)
        out.append(g @ (res.sum_q / n_per / r32.astype(np.float64)))
    rv = np.float64(ph.rho.reshape(-1)[v])
    # the central difference of J = sum_u g_u D_u over the density actually used
    return (out[0] - out[1]) / (rv * (1.0 + h) - rv * (1.0 - h))


@pytest.mark.parametrize("v", [5, 37])
def test_adjoint_matches_central_differences(v):
    ph, src, g = small_phantom()
    n_batches, n_per, h = 8, 12_500, 0.1
    N = n_batches * n_per
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, n_batches)) as pool:
        fd = np.array(pool.map(_fd_batch, [(k, v, n_per, h) for k in range(n_batches)]))
    gm, gv, _ = O.adjoint(ph, src, KERMA, g, N, seed=5, n_batches=20, rho_maj=RHO_MAJ)
    fd_m, fd_se = fd.mean(), fd.std(ddof=1) / np.sqrt(n_batches)
    sig = np.sqrt(gv[v] + fd_se ** 2)
    assert abs(gm[v] - fd_m) < 4.0 * sig, (gm[v], fd_m, sig)
    # power: the explicit -g D / rho term alone is many sigma, so dropping it
    # (or the score term it nearly cancels) would fail this test
    r = O.run(ph, src, KERMA, N, seed=5, n_batches=20, rho_maj=RHO_MAJ)
    D = r.sum_q / N / ph.rho.reshape(-1).astype(np.float64)
    explicit = g[v] * D[v] / ph.rho.reshape(-1)[v]
    assert abs(explicit) > 10.0 * sig


def test_majorant_below_maximum_is_rejected():
    ph, src, _ = small_phantom()
    with pytest.raises(ValueError):
        O.run(ph, src, KERMA, 10, rho_maj=[0.5, 0.5])
