"""The parity statistics themselves: the batch permutation gate keeps its size
under correlated voxels and has power against a small planted bias.

The planted mistakes live in the oracle's output on the CPU (a scaled dose),
never in the CUDA path."""
import numpy as np

import oracle as O
import synthetic as S
from parity import permutation_gate


def correlated_batches(rng, K, n, corr_len, scale=1.0):
    # smooth (spatially correlated) noise around a profile, per batch
    x = np.arange(n)
    prof = 1.0 + np.exp(-((x - n / 2) / (n / 6)) ** 2)
    ker = np.exp(-0.5 * (np.arange(-3 * corr_len, 3 * corr_len + 1) / corr_len) ** 2)
    out = []
    for _ in range(K):
        e = np.convolve(rng.normal(size=n + len(ker) - 1), ker, "valid")
        out.append(scale * prof * (1.0 + 0.05 * e / ker.sum() ** 0.5))
    return np.array(out)


def test_permutation_gate_size_under_correlation():
    rng = np.random.default_rng(3)
    passes = 0
    textbook_fail = 0
    for trial in range(40):
        a = correlated_batches(rng, 20, 400, 8)
        b = correlated_batches(rng, 20, 400, 8)
        r = permutation_gate(a, b, thr=0.1, n_perm=300, seed=trial)
        passes += r["pass"]
        textbook_fail += r["p_chi2_textbook"] < 0.01
    # at alpha = 0.01 on two statistics, nearly all null comparisons pass,
    # while the independent-voxel chi-square rejects a large share of them
    assert passes >= 36
    assert textbook_fail >= 8


def test_permutation_gate_detects_small_bias():
    rng = np.random.default_rng(4)
    fails = 0
    for trial in range(10):
        a = correlated_batches(rng, 20, 400, 2)
        b = correlated_batches(rng, 20, 400, 2, scale=1.02)
        fails += not permutation_gate(a, b, thr=0.1, n_perm=300, seed=trial)["pass"]
    assert fails >= 9


def test_oracle_against_itself_and_a_planted_bias():
    w = S.workload_water_pencil()
    K, nk = 12, 1500
    run = lambda seed, first: O.run(w.phantom, w.source, w.transport, nk, seed=seed,
                                    first_hist=first, n_batches=2, n_threads=4).dose
    A = np.array([run(21, k * nk) for k in range(K)])
    B = np.array([run(22, k * nk) for k in range(K)])
    assert permutation_gate(A, B, thr=0.1, n_perm=500)["pass"]
    # a 6 % dose error planted in one oracle run is rejected
    assert not permutation_gate(A, 1.06 * B, thr=0.1, n_perm=500)["pass"]


def test_selection_on_the_pooled_mean_keeps_the_gate_exact_for_sparse_voxels():
    """Two engines drawn from one distribution, with sparsely populated voxels
    (0.2-3 compound events per batch, as at the configured sizes): the gate
    chooses its voxels on the mean of all batches and passes; choosing them
    on either engine's own mean (a voxel enters when one engine fluctuated
    high) inflates the observed chi-square beyond every reassignment and
    rejects identical engines."""
    from parity import batch_stats, permutation_gate
    rng = np.random.default_rng(1)
    nv, K = 50_000, 20
    lam = np.linspace(0.2, 3.0, nv)

    def batches():
        n = rng.poisson(lam, (K, nv))
        return rng.gamma(np.maximum(n, 1e-9), 1.0) * (n > 0)
    A, B = batches(), batches()
    assert permutation_gate(A, B, thr=0.1, n_perm=200)["pass"]
    mg, _ = batch_stats(A)
    mo, _ = batch_stats(B)
    dmax = max(mg.max(), mo.max())
    biased = (mg >= 0.1 * dmax) | (mo >= 0.1 * dmax)
    assert not permutation_gate(A, B, thr=0.1, n_perm=200, sel=biased)["pass"]
