"""Statistical comparison of two dose estimates (test infrastructure).

The paper compares codes bin by bin with 2-sigma error bars (Sec. 5.2) and by
the z-score histogram of voxels above 0.1 % of the maximum (Sec. 5.4). The
parity gate here: on voxels with dose >= thr * max, at least 95 % within two
combined standard deviations, and a global chi-square p-value > 0.01.

Both estimates must have the same number of histories (independent seeds): with
variances estimated from the data, a well-sampled estimate compared with a
sparsely sampled one gives a skewed, biased z even without any physics
difference. The gated voxels must also be well populated (relative sigma of a
few per cent): with ~15 events per voxel the noise of the variance estimates
alone inflates chi-square by 3-6 %, enough to fail p > 0.01 for two runs of the
same engine.
"""
import math

import numpy as np
from scipy import stats


def compare(d1, v1, d2, v2, thr=0.1):
    """z-scores of two dose estimates on the voxels whose dose -- estimated by
    the mean of the two, which is independent of their difference -- is at
    least thr of the maximum. (Selecting on either estimate alone would pick
    voxels where one of them fluctuated high, and inflate the differences of
    sparsely populated voxels.)"""
    d1, v1, d2, v2 = (np.asarray(x, np.float64).ravel() for x in (d1, v1, d2, v2))
    dm = 0.5 * (d1 + d2)
    sel = dm >= thr * dm.max()
    sc = np.sqrt(v1[sel] + v2[sel])
    ok = sc > 0
    z = (d1[sel][ok] - d2[sel][ok]) / sc[ok]
    n = int(z.size)
    chi2 = float(np.sum(z * z))
    p = float(stats.chi2.sf(chi2, n)) if n else float("nan")
    out = {
        "n_vox": n,
        "frac_2sigma": float(np.mean(np.abs(z) <= 2.0)) if n else float("nan"),
        "chi2": chi2,
        "dof": n,
        "p": p,
        "z_mean": float(z.mean()) if n else float("nan"),
        "z_std": float(z.std()) if n else float("nan"),
        "max_abs_z": float(np.abs(z).max()) if n else float("nan"),
    }
    out["literal_pass"] = literal_gate(out) if n else False
    return out


def outside_consistent(res, alpha=0.01):
    """Binomial reading of the 95 % rule: the number of voxels outside two
    combined sigma is consistent (upper tail p > alpha) with the 4.55 % that a
    standard normal puts there. With few gated voxels a literal 95 % bar fails
    a perfect engine often (80 voxels: about 30 % of the time)."""
    n = res["n_vox"]
    k = int(round((1.0 - res["frac_2sigma"]) * n))
    return float(stats.binom.sf(k - 1, n, 2 * stats.norm.sf(2.0))) > alpha


def literal_gate(res, min_frac=0.95, min_p=0.01, min_vox=10):
    """The parity gate exactly as written (no calibration): at least 95 % of
    the gated voxels within two combined sigma and the textbook chi-square
    (dof = number of voxels) p-value above 0.01. It assumes independent,
    normal z-scores with exactly known variances; for a perfect engine the
    expected fraction within 2 sigma is 95.45 %, so it is a sharp test only
    with many gated voxels (about 2e4 for a false-failure rate near 0.1 %)
    and variances estimated from many batches (or history by history)."""
    return bool(res["n_vox"] >= min_vox and res["frac_2sigma"] >= min_frac and res["p"] > min_p)


def gate(res, min_frac=0.95, min_p=0.01, min_vox=10):
    """>= 95 % of the gated voxels within 2 combined sigma (or, for a small
    voxel count, a count outside 2 sigma consistent with a normal) and a
    global chi-square p-value > 0.01."""
    frac_ok = res["frac_2sigma"] >= min_frac or outside_consistent(res)
    return res["n_vox"] >= min_vox and frac_ok and res["p"] > min_p


def rel_uncertainty(dose, var, thr=0.5):
    """Mean relative standard deviation over voxels with dose >= thr * max."""
    d = np.asarray(dose).ravel()
    s = np.sqrt(np.asarray(var).ravel())
    sel = d >= thr * d.max()
    return float(np.mean(s[sel] / d[sel]))


def batch_stats(B):
    """Per-voxel mean and variance of the mean from K independent batch means (K, nvox)."""
    B = np.asarray(B, np.float64)
    K = B.shape[0]
    m = B.mean(0)
    v = B.var(0, ddof=1) / K
    return m, v


def permutation_gate(Bg, Bo, thr=0.1, n_perm=2000, seed=0, alpha=0.01, sel=None):
    """Parity of two engines from K independent batch means each (arrays
    (K, nvox) of dose per batch). The statistics are those of ``compare``
    (chi-square over the voxels above thr * max, fraction within two combined
    sigma); their null distribution is obtained by randomly reassigning the 2K
    batches between the two engines. Voxel doses are correlated (one track
    deposits in many voxels), so the chi-square of independent voxels is not
    chi-square distributed; the permutation null is exact whatever the
    correlation, because under parity the 2K batches are exchangeable.
    Passes when the chi-square is not in the upper alpha tail and the 2-sigma
    fraction is at least 95 % or not in the lower alpha tail of its null, and
    the mean z-score (the first moment of the paper's z-score histogram check,
    which a uniform dose-scale error moves) is not in either alpha/2 tail.
    The gated voxels are chosen on the mean of all 2K batches, which every
    reassignment leaves unchanged: a selection on either engine's own mean
    would favour voxels where that engine fluctuated high, which the
    permutation null does not reproduce (with sparsely populated voxels this
    alone rejected two runs of the same engine).
    ``sel`` (a boolean voxel mask) replaces the threshold selection, e.g. for
    signed quantities such as gradients."""
    Bg = np.asarray(Bg, np.float64)
    Bo = np.asarray(Bo, np.float64)
    K = Bg.shape[0]
    allb = np.concatenate([Bg, Bo], 0)
    if sel is None:
        pooled = allb.mean(0)
        sel = pooled >= thr * pooled.max()
    X = allb[:, sel]

    def stat(a, b):
        ma, va = a.mean(0), a.var(0, ddof=1) / a.shape[0]
        mb, vb = b.mean(0), b.var(0, ddof=1) / b.shape[0]
        sc = np.sqrt(va + vb)
        ok = sc > 0
        z = (ma[ok] - mb[ok]) / sc[ok]
        return float(np.sum(z * z)), float(np.mean(np.abs(z) <= 2.0)), z

    chi2, frac, z = stat(X[:K], X[K:])
    zm = float(z.mean())
    rng = np.random.default_rng(seed)
    cn, fn, mn = np.empty(n_perm), np.empty(n_perm), np.empty(n_perm)
    for i in range(n_perm):
        idx = rng.permutation(2 * K)
        cn[i], fn[i], zp = stat(X[idx[:K]], X[idx[K:]])
        mn[i] = zp.mean()
    p_chi2 = float((1 + np.sum(cn >= chi2)) / (n_perm + 1))
    p_frac = float((1 + np.sum(fn <= frac)) / (n_perm + 1))
    p_zm = float((1 + np.sum(np.abs(mn) >= abs(zm))) / (n_perm + 1))
    res = {"n_vox": int(sel.sum()), "K": K, "chi2_per_dof": chi2 / max(1, z.size),
           "p_chi2_perm": p_chi2, "frac_2sigma": frac, "p_frac_perm": p_frac,
           "z_mean": zm, "p_zmean_perm": p_zm, "z_std": float(z.std()),
           "null_chi2_per_dof_median": float(np.median(cn)) / max(1, z.size),
           "p_chi2_textbook": float(stats.chi2.sf(chi2, z.size))}
    res["pass"] = bool(res["n_vox"] >= 10 and p_chi2 > alpha and p_zm > alpha
                       and (frac >= 0.95 or p_frac > alpha))
    # the gate as written, on the same z-scores (batch variances from K batches:
    # t-distributed, so this reading fails correct engines at small K)
    res["literal_pass"] = bool(res["n_vox"] >= 10 and frac >= 0.95 and res["p_chi2_textbook"] > 0.01)
    return res


def dual_gate(Bg, Bo, dg, vg, do, vo, thr=0.1, n_perm=1000, seed=0):
    """Both readings of the parity gate on one data set. Bg, Bo: K independent
    batch doses per engine (the permutation gate, exact under correlated
    voxels); (dg, vg), (do, vo): each engine's pooled dose and its variance
    estimated accurately -- from about a thousand batches (GPU batch
    estimator) or history by history (the oracle's Eq. 1-2) -- for the
    literal gate (>= 95 % within 2 sigma, textbook chi-square p > 0.01).
    Returns the permutation result with the literal comparison under
    "literal" and its verdict in "literal_pass"."""
    res = permutation_gate(Bg, Bo, thr=thr, n_perm=n_perm, seed=seed)
    lit = compare(dg, vg, do, vo, thr=thr)
    res["literal"] = {k: lit[k] for k in ("n_vox", "frac_2sigma", "chi2", "dof", "p", "z_mean",
                                           "z_std")}
    res["literal_pass"] = lit["literal_pass"]
    return res
