"""Statistical comparison of two dose estimates (test infrastructure).

The paper compares codes bin by bin with 2-sigma error bars (Sec. 5.2) and by
the z-score histogram of voxels above 0.1 % of the maximum (Sec. 5.4). The
parity gate here: on voxels with dose >= thr * max, at least 95 % within two
combined standard deviations, and a global chi-square p-value > 0.01.
"""
import math

import numpy as np
from scipy import stats


def compare(d1, v1, d2, v2, thr=0.1):
    d1, v1, d2, v2 = (np.asarray(x, np.float64).ravel() for x in (d1, v1, d2, v2))
    dmax = max(d1.max(), d2.max())
    sel = (d1 >= thr * dmax) | (d2 >= thr * dmax)
    sc = np.sqrt(v1[sel] + v2[sel])
    ok = sc > 0
    z = (d1[sel][ok] - d2[sel][ok]) / sc[ok]
    n = int(z.size)
    chi2 = float(np.sum(z * z))
    p = float(stats.chi2.sf(chi2, n)) if n else float("nan")
    return {
        "n_vox": n,
        "frac_2sigma": float(np.mean(np.abs(z) <= 2.0)) if n else float("nan"),
        "chi2": chi2,
        "dof": n,
        "p": p,
        "z_mean": float(z.mean()) if n else float("nan"),
        "z_std": float(z.std()) if n else float("nan"),
        "max_abs_z": float(np.abs(z).max()) if n else float("nan"),
    }


def gate(res, min_frac=0.95, min_p=0.01, min_vox=10):
    return res["n_vox"] >= min_vox and res["frac_2sigma"] >= min_frac and res["p"] > min_p


def rel_uncertainty(dose, var, thr=0.5):
    """Mean relative standard deviation over voxels with dose >= thr * max."""
    d = np.asarray(dose).ravel()
    s = np.sqrt(np.asarray(var).ravel())
    sel = d >= thr * d.max()
    return float(np.mean(s[sel] / d[sel]))
