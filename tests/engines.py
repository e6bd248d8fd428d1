"""Runs of both engines for the two-verdict parity comparison (test
infrastructure, shared by the GPU tests and the smoke check).

Each engine runs K independent sets of nk histories (disjoint history ids):
their K doses feed the permutation gate; their pooled tally -- for the GPU,
the K runs' moments added into one tally through gbmc_add_moments, so the
variance comes from K times batches_per_run batches; for the oracle, the
history-by-history sums of Eq. 1-2 -- gives the accurately estimated variance
that the literal gate needs.
"""
import numpy as np

import oracle as O


def gpu_dual(w, K, nk, seed, kernel=0, batches_per_run=50, device=0, **kw):
    """(K batch doses, pooled dose, pooled variance, summed statistics)."""
    import paper_2003_00796_gb300 as G
    e = G.Engine(device, kernel=kernel, n_batches=batches_per_run, **kw).setup(w)
    B, s1, s2, N, Kb = [], 0.0, 0.0, 0, 0
    tot = {}
    for k in range(K):
        e.reset()
        e.run(nk, seed=seed, first_hist=k * nk)
        B.append(e.dose()[0])
        a1, a2, n, kb = e.moments()
        s1, s2, N, Kb = s1 + a1, s2 + a2, N + n, Kb + kb
        st = e.stats()
        for key, val in st.items():
            if key == "error_flags":
                tot[key] = tot.get(key, 0) | val
            elif isinstance(val, (int, float)) and not key.endswith("_ms"):
                tot[key] = tot.get(key, 0) + val
    e.reset()
    e.add_moments(s1, s2, N, Kb)
    d, v = e.dose()
    tot["pooled_batches"] = Kb
    e.close()
    return np.array(B), d, v, tot


def oracle_dual(w, K, nk, seed, n_threads):
    """(K batch doses, pooled dose, its history-by-history variance (Eq. 2))."""
    B, acc = [], None
    for k in range(K):
        r = O.run(w.phantom, w.source, w.transport, nk, seed=seed, first_hist=k * nk,
                  n_batches=max(2, n_threads), n_threads=n_threads, vr=getattr(w, "vr", None))
        B.append(r.dose)
        acc = r if acc is None else O.OracleResult(
            acc.n_hist + r.n_hist, acc.n_batches + r.n_batches, acc.sum_q + r.sum_q,
            acc.sum_q2 + r.sum_q2, acc.batch_s1 + r.batch_s1, acc.batch_s2 + r.batch_s2,
            r.stats, r.mass)
    return np.array(B), acc.dose, acc.dose_sigma ** 2
