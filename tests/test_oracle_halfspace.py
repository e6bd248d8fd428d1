"""The paper's kernel-throughput settings (Sec. 6.1: vacuum / water half-space,
point source aimed at the plane) on the oracle: each kind tracks exactly the
particle types it names, every history closes its energy ledger in FP64, and
the 1 MeV photon kinds attenuate like exp(-mu z) before their first real
interaction (the uncollided fraction through the whole block)."""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S


@pytest.mark.parametrize("kind", S.HALFSPACE_KINDS)
def test_halfspace_kinds(kind):
    w = S.workload_halfspace(kind, 0, n=16, d=2e-4 if kind == "e40keV" else 1.0)
    n = 300 if kind != "g1MeV" else 5000
    r = O.run(w.phantom, w.source, w.transport, n, seed=3, n_batches=4)
    st = r.stats
    assert st["n_hist"] == n
    assert st["max_ledger_rel"] < 1e-9
    assert st["e_dep"] + st["e_esc"] == pytest.approx(st["e_src"], rel=1e-9)
    if kind == "e40keV":
        assert st["n_tent"] == 0 and st["n_e_steps"] > 50 * n
        assert st["e_src"] == pytest.approx(0.040 * n, rel=1e-12)
    else:
        assert st["n_tent"] >= n
        assert (st["n_e_steps"] == 0) == (kind == "g1MeV")


def test_halfspace_uncollided_fraction():
    """1 MeV photons through the 16 cm deep water block: the fraction with no
    real interaction is exp(-mu 16 cm) (binomial, 4 sigma), i.e. the source
    sits on the plane and aims along its normal."""
    w = S.workload_halfspace("g1MeV", 0, n=16, d=1.0)
    P = O.Problem(w.phantom, w.source, w.transport)
    n = 40_000
    xyz, typ = P.first_interactions(25, 0, n)
    mu = O.lib().or_mu_total(O.material(S.water()), 1.0)
    p = math.exp(-mu * 16.0)
    frac = float(np.mean(typ == 0))
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n)
    hit = typ != 0
    # first interactions lie on the beam axis, at the face centre's voxel centre
    np.testing.assert_allclose(xyz[hit, 0], 8.5, atol=1e-12)
    np.testing.assert_allclose(xyz[hit, 1], 8.5, atol=1e-12)
    # depth of the first interaction: exponential with rate mu, truncated at 16 cm
    z = xyz[hit, 2]
    mean_exact = 1.0 / mu - 16.0 * p / (1.0 - p)
    assert abs(z.mean() - mean_exact) < 4 * z.std() / math.sqrt(len(z))
