"""Pins of the oracle's event selection and kinematics against what physics and
mathematics fix, independently of the oracle's own formulas (Sec. 5.1 of the
paper tests each interaction routine in isolation against its model):

* photon interaction type: at a real collision the type is Compton, PE,
  Rayleigh or pair with probability mu_i(E) / mu(E) at the photon's current
  energy -- multinomial tests on the first and second interactions of
  primary photons (the second after a Compton energy loss);
* class II hard events: the counts of hard elastic, inelastic and
  bremsstrahlung events and of delta (null) events have mean equal to their
  compensators, the integrals of the partial cross sections (and of the step
  majorant minus their sum) over the mass thickness the tracks travelled at
  their CSDA energy -- a martingale identity that holds whatever the tracks
  do;
* two-body kinematics of hard inelastic collisions: energy and momentum
  conservation for an electron at rest;
* the screened Rutherford (Wentzel) law: its large-angle limit is the
  textbook unscreened Rutherford cross section (with Z(Z+1) for the atomic
  electrons), and its screening parameter lies within Moliere's stated
  accuracy of the Born-approximation screening angle computed here from the
  Thomas-Fermi atom (Moliere's three-exponential fit of the Thomas-Fermi
  function, Thomas-Fermi radius (9 pi^2 / 128)^(1/3) a_0 Z^(-1/3)).

Each pin is shown to fail when a plausible mistake is planted in a copy of the
oracle (``oracle.planted``): the checks below are functions so that the same
check runs on the oracle and on the planted copy.
"""
import ctypes as C
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
import synthetic as S

MEC2 = 0.51099895
ALPHA = 1 / 137.035999084
RE = 2.8179403262e-13


def slab(material, side=400.0):
    """One voxel of side cm: a homogeneous medium in which almost every primary
    interacts before it leaves."""
    return S.Phantom(np.zeros((1, 1, 1), np.uint8), np.full((1, 1, 1), material.rho, np.float32),
                     side, side, side, [material])


def partials(material, E):
    L = O.lib()
    M = C.byref(O.material(material))
    p = np.array([L.or_mu_compton(M, E), L.or_mu_pe(M, E), L.or_mu_rayleigh(M, E),
                  L.or_mu_pair(M, E)])
    return p / p.sum()


# ---------------------------------------------------------------------------
# (a) photon interaction type
# ---------------------------------------------------------------------------

TYPE_CASES = [(S.water(), 0.03), (S.water(), 1.0), (S.water(), 10.0),
              (S.bone(), 0.03), (S.bone(), 1.0), (S.bone(), 10.0)]


def first_type_pvalues(n=20_000):
    """Multinomial chi-square p-values of the first-interaction type counts
    against mu_i / mu at the source energy, one per (material, energy)."""
    expected = [partials(m, E) for m, E in TYPE_CASES]   # closed forms, pinned elsewhere
    out = []
    for (m, E), p in zip(TYPE_CASES, expected):
        src = S.Source(S.PHOTON, 0, 200.0, 200.0, 0.0, 0.0, E)
        P = O.Problem(slab(m), src, S.Transport(eabs_g=1e-3))
        _, typ = P.first_interactions(seed=17, first=0, n=n)
        t = typ[typ > 0]
        obs = np.array([np.sum(t == k) for k in (1, 2, 3, 4)], float)
        keep = p > 0
        exp = p[keep] * t.size
        chi2 = float(np.sum((obs[keep] - exp) ** 2 / exp))
        out.append((m.name, E, stats.chi2.sf(chi2, keep.sum() - 1), obs[~keep].sum()))
    return out


def second_type_zscores(n=40_000):
    """Second real interaction of 100 keV primary photons in bone (after a
    Compton or Rayleigh event, at a spread of lower energies): per type,
    (count - sum_j p_i(E_j)) / sqrt(sum_j p_i (1 - p_i)) with p_i(E_j) the
    share of type i at the energy E_j the photon had before that interaction."""
    m = S.bone()
    src = S.Source(S.PHOTON, 0, 200.0, 200.0, 0.0, 0.0, 0.1)
    P = O.Problem(slab(m), src, S.Transport(eabs_g=1e-3))
    _, E, typ = P.nth_interactions(2, seed=23, first=0, n=n)
    sel = typ > 0
    E, typ = E[sel], typ[sel]
    p = np.array([partials(m, e) for e in E])   # evaluated with the unplanted oracle
    return E, typ, p


def z_of(typ, p):
    z = []
    for k in range(3):
        ind = (typ == k + 1).astype(float)
        z.append(float((ind - p[:, k]).sum() / math.sqrt((p[:, k] * (1 - p[:, k])).sum())))
    return z


def test_first_interaction_type_follows_partial_attenuation():
    for name, E, pval, impossible in first_type_pvalues():
        assert impossible == 0, (name, E)     # no pair below threshold
        assert pval > 1e-3, (name, E, pval)


def test_second_interaction_type_uses_the_current_energy():
    E, typ, p = second_type_zscores()
    assert E.min() < 0.08 and E.max() <= 0.1 + 1e-12   # energies after a first scatter
    for k, z in enumerate(z_of(typ, p)):
        assert abs(z) < 4.0, (k, z)


PLANT_SWAP_PE_RAYLEIGH = [(
    "int type = (c < pc) ? 1 : (c < pc + pp) ? 2 : (c < pc + pp + pr) ? 3 : 4;",
    "int type = (c < pc) ? 1 : (c < pc + pr) ? 2 : (c < pc + pp + pr) ? 3 : 4;")]
PLANT_PE_AT_SOURCE_ENERGY = [(
    "const double pc = or_mu_compton(mat, E), pp = or_mu_pe(mat, E);",
    "const double pc = or_mu_compton(mat, E), pp = or_mu_pe(mat, p->src.energy);")]


def test_planted_type_mistakes_fail_the_type_pins():
    with O.planted(PLANT_SWAP_PE_RAYLEIGH, "swap_pe_ray"):
        res = first_type_pvalues(n=20_000)
    assert min(pv for _, _, pv, _ in res) < 1e-6
    E, _, p = second_type_zscores(n=30_000)
    with O.planted(PLANT_PE_AT_SOURCE_ENERGY, "pe_src_energy"):
        _, E2, typ2 = O.Problem(slab(S.bone()), S.Source(S.PHOTON, 0, 200.0, 200.0, 0.0, 0.0, 0.1),
                                S.Transport(eabs_g=1e-3)).nth_interactions(2, seed=23, first=0, n=30_000)
    sel = typ2 > 0
    p2 = np.array([partials(S.bone(), e) for e in E2[sel]])
    assert max(abs(z) for z in z_of(typ2[sel], p2)) > 6.0


# ---------------------------------------------------------------------------
# (b) class II hard events: counts against their compensators
# ---------------------------------------------------------------------------

def hard_event_z(n=3000, energy=3.0, particle=S.ELECTRON, materials=None, seed=31):
    """Electrons (or positrons) through a water/bone slab stack (material
    changes truncate steps, voxel crossings do not), instrumented: z-scores
    (count - compensator) / sqrt(compensator) of the hard elastic,
    inelastic, bremsstrahlung and delta events."""
    mats = materials or [S.water(), S.bone()]
    nz = 16
    mat = np.zeros((nz, 8, 8), np.uint8)
    mat[4:8] = 1 if len(mats) > 1 else 0
    mat[12:] = 1 if len(mats) > 1 else 0
    rho = np.array([m.rho for m in mats], np.float32)[mat]
    ph = S.Phantom(mat, rho, 2.0, 2.0, 0.25, mats)
    src = S.Source(particle, 0, 8.0, 8.0, 0.0, 0.0, energy)
    r = O.run(ph, src, S.Transport(), n, seed=seed, n_batches=8, n_threads=8, instrument=True)
    st = r.stats
    comp = {"el": st["i_el"], "inel": st["i_inel"], "br": st["i_br"],
            "delta": st["i_hat"] - st["i_el"] - st["i_inel"] - st["i_br"]}
    cnt = {"el": st["n_hard_el"], "inel": st["n_hard_inel"], "br": st["n_hard_br"],
           "delta": st["n_delta"]}
    return {k: ((cnt[k] - comp[k]) / math.sqrt(max(comp[k], 1.0)), cnt[k], comp[k]) for k in comp}


@pytest.mark.parametrize("particle,energy", [(S.ELECTRON, 3.0), (S.ELECTRON, 15.0),
                                             (S.POSITRON, 3.0)])
def test_hard_event_counts_match_their_compensators(particle, energy):
    z = hard_event_z(particle=particle, energy=energy)
    for k, (zz, cnt, comp) in z.items():
        assert comp > 200, (k, comp)             # every kind of event is exercised
        assert abs(zz) < 4.0, (k, zz, cnt, comp)


PLANT_SWAP_INEL_BREMS = [("    } else if (c < sel + sin_) {\n      w->st.n_hard_inel++;",
                          "    } else if (c < sel + sbr) {\n      w->st.n_hard_inel++;")]
PLANT_NO_DELTA = [("    const double c = su[4] * smaj;",
                   "    const double c = su[4] * (sel + sin_ + sbr);")]
PLANT_STEP_START_ENERGY = [("    hard_xs(p, t.m, pos, e->E, &sel, &sin_, &sbr);",
                            "    hard_xs(p, t.m, pos, T0, &sel, &sin_, &sbr);")]


@pytest.mark.parametrize("plant,tag", [(PLANT_SWAP_INEL_BREMS, "swap_inel_br"),
                                       (PLANT_NO_DELTA, "no_delta"),
                                       (PLANT_STEP_START_ENERGY, "t0_energy")])
def test_planted_hard_event_mistakes_fail_the_compensator_pin(plant, tag):
    with O.planted(plant, tag):
        z = hard_event_z()
    assert max(abs(zz) for zz, _, _ in z.values()) > 6.0, z


# ---------------------------------------------------------------------------
# (c) two-body kinematics of hard inelastic collisions
# ---------------------------------------------------------------------------

def momentum_residual(n=2000, seed=5):
    """Largest relative violation of momentum conservation
    p(T) u = p(T - W) u' + p(W) u_d over random collisions, and of the
    opposite-azimuth condition (u, u', u_d coplanar)."""
    rng = np.random.default_rng(seed)
    L = O.lib()
    worst, worst_plane = 0.0, 0.0

    def p_of(T):
        return math.sqrt(T * (T + 2 * MEC2))

    for _ in range(n):
        T = math.exp(rng.uniform(math.log(0.03), math.log(20.0)))
        W = rng.uniform(0.0, 1.0) * T * 0.999 + 1e-4 * T
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        phi = rng.uniform(0, 2 * math.pi)
        ua = (C.c_double * 3)(*u)
        up, ud = (C.c_double * 3)(), (C.c_double * 3)()
        L.or_binary_collision(T, W, phi, ua, up, ud)
        up, ud = np.array(up[:]), np.array(ud[:])
        res = p_of(T) * u - p_of(T - W) * up - p_of(W) * ud
        worst = max(worst, float(np.linalg.norm(res)) / p_of(T))
        worst_plane = max(worst_plane, abs(float(np.dot(np.cross(up, ud), u))))
    return worst, worst_plane


def test_two_body_kinematics_conserve_momentum():
    worst, plane = momentum_residual()
    assert worst < 1e-12 and plane < 1e-12, (worst, plane)


def test_planted_kinematics_mistake_fails_momentum_pin():
    plant = [("  rotate(ud, cd, phi + PI);", "  rotate(ud, cp, phi + PI);")]
    with O.planted(plant, "cd_cp"):
        worst, _ = momentum_residual(n=300)
    assert worst > 1e-3


# ---------------------------------------------------------------------------
# (d) screened Rutherford (Wentzel) elastic scattering
# ---------------------------------------------------------------------------

def oracle_screening(Z, T):
    """The oracle's screening parameter A, read off its DCS:
    dcs(mu = 1) / dcs(mu = -1) = ((1 + A) / A)^2."""
    L = O.lib()
    r = L.or_elastic_dcs(Z, T, 1.0) / L.or_elastic_dcs(Z, T, -1.0)
    return 1.0 / (math.sqrt(r) - 1.0)


def rutherford_ratio(Z, T, theta):
    """Oracle DCS per steradian over the textbook unscreened Rutherford cross
    section (Z(Z+1) r_e^2 (m c^2)^2 / (4 (p beta c)^2 sin^4(theta / 2)), with
    p c = sqrt(T (T + 2 m c^2)) and beta = p c / (T + m c^2)), with the
    oracle's own screening factor ((1 - mu) / (1 - mu + 2A))^2 divided out
    (below 1e-3 of a correction except for heavy atoms at low energy), so that
    the prefactor is compared alone."""
    pc = math.sqrt(T * (T + 2 * MEC2))
    pbc = pc * pc / (T + MEC2)
    ruth = Z * (Z + 1) * (RE * MEC2) ** 2 / (4 * pbc ** 2 * math.sin(theta / 2) ** 4)
    x = 1.0 - math.cos(theta)
    screen = (x / (x + 2.0 * oracle_screening(Z, T))) ** 2
    return O.lib().or_elastic_dcs(Z, T, math.cos(theta)) / (2 * math.pi) / ruth / screen


def screening_ratio(Z, T):
    """The oracle's screening parameter A (from its DCS: dcs(mu=1)/dcs(mu=-1)
    = ((1 + A)/A)^2) over chi_a^2 / 4, chi_a the Born-approximation screening
    angle of the Thomas-Fermi atom: Moliere's definition
    -ln chi_a = lim_K [int_0^K q(chi) dchi/chi - ln K] + 1/2 for the
    screening factor q of the DCS, here of the potential
    (Z e^2 / r) sum_i a_i exp(-b_i r / a_TF) (Moliere's fit of the
    Thomas-Fermi function: a = 0.35, 0.55, 0.10; b = 0.3, 1.2, 6.0),
    chi in units of chi_0 = lambda / a_TF, lambda the reduced de Broglie
    wavelength, a_TF = (9 pi^2 / 128)^(1/3) a_0 Z^(-1/3)."""
    A = oracle_screening(Z, T)
    a, b = (0.35, 0.55, 0.10), (0.3, 1.2, 6.0)

    def q(x):
        return sum(ai * x * x / (x * x + bi * bi) for ai, bi in zip(a, b)) ** 2
    i1 = integrate.quad(lambda x: q(x) / x, 0.0, 1.0, limit=400)[0]
    i2 = integrate.quad(lambda x: (q(x) - 1.0) / x, 1.0, np.inf, limit=400)[0]
    chi_a_over_chi0 = math.exp(-(i1 + i2 + 0.5))
    c_tf = (9 * math.pi ** 2 / 128) ** (1 / 3)          # Thomas-Fermi radius in a_0 Z^(-1/3)
    p_mc = math.sqrt(T * (T + 2 * MEC2)) / MEC2          # momentum in m c
    chi0 = ALPHA * Z ** (1 / 3) / (c_tf * p_mc)          # lambda / a_TF, a_0 = lambda_C / alpha
    return A / (0.25 * (chi_a_over_chi0 * chi0) ** 2)


def test_elastic_large_angle_limit_is_rutherford():
    for Z in (1, 6, 8, 20, 82):
        for T in (0.05, 1.0, 20.0):
            for th in (math.pi / 2, 2.5, math.pi):
                assert rutherford_ratio(Z, T, th) == pytest.approx(1.0, rel=1e-9), (Z, T, th)


def test_elastic_screening_matches_thomas_fermi_born_value():
    # small alpha Z / beta: Moliere's screening formula reduces to its Born
    # limit, which it reproduces to a few per cent (1.13 against 1.172 here)
    for Z in (6, 8):
        for T in (5.0, 20.0):
            assert screening_ratio(Z, T) == pytest.approx(1.0, abs=0.05), (Z, T)


def test_planted_elastic_mistakes_fail_the_wentzel_pins():
    with O.planted([("  *C = z * (z + 1.0) * RE * RE * f * f;", "  *C = z * z * RE * RE * f * f;")], "c_z2"):
        assert abs(rutherford_ratio(8, 1.0, math.pi) - 1.0) > 0.05
    with O.planted([("(0.885 * sqrt(p2))", "(0.80 * sqrt(p2))")], "tf_radius"):
        assert abs(screening_ratio(8, 20.0) - 1.0) > 0.1
    with O.planted([("(1.13 + 3.76", "(1.30 + 3.76")], "moliere_113"):
        assert abs(screening_ratio(8, 20.0) - 1.0) > 0.1
