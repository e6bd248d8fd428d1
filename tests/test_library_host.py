"""Host-side checks of the CUDA library that need no GPU.

* libgbmc.so loads and exports every entry point declared in include/gbmc.h;
* the FP32 log-log tables that the kernels interpolate (built from the closed
  forms in FP64 by the library's own host code) agree with the oracle's
  independent FP64 evaluation of the same quantities;
* the Walker alias table reproduces the source bin weights exactly;
* argument validation of the C ABI.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
import paper_2003_00796_gb300 as G
import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gbmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gbmc_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = G.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", G._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s(gbmc_\w+)", out))
    assert set(names) <= exported


def test_checked_library_has_the_same_abi():
    """libgbmc_checked.so (GBMC_CHECKED build) exports every declared symbol,
    says which variant it is, loads beside libgbmc.so, and rejects bad
    arguments of gbmc_check_index before touching the device."""
    Lc, L = G.lib(checked=True), G.lib(checked=False)
    out = subprocess.run(["nm", "-D", "--defined-only", G._build.LIB_CHECKED], capture_output=True,
                         text=True).stdout
    assert set(declared_symbols()) <= set(re.findall(r"\s[TW]\s(gbmc_\w+)", out))
    assert (Lc.gbmc_build_checked(), L.gbmc_build_checked()) == (1, 0)
    one = np.zeros(1, np.int32)
    b = np.ones(1, np.int64)
    f = np.zeros(1, np.uint32)
    for lib_ in (L, Lc):
        assert lib_.gbmc_check_index(0, one.ctypes.data, b.ctypes.data, -1, one.ctypes.data,
                                     f.ctypes.data) == 1
        assert lib_.gbmc_check_index(0, None, b.ctypes.data, 1, one.ctypes.data, f.ctypes.data) == 1
        assert lib_.gbmc_check_index(0, None, None, 0, None, None) == 0
    # host-side table code is the same in both
    mats = [S.water(), S.bone()]
    x = np.geomspace(0.02, 15.0, 50)
    vals = []
    for checked in (False, True):
        e = G.Engine(device=-1, checked=checked)
        assert e.checked == checked
        e.set_materials(mats, S.Transport(), 20.0)
        vals.append(e.table_eval(0, 1, x))
        e.close()
    np.testing.assert_array_equal(vals[0], vals[1])


def test_memory_limit_calls_on_a_host_context():
    """gbmc_set_mem_limit / gbmc_mem_info: a host-only context holds no device
    buffers, so its count stays 0 whatever it builds; null arguments are
    rejected."""
    e = G.Engine(device=-1)
    assert e.mem_info() == (0, 0)
    e.set_mem_limit(123)
    e.set_materials([S.water()], S.Transport(), 2.0)
    assert e.mem_info() == (0, 123)
    L = G.lib()
    u = C.c_uint64()
    assert L.gbmc_set_mem_limit(None, 1) == 1
    assert L.gbmc_mem_info(None, C.byref(u), C.byref(u)) == 1
    assert L.gbmc_mem_info(e._h, None, C.byref(u)) == 1
    e.close()


def test_kernels_are_built_for_sm_103a():
    out = subprocess.run(["cuobjdump", "--list-elf", G._build.LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


@pytest.fixture(scope="module")
def host_engine():
    e = G.Engine(device=-1)
    mats = [S.water(), S.bone(), S.lung(), S.air()]
    e.set_materials(mats, S.Transport(), 20.0)
    return e, mats


QUANT = [
    (0, "or_mu_total"), (1, "or_mu_compton"), (2, "or_mu_pe"), (3, "or_mu_rayleigh"),
]


@pytest.mark.parametrize("q,fn", QUANT)
def test_photon_tables_vs_oracle(host_engine, q, fn):
    e, mats = host_engine
    L = O.lib()
    E = np.geomspace(0.0101, 19.5, 400)
    for m, mat in enumerate(mats):
        ref = np.array([getattr(L, fn)(C.byref(O.material(mat)), x) for x in E])
        got = e.table_eval(q, m, E)
        # 1e-4, except the total at the photoelectric/Compton crossover (largest
        # curvature of log mu in log E: 1.6e-4 at 384 nodes); the pair kink sits
        # on a node
        np.testing.assert_allclose(got, ref, rtol=2e-4 if q == 0 else 1e-4)


def test_electron_tables_vs_oracle(host_engine):
    e, mats = host_engine
    L = O.lib()
    tp = S.Transport()
    T = np.geomspace(0.1, 19.5, 300)
    for m, mat in enumerate(mats):
        M = C.byref(O.material(mat))
        for q, ref in [
            (4, [L.or_sig_el_hard(M, t, tp.c1) for t in T]),
            (5, [L.or_sig_inel(M, 0, t, tp.wcc) for t in T]),
            (6, [L.or_sig_inel(M, 1, t, tp.wcc) for t in T]),
            (7, [L.or_sig_brems(M, t, tp.wcr) for t in T]),
            (8, [L.or_sig1_soft(M, t, tp.c1) for t in T]),
        ]:
            np.testing.assert_allclose(e.table_eval(q, m, T), ref, rtol=1e-4, err_msg=f"q={q} m={m}")
        xc = e.table_eval(9, m, T)
        ref = np.array([L.or_el_xc(M, t, tp.c1) for t in T])
        np.testing.assert_allclose(xc, ref, rtol=1e-4, atol=1e-7)


def test_summed_hard_table_bounds_its_parts(host_engine):
    """The step majorant of analog runs interpolates the summed hard cross
    section (elastic + inelastic + bremsstrahlung) in one table; between nodes
    it must not fall below the sum of the parts as the event choice
    interpolates them (else hard events would be lost), and it must stay close
    to it (else steps would be wasted on delta events)."""
    e, mats = host_engine
    L = O.lib()
    tp = S.Transport()
    T = np.geomspace(1.2e-3, 19.5, 20000)
    for m, mat in enumerate(mats):
        M = C.byref(O.material(mat))
        for s_, q_in, q_sum in ((0, 5, 104), (1, 6, 105)):
            parts = e.table_eval(4, m, T) + e.table_eval(q_in, m, T) + e.table_eval(7, m, T)
            tot = e.table_eval(q_sum, m, T)
            live = parts > 1e-20
            assert np.all(tot[live] >= parts[live] * (1.0 - 1e-6)), (m, s_)
            assert np.max(tot[live] / parts[live]) < 1.01, (m, s_)
            # and it is the closed-form sum at the nodes' accuracy
            Tc = np.geomspace(0.1, 19.5, 50)
            ref = [L.or_sig_el_hard(M, t, tp.c1) + L.or_sig_inel(M, s_, t, tp.wcc) +
                   L.or_sig_brems(M, t, tp.wcr) for t in Tc]
            np.testing.assert_allclose(e.table_eval(q_sum, m, Tc), ref, rtol=1e-4)


def test_range_tables_vs_oracle(host_engine):
    """CSDA range differences and the inverse range, against the oracle's
    Gauss-Legendre integrals of 1/S."""
    e, mats = host_engine
    ph = S.water_cube(4, 1.0)
    ph.materials = mats
    P = O.Problem(ph, S.Source(), S.Transport())
    T = np.geomspace(0.1, 19.0, 120)
    for m in range(len(mats)):
        for pos in (0, 1):
            got = e.table_eval(10 + pos, m, T)          # R'(T) with the library's offset
            ref = np.array([P.range(m, pos, t) for t in T])
            # differences remove the offset convention
            d_got = got[1:] - got[0]
            d_ref = ref[1:] - ref[0]
            np.testing.assert_allclose(d_got, d_ref, rtol=5e-4)
            # inverse range: R'^-1(R'(T)) = T
            back = e.table_eval(101 + pos, m, got)
            np.testing.assert_allclose(back, T, rtol=1e-4)
            # the energy after a step of 5 % CSDA loss (the oracle's mass
            # thickness for it, through the library's range and inverse-range
            # tables): 1e-4 of the energy, 1e-3 of the loss itself
            T0 = T[T > 0.105]
            t = np.array([P.range(m, pos, x) - P.range(m, pos, 0.95 * x) for x in T0])
            E1 = e.table_eval(101 + pos, m, e.table_eval(10 + pos, m, T0) - t)
            np.testing.assert_allclose(E1, 0.95 * T0, rtol=1e-4)
            np.testing.assert_allclose(T0 - E1, 0.05 * T0, rtol=1e-3)


def test_soft_aprime_table_vs_oracle(host_engine):
    e, _ = host_engine
    L = O.lib()
    mb = np.geomspace(2e-9, 0.999, 200)
    ref = np.array([L.or_soft_aprime(x) for x in mb])
    np.testing.assert_allclose(e.table_eval(103, 0, mb), ref, rtol=1e-4)


def test_alias_table_reproduces_weights():
    edges, w = S.kramers_spectrum(6.0, 0.1, 64)
    prob, alias = G.build_alias(w)
    n = len(w)
    mass = prob.astype(np.float64) / n
    for i in range(n):
        mass[alias[i]] += (1.0 - prob[i]) / n
    np.testing.assert_allclose(mass, w / w.sum(), rtol=0, atol=2e-7)
    assert np.all((alias >= 0) & (alias < n))
    # degenerate: a single bin, and zero weights
    p1, a1 = G.build_alias([3.0])
    assert p1[0] == 1.0 and a1[0] == 0
    p2, a2 = G.build_alias([0.0, 1.0, 0.0])
    m2 = p2.astype(np.float64) / 3
    for i in range(3):
        m2[a2[i]] += (1.0 - p2[i]) / 3
    np.testing.assert_allclose(m2, [0, 1, 0], atol=1e-7)
    with pytest.raises(G.GbmcError):
        G.build_alias([0.0, 0.0])
    with pytest.raises(G.GbmcError):
        G.build_alias([1.0, -1.0])


def test_argument_validation_host_only():
    e = G.Engine(device=-1)
    with pytest.raises(G.GbmcError) as ex:
        e.set_materials([S.water()] * 5, S.Transport(), 2.0)     # too many materials
    assert ex.value.status == 1
    with pytest.raises(G.GbmcError):
        e.set_materials([S.water()], S.Transport(c1=0.0), 2.0)
    bad = S.Material("x", [1], [1.0], 10.0, 1.0)
    bad.Z = [0]
    with pytest.raises(G.GbmcError):
        e.set_materials([bad], S.Transport(), 2.0)
    e.set_materials([S.water()], S.Transport(), 2.0)
    # host-only contexts cannot load phantoms or run
    with pytest.raises(G.GbmcError) as ex:
        e.load_phantom(S.water_cube(4, 1.0))
    assert ex.value.status == 4
    with pytest.raises(G.GbmcError):
        e.run(10)
    with pytest.raises(G.GbmcError):
        G.Engine(device=-1, n_batches=1)
    # more batches than a particle record can carry / the flush can weight
    with pytest.raises(G.GbmcError) as ex:
        G.Engine(device=-1, n_batches=1025)
    assert ex.value.status == 1
    G.Engine(device=-1, n_batches=1024).close()
    # the moments and the allocation-free flags need a device context
    with pytest.raises(G.GbmcError) as ex:
        e.moments()
    assert ex.value.status == 4
    with pytest.raises(G.GbmcError) as ex:
        e.noalloc_flags(stream=0)
    assert ex.value.status == 4


def test_stack_capacity_option_is_the_compiled_one():
    """The per-thread stack holds 48 records (a compile-time constant of the
    plain and drain kernels): options asking for another capacity are refused
    instead of being ignored."""
    L = G.lib()
    for cap, want in ((0, 0), (48, 0), (7, 1), (64, 1)):
        h = C.c_void_p()
        opt = G.gbmc_options(0, 8, 0, 0, cap, 0, 0, 0, 0, 0, 0)
        assert L.gbmc_create(C.byref(h), -1, C.byref(opt)) == want, cap
        if h:
            L.gbmc_destroy(h)
