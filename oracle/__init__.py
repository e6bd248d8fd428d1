"""CPU oracle for voxel dose Monte Carlo -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product path (the CUDA library and its Python
binding) never does, and this package imports nothing from it.

The C source ``gbmc_oracle.c`` is a plain FP64 serial (or thread-per-batch)
transport code written from the physics reading; this module builds it with
gcc and exposes it through ctypes, plus the paper's tally estimators:

* Eq. 1-2 (history by history): Q = sum q / N, Q2 = sum q^2 / N,
  sigma_Q = sqrt((Q2 - Q^2) / N) -- Eq. 2 as printed lacks the square root;
  the square root of the bracket over N is the reading used (the standard
  estimator of the standard deviation of a mean).
* Eq. 3 (threads): per-thread counters summed, then Eq. 1-2 with N = N_t.
* The batch estimator that the GPU uses: with batch totals B_k of n_k
  histories, var(mean) = (sum_k B_k^2 / n_k - N mean^2) / (N (K - 1)).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgbmc_oracle.so")
_lock = threading.Lock()
_lib = None

MEC2 = 0.51099895
OR_MAX_EL = 8
OR_MAX_MAT = 8


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libgbmc_oracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-1] + "h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Material(C.Structure):
    _fields_ = [("n_el", C.c_int), ("Z", C.c_int * OR_MAX_EL), ("A", C.c_double * OR_MAX_EL),
                ("w", C.c_double * OR_MAX_EL), ("I_eV", C.c_double)]


class TransportC(C.Structure):
    _fields_ = [("eabs_g", C.c_double), ("eabs_e", C.c_double), ("wcc", C.c_double),
                ("wcr", C.c_double), ("c1", C.c_double), ("step_frac", C.c_double),
                ("step_vox", C.c_double)]


class VRC(C.Structure):
    _fields_ = [("f_inel", C.c_double), ("f_brems", C.c_double), ("w_lo", C.c_double),
                ("w_hi", C.c_double), ("n_split_brems", C.c_int)]


class SourceC(C.Structure):
    _fields_ = [("particle", C.c_int), ("shape", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("hx", C.c_double), ("hy", C.c_double), ("energy", C.c_double),
                ("n_bins", C.c_int), ("edges", C.POINTER(C.c_double)),
                ("weights", C.POINTER(C.c_double))]


class PhantomC(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("mat", C.POINTER(C.c_uint8)),
                ("rho", C.POINTER(C.c_float))]


class TallyC(C.Structure):
    _fields_ = [("sum_q", C.POINTER(C.c_double)), ("sum_q2", C.POINTER(C.c_double)),
                ("batch_s1", C.POINTER(C.c_double)), ("batch_s2", C.POINTER(C.c_double))]


_STAT_FIELDS = ["n_hist", "n_batches", "n_tent", "n_real", "n_compton", "n_pe", "n_rayleigh",
                "n_pair", "n_e_steps", "n_cross", "n_hard_el", "n_hard_inel", "n_hard_br",
                "n_delta", "n_annih", "n_escape", "n_particles"]


class StatsC(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in _STAT_FIELDS] + [
        ("e_src", C.c_double), ("e_dep", C.c_double), ("e_esc", C.c_double),
        ("max_ledger_rel", C.c_double), ("e_path", C.c_double),
        ("e_path_absorbed", C.c_double), ("n_e_absorbed", C.c_uint64),
        ("i_el", C.c_double), ("i_inel", C.c_double), ("i_br", C.c_double), ("i_hat", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


def _load(path):
    """ctypes handle of an oracle library with every signature declared."""
    L = C.CDLL(path)
    d, u64, u32, i32 = C.c_double, C.c_uint64, C.c_uint32, C.c_int
    pd, pm = C.POINTER(C.c_double), C.POINTER(Material)
    sig = {
        "or_philox4x32_10": (None, [C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]),
        "or_mix64": (u64, [u64, u64]),
        "or_uniform": (d, [u64, u32, u32, u64, u32]),
        "or_sigma_kn": (d, [d]),
        "or_rayleigh_I": (d, [d]),
        "or_mu_compton": (d, [pm, d]), "or_mu_pe": (d, [pm, d]),
        "or_mu_rayleigh": (d, [pm, d]), "or_mu_pair": (d, [pm, d]),
        "or_mu_total": (d, [pm, d]), "or_electron_density": (d, [pm]),
        "or_s_col": (d, [pm, i32, d]), "or_s_restricted": (d, [pm, i32, d, d, d]),
        "or_sig_inel": (d, [pm, i32, d, d]), "or_inv_x0": (d, [pm]),
        "or_sig_brems": (d, [pm, d, d]), "or_sig_el_hard": (d, [pm, d, d]),
        "or_sig1_soft": (d, [pm, d, d]), "or_soft_aprime": (d, [d]),
        "or_el_xc": (d, [pm, d, d]),
        "or_problem_create": (C.c_void_p, [pm, i32, C.POINTER(TransportC),
                                           C.POINTER(PhantomC), C.POINTER(SourceC)]),
        "or_problem_destroy": (None, [C.c_void_p]),
        "or_range": (d, [C.c_void_p, i32, i32, d]),
        "or_range_inv": (d, [C.c_void_p, i32, i32, d]),
        "or_sample_compton": (None, [d, i32, u64, pd, pd]),
        "or_sample_rayleigh": (None, [pm, d, i32, u64, pd]),
        "or_sample_pair_split": (None, [i32, u64, pd]),
        "or_sample_moller": (None, [d, d, i32, u64, pd]),
        "or_sample_el_hard": (None, [pm, d, d, i32, u64, pd]),
        "or_sample_soft": (None, [d, i32, u64, pd]),
        "or_sample_source_energy": (None, [C.POINTER(SourceC), i32, u64, pd]),
        "or_sample_annihilation": (None, [i32, u64, pd, pd, pd, pd]),
        "or_compton_kinematics": (None, [d, d, d, d, pd, pd, pd]),
        "or_ray_chords": (i32, [C.POINTER(PhantomC), pd, pd, d, i32,
                                C.POINTER(C.c_int64), pd]),
        "or_run": (i32, [C.c_void_p, u64, u32, u64, u64, i32, i32,
                         C.POINTER(TallyC), C.POINTER(StatsC)]),
        "or_first_interactions": (i32, [C.c_void_p, u64, u32, u64, u64, pd,
                                        C.POINTER(C.c_int)]),
        "or_problem_set_majorant": (i32, [C.c_void_p, pd]),
        "or_problem_set_vr": (i32, [C.c_void_p, C.POINTER(VRC)]),
        "or_adjoint": (i32, [C.c_void_p, u64, u32, u64, u64, i32, pd, pd, pd,
                             C.POINTER(StatsC)]),
        "or_lr_primary": (i32, [C.c_void_p, u64, u32, u64, u64, C.c_int64, pd, pd]),
        "or_nth_interactions": (i32, [C.c_void_p, u64, u32, u64, u64, i32, pd, pd,
                                      C.POINTER(C.c_int)]),
        "or_problem_set_instrument": (i32, [C.c_void_p, i32]),
        "or_binary_collision": (None, [d, d, d, pd, pd, pd]),
        "or_elastic_dcs": (d, [i32, d, d]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


@contextlib.contextmanager
def planted(replacements, tag: str):
    """Test infrastructure: run the enclosed code against a copy of the oracle
    built with a planted mistake. ``replacements`` is a list of (old, new)
    source strings, each old string occurring exactly once in gbmc_oracle.c.
    Used to show that a pin fails when the oracle it pins is wrong."""
    global _lib
    src = open(_SRC).read()
    for old, new in replacements:
        if src.count(old) != 1:
            raise ValueError(f"planted mistake: {old!r} occurs {src.count(old)} times")
        src = src.replace(old, new)
    os.makedirs(_BUILD, exist_ok=True)
    csrc = os.path.join(_BUILD, f"planted_{tag}.c")
    so = os.path.join(_BUILD, f"planted_{tag}_{os.getpid()}.so")
    with open(csrc, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-I", _HERE, "-o", so, csrc,
                    "-lm", "-lpthread"], check=True)
    with _lock:
        saved = _lib
        _lib = _load(so)
    try:
        yield _lib
    finally:
        with _lock:
            _lib = saved


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def material(m) -> Material:
    """ctypes material from any object with Z, A, w, I_eV."""
    M = Material()
    M.n_el = len(m.Z)
    for i, (z, a, w) in enumerate(zip(m.Z, m.A, m.w)):
        M.Z[i], M.A[i], M.w[i] = int(z), float(a), float(w)
    M.I_eV = float(m.I_eV)
    return M


def transport(t) -> TransportC:
    return TransportC(t.eabs_g, t.eabs_e, t.wcc, t.wcr, t.c1, t.step_frac, t.step_vox)


class Problem:
    """An initialised oracle problem (materials, transport cut-offs, phantom, source)."""

    def __init__(self, phantom, source, tp, rho_maj=None, vr=None, instrument=False):
        L = lib()
        self._mats = (Material * len(phantom.materials))(*[material(m) for m in phantom.materials])
        self._tp = transport(tp)
        self._mat = np.ascontiguousarray(phantom.mat, dtype=np.uint8)
        self._rho = np.ascontiguousarray(phantom.rho, dtype=np.float32)
        nx, ny, nz = phantom.shape
        self.phantom = phantom
        self._ph = PhantomC(nx, ny, nz, phantom.dx, phantom.dy, phantom.dz,
                            self._mat.ctypes.data_as(C.POINTER(C.c_uint8)),
                            self._rho.ctypes.data_as(C.POINTER(C.c_float)))
        self._src, self._keep = source_c(source)
        self._p = L.or_problem_create(self._mats, len(phantom.materials), C.byref(self._tp),
                                      C.byref(self._ph), C.byref(self._src))
        if not self._p:
            raise RuntimeError("or_problem_create failed")
        if rho_maj is not None:
            rm = np.ascontiguousarray(rho_maj, dtype=np.float64)
            if L.or_problem_set_majorant(self._p, _dptr(rm)) != 0:
                raise ValueError("majorant densities below the phantom's maxima")
        if vr is not None:
            self._vr = VRC(vr.f_inel, vr.f_brems, vr.w_lo, vr.w_hi, vr.n_split_brems)
            if L.or_problem_set_vr(self._p, C.byref(self._vr)) != 0:
                raise ValueError("variance-reduction parameters out of range")
        if instrument:
            L.or_problem_set_instrument(self._p, 1)

    def __del__(self):
        try:
            if self._p:
                lib().or_problem_destroy(self._p)
                self._p = None
        except Exception:
            pass

    def range(self, mat: int, positron: int, T: float) -> float:
        return lib().or_range(self._p, mat, positron, T)

    def range_inv(self, mat: int, positron: int, r: float) -> float:
        return lib().or_range_inv(self._p, mat, positron, r)

    def first_interactions(self, seed, first, n, job=0):
        xyz = np.zeros((n, 3))
        typ = np.zeros(n, np.int32)
        lib().or_first_interactions(self._p, seed, job, first, n, _dptr(xyz),
                                    typ.ctypes.data_as(C.POINTER(C.c_int)))
        return xyz, typ

    def nth_interactions(self, k, seed, first, n, job=0):
        """Position, energy before it and type of the k-th real interaction of
        each history's primary photon (type 0: it had fewer)."""
        xyz = np.zeros((n, 3))
        E = np.zeros(n)
        typ = np.zeros(n, np.int32)
        lib().or_nth_interactions(self._p, seed, job, first, n, k, _dptr(xyz), _dptr(E),
                                  typ.ctypes.data_as(C.POINTER(C.c_int)))
        return xyz, E, typ


def source_c(s):
    edges = weights = None
    keep = []
    sc = SourceC(int(s.particle), int(s.shape), s.x0, s.y0, s.hx, s.hy, float(s.energy), 0, None, None)
    if s.edges is not None:
        edges = np.ascontiguousarray(s.edges, np.float64)
        weights = np.ascontiguousarray(s.weights, np.float64)
        keep = [edges, weights]
        sc.n_bins = len(weights)
        sc.edges = _dptr(edges)
        sc.weights = _dptr(weights)
    return sc, keep


@dataclass
class OracleResult:
    n_hist: int
    n_batches: int
    sum_q: np.ndarray
    sum_q2: np.ndarray
    batch_s1: np.ndarray
    batch_s2: np.ndarray
    stats: dict
    mass: np.ndarray  # rho * V per voxel, g

    @property
    def edep_mean(self):
        """Eq. 1: mean energy deposited per history in each voxel (MeV)."""
        return self.sum_q / self.n_hist

    @property
    def edep_sigma_history(self):
        """Eq. 2 (square-root reading): sigma of the mean per voxel (MeV)."""
        N = self.n_hist
        q = self.sum_q / N
        q2 = self.sum_q2 / N
        return np.sqrt(np.maximum(q2 - q * q, 0.0) / N)

    @property
    def edep_sigma_batch(self):
        """Batch estimator: var = (sum B^2/n - N mean^2) / (N (K - 1))."""
        N, K = self.n_hist, self.n_batches
        q = self.sum_q / N
        var = (self.batch_s2 - N * q * q) / (N * max(K - 1, 1))
        return np.sqrt(np.maximum(var, 0.0))

    @property
    def dose(self):
        """MeV/g per history."""
        return self.edep_mean / self.mass

    @property
    def dose_sigma(self):
        return self.edep_sigma_history / self.mass

    @property
    def dose_sigma_batch(self):
        return self.edep_sigma_batch / self.mass


def run(phantom, source, tp, n_hist: int, seed: int = 1, first_hist: int = 0,
        n_batches: int = 40, n_threads: int = 1, job: int = 0, rho_maj=None,
        vr=None, instrument: bool = False) -> OracleResult:
    """Run the oracle on [first_hist, first_hist + n_hist) and return its tallies.
    ``rho_maj``: per-material densities fixing the photon majorant; ``vr``:
    variance reduction (a ``synthetic.VR``); ``instrument``: accumulate the
    hard-event compensators in the statistics (slow)."""
    P = Problem(phantom, source, tp, rho_maj, vr, instrument)
    nv = phantom.n_vox
    arrs = [np.zeros(nv) for _ in range(4)]
    T = TallyC(*[_dptr(a) for a in arrs])
    st = StatsC()
    rc = lib().or_run(P._p, seed, job, first_hist, n_hist, n_batches, n_threads,
                      C.byref(T), C.byref(st))
    if rc != 0:
        raise RuntimeError(f"or_run failed ({rc})")
    mass = (phantom.rho.astype(np.float64) * phantom.dx * phantom.dy * phantom.dz).reshape(-1)
    kb = min(n_batches, n_hist)
    return OracleResult(n_hist, kb, arrs[0], arrs[1], arrs[2], arrs[3], st.as_dict(), mass)


def adjoint(phantom, source, tp, g, n_hist: int, seed: int = 1, first_hist: int = 0,
            n_batches: int = 20, rho_maj=None, job: int = 0, vr=None):
    """Likelihood-ratio dL/drho per voxel for g = dL/dD (D in MeV/g per history).
    Returns (mean, variance of the mean, stats). Analog histories only: a
    ``vr`` with variance reduction is refused."""
    P = Problem(phantom, source, tp, rho_maj, vr)
    nv = phantom.n_vox
    gg = None
    if g is not None:   # None: the score alone (G_h = 1, no explicit term)
        gg = np.ascontiguousarray(np.asarray(g, np.float64).reshape(-1))
        if gg.size != nv:
            raise ValueError("g must have one value per voxel")
    s1, s2 = np.zeros(nv), np.zeros(nv)
    st = StatsC()
    rc = lib().or_adjoint(P._p, seed, job, first_hist, n_hist, n_batches,
                          _dptr(gg) if gg is not None else None,
                          _dptr(s1), _dptr(s2), C.byref(st))
    if rc != 0:
        raise RuntimeError(f"or_adjoint failed ({rc})")
    K = min(n_batches, n_hist)
    m = s1 / n_hist
    var = np.maximum((s2 - n_hist * m * m) / (n_hist * max(K - 1, 1)), 0.0)
    return m, var, st.as_dict()


def lr_primary(phantom, source, tp, n_hist: int, target: int = -1, seed: int = 1, rho_maj=None):
    """Score-function estimate of dP/drho_v for the event "the primary photon's
    first real interaction is in voxel ``target``" (-1: it leaves uncollided),
    and its variance of the mean (test functionals with closed forms)."""
    P = Problem(phantom, source, tp, rho_maj)
    nv = phantom.n_vox
    s1, s2 = np.zeros(nv), np.zeros(nv)
    rc = lib().or_lr_primary(P._p, seed, 0, 0, n_hist, target, _dptr(s1), _dptr(s2))
    if rc != 0:
        raise RuntimeError(f"or_lr_primary failed ({rc})")
    m = s1 / n_hist
    return m, np.maximum(s2 / n_hist - m * m, 0.0) / n_hist
