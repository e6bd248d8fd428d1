"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module builds the *inputs* of a transport run -- material compositions,
voxel phantoms, source descriptions and batched job lists -- and nothing else.
It holds none of the transport arithmetic (no cross sections, no sampling of
interactions, no tallies), so that the GPU library and the CPU oracle, which
both consume these arrays, stay independent of one another.

The paper (Sec. 4.2.1 state samplers, Sec. 4.2.2 voxelised geometries, Sec. 4.4
CT calibration curve) describes these components only structurally; the
concrete recipes below are the synthetic stand-ins for its patient CT and
PENELOPE example geometries, which are not available here.

Every generator is deterministic given its seed (numpy's Philox bit generator).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Elements and materials (input data: compositions, densities, I-values)
# ---------------------------------------------------------------------------

# Standard atomic weights (g/mol) of the elements used by the synthetic tissues.
ATOMIC_WEIGHT = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 15: 30.974,
                 18: 39.948, 20: 40.078}


@dataclass
class Material:
    """A homogeneous mixture given by element mass fractions.

    ``Z``/``A``/``w`` are the atomic numbers, atomic weights (g/mol) and mass
    fractions (summing to 1); ``I_eV`` is the mean excitation energy used by the
    Bethe stopping power; ``rho`` is the nominal density in g/cm^3 (phantoms may
    override it voxel by voxel).
    """
    name: str
    Z: List[int]
    w: List[float]
    I_eV: float
    rho: float
    A: List[float] = field(default_factory=list)

    def __post_init__(self):
        if not self.A:
            self.A = [ATOMIC_WEIGHT[z] for z in self.Z]
        s = float(sum(self.w))
        self.w = [float(x) / s for x in self.w]


def water() -> Material:
    return Material("water", [1, 8], [0.1119, 0.8881], 75.0, 1.00)


def lung() -> Material:
    # lung is water composition at lung density
    return Material("lung", [1, 8], [0.1119, 0.8881], 75.0, 0.26)


def bone() -> Material:
    # simplified cortical bone (Mg and S folded into Ca)
    return Material("bone", [1, 6, 7, 8, 15, 20],
                    [0.064, 0.278, 0.027, 0.410, 0.070, 0.151], 106.0, 1.85)


def air() -> Material:
    return Material("air", [7, 8, 18], [0.755, 0.232, 0.013], 85.7, 0.0012)


# ---------------------------------------------------------------------------
# Transport parameters and sources
# ---------------------------------------------------------------------------

@dataclass
class Transport:
    """Absorption energies and class II cut-offs (MeV, rad).

    ``eabs_g``/``eabs_e``: photon / e+- absorption energies; ``wcc``/``wcr``:
    hard inelastic / hard bremsstrahlung energy-loss cut-offs; ``c1``: the
    hard elastic mean free path is max(lambda_el, c1 * lambda_1) (PENELOPE's
    C1 parameter); ``step_frac``: largest fractional CSDA energy loss per step;
    ``step_vox``: largest step in voxel widths.
    """
    eabs_g: float = 0.010
    eabs_e: float = 0.100
    wcc: float = 0.010
    wcr: float = 0.010
    c1: float = 0.05
    step_frac: float = 0.05
    step_vox: float = 4.0


@dataclass
class VR:
    """Variance reduction (Sec. 5.2's 40 keV electron example forces hard
    bremsstrahlung x2000 and hard inelastic collisions x200 and splits
    bremsstrahlung photons in two). ``f_inel``/``f_brems``: interaction
    forcing factors for electrons and positrons whose weight lies in
    [``w_lo``, ``w_hi``]; ``n_split_brems``: copies of each bremsstrahlung
    photon."""
    f_inel: float = 1.0
    f_brems: float = 1.0
    w_lo: float = 0.1
    w_hi: float = 2.0
    n_split_brems: int = 1


PHOTON, ELECTRON, POSITRON = 0, 1, 2


@dataclass
class Source:
    """Primary-particle state sampler (Sec. 4.2.1): position, direction, energy.

    Primaries start on the z = 0 face moving along +z. ``shape`` 0 is a pencil
    at (x0, y0); shape 1 is a uniform rectangle of half widths (hx, hy) centred
    on (x0, y0). Energy is ``energy`` (MeV) when ``edges`` is None, otherwise a
    binned spectrum with bin ``edges`` (n+1 values) and bin ``weights`` (n),
    uniform inside each bin.
    """
    particle: int = PHOTON
    shape: int = 0
    x0: float = 0.0
    y0: float = 0.0
    hx: float = 0.0
    hy: float = 0.0
    energy: float = 1.0
    edges: Optional[np.ndarray] = None
    weights: Optional[np.ndarray] = None

    def max_energy(self) -> float:
        return float(self.edges[-1]) if self.edges is not None else float(self.energy)


def kramers_spectrum(e0: float = 6.0, lo: float = 0.1, nbins: int = 64):
    """Thick-target (Kramers) bremsstrahlung shape dN/dE ~ (E0 - E)/E, binned.

    Equal-width bins over [lo, e0]; each bin's weight is the integral of the
    shape over the bin, E0 ln(b/a) - (b - a). Returns (edges, weights) with the
    weights normalised to sum 1.
    """
    edges = np.linspace(lo, e0, nbins + 1)
    a, b = edges[:-1], edges[1:]
    wts = e0 * np.log(b / a) - (b - a)
    return edges, wts / wts.sum()


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------

@dataclass
class Phantom:
    """Voxel phantom: ``mat`` (uint8 material index) and ``rho`` (float32 g/cm^3),
    both C-ordered as [iz][iy][ix], with voxel sizes (dx, dy, dz) in cm; the grid
    occupies [0, nx dx] x [0, ny dy] x [0, nz dz] and is surrounded by vacuum."""
    mat: np.ndarray
    rho: np.ndarray
    dx: float
    dy: float
    dz: float
    materials: List[Material]

    @property
    def shape(self):
        nz, ny, nx = self.mat.shape
        return nx, ny, nz

    @property
    def n_vox(self) -> int:
        return int(self.mat.size)


def water_cube(n: int = 20, d: float = 0.5) -> Phantom:
    """Homogeneous water cube of n^3 voxels of side d cm."""
    mat = np.zeros((n, n, n), np.uint8)
    rho = np.full((n, n, n), 1.0, np.float32)
    return Phantom(mat, rho, d, d, d, [water()])


def slab_phantom(nxy: int, dz_list: Sequence[float], mats: Sequence[int],
                 materials: List[Material], d: float = 0.5,
                 rhos: Optional[Sequence[float]] = None) -> Phantom:
    """Laterally uniform stack of slabs along z; ``dz_list`` gives the number of
    voxels of each slab, ``mats`` its material index."""
    layers_m, layers_r = [], []
    for i, (nzs, m) in enumerate(zip(dz_list, mats)):
        r = materials[m].rho if rhos is None else rhos[i]
        layers_m += [m] * int(nzs)
        layers_r += [r] * int(nzs)
    nz = len(layers_m)
    mat = np.empty((nz, nxy, nxy), np.uint8)
    rho = np.empty((nz, nxy, nxy), np.float32)
    for k in range(nz):
        mat[k] = layers_m[k]
        rho[k] = layers_r[k]
    return Phantom(mat, rho, d, d, d, materials)


def gaussian_random_field(n: int, d: float, corr_len: float, seed: int,
                          stream: int = 0) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field on an n^3 grid.

    White N(0,1) noise is smoothed by a separable Gaussian kernel of standard
    deviation corr_len/sqrt(2) (so the field's covariance is
    exp(-r^2/(2 corr_len^2))), with periodic boundaries, then standardised.
    Returned as float64 [iz][iy][ix].
    """
    rng = np.random.Generator(np.random.Philox(key=[seed, stream]))
    g = rng.standard_normal((n, n, n))
    s_vox = (corr_len / np.sqrt(2.0)) / d
    k = np.fft.fftfreq(n)
    kern = np.exp(-2.0 * (np.pi * k * s_vox) ** 2)  # FT of a unit-area Gaussian
    G = np.fft.fftn(g)
    G *= kern[:, None, None] * kern[None, :, None] * kern[None, None, :]
    f = np.real(np.fft.ifftn(G))
    f -= f.mean()
    f /= f.std()
    return f


def grf_three_material(n: int = 128, d: float = 0.2, seed: int = 2,
                       corr_len: float = 1.5) -> Phantom:
    """Water/bone/lung phantom by thresholding a Gaussian random field.

    lung where g < -0.84 (about 20 %), bone where g > 1.04 (about 15 %), water
    elsewhere; each material at its nominal density (1.00 / 1.85 / 0.26).
    Material indices: 0 water, 1 bone, 2 lung.
    """
    g = gaussian_random_field(n, d, corr_len, seed)
    mats = [water(), bone(), lung()]
    mat = np.zeros(g.shape, np.uint8)
    mat[g > 1.04] = 1
    mat[g < -0.84] = 2
    rho = np.array([m.rho for m in mats], np.float32)[mat]
    return Phantom(mat, rho, d, d, d, mats)


# piecewise-linear CT calibration curve (HU -> g/cm^3), Sec. 4.4's user curve
HU_RAMP = ((-1000.0, 0.0012), (-200.0, 0.80), (0.0, 1.00), (200.0, 1.10), (1500.0, 1.90))


def hu_to_density(hu: np.ndarray) -> np.ndarray:
    xs = np.array([p[0] for p in HU_RAMP])
    ys = np.array([p[1] for p in HU_RAMP])
    return np.interp(hu, xs, ys)


def hu_to_material(hu: np.ndarray) -> np.ndarray:
    """air < -900 <= lung < -200 <= water < 200 <= bone -> indices 0..3."""
    m = np.full(hu.shape, 2, np.uint8)  # water
    m[hu < -200.0] = 1
    m[hu < -900.0] = 0
    m[hu >= 200.0] = 3
    return m


def ct_phantom(n: int = 256, d: float = 0.1, seed: int = 3,
               corr_len: float = 1.5) -> Phantom:
    """CT-like phantom: GRF -> HU = clamp(-100 + 450 g, -1000, 1500) -> ramp.

    Material indices: 0 air, 1 lung, 2 water, 3 bone; densities from the ramp.
    """
    g = gaussian_random_field(n, d, corr_len, seed)
    hu = np.clip(-100.0 + 450.0 * g, -1000.0, 1500.0)
    rho = hu_to_density(hu).astype(np.float32)
    mat = hu_to_material(hu)
    mats = [air(), lung(), water(), bone()]
    return Phantom(mat, rho, d, d, d, mats)


def crop(ph: Phantom, n: int) -> Phantom:
    """Central n^3 crop of a phantom (used for small-size oracle comparisons)."""
    nx, ny, nz = ph.shape
    ox, oy, oz = (nx - n) // 2, (ny - n) // 2, (nz - n) // 2
    return Phantom(np.ascontiguousarray(ph.mat[oz:oz + n, oy:oy + n, ox:ox + n]),
                   np.ascontiguousarray(ph.rho[oz:oz + n, oy:oy + n, ox:ox + n]),
                   ph.dx, ph.dy, ph.dz, ph.materials)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    phantom: Phantom
    source: Source
    transport: Transport
    n_hist: int
    seed: int
    vr: Optional["VR"] = None


def workload_water_pencil(n_hist: int = 100_000) -> Workload:
    """1 MeV photon pencil beam on the face centre of a 10 cm water cube (20^3, 5 mm)."""
    ph = water_cube(20, 0.5)
    src = Source(PHOTON, 0, 5.0, 5.0, 0.0, 0.0, 1.0)
    return Workload("water20_pencil_1MeV", ph, src, Transport(), n_hist, 1)


def workload_grf_spectrum(n: int = 128, n_hist: int = 100_000_000) -> Workload:
    """128^3 x 2 mm water/bone/lung GRF phantom, 10x10 cm photon field, 0.1-6 MeV
    Kramers spectrum (64 bins)."""
    ph = grf_three_material(n, 0.2, seed=2)
    edges, wts = kramers_spectrum(6.0, 0.1, 64)
    L = n * 0.2
    src = Source(PHOTON, 1, L / 2, L / 2, 5.0, 5.0, 6.0, edges, wts)
    return Workload(f"grf{n}_2mm_photon_field_kramers6MeV", ph, src, Transport(), n_hist, 1)


def workload_ct_electron(n: int = 256, n_hist: int = 50_000_000) -> Workload:
    """256^3 x 1 mm CT-like phantom (4 materials), 20 MeV electron 5x5 cm beam."""
    ph = ct_phantom(n, 0.1, seed=3)
    L = n * 0.1
    src = Source(ELECTRON, 1, L / 2, L / 2, 2.5, 2.5, 20.0)
    return Workload(f"ct{n}_1mm_electron_20MeV", ph, src, Transport(), n_hist, 1)


HALFSPACE_KINDS = ("e40keV", "g1MeV", "g1MeV_e100keV")


def workload_halfspace(kind: str, n_hist: int = 10_000_000, n: int = 64,
                       d: float = 1.0) -> Workload:
    """The paper's kernel-throughput tests (Sec. 6.1): vacuum / water half-space,
    a monoenergetic point source in the vacuum aimed perpendicularly at the
    plane. The half-space is an n^3 water block of voxel d (cm; 64 cm deep by
    default, past which 1 MeV photons are attenuated by e^-4.5) whose z = 0 face
    is the plane; the source emits along +z from the face centre (a voxel
    centre). Three kinds:

    * ``e40keV``: 40 keV electrons, electrons absorbed below 1 keV, photons
      never tracked (absorbed where they are made);
    * ``g1MeV``: 1 MeV photons absorbed below 1 keV, electrons never tracked;
    * ``g1MeV_e100keV``: as ``g1MeV`` with electrons tracked down to 100 keV.

    W_cc = W_cr = 1 keV and C1 = 0.05 (the paper's settings for its 40 keV
    electron disc example); "never tracked" is an absorption energy above
    every energy in the problem."""
    if kind not in HALFSPACE_KINDS:
        raise ValueError(f"unknown half-space kind {kind!r}")
    ph = water_cube(n, d)
    c = (n // 2 + 0.5) * d
    never = 1e3
    if kind == "e40keV":
        src = Source(ELECTRON, 0, c, c, 0.0, 0.0, 0.040)
        tp = Transport(eabs_g=never, eabs_e=1e-3, wcc=1e-3, wcr=1e-3)
    elif kind == "g1MeV":
        src = Source(PHOTON, 0, c, c, 0.0, 0.0, 1.0)
        tp = Transport(eabs_g=1e-3, eabs_e=never, wcc=1e-3, wcr=1e-3)
    else:
        src = Source(PHOTON, 0, c, c, 0.0, 0.0, 1.0)
        tp = Transport(eabs_g=1e-3, eabs_e=0.100, wcc=1e-3, wcr=1e-3)
    return Workload(f"halfspace_{kind}_water{n}_{d * 10:g}mm", ph, src, tp, n_hist, 1)


def workload_beam_vr(n_hist: int = 10_000_000, n: int = 64, d: float = 0.1) -> Workload:
    """1 MeV electron pencil on the face centre of an n^3 water cube of voxel d
    (cm), photons tracked to 1 keV, electrons to 20 keV, W_cc = W_cr = 5 keV:
    a dose made by the electrons down to their range (4.4 mm) and a
    bremsstrahlung tail beyond it, the region that bremsstrahlung forcing and
    splitting (variance reduction) serve."""
    ph = water_cube(n, d)
    c = (n // 2 + 0.5) * d
    src = Source(ELECTRON, 0, c, c, 0.0, 0.0, 1.0)
    tp = Transport(eabs_g=1e-3, eabs_e=0.02, wcc=0.005, wcr=0.005)
    return Workload(f"beam_e1MeV_water{n}_{d * 10:g}mm", ph, src, tp, n_hist, 1)


def batched_jobs(n_jobs: int = 64, seed: int = 4, hist_scale: float = 1.0):
    """Uneven batched jobs: cube side log-uniform in [32, 192], voxel size in
    {1,2,3,4} mm, GRF 3-material phantom with per-job seed, photon or electron
    (p = 1/2) mono source with energy log-uniform in [0.1, 18] MeV, histories
    log-uniform in [1e5, 2e7] (times ``hist_scale``)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 99]))
    jobs = []
    for j in range(n_jobs):
        n = int(round(np.exp(rng.uniform(np.log(32), np.log(192)))))
        d = float(rng.integers(1, 5)) * 0.1
        part = PHOTON if rng.uniform() < 0.5 else ELECTRON
        e = float(np.exp(rng.uniform(np.log(0.1), np.log(18.0))))
        nh = int(round(np.exp(rng.uniform(np.log(1e5), np.log(2e7))) * hist_scale))
        ph = grf_three_material(n, d, seed=1000 + j, corr_len=1.5)
        L = n * d
        src = Source(part, 1, L / 2, L / 2, L / 4, L / 4, e)
        jobs.append(Workload(f"job{j}", ph, src, Transport(), max(nh, 1), 1000 + j))
    return jobs


def density_perturbation(shape, seed: int = 5, amp: float = 0.05) -> np.ndarray:
    """Seeded multiplicative density perturbation 1 + amp * g', g' ~ N(0, 1)
    independently per voxel (Philox stream `seed`), float32 of `shape`."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 77]))
    return (1.0 + amp * rng.standard_normal(shape)).astype(np.float32)


def workload_differentiable(n: int = 128, n_hist: int = 10_000_000):
    """The 128^3 three-material GRF phantom with the 0.1-6 MeV Kramers field and
    the target densities rho * (1 + 0.05 g') (seed 5) whose dose is the target
    of the loss L = sum (D - T)^2. Returns (workload, target density array)."""
    w = workload_grf_spectrum(n, n_hist)
    w.name = f"grf{n}_2mm_kramers6MeV_adjoint"
    return w, (w.phantom.rho * density_perturbation(w.phantom.rho.shape)).astype(np.float32)


# ---------------------------------------------------------------------------
# JSON presets of the five configurations (synthetic/presets/*.json): the same
# recipes as the workload_* functions above, written out as data
# ---------------------------------------------------------------------------
PRESET_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "presets")
_PARTICLES = {"photon": PHOTON, "electron": ELECTRON, "positron": POSITRON}


def preset_names():
    return sorted(f[:-5] for f in os.listdir(PRESET_DIR) if f.endswith(".json"))


def _preset_phantom(p) -> Phantom:
    kind = p["kind"]
    if kind == "water_cube":
        return water_cube(p["n"], p["d"])
    if kind == "grf_three_material":
        return grf_three_material(p["n"], p["d"], seed=p["seed"], corr_len=p["corr_len"])
    if kind == "ct_phantom":
        return ct_phantom(p["n"], p["d"], seed=p["seed"], corr_len=p["corr_len"])
    raise ValueError(f"unknown phantom kind {kind!r}")


def _preset_source(s, ph: Phantom) -> Source:
    nx, ny, _ = ph.shape
    x0, y0 = (nx * ph.dx / 2, ny * ph.dy / 2) if s.get("centred") else (s["x0"], s["y0"])
    shape = {"pencil": 0, "field": 1}[s["shape"]]
    edges = wts = None
    energy = s.get("energy")
    if "spectrum" in s:
        sp = s["spectrum"]
        if sp["kind"] != "kramers":
            raise ValueError(f"unknown spectrum kind {sp['kind']!r}")
        edges, wts = kramers_spectrum(sp["e0"], sp["lo"], sp["bins"])
        energy = sp["e0"]
    return Source(_PARTICLES[s["particle"]], shape, x0, y0, s.get("hx", 0.0), s.get("hy", 0.0),
                  energy, edges, wts)


def load_preset(name: str, **override):
    """Build a configuration from its JSON preset (a file name under
    synthetic/presets, with or without .json, or a path). Returns a Workload;
    a batched preset returns the list of job Workloads (``override`` may set
    n_jobs, seed, hist_scale); a differentiable one returns (Workload, target
    densities). Other ``override`` keys replace top-level fields (n_hist, seed)."""
    path = name if os.path.sep in name else os.path.join(PRESET_DIR, name if name.endswith(".json")
                                                           else name + ".json")
    with open(path) as f:
        p = json.load(f)
    if "batched" in p:
        b = dict(p["batched"], **override)
        return batched_jobs(b["n_jobs"], b["seed"], b["hist_scale"])
    if "base" in p:
        w = load_preset(os.path.join(os.path.dirname(path), p["base"]),
                        n_hist=override.get("n_hist", p["n_hist"]))
        w.name = p["name"]
        q = p["perturbation"]
        return w, (w.phantom.rho * density_perturbation(w.phantom.rho.shape, seed=q["seed"],
                                                        amp=q["amp"])).astype(np.float32)
    p = dict(p, **override)
    ph = _preset_phantom(p["phantom"])
    return Workload(p["name"], ph, _preset_source(p["source"], ph), Transport(**p["transport"]),
                    int(p["n_hist"]), int(p["seed"]))
