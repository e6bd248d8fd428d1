"""Python binding of the GB300 voxel dose Monte Carlo library (libgbmc.so).

Argument marshalling only: every step of the transport runs in the CUDA
library behind the C ABI of ``include/gbmc.h``. The raw entry points are
exposed under their C names (``gbmc_create``, ``gbmc_run``, ...); ``Engine``
is a convenience wrapper that converts numpy arrays / torch tensors and the
dataclasses of ``synthetic`` (or any objects with the same attributes).

There is no CPU fallback: importing this package raises if the shared library
is missing and cannot be built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_libs = {}

MAX_MAT, MAX_EL, MAX_BINS = 4, 8, 256
PTR_HOST, PTR_DEVICE = 0, 1
KERNEL_PLAIN, KERNEL_WAVEFRONT = 0, 1
STATUS = {0: "GBMC_OK", 1: "GBMC_ERR_ARG", 2: "GBMC_ERR_CUDA", 3: "GBMC_ERR_OOM",
          4: "GBMC_ERR_STATE", 5: "GBMC_ERR_DEVICE_LIMIT", 6: "GBMC_ERR_STACK",
          7: "GBMC_ERR_BOUNDS"}
FLAG_BOUNDS = 128   # error_flags bit of an index out of range (checked library)


class gbmc_material(C.Structure):
    _fields_ = [("n_el", C.c_int), ("Z", C.c_int * MAX_EL), ("A", C.c_double * MAX_EL),
                ("w", C.c_double * MAX_EL), ("I_eV", C.c_double)]


class gbmc_transport(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("eabs_g", "eabs_e", "wcc", "wcr", "c1", "step_frac", "step_vox")]


class gbmc_source(C.Structure):
    _fields_ = [("particle", C.c_int), ("shape", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("hx", C.c_double), ("hy", C.c_double), ("energy", C.c_double), ("n_bins", C.c_int),
                ("edges", C.POINTER(C.c_double)), ("weights", C.POINTER(C.c_double))]


class gbmc_job(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("mat", C.c_void_p), ("rho", C.c_void_p), ("src", gbmc_source),
                ("n_hist", C.c_uint64), ("first_hist", C.c_uint64), ("seed", C.c_uint64)]


class gbmc_vr(C.Structure):
    _fields_ = [("f_inel", C.c_double), ("f_brems", C.c_double), ("w_lo", C.c_double),
                ("w_hi", C.c_double), ("n_split_brems", C.c_int)]


class gbmc_options(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("kernel", "n_batches", "block", "blocks_per_sm",
                                       "stack_cap", "queue_cap", "timing", "photon_budget",
                                       "charged_budget", "pass_target", "ledger_check")]


class gbmc_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("n_hist", "n_batches", "n_tent", "n_real", "n_e_steps",
                                          "n_cross", "n_hard", "n_particles")] + [
        ("e_src", C.c_double), ("e_dep", C.c_double), ("e_esc", C.c_double),
        ("e_pair_net", C.c_double), ("error_flags", C.c_uint32), ("reserved", C.c_uint32),
        ("last_run_ms", C.c_double), ("transport_ms", C.c_double), ("flush_ms", C.c_double),
        ("n_transport_launches", C.c_uint64), ("n_flush_launches", C.c_uint64),
        ("photon_ms", C.c_double), ("n_photon_launches", C.c_uint64),
        ("n_kernel_launches", C.c_uint64), ("n_passes", C.c_uint64),
        ("n_graph_launches", C.c_uint64), ("max_ledger_rel", C.c_double),
        ("n_ledger_checked", C.c_uint64), ("drain_ms", C.c_double), ("n_drain_launches", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class GbmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def checked_default() -> bool:
    """True when the environment variable GBMC_CHECKED selects the checked
    library for every engine of the process."""
    return os.environ.get("GBMC_CHECKED", "0") not in ("", "0")


def lib(checked=None):
    """Load libgbmc.so, or with ``checked`` the checked build
    libgbmc_checked.so (index checks in every kernel; default: the
    GBMC_CHECKED environment variable), building it with nvcc if it is
    missing or stale. Both can be loaded in one process."""
    if checked is None:
        checked = checked_default()
    checked = bool(checked)
    with _lock:
        L = _libs.get(checked)
        if L is None:
            path = _build.lib_path(checked)
            if not _build.up_to_date(checked):
                path = _build.build(checked=checked)
            L = C.CDLL(path)
            P, vp, i32, u32, u64, d = C.POINTER, C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double
            sig = {
                "gbmc_create": (i32, [P(vp), i32, P(gbmc_options)]),
                "gbmc_set_materials": (i32, [vp, P(gbmc_material), i32, P(gbmc_transport), d]),
                "gbmc_load_phantom": (i32, [vp, i32, i32, i32, d, d, d, vp, vp, i32]),
                "gbmc_set_source": (i32, [vp, P(gbmc_source)]),
                "gbmc_run": (i32, [vp, u64, u64, u64, vp]),
                "gbmc_get_dose": (i32, [vp, vp, vp, i32]),
                "gbmc_get_edep": (i32, [vp, vp, vp, i32]),
                "gbmc_get_stats": (i32, [vp, P(gbmc_stats)]),
                "gbmc_reset_tally": (i32, [vp]),
                "gbmc_last_error": (C.c_char_p, [vp]),
                "gbmc_destroy": (None, [vp]),
                "gbmc_philox_fill": (i32, [i32, u32, u32, u32, u32, u32, u32, vp, i32]),
                "gbmc_first_interactions": (i32, [vp, u64, u64, i32, vp, vp]),
                "gbmc_build_alias": (i32, [P(d), i32, P(C.c_float), P(C.c_int)]),
                "gbmc_table_eval": (i32, [vp, i32, i32, P(d), i32, P(d)]),
                "gbmc_run_noalloc": (i32, [vp, u64, u64, u64, i32, vp, vp, vp]),
                "gbmc_set_majorant": (i32, [vp, P(d), i32]),
                "gbmc_set_vr": (i32, [vp, P(gbmc_vr)]),
                "gbmc_run_batch": (i32, [vp, P(gbmc_job), i32, vp]),
                "gbmc_get_job_dose": (i32, [vp, i32, vp, vp, i32]),
                "gbmc_autotune": (i32, [vp, P(gbmc_job), i32, u64, u64, vp, P(gbmc_options)]),
                "gbmc_adjoint": (i32, [vp, vp, i32, u64, u64, u64, vp, vp, i32, vp]),
                "gbmc_get_moments": (i32, [vp, vp, vp, P(u64), P(u64), i32]),
                "gbmc_add_moments": (i32, [vp, vp, vp, u64, u64, i32]),
                "gbmc_noalloc_flags": (i32, [vp, vp, P(u32)]),
                "gbmc_probe_peak": (i32, [i32, i32, i32, P(d), P(d)]),
                "gbmc_build_checked": (i32, []),
                "gbmc_set_mem_limit": (i32, [vp, u64]),
                "gbmc_mem_info": (i32, [vp, P(u64), P(u64)]),
                "gbmc_check_index": (i32, [i32, vp, vp, i32, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _libs[checked] = L
    return L


# the raw C entry points under their own names
def __getattr__(name):
    if name.startswith("gbmc_"):
        return getattr(lib(), name)
    raise AttributeError(name)


def _material(m) -> gbmc_material:
    M = gbmc_material()
    M.n_el = len(m.Z)
    for i, (z, a, w) in enumerate(zip(m.Z, m.A, m.w)):
        M.Z[i], M.A[i], M.w[i] = int(z), float(a), float(w)
    M.I_eV = float(m.I_eV)
    return M


def _ptr(x):
    """(address, ptr_kind) of a contiguous numpy array or torch tensor."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (PTR_DEVICE if x.is_cuda else PTR_HOST)
    return x.ctypes.data, PTR_HOST


class Engine:
    """One library context: materials + phantom + source, then runs.

    ``device=-1`` makes a host-only context (tables and host helpers only).
    ``checked=True`` runs it on the checked library (index checks in every
    kernel, GBMC_ERR_BOUNDS on a violation); None follows GBMC_CHECKED.
    """

    def __init__(self, device: int = 0, kernel: int = KERNEL_PLAIN, n_batches: int = 40,
                 block: int = 0, blocks_per_sm: int = 0, queue_cap: int = 0, timing: bool = False,
                 photon_budget: int = 0, charged_budget: int = 0, pass_target: int = 0,
                 ledger_check: bool = False, checked=None):
        self.L = lib(checked)
        self.checked = bool(self.L.gbmc_build_checked())
        self._h = C.c_void_p()
        opt = gbmc_options(kernel, n_batches, block, blocks_per_sm, 0, queue_cap, int(timing),
                           photon_budget, charged_budget, pass_target, int(ledger_check))
        self._check(self.L.gbmc_create(C.byref(self._h), device, C.byref(opt)), "gbmc_create")
        self.device = device
        self.nvox = 0
        self.shape = None

    def _check(self, st, what):
        if st != 0:
            msg = self.L.gbmc_last_error(self._h).decode() if self._h else ""
            raise GbmcError(st, f"{what}: {msg}")

    def close(self):
        if self._h:
            self.L.gbmc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_materials(self, materials, tp, e_max: float):
        arr = (gbmc_material * len(materials))(*[_material(m) for m in materials])
        t = gbmc_transport(tp.eabs_g, tp.eabs_e, tp.wcc, tp.wcr, tp.c1, tp.step_frac, tp.step_vox)
        self._check(self.L.gbmc_set_materials(self._h, arr, len(materials), C.byref(t), e_max),
                    "gbmc_set_materials")

    def load_phantom(self, ph, mat=None, rho=None):
        """``ph``: object with shape, dx, dy, dz; ``mat``/``rho`` override its
        arrays (e.g. torch CUDA tensors, passed as device pointers)."""
        mat = ph.mat if mat is None else mat
        rho = ph.rho if rho is None else rho
        if not hasattr(mat, "data_ptr"):
            mat = np.ascontiguousarray(mat, np.uint8)
            rho = np.ascontiguousarray(rho, np.float32)
        self._keep = (mat, rho)
        pm, km = _ptr(mat)
        pr, kr = _ptr(rho)
        if km != kr:
            raise ValueError("mat and rho must live in the same memory")
        nx, ny, nz = ph.shape
        self._check(self.L.gbmc_load_phantom(self._h, nx, ny, nz, ph.dx, ph.dy, ph.dz, pm, pr, km),
                    "gbmc_load_phantom")
        self.nvox = nx * ny * nz
        self.shape = (nz, ny, nx)

    @staticmethod
    def _source(s, keep):
        src = gbmc_source(int(s.particle), int(s.shape), s.x0, s.y0, s.hx, s.hy, float(s.energy), 0,
                          None, None)
        if s.edges is not None:
            e = np.ascontiguousarray(s.edges, np.float64)
            w = np.ascontiguousarray(s.weights, np.float64)
            keep.append((e, w))
            src.n_bins = len(w)
            src.edges = e.ctypes.data_as(C.POINTER(C.c_double))
            src.weights = w.ctypes.data_as(C.POINTER(C.c_double))
        return src

    def set_source(self, s):
        keep = []
        src = self._source(s, keep)
        self._src_keep = keep
        self._check(self.L.gbmc_set_source(self._h, C.byref(src)), "gbmc_set_source")

    def run_batch(self, jobs, stream=None):
        """Batched run of jobs: a list of (phantom, source, n_hist, seed[, first_hist])
        tuples; every job's phantom uses the context's materials. Returns the
        number of jobs; doses via job_dose(j)."""
        keep = []
        arr = self._jobs(jobs, keep)
        self._batch_shapes = [tuple(jb[0].mat.shape) for jb in jobs]
        self._check(self.L.gbmc_run_batch(self._h, arr, len(jobs), self._stream(stream)), "gbmc_run_batch")
        return len(jobs)

    def _jobs(self, jobs, keep):
        arr = (gbmc_job * len(jobs))()
        for j, jb in enumerate(jobs):
            ph, src, n, seed = jb[:4]
            first = jb[4] if len(jb) > 4 else 0
            mat = np.ascontiguousarray(ph.mat, np.uint8)
            rho = np.ascontiguousarray(ph.rho, np.float32)
            keep += [mat, rho]
            nx, ny, nz = ph.shape
            arr[j] = gbmc_job(nx, ny, nz, ph.dx, ph.dy, ph.dz, mat.ctypes.data, rho.ctypes.data,
                              self._source(src, keep), int(n), int(first), int(seed))
        return arr

    def autotune(self, n_trial: int, seed: int = 1, jobs=None, stream=None) -> dict:
        """Pick the wavefront options by timing trial runs (see gbmc_autotune);
        returns the chosen options as a dict."""
        keep = []
        arr = self._jobs(jobs, keep) if jobs else None
        if jobs:
            self._batch_shapes = [tuple(jb[0].mat.shape) for jb in jobs]
        out = gbmc_options()
        self._check(self.L.gbmc_autotune(self._h, arr, len(jobs) if jobs else 0, n_trial, seed,
                                         self._stream(stream), C.byref(out)), "gbmc_autotune")
        return {f: getattr(out, f) for f, _ in out._fields_}

    def job_dose(self, j: int, out=None, var=None):
        """(dose, variance) in MeV/g per history of job j of the last batched run."""
        nv = int(np.prod(self._batch_shapes[j]))
        if out is None:
            out = np.zeros(nv)
            var = np.zeros(nv) if var is None else var
        po, ko = _ptr(out)
        pv = _ptr(var)[0] if var is not None else None
        self._check(self.L.gbmc_get_job_dose(self._h, j, po, pv, ko), "gbmc_get_job_dose")
        return out, var

    def setup(self, workload_or_phantom, source=None, tp=None, e_max=None):
        """Materials, phantom and source from a synthetic Workload (or parts)."""
        vr = None
        if source is None:
            w = workload_or_phantom
            ph, source, tp, vr = w.phantom, w.source, w.transport, getattr(w, "vr", None)
        else:
            ph = workload_or_phantom
        self.set_materials(ph.materials, tp, e_max or max(1.1, source.max_energy() * 1.02))
        self.load_phantom(ph)
        self.set_source(source)
        self.set_vr(vr)
        return self

    def set_vr(self, vr=None):
        """Variance reduction (interaction forcing, bremsstrahlung splitting)
        from a ``synthetic.VR``-like object; None switches it off."""
        if vr is None:
            self._check(self.L.gbmc_set_vr(self._h, None), "gbmc_set_vr")
            return
        v = gbmc_vr(vr.f_inel, vr.f_brems, vr.w_lo, vr.w_hi, int(vr.n_split_brems))
        self._check(self.L.gbmc_set_vr(self._h, C.byref(v)), "gbmc_set_vr")

    @staticmethod
    def _stream(stream):
        s = stream
        if s is None:
            try:
                import torch
                s = torch.cuda.current_stream().cuda_stream
            except Exception:
                s = 0
        elif hasattr(s, "cuda_stream"):
            s = s.cuda_stream
        return C.c_void_p(s)

    def run(self, n_hist: int, seed: int = 1, first_hist: int = 0, stream=None):
        self._check(self.L.gbmc_run(self._h, n_hist, seed, first_hist, self._stream(stream)),
                    "gbmc_run")

    def set_majorant(self, rho_maj=None):
        """Fix the photon majorant from per-material densities (None: the
        phantom's maxima)."""
        if rho_maj is None:
            self._check(self.L.gbmc_set_majorant(self._h, None, 0), "gbmc_set_majorant")
            return
        a = np.ascontiguousarray(rho_maj, np.float64)
        self._check(self.L.gbmc_set_majorant(self._h, a.ctypes.data_as(C.POINTER(C.c_double)),
                                             len(a)), "gbmc_set_majorant")

    def adjoint(self, dL_dD, n_hist: int, seed: int = 1, first_hist: int = 0, out=None, var=None,
                stream=None):
        """dL/drho per voxel (and the variance of that mean) for dL_dD = dL/dD,
        by the path-replay adjoint. Arrays: numpy (host) or torch (CUDA)."""
        if out is None:
            out = np.zeros(self.nvox)
            var = np.zeros(self.nvox) if var is None else var
        pg, kg = _ptr(dL_dD)
        po, ko = _ptr(out)
        pv = _ptr(var)[0] if var is not None else None
        if var is not None and _ptr(var)[1] != ko:
            raise ValueError("out and var must live in the same memory")
        self._check(self.L.gbmc_adjoint(self._h, pg, kg, n_hist, seed, first_hist, po, pv, ko,
                                        self._stream(stream)), "gbmc_adjoint")
        return out, var

    def _get(self, fn, out=None, var=None):
        if out is None:
            out = np.zeros(self.nvox)
            var = np.zeros(self.nvox)
        po, ko = _ptr(out)
        pv = _ptr(var)[0] if var is not None else None
        self._check(fn(self._h, po, pv, ko), fn.__name__)
        return out, var

    def dose(self, out=None, var=None):
        """(dose, variance) in MeV/g per history, as flat arrays."""
        return self._get(self.L.gbmc_get_dose, out, var)

    def edep(self, out=None, var=None):
        """(mean energy per history, variance) per voxel in MeV."""
        return self._get(self.L.gbmc_get_edep, out, var)

    def stats(self, check=True) -> dict:
        st = gbmc_stats()
        r = self.L.gbmc_get_stats(self._h, C.byref(st))
        if check:
            self._check(r, "gbmc_get_stats")
        d = st.as_dict()
        d["status"] = r
        return d

    def reset(self):
        self._check(self.L.gbmc_reset_tally(self._h), "gbmc_reset_tally")

    def moments(self, s1=None, s2=None):
        """The tally's moments: per voxel S1 = sum_k B_k and S2 = sum_k B_k^2 / n_k
        over its batches, with its history and batch counts. ``s1``/``s2``:
        numpy arrays or torch tensors of nvox float64 to fill (default: new
        numpy arrays). Returns (s1, s2, n_hist, n_batches)."""
        if s1 is None:
            s1, s2 = np.zeros(self.nvox), np.zeros(self.nvox)
        self._check_f64(s1, s2)
        p1, k1 = _ptr(s1)
        p2, k2 = _ptr(s2)
        if k1 != k2:
            raise ValueError("s1 and s2 must live in the same memory")
        n, k = C.c_uint64(), C.c_uint64()
        self._check(self.L.gbmc_get_moments(self._h, p1, p2, C.byref(n), C.byref(k), k1),
                    "gbmc_get_moments")
        return s1, s2, int(n.value), int(k.value)

    def add_moments(self, s1, s2, n_hist: int, n_batches: int):
        """Add another tally's moments (e.g. the all-reduced sums of every rank)
        to this tally; dose() then reports the combined estimate."""
        if not hasattr(s1, "data_ptr"):
            s1 = np.ascontiguousarray(s1, np.float64)
            s2 = np.ascontiguousarray(s2, np.float64)
        self._check_f64(s1, s2)
        p1, k1 = _ptr(s1)
        p2, k2 = _ptr(s2)
        if k1 != k2:
            raise ValueError("s1 and s2 must live in the same memory")
        self._keep_m = (s1, s2)
        self._check(self.L.gbmc_add_moments(self._h, p1, p2, int(n_hist), int(n_batches), k1),
                    "gbmc_add_moments")

    def set_mem_limit(self, limit_bytes: int):
        """Cap the device memory of this context's problem-sized buffers
        (gbmc_set_mem_limit; 0 = no limit): allocations beyond it fail with
        GBMC_ERR_OOM."""
        self._check(self.L.gbmc_set_mem_limit(self._h, int(limit_bytes)), "gbmc_set_mem_limit")

    def mem_info(self):
        """(bytes held by the problem-sized buffers, limit) (gbmc_mem_info)."""
        held, lim = C.c_uint64(), C.c_uint64()
        self._check(self.L.gbmc_mem_info(self._h, C.byref(held), C.byref(lim)), "gbmc_mem_info")
        return int(held.value), int(lim.value)

    def checkpoint(self, path, next_hist: int, seed: int, **meta):
        """Save the tally to ``path`` (numpy .npz): its moments (gbmc_get_moments),
        the phantom's shape, the next history id and the seed, plus any
        ``meta`` values. With a counter-based generator keyed by history id, a
        run resumed from it (resume(), then run(n, seed, first_hist=next_hist))
        continues exactly the histories an uninterrupted run would make."""
        s1, s2, n, k = self.moments()
        with open(path, "wb") as f:   # exactly `path` (np.savez would append .npz to a bare name)
            np.savez(f, s1=s1, s2=s2, n_hist=n, n_batches=k, shape=np.asarray(self.shape),
                     next_hist=int(next_hist), seed=int(seed), version=1, **meta)

    def resume(self, path) -> dict:
        """Add a checkpoint's moments to this tally (set up with the same
        materials, phantom and source; the phantom's shape is checked) and
        return its fields: next_hist, seed and the saved ``meta`` values."""
        with np.load(path) as z:
            f = {k: z[k] for k in z.files}
        if int(f.get("version", 0)) != 1:
            raise ValueError(f"{path}: not a checkpoint of this library")
        if tuple(int(v) for v in f["shape"]) != tuple(self.shape or ()):
            raise ValueError(f"{path}: phantom shape {tuple(f['shape'])} != {self.shape}")
        self.add_moments(f["s1"], f["s2"], int(f["n_hist"]), int(f["n_batches"]))
        out = {k: (v.item() if v.ndim == 0 else v) for k, v in f.items()
               if k not in ("s1", "s2", "shape", "version", "n_hist", "n_batches")}
        return out

    def _check_f64(self, *arrs):
        for a in arrs:
            n = a.numel() if hasattr(a, "numel") else a.size
            dt = str(a.dtype)
            if "float64" not in dt or n != self.nvox:
                raise ValueError(f"need {self.nvox} float64 values, got {n} of {dt}")

    def run_noalloc(self, n_hist: int, sum_, sum2, seed: int = 1, first_hist: int = 0,
                    n_batches: int = 40, stream=None):
        """Allocation-free run: adds the batch sums into caller device buffers
        ``sum_`` and ``sum2`` (contiguous torch float64 CUDA tensors of nvox
        elements on this engine's device)."""
        for t in (sum_, sum2):
            if not hasattr(t, "data_ptr") or not t.is_cuda or not t.is_contiguous():
                raise ValueError("sum and sum2 must be contiguous CUDA tensors")
            if t.device.index != self.device:
                raise ValueError(f"sum and sum2 must be on cuda:{self.device}")
        self._check_f64(sum_, sum2)
        self._check(self.L.gbmc_run_noalloc(self._h, n_hist, seed, first_hist, n_batches,
                                            sum_.data_ptr(), sum2.data_ptr(), self._stream(stream)),
                    "gbmc_run_noalloc")

    def noalloc_flags(self, stream=None) -> int:
        """Error flags of the last allocation-free run on this device (0: complete)."""
        f = C.c_uint32()
        self._check(self.L.gbmc_noalloc_flags(self._h, self._stream(stream), C.byref(f)),
                    "gbmc_noalloc_flags")
        return int(f.value)

    def first_interactions(self, n: int, seed: int, first_hist: int = 0):
        xyz = np.zeros((n, 3))
        typ = np.zeros(n, np.int32)
        self._check(self.L.gbmc_first_interactions(self._h, seed, first_hist, n, xyz.ctypes.data,
                                                   typ.ctypes.data), "gbmc_first_interactions")
        return xyz, typ

    def table_eval(self, q: int, m: int, x) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros_like(x)
        self._check(self.L.gbmc_table_eval(self._h, q, m, x.ctypes.data_as(C.POINTER(C.c_double)),
                                           len(x), out.ctypes.data_as(C.POINTER(C.c_double))),
                    "gbmc_table_eval")
        return out


def philox_fill(c, k, n: int, device: int = 0) -> np.ndarray:
    """Device Philox4x32-10 words for counters (c0 + i, c1, c2, c3), key k."""
    out = np.zeros((n, 4), np.uint32)
    st = lib().gbmc_philox_fill(device, c[0], c[1], c[2], c[3], k[0], k[1], out.ctypes.data, n)
    if st != 0:
        raise GbmcError(st, "gbmc_philox_fill")
    return out


PROBES = {"ffma": 0, "imad": 1, "lg2": 2, "ex2": 3, "sin": 4, "l2_atomic": 5}


def probe_peak(kind: str, iters: int, device: int = 0):
    """(operations, milliseconds) of one timed launch of a pipe-peak probe
    (gbmc_probe_peak): ``kind`` one of PROBES."""
    ops, ms = C.c_double(), C.c_double()
    st = lib().gbmc_probe_peak(device, PROBES[kind], int(iters), C.byref(ops), C.byref(ms))
    if st != 0:
        raise GbmcError(st, "gbmc_probe_peak")
    return ops.value, ms.value


def build_alias(weights):
    w = np.ascontiguousarray(weights, np.float64)
    prob = np.zeros(len(w), np.float32)
    alias = np.zeros(len(w), np.int32)
    st = lib().gbmc_build_alias(w.ctypes.data_as(C.POINTER(C.c_double)), len(w),
                                prob.ctypes.data_as(C.POINTER(C.c_float)),
                                alias.ctypes.data_as(C.POINTER(C.c_int)))
    if st != 0:
        raise GbmcError(st, "gbmc_build_alias")
    return prob, alias


def check_index(idx, bound, device: int = 0, checked=None):
    """The checked build's index test run on the device (gbmc_check_index):
    for each pair (idx[i], bound[i]) the index the kernels would use and the
    error bits recorded (FLAG_BOUNDS when out of range, checked library only)."""
    idx = np.ascontiguousarray(idx, np.int32)
    bound = np.ascontiguousarray(bound, np.int64)
    if idx.shape != bound.shape or idx.ndim != 1:
        raise ValueError("idx and bound must be 1-D arrays of one length")
    out = np.zeros_like(idx)
    flags = np.zeros(len(idx), np.uint32)
    st = lib(checked).gbmc_check_index(device, idx.ctypes.data, bound.ctypes.data, len(idx),
                                       out.ctypes.data, flags.ctypes.data)
    if st != 0:
        raise GbmcError(st, "gbmc_check_index")
    return out, flags
