#!/usr/bin/env python3
"""Throughput benchmark: primary histories/s of the voxel dose Monte Carlo on
one GB300, on the 128^3 x 2 mm water/bone/lung phantom with a 10x10 cm field of
the 0.1-6 MeV Kramers spectrum (coupled photon/electron/positron transport).

One step = one gbmc_run of --hist-per-step histories (40 batches, i.e. 40
transport launches + 40 tally flushes). Prints one JSON line (rank 0).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl gbmc|reference]

--impl reference times the CPU oracle (the deliberately plain FP64 reference
implementation) on the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

# ---------------------------------------------------------------------------
# Roofline. Nothing on the path is a dense contraction and its working set is
# on chip (tables in shared memory, phantoms in L2), so the transport kernels
# are bound by the plain ALU pipes: FP32/INT32 issue, the half-rate 32-bit
# integer multiply (the Philox rounds), and the special-function unit (log,
# exp, reciprocal, square root, sine/cosine). Their peaks are MEASURED on the
# GPU at run time by the library's probes (gbmc_probe_peak), at the clock the
# GPU runs; the nominal issue rate (152 SMs x 4 schedulers x 32 lanes x
# 2.07 GHz = 40.28 T thread-instructions/s) is shown beside them.
# ---------------------------------------------------------------------------
ALU_PEAK_NOMINAL = 152 * 4 * 32 * 2.070e9

# Device-instruction budget (the issue view, "issue_frac"): thread
# instructions per event counted by hand from the device code, including its
# address arithmetic and queue handling.
OP_BUDGET = {            # thread-instructions per event
    "n_tent": 100,       # Woodcock step: 2 draws (1/2 Philox block), log, divide, locate, 2 loads
    "n_real": 300,       # type choice (3 lookups + draw) + KN sampling + rotation + child
    "n_e_steps": 350,    # ~12 table lookups, 3 draws, soft deflection, rotation, step control
    "n_cross": 55,       # face distances, position, inverse-range lookup, scoring
    "n_hard": 175,       # type choice, sampling, rotation / secondary
    "n_particles": 40,   # primary sampling / stack pop
}

# Algorithmic budget (the method's own arithmetic per event, counted from the
# oracle's code with each cross section read from the FP32 log-log tables of
# the method): (alu, imul, sfu) = simple FP32/INT operations, 32-bit integer
# multiplies, special-function operations. One table lookup at a known grid
# position = (2 alu, 0, 1 exp2); a grid position = (4 alu, 0, 1 log2).
# Philox4x32-10 block (4 uniforms): 10 rounds x (2 multiplies, 4 xor, 2 key
# adds) + 4 x (shift, scale) = (68, 20, 0).
PHILOX = (68, 20, 0)


def _add(*terms):
    out = [0.0, 0.0, 0.0]
    for w, t in terms:
        for i in range(3):
            out[i] += w * t[i]
    return tuple(out)


ALGO_BUDGET = {
    # one Woodcock flight: a Philox block, -ln u (log2 + mul), / majorant
    # (rcp + mul), position (3 fma), locate (3 x mul, floor, convert, tie
    # test, 2 bounds), voxel index (2 imul), acceptance (pick, mul, compare)
    "tent": _add((1, PHILOX), (1, (27, 2, 2))),
    # type choice at a real collision: 3 lookups, c = u mu, 3 compares
    "real_select": (10, 0, 3),
    # the photon's new energy after a Compton event: grid position, the
    # majorant and 3 materials' totals
    "real_new_energy": (12, 0, 5),
    # Compton (Butcher-Messel): set-up (k, 1/(1+2k), ln(1+2k); 6 alu 2 sfu),
    # 1.6 trials of 3 uniforms (3/4 Philox) + eps (exp or sqrt) + (1-eps)/(k eps)
    # + sin^2 + g (1 rcp) + accept; azimuth sincos; rotation (20 alu, sqrt +
    # rsqrt); electron direction from momentum (12 alu, rsqrt); child path
    # (64-bit mix: 8 imul, 10 alu)
    "compton": _add((1, (6, 0, 2)), (1.6, _add((0.75, PHILOX), (1, (12, 0, 3)))),
                    (1, (2, 0, 2)), (1, (20, 0, 2)), (1, (14, 0, 1)), (1, (10, 8, 0))),
    # photoelectric: the child electron
    "pe": (10, 8, 0),
    # Rayleigh: element weights (4 elements: 3 alu + rcp each), 1.3 trials of
    # 3 uniforms + element pick (8) + t (4 alu, rcp) + accept (4), azimuth,
    # rotation
    "rayleigh": _add((1, (12, 0, 4)), (1.3, _add((0.75, PHILOX), (1, (16, 0, 1)))),
                     (1, (22, 0, 4))),
    # pair: FP64 CDF inversion (6 Newton steps of 8 ops + a division), 2 children
    "pair": (68, 16, 6),
    # class II step: 2 Philox blocks; grid position of T0; step control (R at
    # T_lo, end-energy position, 2 hard-table lookups, max, -ln u / majorant,
    # hinge position); DDA set-up (3 rcp) and two segments (face distances,
    # argmin, position: 20 alu each); end-of-step energy (inverse range:
    # log2 + position + lookup) and deposit; hinge: sigma_1 lookup,
    # 1 - exp(-t sigma_1), logit (rcp + log2), A' lookup, inversion (rcp),
    # azimuth (sincos), rotation
    "e_step": _add((2, PHILOX), (1, (4, 0, 1)), (1, (24, 0, 8)), (1, (40, 0, 3)),
                   (1, (8, 0, 2)), (1, (37, 0, 10))),
    # voxel crossing: face distances (12), argmin (4), position (4),
    # inverse-range settle (log2 + position + lookup), deposit (2), voxel
    # index (4), material compare (1)
    "cross": (33, 0, 2),
    # selection at a hard event: grid position, 3 lookups, compares
    "hard_select": (14, 0, 4),
    # hard elastic: element pick (9), screening (6 alu, rcp), inversion
    # (4 alu, 2 sfu), azimuth, rotation, cut-off lookup
    "hard_el": (43, 0, 7),
    # hard inelastic (Moller): 1.2 trials of 2 uniforms + 12 alu + 2 sfu;
    # two-body kinematics (8 alu, 2 rcp, 2 sqrt); azimuth (1 uniform, sincos);
    # two rotations; child
    "hard_inel": _add((1.2, _add((0.5, PHILOX), (1, (12, 0, 2)))), (1, (8, 0, 4)),
                      (0.25, PHILOX), (1, (0, 0, 2)), (1, (40, 0, 4)), (1, (10, 8, 0))),
    # hard bremsstrahlung: 1 uniform, W = W_cr exp(u ln(T / W_cr)), child
    "hard_br": _add((0.25, PHILOX), (1, (3, 0, 2)), (1, (10, 8, 0))),
    # a particle's start: primary position and energy (1 Philox block, alias
    # arithmetic, batch index) or a secondary's record
    "particle": _add((0.5, PHILOX), (1, (20, 0, 0))),
}


def event_mix(ost):
    """Shares of the photon interaction types and of the hard-event kinds in
    the oracle's statistics of the same workload (the method's event mix)."""
    nr = max(1, ost["n_compton"] + ost["n_pe"] + ost["n_rayleigh"] + ost["n_pair"])
    nh = max(1, ost["n_hard_el"] + ost["n_hard_inel"] + ost["n_hard_br"] + ost["n_delta"])
    return {"compton": ost["n_compton"] / nr, "pe": ost["n_pe"] / nr,
            "rayleigh": ost["n_rayleigh"] / nr, "pair": ost["n_pair"] / nr,
            "hard_el": ost["n_hard_el"] / nh, "hard_inel": ost["n_hard_inel"] / nh,
            "hard_br": ost["n_hard_br"] / nh, "delta": ost["n_delta"] / nh}


def algorithmic_ops(st, mix, kernel):
    """(alu, imul, sfu) operations the method needs for the events counted in
    the GPU statistics st, for one kernel's share of the work: "charged"
    (class II steps, crossings, hard-event selection and elastic events),
    "knock" (hard inelastic and bremsstrahlung events), "photon" (flights and
    interactions) or "all"."""
    B = ALGO_BUDGET
    f = mix
    parts = []
    if kernel in ("photon", "all"):
        real = _add((f["compton"], _add((1, B["compton"]), (1, B["real_new_energy"]))),
                    (f["pe"], B["pe"]), (f["rayleigh"], B["rayleigh"]), (f["pair"], B["pair"]),
                    (1, B["real_select"]))
        parts += [(st["n_tent"], B["tent"]), (st["n_real"], real)]
    if kernel in ("charged", "all"):
        parts += [(st["n_e_steps"], B["e_step"]), (st["n_cross"], B["cross"]),
                  (st["n_hard"], _add((1, B["hard_select"]), (f["hard_el"], B["hard_el"])))]
    if kernel in ("knock", "all"):
        parts += [(st["n_hard"], _add((f["hard_inel"], B["hard_inel"]), (f["hard_br"], B["hard_br"])))]
    if kernel == "all":
        parts += [(st["n_particles"], B["particle"])]
    return _add(*parts)


def pipe_roofline(ops, seconds, peaks):
    """Fraction of the pipe roofline: the lower bound on the time of these
    operations (each pipe at its measured peak, and all of them through the
    one-instruction-per-scheduler-per-clock issue, measured by the FFMA probe)
    over the measured time; the binding pipe's achieved and peak rates."""
    alu, imul, sfu = ops
    t = {"fp32_int_alu": alu / peaks["ffma"], "int_mul": imul / peaks["imad"],
         "sfu": sfu / peaks["lg2"], "issue": (alu + imul + sfu) / peaks["ffma"]}
    bind = max(t, key=t.get)
    rate = {"fp32_int_alu": alu, "int_mul": imul, "sfu": sfu, "issue": alu + imul + sfu}[bind]
    peak = {"fp32_int_alu": peaks["ffma"], "int_mul": peaks["imad"], "sfu": peaks["lg2"],
            "issue": peaks["ffma"]}[bind]
    return {"pipe": bind, "achieved": rate / seconds, "peak": peak, "frac": t[bind] / seconds,
            "per_pipe_frac": {k: v / seconds for k, v in t.items()}}


def measure_peaks(local):
    """The library's pipe probes on this GPU, each launch about 20 ms, with the
    SM clock sampled meanwhile: operations per second (thread level)."""
    import paper_2003_00796_gb300 as G
    clk = ClockSampler(local)
    clk.start()
    out = {}
    for kind, it in (("ffma", 2000), ("imad", 2000), ("lg2", 500), ("ex2", 500), ("sin", 500),
                     ("l2_atomic", 200)):
        ops, ms = G.probe_peak(kind, it, local)
        it = max(1, int(it * 20.0 / max(ms, 1e-3)))
        ops, ms = G.probe_peak(kind, it, local)
        out[kind] = ops / (ms * 1e-3)
    out["clocks"] = clk.stop()
    return out


WORKLOADS = {
    "grf128": lambda n: S.workload_grf_spectrum(128, n),
    "water20": lambda n: S.workload_water_pencil(n),
    "ct256": lambda n: S.workload_ct_electron(256, n),
    "halfspace_e40keV": lambda n: S.workload_halfspace("e40keV", n),
    "halfspace_g1MeV": lambda n: S.workload_halfspace("g1MeV", n),
    "halfspace_g1MeV_e100keV": lambda n: S.workload_halfspace("g1MeV_e100keV", n),
    "beam_e1MeV": lambda n: S.workload_beam_vr(n),
}


def tail_uncertainty(dose, var, depth_axis_len):
    """Mean relative sigma over the bremsstrahlung tail: the depth slabs beyond
    the first one after the peak whose lateral-summed dose is below 0.1 % of
    the largest slab (beyond the electrons' reach, where photons deposit
    alone), voxels there with dose >= 10 % of the tail's maximum."""
    d = dose.reshape(depth_axis_len, -1)
    v = var.reshape(depth_axis_len, -1)
    prof = d.sum(1)
    peak = int(np.argmax(prof))
    low = np.nonzero(prof[peak:] < 1e-3 * prof.max())[0]
    tail = np.zeros(depth_axis_len, bool)
    if low.size:
        tail[peak + int(low[0]):] = True
    dt, vt = d[tail].ravel(), v[tail].ravel()
    if dt.size == 0 or dt.max() <= 0:
        return float("nan"), 0
    sel = dt >= 0.1 * dt.max()
    return float(np.mean(np.sqrt(vt[sel]) / dt[sel])), int(sel.sum())


def src_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2003_00796_gb300", "csrc", "*"))):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def transport_src_hash() -> str:
    """Hash of the code the transport kernels are compiled from (the wavefront
    kernels, the device physics, the data layout and the ABI header), with
    comments and blank space removed: a traffic figure taken by ncu stays
    valid while that code is unchanged."""
    import re
    h = hashlib.sha256()
    for f in ("paper_2003_00796_gb300/csrc/k_wavefront.cu", "paper_2003_00796_gb300/csrc/transport.cuh",
              "paper_2003_00796_gb300/csrc/gbmc_common.cuh", "paper_2003_00796_gb300/csrc/gbmc_internal.h",
              "include/gbmc.h"):
        code = open(os.path.join(ROOT, f)).read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, val in zip(names, p[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rel_uncertainty(dose, var, thr=0.5):
    sel = dose >= thr * dose.max()
    return float(np.mean(np.sqrt(var[sel]) / dose[sel]))


def cpu_baseline(w, target_s: float = 15.0):
    """The oracle as it stands, on all host cores, on a bounded sample."""
    import oracle as O
    nth = os.cpu_count() or 1
    # size the sample from a short calibration run, and once more from the
    # sample itself if it came out well short of the target (the calibration
    # carries the oracle's fixed set-up cost)
    n_next, n, dt = 64 * nth, 0, 0.0
    for attempt in range(3):
        n = n_next
        t0 = time.perf_counter()
        r = O.run(w.phantom, w.source, w.transport, n, seed=78 + attempt, first_hist=10_000_000,
                  n_batches=max(nth, 8), n_threads=nth, vr=w.vr)
        dt = time.perf_counter() - t0
        stats = r.stats
        if attempt > 0 and dt >= 0.5 * target_s:
            break
        n_next = int(max(nth * 8, n * target_s / max(dt, 1e-3)))
    # one thread as well (the oracle's serial mode), on a sample that takes about a fifth of the time
    n1 = max(8, n // (5 * nth))
    t0 = time.perf_counter()
    O.run(w.phantom, w.source, w.transport, n1, seed=90, first_hist=20_000_000,
          n_batches=8, n_threads=1, vr=w.vr)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": "histories/s", "cores": nth, "kind": "oracle",
            "sample": f"{n} histories of the same workload (FP64 serial code, one thread per "
                      f"batch on {nth} host threads), {dt:.1f} s",
            "serial_value": n1 / dt1,
            "serial_sample": f"{n1} histories on one host thread, {dt1:.1f} s",
            "oracle_stats": stats}


def measure_adjoint(args, w, G, local, stream, tuning, first_of, barrier, dist, plain_rate):
    """Forward + path-replay adjoint per step for the differentiable workload on
    this phantom: L = sum (D - T)^2, T the dose of the densities
    rho (1 + 0.05 g') (seed 5), dL/dD = 2 (D - T) formed on the device from
    this step's dose, then dL/drho from as many adjoint histories. Timed with
    CUDA events on the run's stream around the whole step."""
    import torch
    n = int(args.hist_per_step)
    ph = w.phantom
    rho_t = (ph.rho * S.density_perturbation(ph.rho.shape)).astype(np.float32)
    rho_maj = [1.2 * float(ph.rho[ph.mat == m].max()) if np.any(ph.mat == m) else 1.0
               for m in range(len(ph.materials))]
    et = G.Engine(local, kernel=G.KERNEL_WAVEFRONT, n_batches=args.batches, **tuning)
    et.setup(S.Workload("target", S.Phantom(ph.mat, rho_t, ph.dx, ph.dy, ph.dz, ph.materials),
                        w.source, w.transport, 0, 1))
    et.run(n, seed=w.seed + 7, stream=stream)
    T = torch.empty(ph.n_vox, dtype=torch.float64, device="cuda")
    et.dose(out=T, var=None)
    et.close()
    e = G.Engine(local, kernel=G.KERNEL_WAVEFRONT, n_batches=args.batches, **tuning).setup(w)
    e.set_majorant(rho_maj)
    D = torch.empty_like(T)
    grad = torch.empty_like(T)

    def step(k):
        e.reset()
        e.run(n, seed=w.seed, first_hist=first_of(k), stream=stream)
        e.dose(out=D, var=None)
        g = 2.0 * (D - T)
        ea.record(stream)
        e.adjoint(g, n, seed=w.seed + 3, first_hist=first_of(k), out=grad, var=None, stream=stream)
        eb.record(stream)

    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup):
        step(k)
    barrier()
    steps = max(1, min(args.steps, 3))
    t_step, t_adj = 0.0, 0.0
    for k in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(args.warmup + k)
        e1.record(stream)
        torch.cuda.synchronize()
        t_step += e0.elapsed_time(e1) / 1e3
        t_adj += ea.elapsed_time(eb) / 1e3
    barrier()
    if dist is not None:
        tt = torch.tensor([t_step, t_adj], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step, t_adj = float(tt[0]), float(tt[1])
    st = e.stats()
    e.close()
    fin = bool(torch.isfinite(grad).all())
    out = {"value": steps * n / t_step, "unit": "histories/s (forward + adjoint, per step "
           "n forward and n adjoint histories)", "steps": steps,
           "ms_per_step": 1e3 * t_step / steps, "adjoint_ms_per_step": 1e3 * t_adj / steps,
           "adjoint_only": steps * n / t_adj, "loss": "sum (D - T)^2, T at rho (1 + 0.05 g')",
           "grad_finite": fin, "majorant": "fixed at 1.2 x max density per material",
           "transport": "coupled e-/e+/photon (electron density dependence not differentiated)"}
    if plain_rate:
        out["vs_plain_kernel"] = out["value"] / plain_rate
    return out


def load_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    if it was taken on the current transport sources."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        if d.get("transport_src_hash") != transport_src_hash():
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def batch_line(args, local, G, scale=1.0, world=1, rank=0, steps=None, warmup=None,
               autotune=True, plain=True):
    """64 independent jobs (phantoms 32^3-192^3 at 1-4 mm, photon or electron
    sources 0.1-18 MeV, 1e5-2e7 histories each at scale 1) in one batched run
    per step: value = all jobs' histories / the batched run's device time (the
    pass loop's one graph launch and the flushes, CUDA events inside the
    library); e2e = the same over the wall time of the gbmc_run_batch call,
    which uploads the 64 phantoms from host memory and allocates their
    tallies. The plain kernel runs the same jobs one by one (device time of
    each gbmc_run) as the metric's baseline. The autotuner picks the wavefront
    options (budgets, queue depth, block shape) on a scaled-down batch first."""
    import torch
    torch.cuda.set_device(local)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    ws = S.batched_jobs(64, seed=4, hist_scale=scale)
    # ranks split the jobs (independent problems: weak scaling, no exchange)
    mine = [w for j, w in enumerate(ws) if j % world == rank]
    jobs = [(w.phantom, w.source, w.n_hist, w.seed) for w in mine]
    n_total = sum(w.n_hist for w in mine)
    e_max = max(w.source.max_energy() for w in ws) * 1.02
    e = G.Engine(local, kernel=G.KERNEL_WAVEFRONT, n_batches=args.batches,
                 blocks_per_sm=args.blocks_per_sm, photon_budget=args.photon_budget,
                 charged_budget=args.charged_budget, pass_target=args.pass_target,
                 queue_cap=args.queue_cap)
    e.set_materials([S.water(), S.bone(), S.lung()], S.Transport(), e_max)
    tuned = None
    if autotune:
        t0 = time.perf_counter()
        tuned = e.autotune(max(1_000_000, n_total // 20), seed=7, jobs=jobs)
        tuned = {k: tuned[k] for k in ("charged_budget", "photon_budget", "pass_target", "block",
                                       "blocks_per_sm")}
        tuned["search_s"] = time.perf_counter() - t0
    for k in range(warmup):
        e.run_batch(jobs)
    e.reset()
    clk = ClockSampler(local)
    clk.start()
    t_dev, t_wall = 0.0, 0.0
    for k in range(steps):
        t0 = time.perf_counter()
        e.run_batch(jobs)
        t_wall += time.perf_counter() - t0
        t_dev += e.stats()["last_run_ms"] / 1e3
    clocks = clk.stop()
    st = e.stats()
    U = []
    for j in range(len(jobs)):
        d, v = e.job_dose(j)
        U.append(rel_uncertainty(d, v, 0.5))
    e.close()
    plain_rate = None
    if plain:
        tp = 0.0
        ep = G.Engine(local, kernel=G.KERNEL_PLAIN, n_batches=args.batches)
        ep.set_materials([S.water(), S.bone(), S.lung()], S.Transport(), e_max)
        for ph, src, n, seed in jobs:
            ep.load_phantom(ph)
            ep.set_source(src)
            ep.reset()
            ep.run(n, seed=seed)
            tp += ep.stats()["last_run_ms"] / 1e3
        ep.close()
        plain_rate = n_total / tp
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_dev, t_wall, float(n_total)], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt[:2], op=dist.ReduceOp.MAX)
        nt = tt[2:].clone()
        dist.all_reduce(nt, op=dist.ReduceOp.SUM)
        t_dev, t_wall, n_all = float(tt[0]), float(tt[1]), int(nt[0])
    else:
        n_all = n_total
    value = steps * n_all / t_dev
    return {
        "workload": f"batch64_grf_32-192cube_1-4mm_photon_electron_0.1-18MeV_x{scale:g}",
        "value": value, "unit": "histories/s", "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_dev / steps, "jobs": len(ws), "histories_per_step": n_all,
        "wall_s_per_step": t_wall / steps,
        "e2e": {"value": steps * n_all / t_wall, "unit": "histories/s",
                "h2d_bytes_per_step": int(sum(p.mat.nbytes + p.rho.nbytes for p, _, _, _ in jobs)),
                "d2h_bytes_per_step": 0},
        "plain_kernel": {"value": plain_rate, "how": "the same jobs one by one, plain kernel"}
        if plain_rate else None,
        "vs_plain_kernel": value / plain_rate if plain_rate else None,
        "autotuned": tuned, "clocks": clocks,
        "uncertainty": {"median_over_jobs_U": float(np.median(U)), "max_U": float(np.max(U))},
        "gpu_launches": int(st["n_kernel_launches"]),
        "pass_loop": {"passes": int(st["n_passes"]), "graph_launches": int(st["n_graph_launches"])},
        "events_per_history": {k: st[k] / max(1, st["n_hist"]) for k in OP_BUDGET},
    }


def run_batch_bench(args, rank, world, local):
    """--workload batch64: the batched run as the main line."""
    import paper_2003_00796_gb300 as G
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle is not run on the "
                              "64-job batch (hours of host time); see the grf128 reference line"}))
        return
    b = batch_line(args, local, G, scale=args.batch_scale, world=world, rank=rank,
                   autotune=args.autotune, plain=not args.no_plain)
    if rank == 0:
        line = {"metric": "primary histories/s at 1% dose uncertainty", "value": b["value"],
                "unit": "histories/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": b["workload"], "jobs": b["jobs"],
                           "histories_per_step": b["histories_per_step"],
                           "batches_per_job": args.batches, "autotuned": b["autotuned"],
                           "pass_loop": "one CUDA-graph launch per run: a device-driven while loop "
                                        "over passes"}}
        line.update({k: b[k] for k in ("wall_s_per_step", "e2e", "plain_kernel", "vs_plain_kernel",
                                       "uncertainty", "gpu_launches", "pass_loop", "clocks",
                                       "events_per_history")})
        print(json.dumps(line))


def roofline_json(algo, issue_achieved, peaks, kname, t_launch, nl, ops, st, traffic):
    """The roofline object: the algorithmic fraction (the method's operations
    over the measured pipe peaks, binding pipe) and, beside it, the issue view
    (device instructions counted by hand over the measured FFMA/issue peak)."""
    issue = {"achieved": issue_achieved / 1e12, "peak": peaks["ffma"] / 1e12,
             "unit": "T thread-instructions/s", "frac": issue_achieved / peaks["ffma"],
             "ops_per_history": ops / max(1, st["n_hist"]),
             "budget": "device instructions per event counted from the device code (OP_BUDGET)"}
    out = {"bound": "alu", "kernel": kname, "launch_ms": 1e3 * t_launch, "launches": int(nl),
           "traffic": traffic, "issue_frac": issue["frac"], "issue": issue,
           "peak_source": "measured on this GPU by gbmc_probe_peak (fma.rn.f32 for FP32/INT issue, "
                          "mad.lo.u32, lg2.approx), at the clock sampled during the probes; "
                          f"nominal issue {ALU_PEAK_NOMINAL / 1e12:.2f} T/s"}
    if algo:
        out.update({"achieved": algo["achieved"] / 1e9, "peak": algo["peak"] / 1e9, "unit": "Gop/s",
                    "frac": algo["frac"], "pipe": algo["pipe"], "per_pipe_frac": algo["per_pipe_frac"],
                    "ops_per_launch": algo["ops_per_launch"],
                    "ops_per_history_all_kernels": dict(zip(("alu", "imul", "sfu"),
                                                            algo["ops_per_history_all_kernels"])),
                    "event_mix": algo["event_mix"],
                    "budget": "the method's operations per event counted from the oracle's code "
                              "(ALGO_BUDGET), event mix from the oracle's run of this workload"})
    else:
        out.update({"achieved": issue["achieved"] * 1e3, "peak": issue["peak"] * 1e3, "unit": "Gop/s",
                    "frac": issue["frac"], "pipe": "issue (device budget: no oracle event mix in this run)"})
    return out


def run_reference(args, w, rank):
    if rank != 0:
        return
    import oracle as O
    nth = os.cpu_count() or 1
    per_step_s = 8.0
    t0 = time.perf_counter()
    O.run(w.phantom, w.source, w.transport, 32 * nth, seed=91, n_batches=nth, n_threads=nth, vr=w.vr)
    dt = time.perf_counter() - t0
    n_step = int(max(nth * 4, 32 * nth * per_step_s / max(dt, 1e-3)))
    for k in range(args.warmup):
        O.run(w.phantom, w.source, w.transport, max(nth * 2, n_step // 8), seed=92,
              first_hist=k * n_step, n_batches=nth, n_threads=nth, vr=w.vr)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.run(w.phantom, w.source, w.transport, n_step, seed=93, first_hist=100_000_000 + k * n_step,
              n_batches=max(nth, 8), n_threads=nth, vr=w.vr)
    T = time.perf_counter() - t0
    v = args.steps * n_step / T
    line = {
        "impl": "reference", "metric": "primary histories/s at 1% dose uncertainty",
        "value": v, "unit": "histories/s", "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "histories_per_step": n_step, "threads": nth},
        "cpu_baseline": {"value": v, "unit": "histories/s", "cores": nth, "kind": "oracle",
                         "sample": f"{n_step} histories per step of {w.name}"},
        "e2e": {"value": v, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbmc", choices=["gbmc", "reference"])
    ap.add_argument("--workload", default="grf128", choices=sorted(WORKLOADS) + ["batch64"],
                    help="batch64: 64 uneven jobs in one batched run (one step = the whole batch)")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="batch64: scale every job's history count")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the wavefront options with the library's autotuner first")
    ap.add_argument("--hist-per-step", type=float, default=1e7)
    ap.add_argument("--kernel", default="wavefront", choices=["plain", "wavefront"])
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain kernel beside it")
    ap.add_argument("--batches", type=int, default=40)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--photon-budget", type=int, default=0, help="wavefront: real photon events per pass")
    ap.add_argument("--charged-budget", type=int, default=0, help="wavefront: class II steps per pass")
    ap.add_argument("--pass-target", type=int, default=0, help="wavefront: particles in flight per pass")
    ap.add_argument("--queue-cap", type=int, default=0, help="wavefront: queue capacity")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward + adjoint line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the ct256 and batch64 sub-lines of the default run")
    ap.add_argument("--extra-hist", type=int, default=10_000_000,
                    help="histories per step of the ct256 sub-line")
    ap.add_argument("--extra-batch-scale", type=float, default=0.25,
                    help="history scale of the batch64 sub-line (1.0 = 2.17e8 histories)")
    ap.add_argument("--vr", default=None,
                    help="variance reduction F_INEL,F_BREMS,N_SPLIT (forcing window [0.1, 2]); "
                         "adds the analog run and the efficiency gain on the bremsstrahlung tail")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n_step = int(args.hist_per_step)
    if args.workload == "batch64":
        return run_batch_bench(args, rank, world, local)
    w = WORKLOADS[args.workload](n_step)
    if args.vr:
        fi, fb, ns = args.vr.split(",")
        w.vr = S.VR(f_inel=float(fi), f_brems=float(fb), n_split_brems=int(ns))
        w.name += f"_vr{fi}-{fb}-{ns}"

    if args.impl == "reference":
        return run_reference(args, w, rank)

    import torch
    import paper_2003_00796_gb300 as G
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    from paper_2003_00796_gb300 import shard

    def first_of(step):
        # step `step` covers world * n_step history ids; this rank takes its share
        return shard.history_range(world * n_step, step * world * n_step, rank, world)[0]
    flush_buf = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    tuning = dict(blocks_per_sm=args.blocks_per_sm, photon_budget=args.photon_budget,
                  charged_budget=args.charged_budget, pass_target=args.pass_target,
                  queue_cap=args.queue_cap)

    tuned = None
    if args.autotune and args.kernel == "wavefront":
        et = G.Engine(local, kernel=G.KERNEL_WAVEFRONT, n_batches=args.batches, **tuning).setup(w)
        tuned = et.autotune(min(n_step, 4_000_000), seed=w.seed + 11, stream=stream)
        et.close()
        for k in ("photon_budget", "charged_budget", "pass_target"):
            tuning[k] = tuned[k]

    def measure(kernel, steps, clocks=None, timing=False, wl=None, n=None, warmup=None):
        """W untimed warm-up steps, then `steps` timed steps (CUDA events on the
        run's stream, L2 flushed between steps outside the events). timing=True
        also times every launch inside the library (passes launched one by one
        instead of run by the graph's device-side loop): used for the per-kernel split.
        wl, n: another workload and histories per step (default: the main ones)."""
        wl = wl or w
        n_run = int(n or n_step)
        warm = args.warmup if warmup is None else warmup

        def first_k(step):
            return shard.history_range(world * n_run, step * world * n_run, rank, world)[0]
        eng = G.Engine(local, kernel=kernel, n_batches=args.batches, timing=timing, **tuning).setup(wl)
        for k in range(warm):
            eng.run(n_run, seed=wl.seed, first_hist=first_k(k), stream=stream)
        barrier()
        eng.reset()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        if clocks:
            clocks.start()
        t_wall = time.perf_counter()
        for k in range(steps):
            flush_buf.zero_()
            ev[k][0].record(stream)
            eng.run(n_run, seed=wl.seed, first_hist=first_k(warm + k), stream=stream)
            ev[k][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
        clk = clocks.stop() if clocks else None
        t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        if dist is not None:
            tt = torch.tensor([t_dev], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_dev = float(tt.item())
        st = eng.stats()
        if dist is not None:   # the one exchange of a sharded run: pooled tally moments
            shard.combine(eng)
        dose, var = eng.dose()
        eng.close()
        return {"t_dev": t_dev, "t_wall": t_wall, "stats": st, "dose": dose, "var": var, "clk": clk,
                "steps": steps}

    kernel = G.KERNEL_PLAIN if args.kernel == "plain" else G.KERNEL_WAVEFRONT
    M = measure(kernel, args.steps, ClockSampler(local))
    st, t_dev, dose, var, clk, t_wall = M["stats"], M["t_dev"], M["dose"], M["var"], M["clk"], M["t_wall"]
    # per-kernel launch times (a separate, per-launch-timed measurement)
    Mt = measure(kernel, max(1, min(args.steps, 3)), timing=True)
    stt = Mt["stats"]
    U = rel_uncertainty(dose, var, 0.5)
    n_total = world * args.steps * n_step      # all ranks (the tally is pooled across them)
    value = n_total / t_dev
    n1 = n_total * (U / 0.01) ** 2
    # roofline of the dominant transport kernel: the charged-particle kernel of
    # the wavefront path (the plain kernel does everything in one launch)
    nl = max(1, stt["n_transport_launches"])
    t_launch = stt["transport_ms"] / 1e3 / nl
    if kernel == G.KERNEL_WAVEFRONT and stt["transport_ms"] >= stt["photon_ms"]:
        ops = sum(OP_BUDGET[k] * stt[k] for k in ("n_e_steps", "n_cross", "n_hard"))
        kname, kpart = "k_wf_charged", "charged"
    elif kernel == G.KERNEL_WAVEFRONT:
        # photon-dominated workload: the photon kernel (its time is reported
        # with the knock kernel's, one knock launch per photon launch)
        ops = sum(OP_BUDGET[k] * stt[k] for k in ("n_tent", "n_real"))
        kname, kpart = "k_wf_photon", "photon"
        nl = max(1, stt["n_photon_launches"] // 2)
        t_launch = stt["photon_ms"] / 1e3 / nl
    else:
        ops = sum(OP_BUDGET[k] * stt[k] for k in OP_BUDGET)
        kname, kpart = "k_plain", "all"
    achieved = ops / nl / t_launch
    peaks = measure_peaks(local)
    plain = None
    if kernel == G.KERNEL_WAVEFRONT and not args.no_plain:
        Mp = measure(G.KERNEL_PLAIN, max(1, min(args.steps, 3)))
        vp = world * max(1, min(args.steps, 3)) * n_step / Mp["t_dev"]
        plain = {"value": vp, "unit": "histories/s", "steps": max(1, min(args.steps, 3)),
                 "ms_per_step": 1e3 * Mp["t_dev"] / max(1, min(args.steps, 3)),
                 "wavefront_over_plain": value / vp}

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI with host buffers (pinned, as a caller
        # that streams phantoms would hold them): phantom upload, run, dose +
        # variance read back, every step
        ph = w.phantom
        mat_h = torch.from_numpy(np.ascontiguousarray(ph.mat)).pin_memory().numpy()
        rho_h = torch.from_numpy(np.ascontiguousarray(ph.rho)).pin_memory().numpy()
        out_d = torch.zeros(ph.n_vox, dtype=torch.float64).pin_memory().numpy()
        out_v = torch.zeros(ph.n_vox, dtype=torch.float64).pin_memory().numpy()
        e2 = G.Engine(local, kernel=kernel, n_batches=args.batches, **tuning)
        e2.set_materials(ph.materials, w.transport, max(1.1, w.source.max_energy() * 1.02))
        e2.set_source(w.source)
        e2.set_vr(w.vr)
        e2.load_phantom(ph, mat_h, rho_h)
        e2.run(n_step, seed=w.seed + 1, stream=stream)
        e2.dose(out_d, out_v)
        barrier()
        k2 = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for k in range(k2):
            e2.load_phantom(ph, mat_h, rho_h)
            e2.run(n_step, seed=w.seed + 1, first_hist=first_of(k), stream=stream)
            e2.dose(out_d, out_v)
        barrier()
        te = time.perf_counter() - t0
        e2.close()
        e2e = {"value": world * k2 * n_step / te, "unit": "histories/s",
               "h2d_bytes_per_step": int(mat_h.nbytes + rho_h.nbytes),
               "d2h_bytes_per_step": int(out_d.nbytes + out_v.nbytes)}

    vr = None
    if w.vr is not None:
        # the same workload analog: time and the bremsstrahlung-tail uncertainty
        # of both, efficiency 1 / (U^2 T) per history
        vr_w = w
        w = S.Workload(w.name, w.phantom, w.source, w.transport, w.n_hist, w.seed, None)
        Ma = measure(kernel, args.steps)
        w = vr_w
        nz = w.phantom.mat.shape[0]
        Ua, na = tail_uncertainty(Ma["dose"], Ma["var"], nz)
        Uv, nv = tail_uncertainty(dose, var, nz)
        va_ = n_total / Ma["t_dev"]
        vr = {"params": {"f_inel": w.vr.f_inel, "f_brems": w.vr.f_brems,
                         "n_split_brems": w.vr.n_split_brems, "w_window": [w.vr.w_lo, w.vr.w_hi]},
              "value_vr": value, "value_analog": va_, "unit": "histories/s",
              "tail_rel_sigma_vr": Uv, "tail_rel_sigma_analog": Ua, "tail_voxels": [nv, na],
              "tail": "slabs from the first one after the peak below 0.1 % of the peak slab on "
                      "(the bremsstrahlung tail), voxels >= 10 % of the tail maximum",
              "efficiency_gain_tail": (Ua * Ua * Ma["t_dev"]) / (Uv * Uv * t_dev),
              "U_ge_50pct_vr": U, "U_ge_50pct_analog": rel_uncertainty(Ma["dose"], Ma["var"], 0.5)}

    adj = None
    if not args.no_adjoint and w.vr is None:
        adj = measure_adjoint(args, w, G, local, stream, tuning, first_of, barrier, dist,
                              plain["value"] / world if plain else None)
        if adj is not None:
            adj["value"] *= world

    # the metric's other configurations, as sub-lines of the same run: the
    # 256^3 CT phantom with the 20 MeV electron beam (wavefront and plain
    # kernels), and the 64-job batch in one batched run (against the same jobs
    # run one by one with the plain kernel)
    extra = {}
    if not args.no_extra and args.workload == "grf128" and args.kernel == "wavefront":
        wc = WORKLOADS["ct256"](args.extra_hist)
        Mc = measure(G.KERNEL_WAVEFRONT, 3, ClockSampler(local), wl=wc, n=args.extra_hist, warmup=2)
        Mcp = measure(G.KERNEL_PLAIN, 2, wl=wc, n=args.extra_hist, warmup=1)
        vc = world * 3 * args.extra_hist / Mc["t_dev"]
        vcp = world * 2 * args.extra_hist / Mcp["t_dev"]
        Uc = rel_uncertainty(Mc["dose"], Mc["var"], 0.5)
        nc1 = world * 3 * args.extra_hist * (Uc / 0.01) ** 2
        extra["ct256"] = {
            "workload": wc.name, "value": vc, "unit": "histories/s", "steps": 3, "warmup": 2,
            "histories_per_step": args.extra_hist, "ms_per_step": 1e3 * Mc["t_dev"] / 3,
            "plain_kernel": {"value": vcp, "ms_per_step": 1e3 * Mcp["t_dev"] / 2, "steps": 2},
            "vs_plain_kernel": vc / vcp, "clocks": Mc["clk"],
            "uncertainty": {"U_mean_rel_sigma_D_ge_50pct": Uc, "histories_to_1pct": nc1,
                            "seconds_to_1pct": nc1 / vc},
            "events_per_history": {k: Mc["stats"][k] / max(1, Mc["stats"]["n_hist"]) for k in OP_BUDGET}}
        if world == 1:
            extra["batch64"] = batch_line(args, local, G, scale=args.extra_batch_scale,
                                          steps=min(args.steps, 5), warmup=min(args.warmup, 2))

    cpu = None
    mix = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
        mix = event_mix(cpu.pop("oracle_stats"))
    # the algorithmic roofline of the dominant kernel: the method's operations
    # for the events its launches processed (event mix counted by the oracle on
    # the same workload) over the pipes' peaks measured on this GPU
    algo = None
    if mix is not None:
        a_ops = algorithmic_ops(stt, mix, kpart)
        algo = pipe_roofline(a_ops, nl * t_launch, peaks)
        algo["ops_per_launch"] = {"alu": a_ops[0] / nl, "imul": a_ops[1] / nl, "sfu": a_ops[2] / nl}
        algo["ops_per_history_all_kernels"] = [x / max(1, stt["n_hist"]) for x in
                                               algorithmic_ops(stt, mix, "all")]
        algo["event_mix"] = mix

    if rank == 0:
        line = {
            "metric": "primary histories/s at 1% dose uncertainty",
            "value": value, "unit": "histories/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "histories_per_step": n_step, "batches": args.batches,
                       "kernel": args.kernel, "blocks_per_sm": args.blocks_per_sm or 3,
                       "photon_budget": tuning["photon_budget"] or 16,
                       "charged_budget": tuning["charged_budget"] or 32,
                       "pass_target": tuning["pass_target"] or "queue_cap/2",
                       "autotuned": tuned is not None,
                       "queue_cap": args.queue_cap or (1 << 24),
                       "l2": "flushed between steps (512 MB write)",
                       "phantom": list(w.phantom.shape), "voxel_mm": w.phantom.dx * 10},
            "uncertainty": {"U_mean_rel_sigma_D_ge_50pct": U, "histories": n_total,
                            "histories_to_1pct": n1, "seconds_to_1pct": n1 / value,
                            "efficiency_1_over_U2T": 1.0 / (U * U * t_dev)},
            "roofline": roofline_json(algo, achieved, peaks, kname, t_launch, nl, ops, stt,
                                      load_traffic(kname, args.workload)),
            "peaks_measured": {k: v for k, v in peaks.items()},
            "configs": extra or None,
            "plain_kernel": plain,
            "cpu_baseline": cpu, "e2e": e2e, "adjoint": adj, "vr": vr, "clocks": clk,
            "gpu_launches": int(st["n_kernel_launches"]),
            "pass_loop": {"passes": int(st["n_passes"]), "graph_launches": int(st["n_graph_launches"]),
                          "loop": "CUDA-graph while loop, condition set by the pass-control kernel"}
            if kernel == G.KERNEL_WAVEFRONT else None,
            "events_per_history": {k: st[k] / max(1, st["n_hist"]) for k in OP_BUDGET},
            "kernel_split_ms": {"steps": Mt["steps"], "transport": stt["transport_ms"],
                                "photon_and_knock": stt["photon_ms"], "drain": stt["drain_ms"],
                                "flush": stt["flush_ms"],
                                "ms_per_step_timed_launches": 1e3 * Mt["t_dev"] / Mt["steps"]},
            "wall_s": t_wall, "src_hash": src_hash(), "transport_src_hash": transport_src_hash(),
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
