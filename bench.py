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
# Roofline: the transport kernel is bound by instruction issue on the plain
# ALUs (FP32 / INT / SFU); no dense contraction, phantom reads hit L2.
# Peak = 152 SMs x 4 schedulers x 32 lanes x 2.070 GHz max SM clock
#      = 40.28e12 thread-instructions/s.
# Algorithmic work = sum over events of a per-event instruction budget counted
# by hand from the device code (transport.cuh).
# ---------------------------------------------------------------------------
ALU_PEAK = 152 * 4 * 32 * 2.070e9
OP_BUDGET = {            # thread-instructions per event
    "n_tent": 100,       # Woodcock step: 2 draws (1/2 Philox block), log, divide, locate, 2 loads
    "n_real": 300,       # type choice (3 lookups + draw) + KN sampling + rotation + child
    "n_e_steps": 350,    # ~12 table lookups, 3 draws, soft deflection, rotation, step control
    "n_cross": 55,       # face distances, position, inverse-range lookup, scoring
    "n_hard": 175,       # type choice, sampling, rotation / secondary
    "n_particles": 40,   # primary sampling / stack pop
}
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
        O.run(w.phantom, w.source, w.transport, n, seed=78 + attempt, first_hist=10_000_000,
              n_batches=max(nth, 8), n_threads=nth, vr=w.vr)
        dt = time.perf_counter() - t0
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
            "serial_sample": f"{n1} histories on one host thread, {dt1:.1f} s"}


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
    if it was taken on the current sources."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        if d.get("src_hash") != src_hash():
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def run_batch_bench(args, rank, world, local):
    """64 independent jobs (phantoms 32^3-192^3 at 1-4 mm, photon or electron
    sources 0.1-18 MeV, 1e5-2e7 histories each) in one batched run per step:
    value = all jobs' histories / the batched run's device time (pass loop and
    flushes, CUDA events inside the library); wall time includes the upload of
    the 64 phantoms and the allocation of their tallies."""
    import torch
    import paper_2003_00796_gb300 as G
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle is not run on the "
                              "64-job batch (hours of host time); see the grf128 reference line"}))
        return
    torch.cuda.set_device(local)
    ws = S.batched_jobs(64, seed=4, hist_scale=args.batch_scale)
    # ranks split the jobs (independent problems: weak scaling, no exchange)
    mine = [w for j, w in enumerate(ws) if j % world == rank]
    jobs = [(w.phantom, w.source, w.n_hist, w.seed) for w in mine]
    n_total = sum(w.n_hist for w in mine)
    e = G.Engine(local, kernel=G.KERNEL_WAVEFRONT, n_batches=args.batches,
                 blocks_per_sm=args.blocks_per_sm, photon_budget=args.photon_budget,
                 charged_budget=args.charged_budget, pass_target=args.pass_target,
                 queue_cap=args.queue_cap)
    e.set_materials([S.water(), S.bone(), S.lung()], S.Transport(),
                    max(w.source.max_energy() for w in ws) * 1.02)
    tuned = None
    if args.autotune:
        tuned = e.autotune(max(1_000_000, n_total // 20), seed=7, jobs=jobs)
    for k in range(args.warmup):
        e.run_batch(jobs)
    e.reset()
    t_dev, t_wall = 0.0, 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        e.run_batch(jobs)
        t_wall += time.perf_counter() - t0
        t_dev += e.stats()["last_run_ms"] / 1e3
    st = e.stats()
    U = []
    for j in range(len(jobs)):
        d, v = e.job_dose(j)
        U.append(rel_uncertainty(d, v, 0.5))
    e.close()
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_dev, t_wall, float(n_total)], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt[:2], op=dist.ReduceOp.MAX)
        nt = tt[2:].clone()
        dist.all_reduce(nt, op=dist.ReduceOp.SUM)
        t_dev, t_wall, n_all = float(tt[0]), float(tt[1]), int(nt[0])
    else:
        n_all = n_total
    if rank == 0:
        line = {
            "metric": "primary histories/s at 1% dose uncertainty", "value": args.steps * n_all / t_dev,
            "unit": "histories/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64_grf_32-192cube_1-4mm_photon_electron_0.1-18MeV",
                       "jobs": len(ws), "histories_per_step": n_all,
                       "batches_per_job": args.batches, "autotuned": tuned,
                       "pass_loop": "one CUDA-graph launch per run: a device-driven while loop over passes"},
            "wall_s_per_step": t_wall / args.steps,
            "e2e": {"value": args.steps * n_all / t_wall, "unit": "histories/s",
                    "h2d_bytes_per_step": int(sum(p.mat.nbytes + p.rho.nbytes for p, _, _, _ in jobs)),
                    "d2h_bytes_per_step": 0},
            "uncertainty": {"median_over_jobs_U": float(np.median(U)), "max_U": float(np.max(U))},
            "gpu_launches": int(st["n_kernel_launches"]),
            "pass_loop": {"passes": int(st["n_passes"]), "graph_launches": int(st["n_graph_launches"])},
            "events_per_history": {k: st[k] / max(1, st["n_hist"]) for k in OP_BUDGET},
        }
        print(json.dumps(line))


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

    def measure(kernel, steps, clocks=None, timing=False):
        """W untimed warm-up steps, then `steps` timed steps (CUDA events on the
        run's stream, L2 flushed between steps outside the events). timing=True
        also times every launch inside the library (passes launched one by one
        instead of run by the graph's device-side loop): used for the per-kernel split."""
        eng = G.Engine(local, kernel=kernel, n_batches=args.batches, timing=timing, **tuning).setup(w)
        for k in range(args.warmup):
            eng.run(n_step, seed=w.seed, first_hist=first_of(k), stream=stream)
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
            eng.run(n_step, seed=w.seed, first_hist=first_of(args.warmup + k), stream=stream)
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
        kname = "k_wf_charged"
    elif kernel == G.KERNEL_WAVEFRONT:
        # photon-dominated workload: the photon kernel (its time is reported
        # with the knock kernel's, one knock launch per photon launch)
        ops = sum(OP_BUDGET[k] * stt[k] for k in ("n_tent", "n_real"))
        kname = "k_wf_photon"
        nl = max(1, stt["n_photon_launches"] // 2)
        t_launch = stt["photon_ms"] / 1e3 / nl
    else:
        ops = sum(OP_BUDGET[k] * stt[k] for k in OP_BUDGET)
        kname = "k_plain"
    achieved = ops / nl / t_launch
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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

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
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": ALU_PEAK / 1e12,
                         "unit": "Tinst/s", "frac": achieved / ALU_PEAK,
                         "traffic": load_traffic(kname, args.workload),
                         "kernel": kname, "launch_ms": 1e3 * t_launch,
                         "launches": int(nl),
                         "ops_per_history": ops / max(1, stt["n_hist"]),
                         "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz (instruction issue)"},
            "plain_kernel": plain,
            "cpu_baseline": cpu, "e2e": e2e, "adjoint": adj, "vr": vr, "clocks": clk,
            "gpu_launches": int(st["n_kernel_launches"]),
            "pass_loop": {"passes": int(st["n_passes"]), "graph_launches": int(st["n_graph_launches"]),
                          "loop": "CUDA-graph while loop, condition set by the pass-control kernel"}
            if kernel == G.KERNEL_WAVEFRONT else None,
            "events_per_history": {k: st[k] / max(1, st["n_hist"]) for k in OP_BUDGET},
            "kernel_split_ms": {"steps": Mt["steps"], "transport": stt["transport_ms"],
                                "photon_and_knock": stt["photon_ms"], "flush": stt["flush_ms"],
                                "ms_per_step_timed_launches": 1e3 * Mt["t_dev"] / Mt["steps"]},
            "wall_s": t_wall, "src_hash": src_hash(),
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
