"""GPU parity at the configured sizes: the wavefront path against the oracle on
the full 128^3 x 2 mm three-material phantom with the 0.1-6 MeV field, on the
full 256^3 x 1 mm CT-like phantom with the 20 MeV electron beam, and a batched
run of uneven jobs (up to 18 MeV, a 160^3 phantom) with every job gated
against the oracle.

At these sizes a practical number of oracle histories leaves most voxels
with a few deposits, so besides the voxel-level comparison the doses are also
compared on blocks of voxels (energy over mass of 4^3 or 8^3 voxels), where
each value is well populated. Both verdicts are printed for every
comparison: the permutation gate (exact under correlated voxels) decides;
the literal gate (>= 95 % within 2 combined sigma, textbook chi-square
p > 0.01) is reported beside it.
"""
import os
import time

import numpy as np
import pytest

import oracle as O
import paper_2003_00796_gb300 as G
import synthetic as S
from engines import gpu_dual, oracle_dual
from parity import dual_gate, permutation_gate

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def blocks(B, ph, f):
    """Dose (energy over mass) of f^3-voxel blocks, per batch: (K, nblocks)."""
    nz, ny, nx = ph.mat.shape
    mass = ph.rho.astype(np.float64)
    B = np.asarray(B).reshape(-1, nz, ny, nx)
    cz, cy, cx = nz // f * f, ny // f * f, nx // f * f
    e = (B * mass)[:, :cz, :cy, :cx].reshape(-1, cz // f, f, cy // f, f, cx // f, f).sum((2, 4, 6))
    m = mass[:cz, :cy, :cx].reshape(cz // f, f, cy // f, f, cx // f, f).sum((1, 3, 5))
    return (e / m).reshape(B.shape[0], -1)


def show(label, res):
    def r(x):
        return round(x, 4) if isinstance(x, float) else x
    out = {k: r(v) for k, v in res.items() if k != "literal"}
    if "literal" in res:
        out["literal"] = {k: r(v) for k, v in res["literal"].items()}
    print(label, out, flush=True)


def full_parity(w, K, nk, f_block, seed, n_perm=200):
    t0 = time.time()
    Bg, dg, vg, st = gpu_dual(w, K, nk, seed=seed, kernel=G.KERNEL_WAVEFRONT)
    t1 = time.time()
    Bo, do, vo = oracle_dual(w, K, nk, seed=seed + 500, n_threads=NTHREADS)
    t2 = time.time()
    vox = dual_gate(Bg, Bo, dg, vg, do, vo, thr=0.1, n_perm=n_perm)
    blk = permutation_gate(blocks(Bg, w.phantom, f_block), blocks(Bo, w.phantom, f_block),
                           thr=0.1, n_perm=1000)
    print(f"{w.name}: {K} x {nk} histories per engine, gpu {t1 - t0:.1f} s, oracle {t2 - t1:.1f} s "
          f"on {NTHREADS} threads, gpu batches pooled {st['pooled_batches']}", flush=True)
    show(f"{w.name} voxels", vox)
    show(f"{w.name} {f_block}^3 blocks", blk)
    assert st["error_flags"] == 0
    return vox, blk


def test_grf128_full_phantom_against_oracle():
    """128^3 x 2 mm water/bone/lung phantom (seed 2), 10 x 10 cm field of the
    0.1-6 MeV Kramers spectrum: 1e6 histories per engine."""
    w = S.workload_grf_spectrum(128, 0)
    vox, blk = full_parity(w, K=20, nk=50_000, f_block=4, seed=101)
    assert vox["n_vox"] > 100_000 and blk["n_vox"] > 2000
    assert vox["pass"] and blk["pass"]


def test_ct256_full_phantom_against_oracle():
    """256^3 x 1 mm CT-like phantom (seed 3, four materials), 20 MeV electron
    5 x 5 cm beam: 2e5 histories per engine."""
    w = S.workload_ct_electron(256, 0)
    vox, blk = full_parity(w, K=20, nk=10_000, f_block=8, seed=202)
    assert blk["n_vox"] > 200
    assert vox["pass"] and blk["pass"]


def test_batched_jobs_each_against_oracle():
    """One batched run of five uneven jobs -- a 160^3 x 1.5 mm phantom with a
    2 MeV photon field, an 18 MeV electron pencil, a 100 keV photon field, a
    1 MeV electron field and a 6 MeV photon pencil on three-material random
    fields -- repeated on 20 disjoint history sets; every job's 20 doses
    against 20 oracle runs of the same job (same phantom, source and seed
    convention: job id = index)."""
    specs = [  # (side, voxel cm, particle, energy MeV, field half width cm, histories per run)
        (160, 0.15, S.PHOTON, 2.0, 3.0, 5000),
        (48, 0.3, S.ELECTRON, 18.0, 0.0, 1000),
        (32, 0.4, S.PHOTON, 0.1, 4.0, 5000),
        (64, 0.2, S.ELECTRON, 1.0, 2.0, 2000),
        (40, 0.1, S.PHOTON, 6.0, 0.0, 5000),
    ]
    jobs = []
    for j, (n, d, part, E, h, nk) in enumerate(specs):
        ph = S.grf_three_material(n, d, seed=40 + j)
        L = n * d
        src = S.Source(part, 1 if h > 0 else 0, L / 2, L / 2, h, h, E)
        jobs.append((ph, src, nk))
    K, seed = 20, 77
    e = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=8)
    e.set_materials([S.water(), S.bone(), S.lung()], S.Transport(), 18.0 * 1.02)
    Bg = [[] for _ in jobs]
    for k in range(K):
        e.run_batch([(ph, src, nk, seed, k * nk) for ph, src, nk in jobs])
        for j in range(len(jobs)):
            Bg[j].append(e.job_dose(j)[0])
    st = e.stats()
    e.close()
    assert st["error_flags"] == 0
    for j, (ph, src, nk) in enumerate(jobs):
        t0 = time.time()
        Bo = [O.run(ph, src, S.Transport(), nk, seed=seed, first_hist=k * nk + 10_000_000, job=j,
                    n_batches=max(2, NTHREADS), n_threads=NTHREADS).dose for k in range(K)]
        res = permutation_gate(np.array(Bg[j]), np.array(Bo), thr=0.1, n_perm=300)
        f = 8 if ph.mat.shape[0] >= 128 else 4
        blk = permutation_gate(blocks(Bg[j], ph, f), blocks(Bo, ph, f), thr=0.1, n_perm=1000)
        print(f"job {j} {ph.mat.shape} {src.energy} MeV particle {src.particle}: "
              f"oracle {time.time() - t0:.1f} s", flush=True)
        show(f"job {j} voxels", res)
        show(f"job {j} {f}^3 blocks", blk)
        assert res["pass"] and blk["pass"], j
