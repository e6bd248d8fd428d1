"""Multi-GPU runs: histories are independent (the paper's processes meet only to
sum their tallies at the end, Sec. 4.3), so a run is split into contiguous
history-id ranges, one per rank, and the only exchange is one FP64 sum of the
per-voxel tally moments after the last run.

Each rank keeps its own batches (K_r of them over N_r histories). From a rank's
batch mean m_r and variance of the mean v_r per voxel the two moments are

    S1_r = N_r m_r
    S2_r = v_r N_r (K_r - 1) + N_r m_r^2      (= sum over its batches of B_k^2 / n_k)

and the pooled result over K = sum K_r batches and N = sum N_r histories is

    m = sum S1_r / N,   v = (sum S2_r - N m^2) / (N (K - 1)),

which is the single-GPU batch estimator applied to all batches of all ranks.
"""
from __future__ import annotations

import numpy as np


def history_range(n_hist: int, first_hist: int, rank: int, world: int) -> tuple[int, int]:
    """(first id, count) of rank's share of [first_hist, first_hist + n_hist):
    rank r takes [first + floor(r N / R), first + floor((r + 1) N / R))."""
    if world < 1 or not 0 <= rank < world or n_hist < 0:
        raise ValueError("need 0 <= rank < world and n_hist >= 0")
    a = (n_hist * rank) // world
    b = (n_hist * (rank + 1)) // world
    return first_hist + a, b - a


def moments(mean: np.ndarray, var: np.ndarray, n_hist: int, n_batches: int):
    """(S1, S2) of one rank from its batch mean and variance of the mean."""
    mean = np.asarray(mean, np.float64)
    var = np.asarray(var, np.float64)
    s1 = n_hist * mean
    s2 = var * n_hist * max(n_batches - 1, 0) + n_hist * mean * mean
    return s1, s2


def pooled(s1: np.ndarray, s2: np.ndarray, n_hist: int, n_batches: int):
    """(mean, variance of the mean) from summed moments."""
    m = s1 / n_hist
    v = (s2 - n_hist * m * m) / (n_hist * max(n_batches - 1, 1))
    return m, np.maximum(v, 0.0)


def combine(mean, var, n_hist: int, n_batches: int, group=None):
    """Sum the tally moments of all ranks (torch.distributed all-reduce of FP64
    tensors: CPU tensors for gloo, CUDA tensors for nccl) and return the pooled
    (mean, variance, histories, batches) on every rank."""
    import torch
    import torch.distributed as dist
    s1, s2 = moments(mean, var, n_hist, n_batches)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = torch.from_numpy(np.concatenate([s1, s2, [float(n_hist), float(n_batches)]])).to(dev)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    nv = s1.size
    n_tot, k_tot = int(round(out[2 * nv])), int(round(out[2 * nv + 1]))
    m, v = pooled(out[:nv], out[nv:2 * nv], n_tot, k_tot)
    return m, v, n_tot, k_tot
