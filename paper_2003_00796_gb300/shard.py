"""Multi-GPU runs: histories are independent (the paper's processes meet only to
sum their tallies at the end, Sec. 4.3), so a run is split into contiguous
history-id ranges, one per rank, and the only exchange is one FP64 sum of the
per-voxel tally moments after the last run.

Each rank keeps its own batches. The library exports a tally's moments
(gbmc_get_moments: per voxel S1 = sum_k B_k and S2 = sum_k B_k^2 / n_k, with
the history and batch counts) and takes summed ones back (gbmc_add_moments);
the estimator itself (mean S1 / N, variance (S2 - N mean^2) / (N (K - 1))) is
the library's, so this module only partitions ids, checks that every rank
reached the exchange, and sums arrays.
"""
from __future__ import annotations

import datetime

import numpy as np


class MissingRanksError(RuntimeError):
    """Some ranks never reached the tally exchange: their histories are missing
    from every pooled result."""

    def __init__(self, missing, spans):
        self.missing = list(missing)
        self.spans = list(spans)
        desc = ", ".join(f"rank {r}: ids [{a}, {a + c})" for r, (a, c) in zip(missing, spans))
        super().__init__(f"ranks that did not reach the tally exchange: {desc}")


def history_range(n_hist: int, first_hist: int, rank: int, world: int) -> tuple[int, int]:
    """(first id, count) of rank's share of [first_hist, first_hist + n_hist):
    rank r takes [first + floor(r N / R), first + floor((r + 1) N / R))."""
    if world < 1 or not 0 <= rank < world or n_hist < 0:
        raise ValueError("need 0 <= rank < world and n_hist >= 0")
    a = (n_hist * rank) // world
    b = (n_hist * (rank + 1)) // world
    return first_hist + a, b - a


def exchange_ready(store, rank: int, world: int, n_hist: int, first_hist: int,
                   timeout_s: float = 30.0, tag: str = "gbmc") -> None:
    """Failure detection on the host, before the collective: every rank
    announces itself in the key-value store of the process group and waits
    (at most timeout_s) for all the others. A rank that died or never got
    here is found by its missing key, and MissingRanksError names the history
    ranges that the pooled tally would lack, instead of the all-reduce
    waiting on a rank that will never join."""
    keys = [f"{tag}/ready/{r}" for r in range(world)]
    store.set(keys[rank], "1")
    try:
        store.wait(keys, datetime.timedelta(seconds=timeout_s))
    except Exception:
        missing = [r for r in range(world) if not store.check([keys[r]])]
        if not missing:
            raise
        raise MissingRanksError(missing, [history_range(n_hist, first_hist, r, world)
                                          for r in missing]) from None


def allreduce_moments(s1, s2, n_hist: int, n_batches: int, group=None):
    """One FP64 sum over all ranks of the tally moments and counts (CPU tensors
    for gloo, CUDA tensors for nccl). Returns the summed (s1, s2, n_hist,
    n_batches) as numpy arrays and ints."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    s1 = torch.as_tensor(s1, dtype=torch.float64).reshape(-1)
    s2 = torch.as_tensor(s2, dtype=torch.float64).reshape(-1)
    cnt = torch.tensor([float(n_hist), float(n_batches)], dtype=torch.float64)
    buf = torch.cat([s1.cpu(), s2.cpu(), cnt]).to(dev)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    nv = s1.numel()
    return out[:nv], out[nv:2 * nv], int(round(out[2 * nv])), int(round(out[2 * nv + 1]))


def combine(engine, group=None, store=None, n_hist: int = 0, first_hist: int = 0,
            timeout_s: float = 30.0):
    """Replace the engine's tally by the pool of every rank's tally: its moments
    (read through the C ABI), summed over the ranks, added back into the reset
    tally. Afterwards engine.dose() gives the pooled dose and variance on every
    rank. With a ``store`` (the process group's key-value store), ranks that
    never reached the exchange are reported (MissingRanksError, naming their
    shares of the n_hist ids from first_hist) before any collective runs.
    Statistics are reset with the tally: read them first."""
    import torch.distributed as dist
    if store is not None:
        exchange_ready(store, dist.get_rank(group), dist.get_world_size(group), n_hist,
                       first_hist, timeout_s)
    s1, s2, n, k = engine.moments()
    S1, S2, N, K = allreduce_moments(s1, s2, n, k, group)
    engine.reset()
    engine.add_moments(S1, S2, N, K)
    return N, K
