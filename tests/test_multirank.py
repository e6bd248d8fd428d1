"""History sharding across ranks and the one end-of-run exchange, on CPU ranks
(gloo, world size 2). Each rank transports its share of the histories with the
oracle; the pooled tally must equal one run over all histories, because the
ranks' batches are exactly the batches of the single run."""
import os
import socket
import tempfile

import numpy as np
import pytest

import synthetic as S
from paper_2003_00796_gb300 import shard

N_TOTAL, K_TOTAL, WORLD = 1600, 8, 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = S.workload_water_pencil(N_TOTAL)
        first, n = shard.history_range(N_TOTAL, 0, rank, world)
        r = O.run(w.phantom, w.source, w.transport, n, seed=3, first_hist=first,
                  n_batches=K_TOTAL // world)
        m, v, n_tot, k_tot = shard.combine(r.edep_mean, r.edep_sigma_batch ** 2, n,
                                           r.n_batches)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), m=m, v=v, n=n_tot, k=k_tot)
    finally:
        dist.destroy_process_group()


def test_history_range_partitions():
    for n in (0, 1, 7, 1000, 12345):
        for world in (1, 2, 3, 8):
            spans = [shard.history_range(n, 17, r, world) for r in range(world)]
            ids = [i for a, c in spans for i in range(a, a + c)]
            assert ids == list(range(17, 17 + n))
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def test_moments_round_trip():
    rng = np.random.default_rng(0)
    m = rng.random(50)
    v = rng.random(50) * 1e-3
    s1, s2 = shard.moments(m, v, 1000, 10)
    m2, v2 = shard.pooled(s1, s2, 1000, 10)
    np.testing.assert_allclose(m2, m, rtol=1e-14)
    np.testing.assert_allclose(v2, v, rtol=1e-9, atol=1e-18)


def test_two_gloo_ranks_pool_to_the_single_run():
    import torch.multiprocessing as mp
    import oracle as O
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(WORLD, _free_port(), d), nprocs=WORLD,
                           start_method="spawn")
        res = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(WORLD)]
    w = S.workload_water_pencil(N_TOTAL)
    one = O.run(w.phantom, w.source, w.transport, N_TOTAL, seed=3, first_hist=0,
                n_batches=K_TOTAL)
    for r in res:   # every rank holds the pooled result
        assert int(r["n"]) == N_TOTAL and int(r["k"]) == K_TOTAL
        np.testing.assert_allclose(r["m"], one.edep_mean, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r["v"], one.edep_sigma_batch ** 2, rtol=1e-8, atol=1e-18)
    assert one.edep_mean.sum() > 0.1


def test_rank_that_raises_is_reported():
    """A rank that fails before the exchange: the launcher reports it instead of
    hanging the other rank (gloo's default timeout is not reached because the
    failing rank's process group is torn down)."""
    import torch.multiprocessing as mp
    with pytest.raises(Exception):
        mp.start_processes(_failing_rank, args=(WORLD, _free_port()), nprocs=WORLD,
                           start_method="spawn")


def _failing_rank(rank, world, port):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    if rank == 1:
        raise RuntimeError("rank 1 fails before the tally exchange")
    shard.combine(np.zeros(4), np.zeros(4), 10, 2)
