"""History sharding across ranks and the one end-of-run exchange, on CPU ranks
(gloo, world size 2). Each rank transports its share of the histories with the
oracle; the summed tally moments must equal those of one run over all
histories, because the ranks' batches are exactly the batches of the single
run. A rank that dies before the exchange is reported by the others, with the
history ranges that are missing, before any collective runs."""
import datetime
import multiprocessing
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


def _init(rank, world, port):
    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                          timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    return store


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle as O
    store = _init(rank, world, port)
    try:
        w = S.workload_water_pencil(N_TOTAL)
        first, n = shard.history_range(N_TOTAL, 0, rank, world)
        r = O.run(w.phantom, w.source, w.transport, n, seed=3, first_hist=first,
                  n_batches=K_TOTAL // world)
        shard.exchange_ready(store, rank, world, N_TOTAL, 0, timeout_s=30)
        s1, s2, n_tot, k_tot = shard.allreduce_moments(r.batch_s1, r.batch_s2, n, r.n_batches)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), s1=s1, s2=s2, n=n_tot, k=k_tot)
    finally:
        dist.destroy_process_group()


def test_history_range_partitions():
    for n in (0, 1, 7, 1000, 12345):
        for world in (1, 2, 3, 8):
            spans = [shard.history_range(n, 17, r, world) for r in range(world)]
            ids = [i for a, c in spans for i in range(a, a + c)]
            assert ids == list(range(17, 17 + n))
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


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
    for r in res:   # every rank holds the summed moments of all batches
        assert int(r["n"]) == N_TOTAL and int(r["k"]) == K_TOTAL
        np.testing.assert_allclose(r["s1"], one.batch_s1, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r["s2"], one.batch_s2, rtol=1e-12, atol=1e-18)
    assert one.batch_s1.sum() > 0.1


def _dying_rank(rank, world, port, out_path):
    """Rank 1 dies between its transport and the exchange; rank 0 must learn it
    on the host and name rank 1's missing history ids."""
    import torch.distributed as dist
    store = _init(rank, world, port)
    if rank == 1:
        os._exit(3)   # dies without reaching the exchange (no clean-up, like a crash)
    try:
        shard.exchange_ready(store, rank, world, N_TOTAL, 100, timeout_s=5)
        msg = "no error"
    except shard.MissingRanksError as e:
        msg = f"{e.missing}|{e.spans}|{e}"
    with open(out_path, "w") as f:
        f.write(msg)
    os._exit(0)


def test_rank_that_dies_is_reported_with_its_missing_histories():
    ctx = multiprocessing.get_context("spawn")
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "rank0.txt")
        port = _free_port()
        ps = [ctx.Process(target=_dying_rank, args=(r, WORLD, port, out)) for r in range(WORLD)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
        for p in ps:
            if p.is_alive():
                p.kill()
        assert ps[1].exitcode == 3
        msg = open(out).read()
    first, n = shard.history_range(N_TOTAL, 100, 1, WORLD)
    assert msg.startswith("[1]|"), msg
    assert f"[{first}, {first + n})" in msg
