"""Tally moments through the C ABI (gbmc_get_moments / gbmc_add_moments): the
exchange of a multi-GPU run (Sec. 4.3: workers sum their counters at the end).
Two contexts that run disjoint halves of the histories, pooled by adding one's
moments into the other, give the tally of one run over all histories: the same
histories in the same batches, so equal up to the order of FP32 atomics."""
import numpy as np
import pytest

import paper_2003_00796_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", [G.KERNEL_PLAIN, G.KERNEL_WAVEFRONT])
def test_pooled_moments_equal_one_run(kernel):
    torch = pytest.importorskip("torch")
    w = S.workload_grf_spectrum(24, 0)
    n, K = 60_000, 10
    one = G.Engine(0, kernel=kernel, n_batches=2 * K).setup(w)
    one.run(n, seed=9)
    m1, v1 = one.edep()
    halves = []
    for r in range(2):
        e = G.Engine(0, kernel=kernel, n_batches=K).setup(w)
        e.run(n // 2, seed=9, first_hist=r * (n // 2))
        halves.append(e)
    # rank 0's moments on the host, rank 1's on the device (both pointer kinds)
    a1, a2, na, ka = halves[0].moments()
    b1 = torch.zeros(w.phantom.n_vox, dtype=torch.float64, device="cuda")
    b2 = torch.zeros_like(b1)
    _, _, nb, kb = halves[1].moments(b1, b2)
    assert (na, ka, nb, kb) == (n // 2, K, n // 2, K)
    pooled = halves[0]
    pooled.reset()
    pooled.add_moments(a1, a2, na, ka)
    pooled.add_moments(b1, b2, nb, kb)
    m, v = pooled.edep()
    big = m1 > 0.01 * m1.max()
    np.testing.assert_allclose(m[big], m1[big], rtol=1e-5)
    np.testing.assert_allclose(v[big], v1[big], rtol=1e-3)
    assert m.sum() == pytest.approx(m1.sum(), rel=1e-6)
    s1, s2, nn, kk = pooled.moments()
    assert (nn, kk) == (n, 2 * K)
    np.testing.assert_allclose(s1, a1 + b1.cpu().numpy(), rtol=1e-12, atol=1e-300)
    with pytest.raises(ValueError):
        pooled.add_moments(a1[:-1], a2[:-1], 1, 1)
    for e in halves + [one]:
        e.close()


def test_combine_over_a_one_rank_group_keeps_the_tally():
    """shard.combine on a world of one (gloo on the host): moments out, summed
    (identity), back in: the dose and its variance are unchanged."""
    import datetime
    import socket
    torch = pytest.importorskip("torch")
    import torch.distributed as dist
    from paper_2003_00796_gb300 import shard
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    store = dist.TCPStore("127.0.0.1", port, 1, True, timeout=datetime.timedelta(seconds=30))
    dist.init_process_group("gloo", store=store, rank=0, world_size=1)
    try:
        w = S.workload_water_pencil(0)
        e = G.Engine(0, n_batches=8).setup(w)
        e.run(20_000, seed=4)
        d0, v0 = e.dose()
        N, K = shard.combine(e, store=store, n_hist=20_000)
        d1, v1 = e.dose()
        assert (N, K) == (20_000, 8)
        np.testing.assert_allclose(d1, d0, rtol=1e-12, atol=0)
        np.testing.assert_allclose(v1, v0, rtol=1e-9, atol=1e-300)
        e.close()
    finally:
        dist.destroy_process_group()


def test_checkpoint_resume_continues_the_run(tmp_path):
    """Checkpoint and resume (the tally's moments saved with the next history
    id and the seed): run the first half, checkpoint, resume in a fresh
    context and run the second half. The histories are keyed by their ids, so
    the result is the tally of one context running both halves -- the same
    histories in the same batches, equal up to the order of FP32 atomics."""
    w = S.workload_grf_spectrum(24, 0)
    n, K = 60_000, 10
    ref = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=K).setup(w)
    ref.run(n // 2, seed=9, first_hist=0)
    ref.run(n // 2, seed=9, first_hist=n // 2)
    a, va = ref.edep()
    ref.close()
    first = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=K).setup(w)
    first.run(n // 2, seed=9)
    path = tmp_path / "tally.npz"
    first.checkpoint(path, next_hist=n // 2, seed=9, workload=w.name)
    first.close()
    e = G.Engine(0, kernel=G.KERNEL_WAVEFRONT, n_batches=K).setup(w)
    f = e.resume(path)
    assert (f["next_hist"], f["seed"], str(f["workload"])) == (n // 2, 9, w.name)
    e.run(n - f["next_hist"], seed=f["seed"], first_hist=f["next_hist"])
    b, vb = e.edep()
    _, _, nn, kk = e.moments()
    assert (nn, kk) == (n, 2 * K)
    big = a > 0.01 * a.max()
    np.testing.assert_allclose(b[big], a[big], rtol=1e-5)
    np.testing.assert_allclose(vb[big], va[big], rtol=1e-3)
    # a checkpoint of another phantom shape is refused before anything is added
    other = G.Engine(0, n_batches=K).setup(S.workload_water_pencil())
    with pytest.raises(ValueError):
        other.resume(path)
    assert other.moments()[2] == 0
    other.close()
    e.close()
