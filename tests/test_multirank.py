"""Multi-rank host logic on CPU (gloo, world size 2): disjoint trajectory shards, and the end-of-job
sum of (sum S, sum S^2, count) per observable reproduces the single-process ensemble exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_total, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as o
    from paper_2107_06147_gb300 import inputs, sharding
    w = inputs.small_parity(N=32, n_traj=n_total, seed=3)
    ids = sharding.shard(n_total, rank, world)
    g = o.Grid(N=32, L=w.grid.L, dt=w.grid.dt)
    inits = [o.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits]
    media = [o.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media]
    obs, _, _ = o.run_batch(g, inits, w.init_idx[ids], media, w.medium_idx[ids], w.seeds[ids], n_threads=1)
    m = sharding.local_moments(obs, w.medium_idx[ids], len(w.media))
    tot = sharding.reduce_moments(m)
    np.save(os.path.join(out_dir, f"ids{rank}.npy"), ids)
    np.save(os.path.join(out_dir, f"tot{rank}.npy"), tot)
    dist.destroy_process_group()


def test_two_rank_shards_and_reduction(tmp_path, oracle_lib):
    n_total = 23
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_total, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    ids = [np.load(tmp_path / f"ids{r}.npy") for r in range(2)]
    assert len(np.intersect1d(ids[0], ids[1])) == 0
    assert np.array_equal(np.sort(np.concatenate(ids)), np.arange(n_total))
    t0, t1 = (np.load(tmp_path / f"tot{r}.npy") for r in range(2))
    assert np.array_equal(t0, t1)
    # the same ensemble computed in one process
    import oracle as o
    from paper_2107_06147_gb300 import inputs, sharding
    w = inputs.small_parity(N=32, n_traj=n_total, seed=3)
    g = o.Grid(N=32, L=w.grid.L, dt=w.grid.dt)
    inits = [o.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits]
    media = [o.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media]
    obs, _, _ = o.run_batch(g, inits, w.init_idx, media, w.medium_idx, w.seeds)
    ref = sharding.local_moments(obs, w.medium_idx, len(w.media))
    np.testing.assert_allclose(t0, ref, rtol=1e-12, atol=1e-300)
    mean, sem = sharding.ensemble(t0)
    assert mean.shape == (len(w.media), 6) and np.all(sem >= 0)


def test_shard_edges():
    from paper_2107_06147_gb300 import sharding
    assert [len(sharding.shard(10, r, 4)) for r in range(4)] == [3, 3, 2, 2]
    assert len(sharding.shard(0, 0, 2)) == 0
    with pytest.raises(ValueError):
        sharding.shard(5, 2, 2)
