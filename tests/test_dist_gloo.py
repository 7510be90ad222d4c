"""Multi-rank host logic on CPU: two gloo ranks shard block columns, reduce the
timed region with a max and merge per-site observables (no GPU involved)."""
import os
import socket

import numpy as np
import pytest

from paper_1309_5994_gb300 import dist


def test_step_sources_partition_all_sites():
    n_sites, batch, world = 256, 16, 4
    seen = []
    for step in range(n_sites // (batch * world)):
        for rank in range(world):
            seen += dist.step_sources(n_sites, batch, rank, world, step)
    assert sorted(seen) == list(range(n_sites))


def test_shard_sites_balanced_cover():
    for n, w in ((256, 3), (7, 4), (1, 2)):
        parts = [dist.shard_sites(n, r, w) for r in range(w)]
        assert sorted(sum(parts, [])) == list(range(n))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1


def test_merge_rejects_conflicts():
    a = np.full((2, 3), np.nan)
    b = np.full((2, 3), np.nan)
    a[0] = 1.0
    b[0] = 2.0
    with pytest.raises(ValueError):
        dist.merge_observables([a, b])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, _ = dist.init("gloo")
    try:
        Nr, Nt = 10, 4
        obs = np.full((3, Nr, Nt), np.nan)
        for i in dist.shard_sites(Nr, r, w):
            obs[:, i, :] = 100.0 * i + np.arange(Nt)
        merged = dist.all_gather_observables(obs)
        dist.barrier()
        m = dist.max_over_ranks(1.5 + r)
        q.put((r, m, merged))
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_merge_and_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = np.stack([np.stack([100.0 * i + np.arange(4) for i in range(10)])] * 3)
    for r, m, merged in out:
        assert m == 2.5
        assert np.array_equal(merged, expect)
