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


class _FakeSolver:
    """Stands in for binding.Solver on CPU: local_greens fills the rows of its sources with a
    value that identifies the site and the iteration, selfenergy_step checks that every row
    arrived and returns a falling measure."""

    def __init__(self, Nr, Nc):
        import torch
        from types import SimpleNamespace
        self.p = SimpleNamespace(Nr=Nr, Nc=Nc)
        self.device = torch.device("cpu")
        self.it = 0
        self.seen = []

    def set_anderson(self, depth):
        self.depth = depth

    def local_greens(self, sources, precision=0, tol=0.0, max_sweeps=0, out=None):
        for s in sources:
            out[s] = complex(s + 1, self.it)
        return out, type("R", (), {"report": {"sweeps": 1}})()

    def selfenergy_step(self, gloc, mix=0.7):
        import torch
        expect = torch.stack([torch.full((self.p.Nc, self.p.Nc), complex(s + 1, self.it), dtype=torch.complex128)
                              for s in range(self.p.Nr)])
        self.seen.append(bool(torch.equal(gloc, expect)))
        self.it += 1
        return 10.0 ** (-self.it)


def _loop_worker(rank, world, port, q):
    import torch.distributed as td
    from paper_1309_5994_gb300.selfconsistency import self_consistent_sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init("gloo")
    try:
        s = _FakeSolver(Nr=5, Nc=3)
        r = self_consistent_sharded(s, mix=0.7, delta_sc=1e-3, max_iter=10, anderson=2)
        q.put((rank, r["iterations"], r["history"], r["sites"], s.seen, s.depth))
    finally:
        td.destroy_process_group()


def test_sharded_self_consistency_exchanges_every_row():
    """Two gloo ranks share the sites of the self-consistency loop; after the row exchange
    both hold every site's local Green's function and take identical steps."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_loop_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, it0, h0, s0, seen0, d0), (r1, it1, h1, s1, seen1, d1) = out
    assert sorted(s0 + s1) == list(range(5)) and not set(s0) & set(s1)
    assert it0 == it1 == 3 and h0 == h1 and all(seen0) and all(seen1) and d0 == d1 == 2
