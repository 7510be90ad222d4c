"""The seeded input recipe: every workload has the documented shape, drive and seed, so the
benchmark, the parity tests and the oracle see the same problems on every machine."""
import numpy as np

import workloads as wl


def test_shapes_of_the_named_workloads():
    cases = [(wl.trapped_4x4_nc64(), 4, 24, 16, 1.0, 0.5), (wl.trapped_16x16_nc256(), 16, 112, 32, 2.0, 0.02),
             (wl.driven_32x32_nc384(), 32, 160, 64, 2.0, 0.005), (wl.driven_24x24_nc256(), 24, 96, 64, 2.0, 0.005)]
    for p, L, Nt, Nm, beta, c in cases:
        assert (p.Lx, p.Ly, p.Nt, p.Nm, p.dt, p.beta, p.trap_c, p.mu) == (L, L, Nt, Nm, 0.05, beta, c, 0.0)
        assert p.U.shape == (L * L, Nt) and p.J.shape == (wl.n_bonds(L, L), Nt)
    assert wl.trapped_16x16_nc256().Nc == 256 and wl.driven_32x32_nc384().Nc == 384


def test_drives():
    t = np.arange(160) * 0.05
    p = wl.driven_32x32_nc384()
    assert np.allclose(p.U, 20.0 * (1.0 + 0.1 * np.sin(20.0 * t))[None, :], rtol=0, atol=1e-13)
    assert np.allclose(p.J, (1.0 - 0.2 * np.sin(20.0 * t))[None, :], rtol=0, atol=1e-13)
    q = wl.trapped_16x16_nc256()
    assert np.all(q.U == 20.0) and np.all(q.J == 1.0)
    a = wl.driven_24x24_nc256(2.0)
    t = np.arange(96) * 0.05
    assert np.allclose(a.U[0], 20.0 * (1.0 + 0.2 * np.sin(20.0 * t)), rtol=0, atol=1e-13)


def test_uneven_batch_is_seeded_and_within_its_ranges():
    a, b = wl.uneven_batch(), wl.uneven_batch()
    assert len(a) == 64
    for p, q in zip(a, b):                     # same seed, same problems
        assert p.name == q.name and np.array_equal(p.U, q.U) and np.array_equal(p.J, q.J)
    for p in a:
        assert 8 <= p.Lx <= 24 and p.Lx == p.Ly
        assert p.Nc in (128, 192, 256) and p.Nm == p.Nc // 4 and 2 * p.Nt + p.Nm == p.Nc
        assert 12.0 <= p.meta["U0"] <= 30.0 and 0.005 <= p.trap_c <= 0.05
        assert 0.0 <= p.meta["phase"] < 2 * np.pi
    assert len({p.Nc for p in a}) == 3


def test_loss_weights_are_seeded_uniform():
    w = wl.loss_weights()
    assert w.shape == (576,) and np.all((w >= 0) & (w < 1)) and np.array_equal(w, wl.loss_weights())
