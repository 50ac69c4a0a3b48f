"""The seeded input generators: the statistics the input recipe states, and
determinism.  No method arithmetic lives in channels.py; these tests pin the
workloads both the GPU path and the oracle read."""
import math

import numpy as np
import pytest

from paper_2304_12745_gb300 import channels as ch


def test_same_seed_same_data_other_seed_other_data():
    for fn in (ch.rayleigh, ch.lognormal, ch.rician_ula):
        a, b, c = fn(16, 4, 32, seed=7), fn(16, 4, 32, seed=7), fn(16, 4, 32, seed=8)
        assert a.dtype == np.complex64 and a.shape == (16, 4, 32) and a.flags.c_contiguous
        assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_prefix_of_a_batch_is_the_smaller_batch():
    for fn in (ch.rayleigh, ch.lognormal):
        assert np.array_equal(fn(10, 4, 16, seed=3)[:5], fn(5, 4, 16, seed=3))


def test_rayleigh_is_cn01():
    H = ch.rayleigh(2048, 8, 64, seed=1)
    assert abs(H.mean()) < 5e-3
    assert H.real.var() == pytest.approx(0.5, rel=0.01)
    assert H.imag.var() == pytest.approx(0.5, rel=0.01)
    assert abs(np.mean(H.real * H.imag)) < 5e-3


def test_lognormal_gains_spread_8_db():
    H = ch.lognormal(2048, 8, 64, seed=2)
    p_db = 10 * np.log10((np.abs(H) ** 2).mean(-1))  # per-user row power
    # 8 dB of shadowing plus ~0.54 dB of estimation noise from 64 antennas
    assert p_db.std() == pytest.approx(math.hypot(8.0, 0.54), abs=0.25)
    assert abs(p_db.mean()) < 0.3
    # within a row the entries stay i.i.d.: the row-normalised power is flat across antennas
    Hn = H / np.sqrt((np.abs(H) ** 2).mean(-1, keepdims=True))
    assert (np.abs(Hn) ** 2).mean((0, 1)) == pytest.approx(np.ones(64), abs=0.05)


def test_rician_unit_power_and_line_of_sight():
    H = ch.rician_ula(4096, 4, 64, seed=3).astype(np.complex128)
    assert (np.abs(H) ** 2).mean() == pytest.approx(1.0, rel=0.01)
    # the LoS term has unit modulus on every antenna and a phase progression
    # pi sin(theta) along the array, so neighbouring antennas are correlated:
    # |E[h_m conj(h_{m+1})]| per user equals kappa / (kappa + 1) > 0
    c = np.abs((H[..., :-1] * H[..., 1:].conj()).mean(-1))
    assert np.median(c) > 0.3
    # kappa_dB ~ U[0, 10]: kappa / (kappa + 1) in [0.5, 0.91], up to estimation noise
    assert np.quantile(c, 0.05) > 0.3 and np.quantile(c, 0.95) < 1.05


def test_targets_and_steps():
    t = ch.targets(3, 8, gamma_db=10.0, sigma_nu=0.5)
    assert t.dtype == np.float32 and np.allclose(t, 0.5 * math.sqrt(10.0))
    assert np.all(ch.targets(2, 4) == 1.0)
    mu = ch.fixed_workload_steps(10)
    assert mu.dtype == np.float32 and mu.shape == (10,)
    assert np.all((mu >= 0.01) & (mu <= 0.1))
    assert np.array_equal(mu, ch.uniform_steps(10, 0.01, 0.1, seed=2))


def test_paper_step_is_the_marchenko_pastur_edge():
    # 1 / (sqrt K + sqrt M)^2; K = 4, M = 32 gives the tiny workload's 0.017057
    assert ch.paper_eta(4, 32) == pytest.approx(0.017057, abs=5e-7)
    assert ch.paper_eta(8, 64) == pytest.approx(1 / (math.sqrt(8) + 8) ** 2)


def test_uneven_shapes_and_packing():
    shapes = ch.uneven_shapes(32768, seed=3)
    assert shapes.dtype == np.int32 and shapes.shape == (32768, 2)
    _, counts = np.unique(shapes[:, 0], return_counts=True)
    assert len(counts) == 4 and np.all(np.abs(counts - 8192) < 400)
    assert {tuple(x) for x in np.unique(shapes, axis=0)} == set(ch.UNEVEN_SHAPES)
    small = ch.uneven_shapes(200, seed=4)
    pool, h_off = ch.uneven_channels(small, seed=4)
    sizes = small[:, 0].astype(np.int64) * small[:, 1]
    assert h_off[0] == 0 and np.array_equal(h_off[1:], np.cumsum(sizes)[:-1])
    assert pool.size == sizes.sum()
    for i, (M, K) in enumerate(ch.UNEVEN_SHAPES):  # each bucket drawn together, in order
        idx = np.nonzero((small[:, 0] == M) & (small[:, 1] == K))[0]
        ref = ch.rician_ula(len(idx), K, M, seed=4 + i)
        for j, b in enumerate(idx):
            assert np.array_equal(pool[h_off[b]:h_off[b] + K * M].reshape(K, M), ref[j])
