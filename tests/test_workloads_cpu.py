"""The seeded input recipe of the workloads (CPU): shapes, ranges, seeds and the structure of
each configuration, so that a change to a generator cannot silently change what the parity tests
and the benchmark run on."""
import numpy as np
import pytest

import workloads as W


def test_shifted_grid_and_time_reversal():
    k = W.SHIFTED_222
    assert k.shape == (8, 3) and np.all(np.abs(k) == 0.25)
    assert len({tuple(r) for r in k}) == 8                  # the whole shifted 2x2x2 grid
    irr = k[:4]
    for r in k[4:]:                                         # the rest are negatives of the first four
        assert any(np.array_equal(r, -q) for q in irr)
    for i in range(4):                                      # and no two of the first four are a pair
        for j in range(4):
            assert not np.array_equal(irr[i], -irr[j])


def test_config1_and_config3_share_the_cell():
    c1, c3 = W.config1(), W.config3()
    assert c1.natom == 4 and c1.nproj == 16 and c1.nband == 16
    assert c1.fft_box == (24, 24, 24) and np.array_equal(c1.kpts, np.zeros((1, 3)))
    assert np.allclose(c1.lattice, 10.0 * np.eye(3)) and c1.ecut == 10.0
    assert np.all(np.abs(c1.D) <= 1.0) and c1.D.shape == (16,)
    assert np.all((c1.pos >= 0) & (c1.pos < 10.0))
    assert np.array_equal(c1.pos, c3.pos) and np.array_equal(c1.D, c3.D) and c3.nband == 1024
    assert (c1.vloc_amp, c1.vloc_sigma, c1.proj_alpha) == (-2.0, 1.0, 0.25)


def test_config2_recipe():
    s = W.config2()
    assert s.natom == 64 and s.nproj == 256 and s.nband == 512 and s.fft_box == (96, 96, 96)
    assert np.array_equal(s.kpts, W.SHIFTED_222[:4])
    d = np.linalg.norm(s.pos[:, None, :] - s.pos[None, :, :], axis=-1)
    assert d[np.triu_indices(64, 1)].min() >= 2.0           # rejection on the raw draws
    assert np.all((s.pos >= 0) & (s.pos < 20.0))


def test_config4_ranges_and_determinism():
    a, b = W.config4(), W.config4()
    assert len(a) == 48
    for s, t in zip(a, b):
        assert np.array_equal(s.pos, t.pos) and np.array_equal(s.D, t.D) and s.ecut == t.ecut
        edge = s.lattice[0, 0]
        assert 8.0 <= edge <= 16.0 and 12.0 <= s.ecut <= 20.0
        assert 8 <= s.natom <= 64 and s.nband == 2 * s.natom
        assert 1 <= len(s.kpts) <= 8 and np.array_equal(s.kpts, W.SHIFTED_222[:len(s.kpts)])
        assert s.fft_box is None                             # default box rule
    nks = [len(s.kpts) for s in a]
    assert sum(nks) == 217                                   # the units the batched tests expect
    assert min(nks) == 1 and max(nks) == 8


def test_config5_arrivals_and_mix():
    reqs = W.config5()
    assert len(reqs) == 200
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential gaps of mean 1/200 s: the sample mean of 200 lies within 30 % with
    # overwhelming probability (and this draw is fixed by the seed)
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.3
    rep = [r for r in reqs if r.repeat_of is not None]
    assert 0.15 < len(rep) / 200 < 0.35
    for i, r in enumerate(reqs):
        if r.repeat_of is not None:
            assert r.repeat_of < i and r.system is reqs[r.repeat_of].system
    fresh = [r.system for r in reqs if r.repeat_of is None]
    small = [s for s in fresh if s.fft_box == (24, 24, 24)]
    assert 0.02 < len(small) / len(fresh) < 0.25              # ~10 % config-1-size systems
    for s in small:
        assert s.natom == 4 and s.nband == 16 and s.ecut == 10.0


def test_overlap_variant_keeps_the_rest():
    s = W.config1()
    q = W.with_overlap(s)
    assert q.Q.shape == (s.nproj,) and np.all((q.Q >= 0) & (q.Q <= 0.5))
    assert np.array_equal(q.pos, s.pos) and np.array_equal(q.D, s.D) and s.Q is None
    assert np.array_equal(W.config1s().Q, q.Q)


def test_random_block_is_seeded():
    a = W.random_block(37, 5, seed=3)
    b = W.random_block(37, 5, seed=3)
    c = W.random_block(37, 5, seed=4)
    assert a.shape == (5, 37) and a.dtype == np.complex128
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert W.random_block(37, 5, seed=3, dtype=np.complex64).dtype == np.complex64
