"""Input generators: determinism, ranges, moments, shapes (not the method)."""
import numpy as np

from synthetic import (SplitMix64, chemistry_integrals, heisenberg_mpo,
                       random_tt_cores, tt_bond_dims, chemistry_mpo)


def test_splitmix_stream_continuation():
    a = SplitMix64(42).uniform_pm1(10)
    g = SplitMix64(42)
    b = np.concatenate([g.uniform_pm1(3), g.uniform_pm1(7)])
    assert np.array_equal(a, b)


def test_splitmix_reference_value():
    # SplitMix64 with state 0: first output of the published generator.
    assert int(SplitMix64(0).next_u64(1)[0]) == 0xE220A8397B1DCDAF


def test_uniform_and_normal_moments():
    u = SplitMix64(7).uniform_pm1(200000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
    z = SplitMix64(7).standard_normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_integral_symmetry():
    h, eri = chemistry_integrals(5, 3)
    assert np.allclose(h, h.T)
    for p in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.array_equal(eri, eri.transpose(p))


def test_tt_dims_clip_to_exact_ranks():
    assert tt_bond_dims([2] * 6, 4) == [1, 2, 4, 4, 4, 2, 1]
    cores = random_tt_cores([4] * 3, 8, 1)
    assert [c.shape for c in cores] == [(1, 4, 4), (4, 4, 4), (4, 4, 1)]


def test_mpo_shapes():
    m = heisenberg_mpo(6)
    assert m[0].shape == (1, 2, 2, 5) and m[-1].shape == (5, 2, 2, 1)
    h, eri = chemistry_integrals(4, 1)
    m = chemistry_mpo(h, eri)
    assert m[0].shape[0] == 1 and m[-1].shape[3] == 1
    assert all(a.shape[3] == b.shape[0] for a, b in zip(m[:-1], m[1:]))
