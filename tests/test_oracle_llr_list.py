"""Pins of the oracle's list-based LLR (Eq. (31)): with the whole state space as the list it is
the exact LLR of Eq. (4); repeated samples do not count twice (the sums run over sets); a single
sample gives +-clip by its bits; two samples that differ in one bit give f(x0) - f(x1) for that
bit; every value lies in [-clip, clip]."""
import itertools

import numpy as np
import pytest

import oracle
import workload


def _target(shape, seed):
    H, y, s2 = workload.generate([shape], seed).channel(0)
    return oracle.Target.from_channel(H, y, s2, shape[2], preconditioned=True, tau=2.0)


@pytest.mark.parametrize("shape", [(2, 2, 4, 6.0), (2, 3, 16, 12.0), (1, 2, 64, 15.0)])
def test_full_list_is_the_exact_llr(shape):
    t = _target(shape, 3)
    states = np.array(list(itertools.product(range(t.L), repeat=t.N)), np.int32)
    np.testing.assert_allclose(t.llr_list(states, 1e9), t.exact_llr(), rtol=1e-12, atol=1e-9)


def test_repeated_samples_count_once():
    t = _target((2, 2, 16, 10.0), 4)
    rng = np.random.default_rng(0)
    base = rng.integers(0, 4, (7, t.N)).astype(np.int32)
    rep = np.concatenate([base, base[[0, 3, 3, 6]]])
    np.testing.assert_array_equal(t.llr_list(rep, 30.0), t.llr_list(base, 30.0))


def test_single_sample_and_one_bit_apart():
    t = _target((2, 2, 16, 10.0), 5)
    k = np.array([[0, 3, 1, 2]], np.int32)
    B = 2
    g = k[0] ^ (k[0] >> 1)
    # bit order: per antenna, the I label bits (MSB first) then the Q label bits
    bits = []
    for a in range(2):
        for dim in (a, 2 + a):
            bits += [(g[dim] >> (B - 1 - p)) & 1 for p in range(B)]
    np.testing.assert_array_equal(t.llr_list(k, 12.5), np.where(np.array(bits) == 0, 12.5, -12.5))
    # flip the LSB of dimension 0's Gray label: level 0 (gray 00) -> level 1 (gray 01)
    k2 = np.array([[0, 3, 1, 2], [1, 3, 1, 2]], np.int32)
    out = t.llr_list(k2, 1e6)
    f0 = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(k2[0]))
    f1 = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(k2[1]))
    assert abs(out[1] - (f0 - f1)) <= 1e-9 * max(1.0, abs(f0 - f1))
    assert np.all(np.abs(np.delete(out, 1)) == 1e6)


def test_values_are_clipped():
    t = _target((2, 2, 4, 30.0), 6)
    states = np.array(list(itertools.product(range(2), repeat=4)), np.int32)
    out = t.llr_list(states, 3.0)
    assert np.all(np.abs(out) <= 3.0) and np.any(np.abs(out) == 3.0)
