"""Pins of the oracle's convergence diagnostics (Sec. III-B): the two-state chain's closed forms,
the spectrum against a general eigen-solver applied to the unsymmetrised matrix, the TV curve
against explicit matrix powers, and, on the enumerable 2x2 QPSK system of Figs. 2-3, the unit
eigenvalue, a rate in (-1, 1) and the paper's finding that the preconditioner lowers the rate at
high SNR."""
import numpy as np
import pytest

import oracle
import oracle.diag as od
import workload


def _two_state(a, b):
    return np.array([[1 - a, a], [b, 1 - b]]), np.array([b, a]) / (a + b)


@pytest.mark.parametrize("a,b", [(0.3, 0.1), (0.9, 0.7), (0.05, 0.6)])
def test_two_state_closed_forms(a, b):
    P, pi = _two_state(a, b)
    np.testing.assert_allclose(od.spectrum(P, pi), [1.0, 1.0 - a - b], atol=1e-14)
    tv = od.tv_curve(P, pi, 12)
    lam = 1.0 - a - b
    np.testing.assert_allclose(tv, abs(0.5 - pi[0]) * np.abs(lam) ** np.arange(13), atol=1e-15)


def _metropolis(S, seed):
    """A reversible chain: Metropolis moves on a random target with a symmetric proposal."""
    rng = np.random.default_rng(seed)
    pi = rng.random(S) + 0.05
    pi /= pi.sum()
    Q = rng.random((S, S))
    Q = Q + Q.T
    np.fill_diagonal(Q, 0.0)
    Q /= Q.sum(1).max() * 1.5
    P = Q * np.minimum(1.0, pi[None, :] / pi[:, None])
    P[np.diag_indices(S)] = 1.0 - P.sum(1)
    return P, pi


@pytest.mark.parametrize("S", [3, 16, 64])
def test_spectrum_matches_a_general_solver(S):
    P, pi = _metropolis(S, S)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-14)
    ref = np.sort(np.linalg.eigvals(P).real)[::-1]
    got = od.spectrum(P, pi)
    np.testing.assert_allclose(got, ref, atol=1e-10)
    assert abs(got[0] - 1.0) < 1e-12 and got[-1] >= -1.0 - 1e-12


def test_tv_curve_is_matrix_powers_and_nonincreasing():
    P, pi = _metropolis(16, 5)
    tv = od.tv_curve(P, pi, 30)
    u = np.full(16, 1.0 / 16)
    for t in (0, 1, 7, 30):
        np.testing.assert_allclose(tv[t], 0.5 * np.abs(u @ np.linalg.matrix_power(P, t) - pi).sum(),
                                   atol=1e-14)
    assert np.all(np.diff(tv) <= 1e-15)


def _rates(snr_db, precond, n=24, seed=1100):
    b = workload.generate([(2, 2, 4, float(snr_db))] * n, seed + int(snr_db))
    out = []
    for ch in range(n):
        H, y, s2 = b.channel(ch)
        t = oracle.Target.from_channel(H, y, s2, 4, preconditioned=precond, tau=2.0)
        P = t.transition_matrix()
        ev = od.spectrum(P, od.stationary(t.all_f() / 2.0))
        assert abs(ev[0] - 1.0) < 1e-10 and -1.0 < ev[1] < 1.0, ev[:3]
        out.append(ev[1])
    return np.array(out)


def test_preconditioner_lowers_the_rate_at_high_snr():
    """Fig. 3: the plain sampler's rate approaches 1 above 8 dB; the preconditioned one stays
    lower. Checked on the medians of 24 channels at 10 dB."""
    assert np.median(_rates(10, True)) < np.median(_rates(10, False))
