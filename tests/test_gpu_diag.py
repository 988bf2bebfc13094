"""Convergence diagnostics on the GPU (Sec. III-B; include/mcmcdet_diag.h) against the oracle:
the exact transition matrix of Eq. (22) entry by entry, the tempered posterior, the spectrum and
the total-variation curve from the uniform start, on the 2x2 QPSK system of Figs. 2-3 at
4..10 dB for both proposals, and on other shapes up to the largest state spaces (256 states; 64
with the spectrum) and 32 receive antennas."""
import numpy as np
import pytest

import oracle
import oracle.diag as od
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _run(shapes, seed, precond, tv_steps=0, eig=False):
    from paper_2407_06042_gb300 import transition_diagnostics
    b = workload.generate(shapes, seed)
    Hd, yd, s2 = H.upload(b)
    nt, nr, qam = shapes[0][:3]
    out = transition_diagnostics(Hd, yd, s2, nt, nr, qam, preconditioned=precond,
                                 tv_steps=tv_steps, eigenvalues=eig)
    return b, {k: v.cpu().numpy() for k, v in out.items()}


def _oracle(b, ch, precond):
    Hc, y, s2 = b.channel(ch)
    s2 = float(np.float32(s2))           # the device reads sigma^2 in FP32
    t = oracle.Target.from_channel(Hc, y, s2, int(b.qam[ch]), preconditioned=precond, tau=2.0)
    P = t.transition_matrix()
    return P, od.stationary(t.all_f() / 2.0)


@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("snr", [4.0, 6.0, 8.0, 10.0])
def test_2x2_qpsk_matches_oracle(snr, precond):
    b, g = _run([(2, 2, 4, snr)] * 6, 1200 + int(snr), precond, tv_steps=40, eig=True)
    for ch in range(6):
        P, pi = _oracle(b, ch, precond)
        np.testing.assert_allclose(g["P"][ch], P, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g["pi"][ch], pi, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g["eig"][ch], od.spectrum(P, pi), rtol=0, atol=1e-10)
        np.testing.assert_allclose(g["tv"][ch], od.tv_curve(P, pi, 40), rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,eig", [((1, 1, 16, 12.0), True), ((1, 1, 64, 20.0), True),
                                       ((1, 2, 4, 3.0), True), ((3, 5, 4, 9.0), True),
                                       ((1, 32, 4, 0.0), True), ((2, 2, 16, 14.0), False),
                                       ((4, 4, 4, 8.0), False)])
@pytest.mark.parametrize("precond", [False, True])
def test_shapes_match_oracle(shape, eig, precond):
    n = 3
    b, g = _run([shape] * n, 1300 + shape[2] + shape[0], precond, tv_steps=10, eig=eig)
    S = g["P"].shape[1]
    for ch in range(n):
        P, pi = _oracle(b, ch, precond)
        assert P.shape == (S, S)
        np.testing.assert_allclose(g["P"][ch], P, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g["P"][ch].sum(1), 1.0, atol=1e-12)
        np.testing.assert_allclose(g["pi"][ch] @ g["P"][ch], g["pi"][ch], atol=1e-12)
        np.testing.assert_allclose(g["tv"][ch], od.tv_curve(P, pi, 10), rtol=0, atol=1e-12)
        if eig:
            np.testing.assert_allclose(g["eig"][ch], od.spectrum(P, pi), rtol=0, atol=1e-10)


def test_preconditioner_lowers_the_rate_on_gpu():
    """Fig. 3 at 10 dB over 100 channel realisations: the median rate of the plain sampler is near
    1 (high-SNR stalling), the preconditioned one's clearly lower."""
    rates = {}
    for precond in (False, True):
        _, g = _run([(2, 2, 4, 10.0)] * 100, 1400, precond, eig=True)
        assert np.all(np.abs(g["eig"][:, 0] - 1.0) < 1e-10)
        rates[precond] = g["eig"][:, 1]
    assert np.median(rates[False]) > 0.98
    assert np.median(rates[True]) < np.median(rates[False]) - 0.05
