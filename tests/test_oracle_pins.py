"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against the mathematics the paper fixes: an independent
library (cuRAND's host Philox, numpy complex arithmetic), a closed form, an identity the paper
proves (detailed balance, Appendix A), the joint proposal of Eq. (12) / Eq. (20) that the
factorised proposal of Eqs. (14)-(17), (21) must reproduce, brute-force enumeration, or the
exact answer a Monte Carlo estimator must converge to (Eq. (4)). A plausible slip anywhere in
the oracle (a dropped factor 1/2, a sign, a swapped forward/reverse proposal, a transposed
embedding) fails at least one of them.
"""
import ctypes
import ctypes.util
import itertools

import numpy as np
import pytest

import oracle
import workload


def _rng(seed=0):
    return np.random.default_rng(seed)


def _channel(nr, nt, seed, snr_db=8.0, qam=4):
    b = workload.generate([(nt, nr, qam, snr_db)], seed)
    return b.channel(0)


# ------------------------------------------------------------------------------------------
# Philox4x32-10
# ------------------------------------------------------------------------------------------
def _curand():
    for name in ("libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host PHILOX4_32_10 generator emits block i of its stream from the counter
    (0, 0, i, 0) under the key (seed lo, seed hi): an independent implementation of the same
    SC'11 generator, called as a library."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(g), 161) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 64
        out = np.zeros(n, np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        cr.curandDestroyGenerator(g)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    mine = np.concatenate([oracle.philox((0, 0, i, 0), key) for i in range(n // 4)])
    np.testing.assert_array_equal(mine, out)


def test_philox_counter_words_all_matter_and_uniform():
    key = (7, 9)
    base = oracle.philox((5, 6, 7, 8), key)
    for j in range(4):
        c = [5, 6, 7, 8]
        c[j] += 1
        assert not np.array_equal(oracle.philox(c, key), base)
    words = np.concatenate([oracle.philox((t, 3, 1, 0), key) for t in range(4000)])
    u = np.array([oracle.uniform(w) for w in words[:4000]])
    assert np.all((u > 0) & (u < 1))
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = ((hist - 200.0) ** 2 / 200.0).sum()
    assert chi2 < 45.0          # 19 dof, p ~ 1e-3


def test_uniform_is_exact_in_fp32():
    for w in [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF, 123456789]:
        u = oracle.uniform(w)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_initial_states_are_uniform_and_independent(qam):
    """Sec. IV-A starts every chain from a random state: the t = 0 levels of oracle_init_state
    are uniform over the L PAM levels (chi-square over 2048 chains x N dimensions), the levels of
    neighbouring dimensions and of neighbouring chains are independent (chi-square of the L^2
    pairs), and other chains, channels and seeds draw other states."""
    from scipy.stats import chi2
    H, y, s2 = _channel(3, 3, 5, qam=qam)
    t = oracle.Target.from_channel(H, y, s2, qam)
    L, N, C = int(round(np.sqrt(qam))), t.N, 2048
    K = np.stack([t.init_state(3, 0, c) for c in range(C)])
    assert K.min() >= 0 and K.max() <= L - 1

    def stat(x, bins):
        cnt = np.bincount(x.ravel(), minlength=bins)
        e = x.size / bins
        return float(((cnt - e) ** 2 / e).sum())
    assert stat(K, L) < chi2.ppf(0.999, L - 1)
    assert stat(K[:, :-1] * L + K[:, 1:], L * L) < chi2.ppf(0.999, L * L - 1)      # dimensions
    assert stat(K[:-1, :] * L + K[1:, :], L * L) < chi2.ppf(0.999, L * L - 1)      # chains
    assert not np.array_equal(t.init_state(3, 1, 0), K[0])
    assert not np.array_equal(t.init_state(4, 0, 0), K[0])
    S = float(L) ** N                                # distinct states among 64 draws
    assert len({tuple(r) for r in K[:64]}) >= 0.8 * S * (1.0 - (1.0 - 1.0 / S) ** 64)


# ------------------------------------------------------------------------------------------
# System model, metric, gradient, preconditioner
# ------------------------------------------------------------------------------------------
def test_real_model_matches_complex_arithmetic():
    H, y, s2 = _channel(5, 3, 11)
    Hr, yr = oracle.real_model(H, y)
    x = _rng(1).standard_normal(3) + 1j * _rng(2).standard_normal(3)
    xr = np.concatenate([x.real, x.imag])
    hx = H @ x
    np.testing.assert_allclose(Hr @ xr, np.concatenate([hx.real, hx.imag]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(yr, np.concatenate([y.real, y.imag]))
    G = H.conj().T @ H
    blk = np.block([[G.real, -G.imag], [G.imag, G.real]])
    np.testing.assert_allclose(Hr.T @ Hr, blk, atol=1e-12)
    z = H.conj().T @ y
    np.testing.assert_allclose(Hr.T @ yr, np.concatenate([z.real, z.imag]), atol=1e-12)


def test_f_is_complex_residual_norm():
    H, y, s2 = _channel(4, 4, 12)
    Hr, yr = oracle.real_model(H, y)
    rng = _rng(3)
    for _ in range(5):
        xc = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        ref = -np.sum(np.abs(y - H @ xc) ** 2) / s2
        got = oracle.f_value(Hr, yr, s2, np.concatenate([xc.real, xc.imag]))
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


def test_gradient_matches_central_differences():
    """f is quadratic, so central differences equal the gradient up to rounding."""
    H, y, s2 = _channel(6, 4, 13, snr_db=15.0)
    Hr, yr = oracle.real_model(H, y)
    x = _rng(4).standard_normal(8) * 0.5
    g = oracle.grad_f(Hr, yr, s2, x)
    h = 1e-3
    fd = np.zeros(8)
    for n in range(8):
        e = np.zeros(8)
        e[n] = h
        fd[n] = (oracle.f_value(Hr, yr, s2, x + e) - oracle.f_value(Hr, yr, s2, x - e)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-6 * np.abs(g).max())


def test_preconditioner_is_damped_inverse():
    H, y, s2 = _channel(8, 8, 14)
    Hr, _ = oracle.real_model(H, y)
    gamma = 0.037
    P = oracle.preconditioner(Hr, gamma)
    A = Hr.T @ Hr + gamma * np.eye(16)
    np.testing.assert_allclose(P @ A, np.eye(16), atol=1e-10)


def test_dmin_is_half_min_distance_of_unit_energy_qam():
    for qc in (4, 16, 64):
        L = int(np.sqrt(qc))
        lv = np.arange(L)
        pts = np.array([complex(2 * a - L + 1, 2 * b - L + 1) for a in lv for b in lv])
        pts = pts / np.sqrt(np.mean(np.abs(pts) ** 2))
        dist = np.abs(pts[:, None] - pts[None, :])
        dmin = dist[dist > 1e-12].min() / 2
        assert abs(oracle.dmin(qc) - dmin) < 1e-14


# ------------------------------------------------------------------------------------------
# Proposal: the factorised softmax must equal the paper's joint definition
# ------------------------------------------------------------------------------------------
def _joint_log_q(t: "oracle.Target", k, kp, precond):
    """log q(x'|x) from the JOINT definition: a Gaussian kernel centred at x + (alpha/2) d with
    variance alpha (Eq. (12)) or alpha*beta with d = M grad (Remark 1, Eq. (20)), normalised
    by brute force over every x' in A^N (Eq. (13))."""
    x = t.values(k)
    g = np.asarray(oracle.grad_f(t.Hr, t.yr, t.sigma2, x)) / t.s.tau
    d = t.P @ g if precond else g
    var = t.s.alpha * (t.s.beta if precond else 1.0)
    centre = x + 0.5 * t.s.alpha * d
    allk = np.array(list(itertools.product(range(t.L), repeat=t.N)))
    allx = (2 * allk - t.L + 1) * t.dmin
    e = -np.sum((allx - centre) ** 2, axis=1) / (2 * var)
    lz = np.logaddexp.reduce(e)
    xp = t.values(kp)
    return -np.sum((xp - centre) ** 2) / (2 * var) - lz


@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("tau", [1.0, 2.0])
def test_factorised_proposal_equals_joint_definition(precond, tau):
    H, y, s2 = _channel(2, 2, 21, snr_db=10.0, qam=16)      # N = 4, L = 4: 256 states
    t = oracle.Target.from_channel(H, y, s2, 16, preconditioned=precond, tau=tau)
    rng = _rng(5)
    for _ in range(6):
        k = rng.integers(0, 4, 4)
        kp = rng.integers(0, 4, 4)
        assert abs(t.log_q(k, kp) - _joint_log_q(t, k, kp, precond)) < 1e-10
    # normalisation over every x'
    k = rng.integers(0, 4, 4)
    tot = np.logaddexp.reduce([t.log_q(k, kp) for kp in itertools.product(range(4), repeat=4)])
    assert abs(tot) < 1e-12


def test_per_antenna_complex_categorical_is_product_of_pam_factors():
    """The per-antenna categorical over the Qc lattice points (2-D Gaussian kernel) equals the
    product of the in-phase and quadrature PAM factors of the stacked real model."""
    H, y, s2 = _channel(3, 1, 22, snr_db=12.0, qam=16)      # one complex antenna: N = 2
    t = oracle.Target.from_channel(H, y, s2, 16, preconditioned=True, tau=2.0)
    k = np.array([1, 2])
    x = t.values(k)
    g = np.asarray(oracle.grad_f(t.Hr, t.yr, t.sigma2, x)) / 2.0
    d = t.P @ g
    centre = complex(*(x + 0.5 * t.s.alpha * d))
    pts = [(a, b) for a in range(4) for b in range(4)]
    e = np.array([-abs(complex(*t.values([a, b])) - centre) ** 2 / (2 * t.s.alpha * t.s.beta)
                  for a, b in pts])
    logp = e - np.logaddexp.reduce(e)
    for (a, b), lp in zip(pts, logp):
        assert abs(t.log_q(k, [a, b]) - lp) < 1e-12


# ------------------------------------------------------------------------------------------
# MH kernel: detailed balance, stationarity, positivity (Appendix A), transition frequencies
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("tau", [1.0, 2.0])
def test_transition_matrix_detailed_balance_2x2_qpsk(precond, tau):
    H, y, s2 = _channel(2, 2, 31, snr_db=8.0, qam=4)        # 16 states (Fig. 2/3 setup)
    t = oracle.Target.from_channel(H, y, s2, 4, preconditioned=precond, tau=tau)
    P = t.transition_matrix()
    f = t.all_f() / tau
    pi = np.exp(f - f.max())
    pi /= pi.sum()
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-13)
    assert np.all(P > 0)                                     # irreducible and aperiodic
    flow = pi[:, None] * P
    np.testing.assert_allclose(flow, flow.T, atol=1e-15, rtol=1e-10)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-14)
    ev = np.sort(np.abs(np.linalg.eigvals(P)))[::-1]
    assert abs(ev[0] - 1) < 1e-12 and ev[1] < 1


def test_two_state_chain_closed_form():
    """A single real BPSK unknown (N = 1): the 2-state chain's second eigenvalue is
    1 - P(+|-) - P(-|+) and its stationary law is exp(f) normalised."""
    Hr = np.array([[0.9], [0.4]])
    yr = np.array([0.5, -0.1])
    s2 = 0.3
    t = oracle.Target(Hr, yr, s2, 2, 1.0, alpha=s2)
    P = t.transition_matrix()
    ev = np.sort(np.linalg.eigvals(P).real)
    assert abs(ev[0] - (1 - P[0, 1] - P[1, 0])) < 1e-14
    f = t.all_f()
    pi = np.exp(f - f.max())
    pi /= pi.sum()
    stat = np.array([P[1, 0], P[0, 1]]) / (P[0, 1] + P[1, 0])
    np.testing.assert_allclose(stat, pi, atol=1e-14)


def test_step_frequencies_match_transition_row():
    """oracle.step from one fixed state, over many independent streams, lands on x' with the
    frequencies of row x of the transition matrix (Eq. (22))."""
    H, y, s2 = _channel(2, 2, 41, snr_db=6.0, qam=4)
    t = oracle.Target.from_channel(H, y, s2, 4, preconditioned=True, tau=1.0)
    P = t.transition_matrix()
    k0 = np.array([0, 1, 1, 0])
    i0 = t.state_index(k0)
    S = 20000
    counts = np.zeros(16)
    for c in range(S):
        kk, _ = t.step(99, 3, c, 1, k0)
        counts[t.state_index(kk)] += 1
    exp_ = P[i0] * S
    mask = exp_ > 5
    chi2 = ((counts[mask] - exp_[mask]) ** 2 / exp_[mask]).sum()
    assert chi2 < 40.0, (chi2, mask.sum())


def test_chains_converge_to_exact_posterior_in_tv():
    """Fig. 2/3 setup: 2x2 QPSK at 8 dB. After 40 transitions the empirical law of the final
    states of S chains is as close to pi (TV) as S iid draws from pi would be."""
    H, y, s2 = _channel(2, 2, 51, snr_db=8.0, qam=4)
    t = oracle.Target.from_channel(H, y, s2, 4, preconditioned=True, tau=1.0)
    f = t.all_f()
    pi = np.exp(f - f.max())
    pi /= pi.sum()
    S = 6000
    counts = np.zeros(16)
    for c in range(S):
        k = t.init_state(5, 0, c)
        k, _ = t.run_chain(5, 0, c, 0, 40, k)
        counts[t.state_index(k)] += 1
    tv = 0.5 * np.abs(counts / S - pi).sum()
    rng = _rng(6)
    iid = [0.5 * np.abs(np.bincount(rng.choice(16, S, p=pi), minlength=16) / S - pi).sum()
           for _ in range(300)]
    assert tv <= np.quantile(iid, 0.99), (tv, np.quantile(iid, 0.99))
    # exact law after 40 steps from the uniform start, via the transition matrix
    P = t.transition_matrix()
    lam2 = np.sort(np.abs(np.linalg.eigvals(P)))[-2]
    assert 0 < lam2 < 1


def test_resume_is_exact():
    H, y, s2 = _channel(4, 4, 61, snr_db=14.0, qam=16)
    t = oracle.Target.from_channel(H, y, s2, 16, preconditioned=True, tau=2.0)
    k0 = t.init_state(0, 2, 7)
    a, _ = t.run_chain(0, 2, 7, 0, 60, k0)
    b, _ = t.run_chain(0, 2, 7, 0, 25, k0)
    b, _ = t.run_chain(0, 2, 7, 25, 35, b)
    np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------------------------------------
# LLRs
# ------------------------------------------------------------------------------------------
def _diag_channel(nt, seed, snr_db, qam):
    rng = _rng(seed)
    h = (rng.standard_normal(nt) + 1j * rng.standard_normal(nt)) * np.sqrt(0.5)
    H = np.diag(h).astype(np.complex64).astype(np.complex128)
    L = int(np.sqrt(qam))
    d = oracle.dmin(qam)
    lev = rng.integers(0, L, (2, nt))
    x = ((2 * lev[0] - L + 1) + 1j * (2 * lev[1] - L + 1)) * d
    s2 = 1.0 / 10 ** (snr_db / 10)
    y = H @ x + (rng.standard_normal(nt) + 1j * rng.standard_normal(nt)) * np.sqrt(s2 / 2)
    return H, y.astype(np.complex64).astype(np.complex128), s2


def _one_dim_llr(H, y, s2, qam):
    """Exact LLRs of a diagonal channel: each real dimension is its own 1-D problem."""
    nt = H.shape[0]
    L = int(np.sqrt(qam))
    B = int(np.log2(L))
    d = oracle.dmin(qam)
    a = (2 * np.arange(L) - L + 1) * d
    g = np.arange(L) ^ (np.arange(L) >> 1)
    out = []
    for i in range(nt):
        h = H[i, i]
        for part in (0, 1):
            # real model row pair of antenna i: y_re = Re h x_re - Im h x_im, y_im = Im h x_re + Re h x_im
            # dimension `part` of x enters |y - h x|^2 through |h|^2 (x_part - xhat_part)^2
            xhat = y[i] / h
            comp = xhat.real if part == 0 else xhat.imag
            f = -np.abs(h) ** 2 * (comp - a) ** 2 / s2
            for bpos in range(B):
                bit = (g >> (B - 1 - bpos)) & 1
                out.append(np.logaddexp.reduce(f[bit == 0]) - np.logaddexp.reduce(f[bit == 1]))
    return np.array(out)


@pytest.mark.parametrize("qam", [4, 16])
def test_exact_llr_of_diagonal_channel_is_one_dimensional(qam):
    H, y, s2 = _diag_channel(2, 71, 9.0, qam)
    t = oracle.Target.from_channel(H, y, s2, qam, preconditioned=False, tau=1.0)
    np.testing.assert_allclose(t.exact_llr(), _one_dim_llr(H, y, s2, qam), rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("tau", [1.0, 2.0, 3.5])
def test_is_llr_exact_for_diagonal_qpsk_with_any_samples(tau):
    """With G diagonal and one bit per dimension, every IS term of Eq. (34) carries the same
    ratio, so the estimate equals the exact LLR whatever the sample list."""
    H, y, s2 = _diag_channel(3, 72, 7.0, 4)
    t = oracle.Target.from_channel(H, y, s2, 4, preconditioned=False, tau=tau)
    samples = _rng(8).integers(0, 2, (17, 6))
    np.testing.assert_allclose(t.llr_is(samples), t.exact_llr(), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("tau", [1.0, 2.0])
def test_is_llr_converges_to_exact_with_iid_tempered_samples(tau):
    """IS-LLR (Eq. (34)) with S iid draws from the tempered target (Eq. (33)), drawn by direct
    enumeration (no MCMC), approaches the exact LLR (Eq. (4)); the error shrinks with S."""
    H, y, s2 = _channel(2, 2, 81, snr_db=9.0, qam=16)
    t = oracle.Target.from_channel(H, y, s2, 16, preconditioned=True, tau=tau)
    f = t.all_f()
    pa = np.exp((f - f.max()) / tau)
    pa /= pa.sum()
    exact = t.exact_llr()
    rng = _rng(9)
    errs = []
    for S in (200, 20000):
        idx = rng.choice(pa.size, S, p=pa)
        samples = np.array([t.state_levels(i) for i in idx])
        errs.append(np.mean(np.abs(t.llr_is(samples) - exact)))
    assert errs[1] < 0.05, errs
    assert errs[1] < errs[0], errs


def test_best_sample_finds_map_on_4x4_16qam():
    """Hard decision (Sec. III-A): the best visited sample equals the exhaustive MAP on most
    channels at the 4x4 16-QAM, 12 dB setting."""
    b = workload.rayleigh_batch(4, 4, 16, [12.0], 6, 1001)
    hits = 0
    for i in range(6):
        H, y, s2 = b.channel(i)
        r = oracle.detect(H, y, s2, 16, chains=32, iterations=100, channel=i)
        t = oracle.Target.from_channel(H, y, s2, 16)
        f = t.all_f()
        assert r["best_f"] <= f.max() + 1e-9
        hits += abs(r["best_f"] - f.max()) < 1e-9
    assert hits >= 5
