"""Pins of the oracle's learned-proposal pieces (an extension with no counterpart in the paper):
the network's backpropagation against central differences, BF16 rounding against torch's, Adam's
first step against its closed form, the features against noise-free closed forms, and the
mixture move and learned warm start against their exact transition laws on enumerable systems."""
import numpy as np
import pytest
import torch

import oracle
import oracle.mlp as mlp
import workload


def _net(qam, rows=7, seed=3):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(qam, seed) + 0.05 * rng.standard_normal(mlp.param_count(qam))
    X = rng.standard_normal((rows, mlp.IN_DIM))
    labels = rng.integers(0, qam, rows)
    return params, X, labels


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_backprop_matches_central_differences(qam):
    params, X, labels = _net(qam)
    loss, g = mlp.loss_and_grad(params, X, labels, qam)
    rng = np.random.default_rng(1)
    idx = rng.choice(params.size, 40, replace=False)
    # every parameter block is sampled: the first and last entries of each
    o = 0
    for _, shp in mlp.shapes(qam):
        n = int(np.prod(shp))
        idx = np.concatenate([idx, [o, o + n - 1]])
        o += n
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        fd = (mlp.loss_and_grad(params + e, X, labels, qam)[0] -
              mlp.loss_and_grad(params - e, X, labels, qam)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_is_cross_entropy_of_softmax():
    params, X, labels = _net(16, rows=5)
    logits, _ = mlp.forward(params, X, 16)
    p = np.exp(logits) / np.exp(logits).sum(1, keepdims=True)
    ref = -np.mean(np.log(p[np.arange(5), labels]))
    assert abs(mlp.loss_and_grad(params, X, labels, 16)[0] - ref) < 1e-12


def test_bf16_rounding():
    u = 2.0 ** -8
    np.testing.assert_array_equal(mlp.bf16([1.0, 1 + u, 1 + 3 * u, -(1 + 3 * u)]),
                                  [1.0, 1.0, 1 + 4 * u, -(1 + 4 * u)])
    rng = np.random.default_rng(0)
    x = rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.2, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01, eps=0.0)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-12)


def test_features_noise_free_closed_forms():
    """y = H x exactly: at x the coordinate-step point r(x) is x itself; with sigma^2 -> 0 the
    preconditioned matched filter is the zero-forcing solution x; on a diagonal channel r(0) is
    y_i / (dmin h_i)."""
    rng = np.random.default_rng(4)
    nt, qam = 3, 16
    H = (rng.standard_normal((5, nt)) + 1j * rng.standard_normal((5, nt))) / np.sqrt(10)
    k = rng.integers(0, 4, 2 * nt)
    d = oracle.dmin(qam)
    xt = 2.0 * k - 3
    x = d * (xt[:nt] + 1j * xt[nt:])
    F = mlp.features(H, H @ x, 1e-12, qam, k)
    np.testing.assert_allclose(F[:, 0] + 1j * F[:, 1], xt[:nt] + 1j * xt[nt:], atol=1e-9)
    np.testing.assert_allclose(F[:, 2] + 1j * F[:, 3], xt[:nt] + 1j * xt[nt:], atol=1e-6)
    np.testing.assert_allclose(F[:, 4], np.log(d * d * (np.abs(H) ** 2).sum(0)), rtol=1e-12)
    h = np.array([0.8 + 0.3j, -0.5 + 0.9j])
    y = np.array([0.2 - 0.1j, 0.4 + 0.7j])
    F0 = mlp.features(np.diag(h), y, 0.05, qam)
    np.testing.assert_allclose(F0[:, 0] + 1j * F0[:, 1], y / h / d, rtol=1e-12)
    np.testing.assert_allclose(F0[:, 5], np.log(0.05))


def _tiny(shape=(2, 2, 4, 6.0), seed=5):
    H, y, s2 = workload.generate([shape], seed).channel(0)
    t = oracle.Target.from_channel(H, y, s2, shape[2], preconditioned=True, tau=2.0)
    params = _net(shape[2], seed=7)[0]
    return t, params


def _exact_row(t, params, lam, x0):
    S = t.n_states()
    states = [t.state_levels(i) for i in range(S)]
    f = t.all_f() / t.s.tau
    nn = [t.nn_logp(params, s) for s in states]
    i0 = t.state_index(x0)
    row = np.zeros(S)
    for j in range(S):
        if j != i0:
            lf = t.mix_log_q(lam, states[i0], nn[i0], states[j])
            lr = t.mix_log_q(lam, states[j], nn[j], states[i0])
            row[j] = np.exp(lf + min(0.0, f[j] - f[i0] + lr - lf))
    row[i0] = 1.0 - row.sum()
    return row, states, nn, f


@pytest.mark.parametrize("shape", [(2, 2, 4, 6.0), (1, 1, 16, 10.0)])
def test_mixture_proposal_is_normalised(shape):
    t, params = _tiny(shape)
    S = t.n_states()
    states = [t.state_levels(i) for i in range(S)]
    for x in states[:4]:
        nn = t.nn_logp(params, x)
        tot = sum(np.exp(t.mix_log_q(0.4, x, nn, s)) for s in states)
        assert abs(tot - 1.0) < 1e-12


def test_mixture_with_zero_weight_is_algorithm1():
    t, params = _tiny((2, 3, 16, 9.0))
    for c in range(30):
        k0 = t.init_state(9, 0, c)
        a, ia = t.step(9, 0, c, 3, k0)
        b, ib = t.mix_step(9, 0, c, 3, k0, 0.0, params)
        np.testing.assert_array_equal(a, b)
        assert abs(ia.log_a - ib.log_a) < 1e-12


@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_mixture_move_frequencies_match_exact_kernel(lam):
    """Exact law of one mixture move from x: q_mix(x'|x) min{1, pi(x') q_mix(x|x') / (pi(x)
    q_mix(x'|x))} for x' != x, with pi the tempered posterior; the network is evaluated at x for
    the forward density and at x' for the reverse one."""
    t, params = _tiny()
    x0 = np.array([1, 0, 0, 1])
    row, states, nn, f = _exact_row(t, params, lam, x0)
    n = 20000
    counts = np.zeros(len(states))
    for c in range(n):
        k, _ = t.mix_step(11, 0, c, 1, x0, lam, params)
        counts[t.state_index(k)] += 1
    exp_ = row * n
    mask = exp_ > 5
    chi2 = ((counts[mask] - exp_[mask]) ** 2 / exp_[mask]).sum()
    assert chi2 < 45.0, chi2       # <= 15 dof, p ~ 1e-4
    assert counts[~mask].sum() <= 20


def test_mixture_kernel_keeps_the_posterior():
    """pi P = pi for the full mixture kernel built from the oracle's own densities."""
    t, params = _tiny()
    S = t.n_states()
    P = np.zeros((S, S))
    for i in range(S):
        P[i], _, _, f = _exact_row(t, params, 0.5, t.state_levels(i))
    pi = np.exp(f - f.max())
    pi /= pi.sum()
    np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-12)


def test_learned_warm_start_draws_from_the_table():
    t, params = _tiny((2, 2, 16, 10.0))
    lp = t.nn_logp(params)
    n = 16000
    counts = np.zeros((2, 16))
    for c in range(n):
        k = t.init_state_learned(3, 1, c, lp)
        counts[np.arange(2), mlp.symbols(k, 2, 4)] += 1
    p = np.exp(lp)
    for i in range(2):
        m = n * p[i] > 5
        chi2 = ((counts[i][m] - n * p[i][m]) ** 2 / (n * p[i][m])).sum()
        assert chi2 < 45.0, (i, chi2)
