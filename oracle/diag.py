"""Convergence diagnostics of the chain from its exact transition matrix -- TEST INFRASTRUCTURE
ONLY (same rule as the rest of ``oracle``: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it).

Sec. III-B: the chain's transition matrix P (Eq. (22), ``Target.transition_matrix``) leaves the
tempered posterior pi ~ exp(f / tau) invariant; its convergence rate r is the second largest
eigenvalue of P, and the distance of the chain's law from pi after t transitions is measured in
total variation (Theorem 1). Plain numpy, FP64; a library eigen-solver is one step.
Pinned in ``tests/test_oracle_diag.py`` (two-state closed forms, a general eigen-solver on the
unsymmetrised matrix, explicit matrix powers, monotonicity)."""
from __future__ import annotations

import numpy as np


def stationary(f_tempered) -> np.ndarray:
    """pi(x) = exp(f_tau(x)) / sum exp(f_tau) over the enumerated states."""
    f = np.asarray(f_tempered, np.float64)
    w = np.exp(f - f.max())
    return w / w.sum()


def spectrum(P, pi) -> np.ndarray:
    """Eigenvalues of a chain reversible w.r.t. pi, descending: those of the symmetric
    D^(1/2) P D^(-1/2), D = diag(pi)."""
    P = np.asarray(P, np.float64)
    s = np.sqrt(np.asarray(pi, np.float64))
    B = (s[:, None] * P) / s[None, :]
    B = 0.5 * (B + B.T)
    return np.sort(np.linalg.eigvalsh(B))[::-1]


def tv_curve(P, pi, steps: int) -> np.ndarray:
    """TV(t) = (1/2) sum_x |p_t(x) - pi(x)|, t = 0..steps, p_0 uniform, p_{t+1} = p_t P."""
    P = np.asarray(P, np.float64)
    pi = np.asarray(pi, np.float64)
    p = np.full(P.shape[0], 1.0 / P.shape[0])
    out = np.empty(steps + 1)
    for t in range(steps + 1):
        out[t] = 0.5 * np.abs(p - pi).sum()
        p = p @ P
    return out
