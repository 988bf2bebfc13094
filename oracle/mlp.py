"""FP64 reference of the learned proposal's network -- TEST INFRASTRUCTURE ONLY.

No counterpart in the paper (its conclusion, Sec. V, names hybrids of model- and data-driven
detection as future work). The network is a per-antenna MLP: 6 features -> 256 -> ReLU -> 256
-> ReLU -> Qc logits over the antenna's constellation points, symbol s = kI * L + kQ with kI, kQ
the in-phase and quadrature level indices. Plain numpy, FP64, written from the definitions
(affine maps, ReLU, softmax cross-entropy, Adam); it shares nothing with the CUDA kernels.

Features of complex antenna i at state x (scaled units of the detector: level values
xt = 2k - (L - 1), Gt = dmin^2 H^T H, zt = dmin H^T y over the stacked real model, real dimensions
i (in-phase) and Nt + i (quadrature)):
    r(x)  = xt + (zt - Gt xt) / diag(Gt)         the current gradient as the point a coordinate
                                                  step reaches (equals zt / diag(Gt) at x = 0)
    wt    = (Gt + (sigma^2 / 2) I)^{-1} zt        the matched filter H^H y under Remark 1's
                                                  preconditioner, in level units
    F_i   = [r_i, r_{Nt+i}, wt_i, wt_{Nt+i}, log Gt_ii, log sigma^2]

The quantised form (quant=True) is the network the tensor-core inference kernel evaluates:
hidden activations and the weights of layers 2 and 3 rounded to BF16 (round to nearest even),
everything else exact.
"""
from __future__ import annotations

import numpy as np

import oracle

HIDDEN = 256
IN_DIM = 6


def shapes(qam: int):
    return [("W1", (HIDDEN, IN_DIM)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
            ("W3", (qam, HIDDEN)), ("b3", (qam,))]


def param_count(qam: int) -> int:
    return int(sum(np.prod(s) for _, s in shapes(qam)))


def unpack(params: np.ndarray, qam: int) -> dict:
    out, o = {}, 0
    for name, shp in shapes(qam):
        n = int(np.prod(shp))
        out[name] = params[o:o + n].reshape(shp)
        o += n
    return out


def init_params(qam: int, seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in shapes(qam):
        if name.startswith("W"):
            bound = np.sqrt(6.0 / shp[1])
            parts.append(rng.uniform(-bound, bound, size=shp).reshape(-1))
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    return np.concatenate(parts)


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64: the float32 value's
    low 16 bits are rounded away."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, X, qam, quant=False):
    P = unpack(np.asarray(params, np.float64), qam)
    X = np.asarray(X, np.float64)
    q = bf16 if quant else (lambda a: a)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = q(np.maximum(a1, 0.0))
    a2 = h1 @ q(P["W2"]).T + P["b2"]
    h2 = q(np.maximum(a2, 0.0))
    return h2 @ q(P["W3"]).T + P["b3"], (X, a1, h1, a2, h2)


def log_softmax(z):
    m = z.max(axis=-1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=-1, keepdims=True))


def loss_and_grad(params, X, labels, qam):
    """Mean over rows of the softmax cross-entropy of the logits against the symbol labels, and
    its gradient with respect to the flat parameter vector (backpropagation written out)."""
    P = unpack(np.asarray(params, np.float64), qam)
    logits, (X, a1, h1, a2, h2) = forward(params, X, qam)
    R = X.shape[0]
    labels = np.asarray(labels)
    lp = log_softmax(logits)
    loss = -lp[np.arange(R), labels].sum() / R
    dlog = np.exp(lp)
    dlog[np.arange(R), labels] -= 1.0
    dlog /= R
    g = {}
    g["W3"] = dlog.T @ h2
    g["b3"] = dlog.sum(axis=0)
    dh2 = dlog @ P["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ P["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return loss, np.concatenate([g[name].reshape(-1) for name, _ in shapes(qam)])


def adam(params, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, ICLR 2015), bias-corrected, step counted from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def features(H, y, sigma2, qam, k=None):
    """Per-antenna features [Nt, 6] of one channel at the state with level indices k (length 2 Nt,
    stacked); k = None is the all-zero point x = 0 used by the warm start."""
    Hr, yr = oracle.real_model(H, y)
    N = Hr.shape[1]
    nt = N // 2
    L = int(round(np.sqrt(qam)))
    d = oracle.dmin(qam)
    Gt = d * d * (Hr.T @ Hr)
    zt = d * (Hr.T @ yr)
    xt = np.zeros(N) if k is None else 2.0 * np.asarray(k, np.float64) - (L - 1)
    g = np.diag(Gt)
    r = xt + (zt - Gt @ xt) / g
    wt = np.linalg.solve(Gt + 0.5 * sigma2 * np.eye(N), zt)
    F = np.zeros((nt, IN_DIM))
    F[:, 0] = r[:nt]
    F[:, 1] = r[nt:]
    F[:, 2] = wt[:nt]
    F[:, 3] = wt[nt:]
    F[:, 4] = np.log(g[:nt])
    F[:, 5] = np.log(sigma2)
    return F


def symbols(k, nt, L):
    """Per-antenna symbol indices s = kI * L + kQ of a stacked level-index vector."""
    k = np.asarray(k)
    return k[..., :nt] * L + k[..., nt:]
