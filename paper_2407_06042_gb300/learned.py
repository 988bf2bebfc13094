"""Training and use of the learned proposal (include/mcmcdet_learned.h).

The paper has no counterpart (Sec. V names model- plus data-driven hybrids as future work). The
network is trained on chain samples that the plain sampler itself generates: for every chain,
the features of its state at a few early transitions (and of the point x = 0) are paired with
the chain's symbol at a later transition, and the network is fitted by softmax cross-entropy
with Adam. Everything that computes runs in the library's kernels (chains, features, forward,
backward, Adam); this module only sequences the calls and moves index arrays.
"""
from __future__ import annotations

import numpy as np

from . import Detector, Mlp


def symbols(flat_states, nt, chains):
    """Per-(channel, chain, antenna) symbol indices kI * L + kQ of an exported state vector, in
    the row order of the detector's features."""
    out = []
    off = 0
    for n_t, L in nt:
        N = 2 * n_t
        s = np.asarray(flat_states[off:off + chains * N], np.int32).reshape(chains, 2, n_t)
        out.append((s[:, 0, :] * L + s[:, 1, :]).reshape(-1))
        off += chains * N
    return np.concatenate(out)


def best_symbols(best_idx, nt, chains):
    """Symbol indices kI * L + kQ of the detector's hard decision (complex Gray labels per
    antenna), repeated for every chain in the row order of the detector's features."""
    out = []
    off = 0
    for n_t, L in nt:
        B = int(np.log2(L))
        g = np.asarray(best_idx[off:off + n_t], np.int64) & 0xFF
        lev = []
        for part in (g >> B, g & (L - 1)):
            k = part.copy()
            k ^= k >> 1
            k ^= k >> 2
            lev.append(k)
        out.append(np.tile(lev[0] * L + lev[1], chains))
        off += n_t
    return np.concatenate(out)


def chain_samples(det: Detector, feature_times, label_time, *, label="chain"):
    """Training rows from the plain sampler on a freshly preprocessed detector: the features of
    every chain at each transition count in feature_times, and of x = 0 (one row per chain and
    antenna), all labelled after label_time transitions with the chain's own symbol
    (label="chain") or with the symbol of the channel's best visited sample (label="best").
    Returns (X [rows x 6] float32 device tensor, labels int32 device tensor)."""
    import torch
    meta = det.batch_meta
    chains = det.cfg.chains
    dims = [(int(n), int(l)) for n, l in zip(meta["nt"], meta["L"])]
    feats = []
    t = 0
    for tf in sorted(feature_times):
        if tf > t:
            det.run_chains(tf - t, t)
            t = tf
        feats.append(det.features())
    det.run_chains(label_time - t, t)
    if label == "best":
        lab = best_symbols(det.estimate()["best_idx"], dims, chains)
    else:
        flat, _ = det.get_chains()
        lab = symbols(flat, dims, chains)
    X0 = det.features(at_zero=True)
    # x = 0 rows, repeated for every chain of the channel (index map built on the host)
    rep, a0 = [], 0
    for n_t, _ in dims:
        rep.append(np.tile(np.arange(a0, a0 + n_t), chains))
        a0 += n_t
    rep = torch.as_tensor(np.concatenate(rep), device=X0.device)
    feats.append(X0.index_select(0, rep))
    X = torch.cat(feats, 0)
    labels = torch.as_tensor(np.tile(lab, len(feats)), dtype=torch.int32, device=X.device)
    return X, labels


def train(mlp: Mlp, X, labels, *, epochs=4, batch=4096, lr=1e-3, seed=0, log_every=0):
    """Adam over shuffled minibatches (permutations drawn on the host). Returns the mean
    training loss of each epoch (read back once per epoch)."""
    import torch
    rows = int(X.shape[0])
    batch = min(batch, mlp.max_rows, rows)
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    acc = torch.zeros(1, dtype=torch.float32, device=X.device)
    hist = []
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(rows).astype(np.int32), device=X.device)
        acc.zero_()
        nb = rows // batch
        for i in range(nb):
            mlp.train_step(X, labels, perm[i * batch:(i + 1) * batch], lr, loss)
            acc += loss
        hist.append(float(acc.item()) / max(nb, 1))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {hist[-1]:.4f}")
    return hist


def hard_bits(best_idx, nt, qam):
    """Bits of the hard decision: per antenna the complex Gray label's log2(Qc) bits, MSB first."""
    out = []
    off = 0
    for n_t, q in zip(nt, qam):
        B2 = int(np.log2(int(q)))
        g = np.asarray(best_idx[off:off + int(n_t)], np.int64) & 0xFF
        out.append(((g[:, None] >> np.arange(B2 - 1, -1, -1)) & 1).reshape(-1))
        off += int(n_t)
    return np.concatenate(out)


def ber_curve(det: Detector, tx_bits, checkpoints, *, learned=False, period=0):
    """Uncoded BER of sign(LLR) and of the hard decision after each checkpoint transition count,
    running from a fresh state: uniform random initial states, or the network's warm start
    (learned=True), with a mixture move at every transition t with t % period == 0 (period > 0).
    The detector must have been preprocessed (and, for learned runs, given a network)."""
    bits = np.asarray(tx_bits).astype(np.int64)
    out = []
    if learned:
        det.init_learned()
    t = 0
    for T in checkpoints:
        if period:
            det.run_mixed(T - t, period, t)
        else:
            det.run_chains(T - t, t)
        t = T
        r = det.estimate()
        hb = hard_bits(r["best_idx"], det.batch_meta["nt"], det.batch_meta["qam"])
        out.append(dict(T=T, ber_llr=float(((r["llr"] < 0).astype(np.int64) != bits).mean()),
                        ber_best=float((hb != bits).mean())))
    return out


def init_params(qam: int, seed: int) -> np.ndarray:
    """He-uniform initial weights (bound sqrt(6 / fan_in), numpy PCG64) and zero biases, in the
    flat layout of include/mcmcdet_learned.h."""
    rng = np.random.default_rng(seed)
    H, F = 256, 6
    parts = []
    for fan_out, fan_in in ((H, F), (H, H), (qam, H)):
        b = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-b, b, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)
