"""Shared helpers of the GPU tests: batch upload, detector set-up, oracle targets, step parity."""
from __future__ import annotations

import numpy as np

import oracle
import workload


def torch_cuda():
    import torch
    return torch


def upload(batch: workload.Batch, device="cuda"):
    torch = torch_cuda()
    H = torch.from_numpy(np.ascontiguousarray(batch.H).view(np.float32).copy()).to(device)
    y = torch.from_numpy(np.ascontiguousarray(batch.y).view(np.float32).copy()).to(device)
    s2 = torch.from_numpy(np.ascontiguousarray(batch.sigma2, np.float32)).to(device)
    torch.cuda.synchronize()
    return H, y, s2


def make_detector(batch: workload.Batch, *, chains, precision="fp32", preconditioned=True,
                  seed=0, tau=2.0, alpha_scale=1.0, host_io=False, **kw):
    from paper_2407_06042_gb300 import Detector
    det = Detector(max_channels=batch.n_channels, max_nt=int(batch.nt.max()),
                   max_nr=int(batch.nr.max()), chains=chains, precision=precision,
                   preconditioned=preconditioned, seed=seed, **kw)
    if host_io:
        H = np.ascontiguousarray(batch.H).view(np.float32)
        y = np.ascontiguousarray(batch.y).view(np.float32)
        s2 = np.ascontiguousarray(batch.sigma2, np.float32)
    else:
        H, y, s2 = upload(batch)
    det.preprocess(batch.nt, batch.nr, batch.qam, H, batch.H_off, y, batch.y_off, s2,
                   alpha_scale=alpha_scale, tau=tau)
    det._inputs = (H, y, s2)
    return det


def split_states(det, batch, flat):
    """Flat chain-state export -> list of [chains, N] arrays per channel."""
    out, off = [], 0
    Np = det.cfg.chains
    for b in range(batch.n_channels):
        N = 2 * int(batch.nt[b])
        out.append(np.asarray(flat[off: off + Np * N], np.int32).reshape(Np, N))
        off += Np * N
    return out


def targets(batch, *, preconditioned=True, tau=2.0, alpha_scale=1.0, channels=None):
    idx = range(batch.n_channels) if channels is None else channels
    res = {}
    for b in idx:
        H, y, s2 = batch.channel(b)
        res[b] = oracle.Target.from_channel(H, y, s2, int(batch.qam[b]),
                                            preconditioned=preconditioned,
                                            alpha_scale=alpha_scale, tau=tau)
    return res


def step_parity(det, batch, tg, *, seed, steps, t0=0, channels=None, w_cat=1e-6, w_acc=1e-6):
    """Runs `steps` single-transition launches; after each, every chain of the checked
    channels is compared with the oracle's transition from the same pre-state. The oracle is
    re-synchronised to the GPU state after every step, so one near-tie never cascades.
    Returns counts of steps, exact matches, excused mismatches and unexcused ones."""
    chans = list(tg.keys()) if channels is None else channels
    flat, _ = det.get_chains()
    cur = split_states(det, batch, flat)
    res = dict(steps=0, mism=0, excused_cat=0, excused_acc=0, bad=0, bad_detail=[],
               min_gap=np.inf)
    for s in range(steps):
        t = t0 + s + 1
        det.run_chains(1, t - 1)
        flat, _ = det.get_chains()
        nxt = split_states(det, batch, flat)
        for b in chans:
            exp, info = tg[b].step_chains(seed, b, t, cur[b])
            diff = np.any(exp != nxt[b], axis=1)
            res["steps"] += exp.shape[0]
            gap = np.abs(info["log_a"] - info["log_u"])
            res["min_gap"] = min(res["min_gap"], float(gap.min()))
            for c in np.nonzero(diff)[0]:
                res["mism"] += 1
                if info["cat_margin"][c] < w_cat:
                    res["excused_cat"] += 1
                elif gap[c] < w_acc:
                    res["excused_acc"] += 1
                else:
                    res["bad"] += 1
                    if len(res["bad_detail"]) < 10:
                        res["bad_detail"].append(dict(t=t, b=b, c=int(c), gap=float(gap[c]),
                                                      margin=float(info["cat_margin"][c]),
                                                      gpu=nxt[b][c].tolist(), exp=exp[c].tolist()))
        cur = nxt
    return res


def levels_from_labels(labels, nt, L):
    """Complex Gray labels per antenna -> stacked real level indices [2 nt]."""
    B = int(np.log2(L))
    lab = np.asarray(labels, np.int64)
    gi, gq = lab >> B, lab & (L - 1)

    def inv_gray(g):
        k = g.copy()
        k ^= k >> 1
        k ^= k >> 2
        return k
    return np.concatenate([inv_gray(gi), inv_gray(gq)])
