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


def states_now(det, batch):
    """Current chain states per channel (states only: nothing in the handle changes)."""
    _, _, n_states = det.sizes()
    flat = np.zeros(n_states, np.int8)
    det.get_chains(states=flat)
    return split_states(det, batch, flat)


def fp64_energy(tg, state):
    """f = -||y - Hx||^2 / sigma^2 of one state (level indices), from the oracle's residual."""
    return oracle.f_value(tg.Hr, tg.yr, tg.sigma2, tg.values(state))


def step_parity(det, batch, tg, *, seed, steps, t0=0, channels=None, w_cat=1e-6, w_acc=1e-6,
                energies=False, label=None):
    """Runs `steps` single-transition launches; after each, every chain of the checked
    channels is compared with the oracle's transition from the same pre-state. The oracle is
    re-synchronised to the GPU state after every step, so one near-tie never cascades.

    Returns counts of steps, exact matches, excused mismatches and unexcused ones, and the
    excused mismatches in bands of the oracle's own margin (< 1e-6, < 1e-4, < window) for
    accept decisions (|log A - log u|) and categorical draws (CDF margin). With a handle created
    with MCMC_ENGINE_TRACE it also returns the largest difference between the kernel's log A and
    the oracle's (Eq. (18)) over the transitions whose proposal is unambiguous (CDF margin above
    1e-3 in every dimension) and whose decision some uniform could flip (log A > -17, log u being
    at least log 2^-24). With energies=True, the tracked energies (which keep accumulating
    over the launches) are compared with the oracle's f of the GPU states after every step:
    the largest relative error is returned. A summary line is appended to the file named by
    MCMC_PARITY_REPORT when that variable is set."""
    chans = list(tg.keys()) if channels is None else channels
    cur = states_now(det, batch)
    Np = det.cfg.chains
    trace = bool(det.cfg.engine & 16)
    res = dict(steps=0, mism=0, excused_cat=0, excused_acc=0, bad=0, bad_detail=[],
               min_gap=np.inf, w_cat=w_cat, w_acc=w_acc,
               bands=dict(acc_1e6=0, acc_1e4=0, acc_win=0, cat_1e6=0, cat_1e4=0, cat_win=0),
               oracle_ties=dict(acc_1e6=0, acc_1e4=0, cat_1e6=0, cat_1e4=0),
               max_dloga=None, dloga_p99=None, energy_rel_max=None)
    dl = []
    erel = 0.0
    for s in range(steps):
        t = t0 + s + 1
        det.run_chains(1, t - 1)
        nxt = states_now(det, batch)
        tr = det.get_trace() if trace else None
        ftr = det.get_tracked()[0] if energies else None
        for b in chans:
            exp, info = tg[b].step_chains(seed, b, t, cur[b])
            diff = np.any(exp != nxt[b], axis=1)
            res["steps"] += exp.shape[0]
            gap = np.abs(info["log_a"] - info["log_u"])
            cm = info["cat_margin"]
            res["min_gap"] = min(res["min_gap"], float(gap.min()))
            res["oracle_ties"]["acc_1e6"] += int((gap < 1e-6).sum())
            res["oracle_ties"]["acc_1e4"] += int((gap < 1e-4).sum())
            res["oracle_ties"]["cat_1e6"] += int((cm < 1e-6).sum())
            res["oracle_ties"]["cat_1e4"] += int((cm < 1e-4).sum())
            if tr is not None:
                # decisions that some uniform could flip: log A above log u's floor, log(2^-24)
                g = tr[b * Np:(b + 1) * Np]
                la = np.minimum(g[:, 0], 0.0)
                ok = (cm > 1e-3) & (info["log_a"] > -17.0)
                if ok.any():
                    dl.append(np.abs(la[ok] - info["log_a"][ok]))
            if ftr is not None:
                for c in range(Np):
                    fx = fp64_energy(tg[b], nxt[b][c])
                    erel = max(erel, abs(ftr[b * Np + c] - fx) / max(abs(fx), 1e-300))
            for c in np.nonzero(diff)[0]:
                res["mism"] += 1
                if cm[c] < w_cat:
                    res["excused_cat"] += 1
                    res["bands"]["cat_1e6" if cm[c] < 1e-6 else "cat_1e4" if cm[c] < 1e-4
                                 else "cat_win"] += 1
                elif gap[c] < w_acc:
                    res["excused_acc"] += 1
                    res["bands"]["acc_1e6" if gap[c] < 1e-6 else "acc_1e4" if gap[c] < 1e-4
                                 else "acc_win"] += 1
                else:
                    res["bad"] += 1
                    if len(res["bad_detail"]) < 10:
                        res["bad_detail"].append(dict(t=t, b=b, c=int(c), gap=float(gap[c]),
                                                      margin=float(cm[c]),
                                                      gpu=nxt[b][c].tolist(), exp=exp[c].tolist()))
        cur = nxt
    if dl:
        d = np.concatenate(dl)
        res["max_dloga"] = float(d.max())
        res["dloga_p99"] = float(np.quantile(d, 0.99))
    if energies:
        res["energy_rel_max"] = erel
    report(label, det, batch, res)
    return res


def report(label, det, batch, res):
    """Appends one JSON line of a parity result to $MCMC_PARITY_REPORT (if set)."""
    import json
    import os
    path = os.environ.get("MCMC_PARITY_REPORT")
    if not path:
        return
    prec = {0: "fp64", 1: "fp32", 2: "mixed"}[det.cfg.precision]
    line = dict(label=label, precision=prec, split_terms=det.cfg.split_terms,
                nt=int(batch.nt.max()), qam=int(batch.qam.max()), chains=det.cfg.chains,
                **{k: v for k, v in res.items() if k != "bad_detail"})
    with open(path, "a") as fh:
        fh.write(json.dumps(line, default=float) + "\n")


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
