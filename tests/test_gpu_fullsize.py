"""Parity at the full benchmark sizes, in the launch configuration bench.py times: 32x32 64-QAM
Rayleigh, SNR 20..32 dB (7 points x 4096 channels), 64 chains, MIXED precision with two split-BF16
terms, autotuned engine, seed 0. Sampled channels spread over the batch are checked against the
FP64 oracle: transition by transition (step mode, MIXED-S2 windows), and after a 200-transition
launch through properties that hold at any size (tracked and best energies equal FP64
evaluations of the exported states, LLRs equal the oracle's IS-LLR of the exported final
states). The same for the 128x128 Kronecker workload (N = 256, thread-block clusters)."""
import numpy as np
import pytest

import oracle
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu

SAMPLED = [0, 1, 4095, 4096, 9000, 14000, 20000, 24575, 28671]


@pytest.fixture(scope="module")
def bench_batch():
    w = workload.WORKLOADS["rayleigh_32x32_64qam"]
    return workload.rayleigh_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], w["per_snr"], w["seed"])


def _det(b, trace=False):
    return H.make_detector(b, chains=64, precision="mixed", split_terms=2, seed=0,
                           engine=16 if trace else 0)


def test_full_size_step_parity(bench_batch):
    b = bench_batch
    assert b.n_channels == 28672
    det = _det(b, trace=True)
    tg = H.targets(b, channels=SAMPLED)
    r = H.step_parity(det, b, tg, seed=0, steps=4, w_cat=6.4e-3, w_acc=6.4e-2, energies=True,
                      label="mixed_headline_fullsize")
    assert r["steps"] == 4 * 64 * len(SAMPLED)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 100), r
    assert r["energy_rel_max"] <= 1e-10, r
    det.destroy()


def test_full_size_run_properties(bench_batch):
    b = bench_batch
    det = _det(b)
    det.run_chains(200)
    out = det.estimate()
    flat, f = det.get_chains()        # FP64 evaluations of the final states
    ftr, _ = det.get_tracked()        # the energies the chains carry (read by the IS-LLR)
    st = H.split_states(det, b, flat)
    tg = H.targets(b, channels=SAMPLED)
    for ch in SAMPLED:
        t = tg[ch]
        # the energies the chains hold after the 200-transition run: FP32 increments from exact
        # initial values, replaced by exact evaluations when the run ends (the default
        # refresh_period 0), so they meet the 1e-5 relative bar with room to spare; the
        # evaluations handed out by get_chains likewise (the drift the increments accumulate
        # without the final evaluation is measured in test_gpu_energy_drift.py)
        for c in range(64):
            fx = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c]))
            assert abs(f[ch * 64 + c] - fx) <= 1e-10 * abs(fx), (ch, c, f[ch * 64 + c], fx)
            assert abs(ftr[ch * 64 + c] - fx) <= 1e-10 * abs(fx), (ch, c, ftr[ch * 64 + c], fx)
        # best sample: its FP64 energy is the reported best_f and no final state beats it
        lab = out["best_idx"][ch * 32:(ch + 1) * 32]
        kb = H.levels_from_labels(lab, 32, 8)
        fb = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(kb))
        assert abs(out["best_f"][ch] - fb) <= 1e-9 * abs(fb) + 1e-9
        finals = [oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c])) for c in range(64)]
        assert fb >= max(finals) - 1e-9 * abs(fb)
        # IS-LLR of the exported final states (Eqs. 34-36) in FP64 vs the GPU's FP32 read-out
        # from the tracked energies: a relative energy error e moves each log weight
        # ((tau - 1) / tau) f by at most e |f| / 2, so each log-sum-exp by as much and an LLR
        # by twice that; the FP32 log-sum-exp adds rounding of the weights' scale
        ref = t.llr_is(st[ch])
        got = out["llr"][ch * 192:(ch + 1) * 192]
        fmax = float(np.abs(f[ch * 64:(ch + 1) * 64]).max())
        np.testing.assert_allclose(got, ref, atol=1e-5 * fmax + 1e-5 * max(1.0, np.abs(ref).max()),
                                   rtol=1e-5)
    det.destroy()


# 128x128 64-QAM Kronecker (rho = 0.5), SNR 26..34 dB, 1024 channels, 256 chains, FP64 energy
# refresh every 50 transitions: the N = 256 workload, which runs on four-CTA thread-block clusters
# (autotuned chain tile).
KRON_SAMPLED = [0, 1, 511, 700, 1023]


@pytest.fixture(scope="module")
def kron_batch():
    w = workload.WORKLOADS["kronecker_128x128_64qam"]
    return workload.kronecker_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], w["total"], w["rho"], w["seed"])


def _kdet(b):
    return H.make_detector(b, chains=256, precision="mixed", split_terms=2, refresh_period=50, seed=0)


def test_kronecker_full_size_step_parity(kron_batch):
    b = kron_batch
    assert b.n_channels == 1024
    det = _kdet(b)
    tg = H.targets(b, channels=KRON_SAMPLED)
    r = H.step_parity(det, b, tg, seed=0, steps=2, w_cat=6.4e-3, w_acc=6.4e-2)
    assert r["steps"] == 2 * 256 * len(KRON_SAMPLED)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 100), r
    det.destroy()


def test_kronecker_full_size_run_properties(kron_batch):
    b = kron_batch
    det = _kdet(b)
    det.run_chains(300)   # the last transition is a refresh point
    out = det.estimate(stats=True)
    flat, f = det.get_chains()
    ftr, _ = det.get_tracked()
    st = H.split_states(det, b, flat)
    tg = H.targets(b, channels=KRON_SAMPLED)
    for ch in KRON_SAMPLED:
        t = tg[ch]
        for c in range(0, 256, 17):
            fx = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c]))
            assert abs(f[ch * 256 + c] - fx) <= 1e-10 * abs(fx), (ch, c, f[ch * 256 + c], fx)
            # the tracked energies right after the refresh (fixed-point digits of Gt)
            assert abs(ftr[ch * 256 + c] - fx) <= 1e-10 * abs(fx), (ch, c, ftr[ch * 256 + c], fx)
        lab = out["best_idx"][ch * 128:(ch + 1) * 128]
        kb = H.levels_from_labels(lab, 128, 8)
        fb = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(kb))
        assert abs(out["best_f"][ch] - fb) <= 1e-9 * abs(fb) + 1e-9
        finals = [oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c])) for c in range(256)]
        assert fb >= max(finals) - 1e-9 * abs(fb)
        ref = t.llr_is(st[ch])
        got = out["llr"][ch * 768:(ch + 1) * 768]
        np.testing.assert_allclose(got, ref, atol=2e-3 * max(1.0, np.abs(ref).max()), rtol=1e-4)
    # between refreshes the energies move by FP32 increments whose products carry the split
    # error 2^-17 of two BF16 terms, relative to the energy scale |y|^2 / sigma^2: the largest
    # correction a refresh made stays within ten such worst-case increments
    scale = max(float(np.sum(np.abs(b.y[b.y_off[i]:b.y_off[i] + b.nr[i]]) ** 2)) / float(b.sigma2[i])
                for i in range(b.n_channels))
    assert out["stats"]["refresh_drift"] <= 10 * 2.0 ** -17 * scale, (out["stats"]["refresh_drift"], scale)
    det.destroy()
