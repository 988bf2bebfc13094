"""Parity at the full benchmark size, in the launch configuration bench.py times: 32x32 64-QAM
Rayleigh, SNR 20..32 dB (7 points x 4096 channels), 64 chains, MIXED precision with two split-BF16
terms, autotuned engine, seed 0. Sampled channels spread over the batch are checked against the
FP64 oracle: transition by transition (step mode, MIXED-S2 windows), and after a 200-transition
launch through properties that hold at any size (tracked and best energies equal FP64
evaluations of the exported states, LLRs equal the oracle's IS-LLR of the exported final
states)."""
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


def _det(b):
    return H.make_detector(b, chains=64, precision="mixed", split_terms=2, seed=0)


def test_full_size_step_parity(bench_batch):
    b = bench_batch
    assert b.n_channels == 28672
    det = _det(b)
    tg = H.targets(b, channels=SAMPLED)
    r = H.step_parity(det, b, tg, seed=0, steps=4, w_cat=6.4e-3, w_acc=6.4e-2)
    assert r["steps"] == 4 * 64 * len(SAMPLED)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 100), r
    det.destroy()


def test_full_size_run_properties(bench_batch):
    b = bench_batch
    det = _det(b)
    det.run_chains(200)
    out = det.estimate()
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b, channels=SAMPLED)
    for ch in SAMPLED:
        t = tg[ch]
        # tracked energies of the final states (FP32 increments, no refresh at this workload)
        # within the 1e-5 relative bar
        for c in range(0, 64, 7):
            fx = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c]))
            assert abs(f[ch * 64 + c] - fx) <= 1e-5 * abs(fx), (ch, c, f[ch * 64 + c], fx)
        # best sample: its FP64 energy is the reported best_f and no final state beats it
        lab = out["best_idx"][ch * 32:(ch + 1) * 32]
        kb = H.levels_from_labels(lab, 32, 8)
        fb = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(kb))
        assert abs(out["best_f"][ch] - fb) <= 1e-9 * abs(fb) + 1e-9
        finals = [oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c])) for c in range(64)]
        assert fb >= max(finals) - 1e-9 * abs(fb)
        # IS-LLR of the exported final states (Eqs. 34-36) in FP64 vs the GPU's FP32 read-out
        ref = t.llr_is(st[ch])
        got = out["llr"][ch * 192:(ch + 1) * 192]
        np.testing.assert_allclose(got, ref, atol=2e-3 * max(1.0, np.abs(ref).max()), rtol=1e-4)
    det.destroy()
