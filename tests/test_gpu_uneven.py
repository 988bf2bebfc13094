"""The uneven batch at full size, in the launch configuration bench.py times: 16 384 channels with
Nt in {8, 16, 32, 64}, Nr in {Nt, 2 Nt}, QPSK / 16-QAM / 64-QAM, SNR U[10, 30] dB, 128 chains,
MIXED precision (two split-BF16 terms), autotuned engines and tiles, seed 0.

Tensor-core channels of N <= 64 of every shape class run in one packed launch whose CTAs pull
work items (largest first) from a device queue; the other classes are launch groups of their own
on parallel branches of one CUDA graph (the default for a batch of several groups). Checked
against the FP64 oracle on channels sampled from every (Nt, QAM) class: transition by transition
(step mode, the MIXED two-term windows) and after a 150-transition run (exact energies, best
energy, IS-LLRs of the exported final states). The packed launch equals one launch per class
chain for chain, and the autotuner's choices are the same for a second batch of the same
classes."""
import numpy as np
import pytest

import oracle
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu

NO_PACK, NO_GRAPH = 32, 64


@pytest.fixture(scope="module")
def batch():
    w = workload.WORKLOADS["uneven_16384"]
    return workload.uneven_batch(w["count"], w["seed"])


def _sample(b, per=1):
    """`per` channels of every (Nt, QAM) class, spread over the batch."""
    out = []
    for nt in (8, 16, 32, 64):
        for q in (4, 16, 64):
            idx = np.nonzero((b.nt == nt) & (b.qam == q))[0]
            if len(idx):
                out += [int(i) for i in idx[np.linspace(0, len(idx) - 1, per).astype(int)]]
    return out


def _det(b, **kw):
    return H.make_detector(b, chains=128, precision="mixed", split_terms=2, seed=0, **kw)


def test_uneven_full_size_groups_and_step_parity(batch):
    b = batch
    assert b.n_channels == 16384
    det = _det(b, engine=16)                      # MCMC_ENGINE_TRACE
    groups = det.launch_groups()
    assert sum(g["items"] for g in groups) > 0
    assert any(g["packed"] for g in groups), groups   # several one-tile classes: one launch
    sample = _sample(b)
    assert len(sample) == 12
    tg = H.targets(b, channels=sample)
    r = H.step_parity(det, b, tg, seed=0, steps=3, w_cat=6.4e-3, w_acc=6.4e-2, energies=True,
                      label="mixed_uneven_fullsize")
    assert r["steps"] == 3 * 128 * len(sample)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 100), r
    assert r["energy_rel_max"] <= 1e-10, r
    det.destroy()


def test_uneven_full_size_run_properties(batch):
    b = batch
    det = _det(b)
    det.run_chains(150)
    out = det.estimate(stats=True)
    flat, f = det.get_chains()
    ftr, _ = det.get_tracked()
    st = H.split_states(det, b, flat)
    sample = _sample(b, per=2)
    tg = H.targets(b, channels=sample)
    ant = np.concatenate([[0], np.cumsum(b.nt)])
    bits = np.concatenate([[0], np.cumsum(b.nt * np.log2(b.qam).astype(int))])
    for ch in sample:
        t = tg[ch]
        for c in range(0, 128, 11):
            fx = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(st[ch][c]))
            assert abs(f[ch * 128 + c] - fx) <= 1e-10 * abs(fx), (ch, c)
            assert abs(ftr[ch * 128 + c] - fx) <= 1e-10 * abs(fx), (ch, c)
        L = int(round(np.sqrt(b.qam[ch])))
        kb = H.levels_from_labels(out["best_idx"][ant[ch]:ant[ch + 1]], int(b.nt[ch]), L)
        fb = oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(kb))
        assert abs(out["best_f"][ch] - fb) <= 1e-9 * abs(fb) + 1e-9
        finals = [oracle.f_value(t.Hr, t.yr, t.sigma2, t.values(s)) for s in st[ch]]
        assert fb >= max(finals) - 1e-6 * abs(fb)
        ref = t.llr_is(st[ch])
        got = out["llr"][bits[ch]:bits[ch + 1]]
        fmax = float(np.abs(f[ch * 128:(ch + 1) * 128]).max())
        np.testing.assert_allclose(got, ref, atol=1e-5 * fmax + 1e-5 * max(1.0, np.abs(ref).max()),
                                   rtol=1e-5)
    assert out["stats"]["transitions"] == 150 * 128 * b.n_channels
    det.destroy()


def test_packed_launch_equals_one_launch_per_class(batch):
    # a 2048-channel slice of the batch (every class present): the packed launch from the work
    # queue, replayed from a graph, against one direct launch per shape class
    b = batch.subset(list(range(2048)))
    outs = []
    for flags in (0, NO_PACK | NO_GRAPH):
        det = _det(b, engine=flags)
        groups = det.launch_groups()
        assert any(g["packed"] for g in groups) == (flags == 0), groups
        det.run_chains(20)
        det.run_chains(10, 20)
        outs.append((det.get_chains()[0], det.estimate()))
        det.destroy()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1]["llr"], outs[1][1]["llr"])
    np.testing.assert_array_equal(outs[0][1]["best_idx"], outs[1][1]["best_idx"])


def test_autotuned_choices_are_stable(batch):
    # the choices made for the first batch of each class (process-wide) hold for the next batch
    b1 = batch.subset(list(range(4096)))
    b2 = batch.subset(list(range(4096, 8192)))
    d1 = _det(b1)
    d2 = _det(b2)
    g1 = {(g["engine"], g["tile"], g["packed"]) for g in d1.launch_groups()}
    g2 = {(g["engine"], g["tile"], g["packed"]) for g in d2.launch_groups()}
    assert g1 == g2, (g1, g2)
    d1.destroy()
    d2.destroy()
