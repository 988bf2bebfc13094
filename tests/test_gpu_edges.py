"""Edge cases of the C ABI on the GPU: empty and oversized batches, zero iterations, the smallest
and largest chain counts, a 1x1 channel, an invalid noise variance, and the learned proposal's
argument and state errors."""
import numpy as np
import pytest

import oracle
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_empty_and_oversized_batches_are_rejected():
    from paper_2407_06042_gb300 import Detector, McmcError
    b = workload.generate([(2, 2, 4, 8.0)] * 3, 31)
    det = Detector(max_channels=2, max_nt=2, max_nr=2, chains=8)
    Hd, yd, s2 = H.upload(b)
    with pytest.raises(McmcError) as e:
        det.preprocess(b.nt[:0], b.nr[:0], b.qam[:0], Hd, b.H_off[:0], yd, b.y_off[:0], s2)
    assert e.value.status == 1
    with pytest.raises(McmcError) as e:                    # 3 channels > max_channels
        det.preprocess(b.nt, b.nr, b.qam, Hd, b.H_off, yd, b.y_off, s2)
    assert e.value.status == 1
    det.destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_iterations_keep_the_initial_states(precision):
    b = workload.generate([(3, 4, 16, 10.0), (2, 2, 4, 6.0)], 32)
    det = H.make_detector(b, chains=8, precision=precision, seed=4)
    det.run_chains(0)
    out = det.estimate()
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b)
    for ch in range(b.n_channels):
        for c in range(8):
            np.testing.assert_array_equal(st[ch][c], tg[ch].init_state(4, ch, c))
        fs = [oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(st[ch][c]))
              for c in range(8)]
        assert abs(out["best_f"][ch] - max(fs)) <= 1e-9 * abs(max(fs))
    det.destroy()


@pytest.mark.parametrize("chains", [4, 1024])
def test_smallest_and_largest_chain_counts(chains):
    b = workload.generate([(4, 4, 16, 12.0), (1, 1, 4, 9.0)], 33)
    det = H.make_detector(b, chains=chains, precision="mixed", split_terms=3, seed=6)
    tg = H.targets(b)
    r = H.step_parity(det, b, tg, seed=6, steps=2, w_cat=2e-4, w_acc=2e-3)
    assert r["steps"] == 2 * chains * 2
    assert r["bad"] == 0, r
    det.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_by_one_channel(precision):
    b = workload.generate([(1, 1, 64, 20.0), (1, 1, 4, 3.0)], 34)
    det = H.make_detector(b, chains=16, precision=precision, seed=7)
    w = (1e-6, 1e-6) if precision == "fp64" else (2e-4, 2e-3)
    r = H.step_parity(det, b, H.targets(b), seed=7, steps=5, w_cat=w[0], w_acc=w[1])
    assert r["bad"] == 0, r
    det.destroy()


def test_nonpositive_noise_variance_is_a_numeric_fault():
    from paper_2407_06042_gb300 import McmcError
    b = workload.generate([(2, 2, 4, 8.0), (2, 2, 4, 8.0)], 35)
    b.sigma2[1] = 0.0
    det = H.make_detector(b, chains=8, precision="fp32")
    det.run_chains(2)
    with pytest.raises(McmcError) as e:
        det.estimate()
    assert e.value.status == 5
    det.destroy()


def test_learned_api_errors():
    from paper_2407_06042_gb300 import McmcError, Mlp
    from paper_2407_06042_gb300 import learned
    b = workload.generate([(2, 2, 16, 8.0)], 36)
    m = Mlp(16, max_rows=64)
    m.set_params(learned.init_params(16, 0))
    d64 = H.make_detector(b, chains=8, precision="fp64")
    with pytest.raises(McmcError) as e:
        d64.set_model(m, 0.5)
    assert e.value.status == 7                             # FP64 handles: plain sampler only
    d64.destroy()
    plain = H.make_detector(b, chains=8, precision="fp32", preconditioned=False)
    with pytest.raises(McmcError) as e:
        plain.features(at_zero=True)
    assert e.value.status == 7                             # needs the preconditioned proposal
    plain.destroy()
    det = H.make_detector(b, chains=8, precision="fp32")
    with pytest.raises(McmcError) as e:
        det.mix_step(1)
    assert e.value.status == 6                             # no network attached
    with pytest.raises(McmcError) as e:
        det.set_model(m, 1.5)
    assert e.value.status == 1
    det.set_model(m, 0.5)
    with pytest.raises(McmcError) as e:
        det.mix_step(0)
    assert e.value.status == 1                             # transitions are numbered from 1
    det.mix_step(1)
    det.set_model(None, 0.0)
    with pytest.raises(McmcError) as e:
        det.init_learned()
    assert e.value.status == 6
    det.destroy()
    m.destroy()
