"""Soft-output variants on the GPU against the oracle (Sec. III-C): the list-based LLR of Eq. (31)
over the distinct final states (mcmc_detect_llr_list), and plain Monte Carlo with tau = 1 (the
IS-LLR of Eq. (34) reduces to it). Includes the degenerate list where every chain holds the same
state, and the argument errors."""
import numpy as np
import pytest

import oracle
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _batch(n=6, snr=14.0, seed=61):
    return workload.rayleigh_batch(4, 4, 16, [snr], n, seed)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-3), ("mixed", 1e-3)])
def test_list_llr_matches_oracle_on_gpu_states(precision, tol):
    b = _batch()
    det = H.make_detector(b, chains=32, precision=precision, seed=3)
    det.run_chains(40)
    llr = det.llr_list(25.0)
    flat, _ = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b)
    nb = 16
    distinct = 0
    for ch in range(b.n_channels):
        ref = tg[ch].llr_list(st[ch], 25.0)
        np.testing.assert_allclose(llr[ch * nb:(ch + 1) * nb], ref, rtol=tol, atol=tol)
        distinct += len({tuple(r) for r in st[ch]})
    assert distinct < 32 * b.n_channels      # repeated states occur: the deduplication is used
    det.destroy()


def test_identical_chains_give_clipped_llrs():
    b = _batch(n=2, seed=62)
    det = H.make_detector(b, chains=8, precision="fp32", seed=1)
    flat, _ = det.get_chains()
    st = H.split_states(det, b, flat)
    same = np.concatenate([np.tile(st[ch][0], 8) for ch in range(2)]).astype(np.int8)
    det.set_chains(same)
    llr = det.llr_list(7.5)
    tg = H.targets(b)
    for ch in range(2):
        np.testing.assert_array_equal(llr[ch * 16:(ch + 1) * 16], tg[ch].llr_list(st[ch][:1], 7.5))
        assert np.all(np.abs(llr[ch * 16:(ch + 1) * 16]) == 7.5)
    det.destroy()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 2e-3)])
def test_plain_monte_carlo_tau_one(precision, tol):
    b = _batch(n=5, seed=63)
    det = H.make_detector(b, chains=32, precision=precision, tau=1.0, seed=4)
    det.run_chains(30)
    out = det.estimate()
    flat, _ = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b, tau=1.0)
    for ch in range(b.n_channels):
        ref = tg[ch].llr_is(st[ch])
        np.testing.assert_allclose(out["llr"][ch * 16:(ch + 1) * 16], ref, rtol=tol, atol=tol)
    det.destroy()


def test_list_llr_argument_errors():
    from paper_2407_06042_gb300 import Detector, McmcError
    det = Detector(max_channels=2, max_nt=4, max_nr=4, chains=8, precision="fp32")
    with pytest.raises(McmcError) as e:
        det.llr_list(5.0, np.zeros(16, np.float32))
    assert e.value.status == 6                       # before preprocess
    det.destroy()
    b = _batch(n=1, seed=64)
    det = H.make_detector(b, chains=8, precision="fp32")
    for bad in (0.0, -1.0, float("inf")):
        with pytest.raises(McmcError) as e:
            det.llr_list(bad)
        assert e.value.status == 1
    det.destroy()
